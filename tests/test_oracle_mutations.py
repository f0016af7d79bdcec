"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/hw_oracle.c (a dropped term, a
wrong sign, a wrong index, a transposed lookup), builds it, and runs the oracle
pin suite against it in a subprocess; the suite must fail.  Everything runs on
the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hw_oracle.c")

MUTATIONS = {
    "grover_weight": ("c = 2.0 / (double)d - ((j == k) ? 1.0 : 0.0);",
                      "c = 1.0 / (double)d - ((j == k) ? 1.0 : 0.0);"),
    "grover_sign": ("c = 2.0 / (double)d - ((j == k) ? 1.0 : 0.0);",
                    "c = ((j == k) ? 1.0 : 0.0) - 2.0 / (double)d;"),
    "fourier_conjugate": ("c = (cos(ang) + I * sin(ang)) / sqrt((double)d);",
                          "c = (cos(ang) - I * sin(ang)) / sqrt((double)d);"),
    "fourier_norm": ("c = (cos(ang) + I * sin(ang)) / sqrt((double)d);",
                     "c = (cos(ang) + I * sin(ang)) / (double)d;"),
    "marked_plus_identity": ("c = (j == k) ? -1.0 : 0.0;", "c = (j == k) ? 1.0 : 0.0;"),
    "shift_identity": ("int64_t b = arc_in_row(row_ptr, head, head[a], v);",
                       "int64_t b = arc_in_row(row_ptr, head, v, head[a]);"),
    "persistent_turns_back": ("int64_t u = ((xw + dx) % L1) * L2 + (yw + dy) % L2;",
                              "int64_t u = ((xw - dx + L1) % L1) * L2 + (yw - dy + L2) % L2;"),
    "persistent_axes_swapped": ("int64_t u = ((xw + dx) % L1) * L2 + (yw + dy) % L2;",
                                "int64_t u = ((xw + dy) % L1) * L2 + (yw + dx) % L2;"),
    "weight_conjugated": ("acc += (w ? w[a] : 1.0) * x[head[a]];", "acc += (w ? conj(w[a]) : 1.0) * x[head[a]];"),
    "weight_ignored": ("acc += (w ? w[a] : 1.0) * x[head[a]];", "acc += x[head[a]];"),
    "arc_weight_not_conjugate": ("w_arc[b] = conj(we[e]);", "w_arc[b] = we[e];"),
    "rev_self": ("rev[a] = find_arc(arcs, num, arcs[a].head, arcs[a].tail);",
                 "rev[a] = find_arc(arcs, num, arcs[a].tail, arcs[a].head);"),
    "ham_gamma_sign": ("acc = -gamma * acc;", "acc = gamma * acc;"),
    "ham_marked_sign": ("if (marked && marked[v]) acc -= x[v];", "if (marked && marked[v]) acc += x[v];"),
    "time_reversed": ("cplx f = -I * tau / (double)k;", "cplx f = I * tau / (double)k;"),
    "series_truncated": ("if (mx < 1e-18) break;", "if (mx < 1e-7) break;"),
    "prob_drops_imag": ("acc += creal(psi[a]) * creal(psi[a]) + cimag(psi[a]) * cimag(psi[a]);\n        p[v] = acc;",
                        "acc += creal(psi[a]) * creal(psi[a]);\n        p[v] = acc;"),
    "record_off_by_one": ("if (record && marked) record[t - 1] = marked_prob_coined(n, row_ptr, marked, psi);",
                          "if (record && marked && t > 1) record[t - 2] = marked_prob_coined(n, row_ptr, marked, psi);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "hw_oracle_mut.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                           "-fcx-fortran-rules", str(mut), "-o", str(lib), "-lm"])
    env = dict(os.environ, HW_ORACLE_LIB_OVERRIDE=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_coined.py"),
                        os.path.join(ROOT, "tests", "test_oracle_ctqw.py"),
                        os.path.join(ROOT, "tests", "test_oracle_persistent.py"),
                        os.path.join(ROOT, "tests", "test_oracle_weighted.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake %r was not caught:\n%s" % (name, r.stdout[-2000:])
