"""The four-term sum of the complex128 Grover coin (sum4.cuh; its three forms
sum4_rn, sum4_rn_flat and sum4_rn_cases), built for the host, against exact
rational arithmetic: when the addends lie within 8 binades
of the largest (and are normal, the result normal) it must equal the exact sum
rounded once to the nearest double (ties to even) -- Python's float() of a
Fraction rounds that way; otherwise it must equal the sequential double sum
((a + b) + c) + d.  CPU only."""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _dbl(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _case(rng, spread):
    e0 = rng.randint(-60, 60)
    xs = []
    for _ in range(4):
        kind = rng.random()
        if kind < 0.05:
            xs.append(rng.choice([0.0, -0.0]))
            continue
        m = rng.getrandbits(52) | (1 << 52)
        if rng.random() < 0.2:
            m |= 0xFFFFFFF   # long runs of ones: carries and ties
        e = e0 - rng.randint(0, spread)
        x = m * 2.0 ** (e - 52)
        xs.append(-x if rng.random() < 0.5 else x)
    return xs


def _exact_path(xs):
    nz = [x for x in xs if x != 0.0]
    if not nz:
        return True
    es = [struct.unpack("<Q", struct.pack("<d", x))[0] >> 52 & 0x7ff for x in nz]
    return max(es) - min(es) <= 8 and min(es) > 0


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_sum4_correctly_rounded(tmp_path):
    exe = tmp_path / "sum4_check"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2406_08186_b300", "csrc"),
                           "-o", str(exe), os.path.join(ROOT, "tests", "sum4_check.cpp")])
    rng = random.Random(7)
    cases = [_case(rng, rng.choice([0, 1, 3, 8, 8, 9, 20])) for _ in range(60000)]
    # hand-made: cancellation to zero, signed zeros, a carry to the next binade, ties
    cases += [[1.0, -1.0, 0.0, -0.0], [-0.0, -0.0, -0.0, -0.0], [0.0, -0.0, -0.0, -0.0],
              [2.0 ** 53 - 1, 2.0 ** 44, 0.0, 0.0], [2.0 ** 53 - 1, 2.0 ** 45, 1.0 * 2 ** 45, 0.0],
              [1.5, 1.5, 1.5, 1.5], [1e300, 1e300, 1e300, 1e300], [5e-324, 1.0, 0.0, 0.0],
              # deep cancellation: the exact sum is a few units of the last place
              [1.0 + 2.0 ** -52, -1.0, 0.0, 0.0], [1.0, -(1.0 - 2.0 ** -53), 0.0, 0.0],
              [3.0, -1.0, -2.0 + 2.0 ** -51, 2.0 ** -8], [-256.0, 255.0, 1.0, 2.0 ** -44]]
    text = "\n".join(" ".join("%016x" % _bits(x) for x in c) for c in cases) + "\n"
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0
    words = [int(h, 16) for h in out.stdout.split()]
    assert len(words) == 3 * len(cases)
    got = [tuple(words[3 * i:3 * i + 3]) for i in range(len(cases))]
    exact_seen = 0
    for c, g in zip(cases, got):
        if _exact_path(c):
            exact = sum((Fraction(x) for x in c), Fraction(0))
            try:
                want = float(exact) if exact != 0 else None
            except OverflowError:
                want = None
            if want is None or want == float("inf") or want == float("-inf") or (want != 0 and abs(want) < 2.2250738585072014e-308):
                # zero result, overflow or subnormal: the sequential sum
                want_bits = _bits(((c[0] + c[1]) + c[2]) + c[3])
                if exact == 0 and any(x != 0.0 for x in c):
                    want_bits = _bits(0.0)
            else:
                want_bits = _bits(want)
                exact_seen += 1
        else:
            want_bits = _bits(((c[0] + c[1]) + c[2]) + c[3])
        assert g == (want_bits,) * 3, (c, [hex(x) for x in g], hex(want_bits))
    assert exact_seen > 20000
