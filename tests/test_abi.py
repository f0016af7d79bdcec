"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
and its host-side graph construction is bit-exact against the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2406_08186_b300 as hw
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hw_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    L = hw.lib()
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value
    assert set(hw.EXPORTS) <= declared


def test_version_and_opts():
    assert "sm_103a" in hw.hw_version()
    o = hw.hw_opts_init()
    assert (o.record_stride, o.taylor_degree, o.taylor_squarings, o.gemm_mode, o.tile) == (1, 0, -1, 0, 0)
    assert (o.u_symmetric, o.addressing, o.shift, o.launch_mode, o.taylor_powers, o.gemm_tiles) == (0,) * 6


def test_opts_struct_matches_header():
    # hw_opts_init writes sizeof(hw_opts) bytes: the binding's struct must
    # carry the header's fields, in order, all int32
    import re
    text = open(os.path.join(ROOT, "include", "hiperwalk_b300.h")).read()
    body = text[text.index("typedef struct hw_opts {"):text.index("} hw_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"int32_t\s+(\w+)\s*;", body)
    assert [f for f, _ in hw.hw_opts._fields_] == fields
    assert ctypes.sizeof(hw.hw_opts) == 4 * len(fields)


def _graphs():
    yield "torus64", synth.torus(64)
    yield "Q10", synth.hypercube(10)
    yield "K40", synth.complete(40)
    yield "star", synth.star(3000)
    yield "er", synth.erdos_renyi(1 << 14, 8 / ((1 << 14) - 1), seed=5)
    yield "er_iso", synth.erdos_renyi(500, 0.002, seed=8, drop_isolated=False)   # degree-0 vertices
    yield "reg3", synth.random_regular(1000, 3, seed=9)


@pytest.mark.parametrize("name,g", list(_graphs()))
def test_arc_basis_bit_exact_vs_oracle(name, g):
    n, eu, ev = g
    row_ptr, col = synth.adjacency_csr(n, eu, ev, scramble_seed=17)
    rp, head, rev = hw.hw_graph_arcs_host(n, row_ptr, col)
    ref = oracle.Arcs(n, eu, ev)
    assert np.array_equal(rp.astype(np.int64), ref.row_ptr)
    assert np.array_equal(head, ref.head)
    assert np.array_equal(rev.astype(np.int64), ref.rev)


@pytest.mark.parametrize("case", ["self_loop", "duplicate", "asymmetric", "out_of_range",
                                  "bad_row_ptr", "n_zero"])
def test_invalid_graphs_rejected(case):
    n = 4
    rp = np.array([0, 1, 2, 3, 4], np.int64)
    col = np.array([1, 0, 3, 2], np.int32)
    if case == "self_loop":
        col = np.array([0, 0, 3, 2], np.int32)
    elif case == "duplicate":
        rp = np.array([0, 2, 4, 5, 6], np.int64)
        col = np.array([1, 1, 0, 0, 3, 2], np.int32)
    elif case == "asymmetric":
        col = np.array([1, 2, 3, 2], np.int32)
    elif case == "out_of_range":
        col = np.array([1, 0, 3, 7], np.int32)
    elif case == "bad_row_ptr":
        rp = np.array([0, 2, 1, 3, 4], np.int64)
    elif case == "n_zero":
        n, rp = 0, np.array([0], np.int64)
    with pytest.raises(hw.HWError) as e:
        hw.hw_graph_arcs_host(n, rp, col)
    assert e.value.status == hw.HW_EINVAL
    assert hw.hw_last_error()


def test_weights_must_be_hermitian_and_finite():
    # host-side validation runs before any device call
    import math
    n, eu, ev = synth.cycle(6)
    rp, col, w = synth.weighted_csr(n, eu, ev, synth.edge_weights(eu.size, seed=1, complex_phase=True))
    bad = w.copy()
    bad[0] = np.conj(bad[0]) * 1.5       # breaks W[v][u] == conj(W[u][v])
    with pytest.raises(hw.HWError) as e:
        hw.hw_graph_csr_weighted(n, rp, col, bad, stream=0)
    assert e.value.status == hw.HW_EINVAL and "Hermitian" in e.value.message
    bad = w.copy()
    bad[2] = complex(math.inf, 0.0)
    with pytest.raises(hw.HWError) as e:
        hw.hw_graph_csr_weighted(n, rp, col, bad, stream=0)
    assert e.value.status == hw.HW_EINVAL and "finite" in e.value.message
    rbad = w.real.copy()
    rbad[3] += 0.5                       # real W must be symmetric
    with pytest.raises(hw.HWError) as e:
        hw.hw_graph_csr_weighted(n, rp, col, rbad, stream=0)
    assert e.value.status == hw.HW_EINVAL
