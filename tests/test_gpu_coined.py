"""GPU parity of the coined walk (Sec. 3.2) against the FP64 oracle.

Tolerances: complex128 amplitudes max-abs <= 1e-12; complex64 probability
vectors L1 <= 1e-3 after 1000 steps.  Cases span several tiles and ragged
tails, degree-0/1 vertices, vertices larger than a tile, marked vertices at
both ends of the vertex range, both coins, batches, in-place calls and records.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL128 = 1e-12
TOL64_L1 = 1e-3


def _torch():
    import torch
    return torch


def run_gpu(hw, g, psi0, steps, coin=0, marked=(), dt=2, record=False, stride=1, inplace=False,
            batch=1):
    """Evolve on the device through the C ABI; returns numpy results."""
    torch = _torch()
    n, eu, ev = g
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    G = hw.hw_graph_csr(n, row_ptr, col)
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    x = torch.from_numpy(np.ascontiguousarray(psi0)).to("cuda", cdt)
    out = x if inplace else torch.empty_like(x)
    rec = None
    if record:
        rec = torch.full(((steps // stride) * batch,), -1.0, dtype=torch.float64, device="cuda")
    hw.hw_coined_evolve(G, coin, list(marked), dt, batch, steps, x, out, rec,
                        opts={"record_stride": stride} if stride != 1 else None)
    prob = torch.empty(n * batch, dtype=torch.float64, device="cuda")
    norm = torch.empty(batch, dtype=torch.float64, device="cuda")
    hw.hw_probability(G, n, dt, batch, out, prob, norm)
    torch.cuda.synchronize()
    res = dict(psi=out.cpu().numpy().astype(np.complex128), prob=prob.cpu().numpy(),
               norm=norm.cpu().numpy(), rec=None if rec is None else rec.cpu().numpy())
    G.free()
    return res


def _graphs():
    yield "torus64", synth.torus(64)
    yield "er_2k", synth.erdos_renyi(2000, 8 / 1999, seed=5)
    yield "er_iso", synth.erdos_renyi(3000, 0.0007, seed=8, drop_isolated=False)  # degrees 0, 1, 2..
    yield "Q9", synth.hypercube(9)
    yield "K1100", synth.complete(1100)          # degree 1099 > one tile
    yield "star", synth.star(2500)               # hub of degree 2499, leaves of degree 1
    yield "reg3", synth.random_regular(5001 * 2, 3, seed=9)


@pytest.mark.parametrize("coin", [0, 1])
@pytest.mark.parametrize("name,g", list(_graphs()))
def test_coined_c128_matches_oracle(hw, name, g, coin):
    if name == "K1100" and coin == 1:
        pytest.skip("O(d^3) oracle per step; the star graph covers Fourier on a large vertex")
    n = g[0]
    ar = oracle.Arcs(*g)
    steps = 2 if name == "K1100" else 37
    psi0 = synth.random_state(ar.num_arcs, seed=31)
    marked = [0, n - 1, n // 3]
    ref, rec_ref = oracle.coined_evolve(ar, psi0, steps, coin, marked, record=True)
    got = run_gpu(hw, g, psi0, steps, coin=coin, marked=marked, record=True)
    assert np.max(np.abs(got["psi"] - ref)) <= TOL128
    assert np.max(np.abs(got["prob"] - oracle.prob_coined(ar, ref))) <= TOL128
    assert np.max(np.abs(got["rec"] - rec_ref)) <= TOL128
    assert abs(got["norm"][0] - 1.0) <= 1e-12


def test_config1_torus64_center_100_steps(hw):
    # 64 x 64 torus, Grover, no mark, 1/2 on the 4 arcs of (32, 32), 100 steps.
    g = synth.torus(64)
    ar = oracle.Arcs(*g)
    psi0 = synth.state_on_vertex_arcs(synth.arc_offsets(*g), 32 * 64 + 32)
    ref = oracle.coined_evolve(ar, psi0, 100)
    got = run_gpu(hw, g, psi0, 100)
    assert np.max(np.abs(got["psi"] - ref)) <= TOL128
    p = got["prob"]
    assert np.max(np.abs(p - oracle.prob_coined(ar, ref))) <= TOL128
    P = p.reshape(64, 64)
    refl = (64 - np.arange(64)) % 64
    assert np.max(np.abs(P - P[refl][:, refl])) < 1e-14


def test_uniform_state_stationary(hw):
    g = synth.erdos_renyi(20000, 8 / 19999, seed=3)
    ar = oracle.Arcs(*g)
    psi0 = synth.uniform_state(ar.num_arcs)
    got = run_gpu(hw, g, psi0, 50)
    assert np.max(np.abs(got["psi"] - psi0)) < 1e-15


def test_cycle_translation(hw):
    N = 1001
    g = synth.cycle(N)
    ar = oracle.Arcs(*g)
    psi0 = synth.random_state(ar.num_arcs, seed=2)
    T = 123
    got = run_gpu(hw, g, psi0, T)["psi"]
    ref = oracle.coined_evolve(ar, psi0, T)   # exact permutation in the oracle
    assert np.max(np.abs(got - ref)) < 1e-15


@pytest.mark.parametrize("steps", [1, 2, 5, 6])
def test_in_place_and_step_parity(hw, steps):
    g = synth.erdos_renyi(3000, 5 / 2999, seed=6)
    ar = oracle.Arcs(*g)
    psi0 = synth.random_state(ar.num_arcs, seed=7)
    ref = oracle.coined_evolve(ar, psi0, steps, marked=[10])
    for inplace in (False, True):
        got = run_gpu(hw, g, psi0, steps, marked=[10], inplace=inplace)
        assert np.max(np.abs(got["psi"] - ref)) <= TOL128


def test_zero_steps_copies(hw):
    g = synth.torus(5)
    psi0 = synth.random_state(100, seed=1)
    got = run_gpu(hw, g, psi0, 0)
    assert np.array_equal(got["psi"], psi0)


def test_record_stride(hw):
    g = synth.torus(40)
    ar = oracle.Arcs(*g)
    psi0 = synth.uniform_state(ar.num_arcs)
    marked = [123, 800]
    _, rec_ref = oracle.coined_evolve(ar, psi0, 60, marked=marked, record=True)
    got = run_gpu(hw, g, psi0, 60, marked=marked, record=True, stride=4)
    assert got["rec"].shape == (15,)
    assert np.max(np.abs(got["rec"] - rec_ref[3::4])) <= TOL128


@pytest.mark.parametrize("name,g,coin", [
    ("torus64_grover", synth.torus(64), 0),      # edge-major, unrolled (degree 4)
    ("torus64_fourier", synth.torus(64), 1),
    ("reg5", synth.random_regular(3001 * 2, 5, seed=3), 0),
    ("Q9", synth.hypercube(9), 0),                # degree 9..16: arc-major lane groups
    ("reg20", synth.random_regular(3000, 20, seed=4), 0),   # degree > 16: edge-major, two passes
    ("Q9_fourier", synth.hypercube(9), 1),        # Fourier above degree 8: arc-major
])
def test_c64_regular_graph_paths(hw, name, g, coin):
    # complex64 on every kernel path of a regular graph, against the FP64 oracle
    ar = oracle.Arcs(*g)
    psi0 = synth.random_state(ar.num_arcs, seed=21)
    marked = [1, g[0] - 2]
    ref, rec_ref = oracle.coined_evolve(ar, psi0, 60, coin_kind=coin, marked=marked, record=True)
    got = run_gpu(hw, g, psi0, 60, coin=coin, marked=marked, dt=1, record=True)
    assert np.max(np.abs(got["psi"] - ref)) < 2e-5
    assert np.sum(np.abs(got["prob"] - oracle.prob_coined(ar, ref))) <= 1e-4
    assert np.max(np.abs(got["rec"] - rec_ref)) < 1e-5


@pytest.mark.parametrize("steps", [1, 2, 5])
def test_in_place_regular_graph(hw, steps):
    # the edge-major path with psi_in == psi_out
    g = synth.random_regular(4000, 4, seed=13)
    ar = oracle.Arcs(*g)
    psi0 = synth.random_state(ar.num_arcs, seed=14)
    ref = oracle.coined_evolve(ar, psi0, steps, marked=[0, 3999])
    for inplace in (False, True):
        got = run_gpu(hw, g, psi0, steps, marked=[0, 3999], inplace=inplace)
        assert np.max(np.abs(got["psi"] - ref)) <= TOL128


def test_c64_probability_l1_after_1000_steps(hw):
    g = synth.erdos_renyi(5000, 8 / 4999, seed=11)
    ar = oracle.Arcs(*g)
    psi0 = synth.random_state(ar.num_arcs, seed=12)
    marked = [17]
    ref, rec_ref = oracle.coined_evolve(ar, psi0, 1000, marked=marked, record=True)
    got = run_gpu(hw, g, psi0, 1000, marked=marked, dt=1, record=True)
    l1 = np.sum(np.abs(got["prob"] - oracle.prob_coined(ar, ref)))
    assert l1 <= TOL64_L1, l1
    assert np.max(np.abs(got["rec"] - rec_ref)) < 1e-4
    assert abs(got["norm"][0] - 1.0) < 1e-4


@pytest.mark.parametrize("dt", [1, 2])
@pytest.mark.parametrize("coin", [0, 1])
def test_batched_matches_oracle_columns(hw, dt, coin):
    g = synth.erdos_renyi(4000, 8 / 3999, seed=13)
    ar = oracle.Arcs(*g)
    B, steps = 5, 25
    psi0 = synth.gaussian_states(ar.num_arcs, B, seed=4)
    marked = [2, ar.n - 1]
    got = run_gpu(hw, g, psi0, steps, coin=coin, marked=marked, dt=dt, record=True, batch=B)
    psi = got["psi"].reshape(ar.num_arcs, B)
    prob = got["prob"].reshape(ar.n, B)
    rec = got["rec"].reshape(steps, B)
    for b in range(B):
        ref, rec_ref = oracle.coined_evolve(ar, psi0[:, b], steps, coin, marked, record=True)
        pref = oracle.prob_coined(ar, ref)
        if dt == 2:
            assert np.max(np.abs(psi[:, b] - ref)) <= TOL128
            assert np.max(np.abs(prob[:, b] - pref)) <= TOL128
            assert np.max(np.abs(rec[:, b] - rec_ref)) <= TOL128
        else:
            assert np.sum(np.abs(prob[:, b] - pref)) <= TOL64_L1
    assert np.max(np.abs(got["norm"] - 1.0)) < (1e-12 if dt == 2 else 1e-4)


def test_device_tables_match_host_build(hw):
    torch = _torch()
    n, eu, ev = synth.erdos_renyi(7000, 6 / 6999, seed=14)
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    G = hw.hw_graph_csr(n, row_ptr, col)
    info = hw.hw_graph_info(G)
    ref = oracle.Arcs(n, eu, ev)
    m = ref.num_arcs
    assert info["n"] == n and info["num_arcs"] == m
    import ctypes
    for key, want in (("d_row_ptr", ref.row_ptr), ("d_head", ref.head), ("d_rev", ref.rev)):
        host = np.empty(want.size, np.int32)
        torch.cuda.synchronize()
        ctypes.CDLL("libcudart.so.13").cudaMemcpy(host.ctypes.data_as(ctypes.c_void_p),
                                                   ctypes.c_void_p(info[key]),
                                                   ctypes.c_size_t(host.nbytes), 2)
        assert np.array_equal(host.astype(np.int64), want.astype(np.int64)), key
    G.free()


def test_invalid_calls_report_errors(hw):
    torch = _torch()
    g = synth.torus(8)
    row_ptr, col = synth.adjacency_csr(*g)
    G = hw.hw_graph_csr(g[0], row_ptr, col)
    x = torch.zeros(G.num_arcs, dtype=torch.complex128, device="cuda")
    rec = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(hw.HWError) as e:
        hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 4, x, x, rec)     # record without marks
    assert e.value.status == hw.HW_EINVAL
    with pytest.raises(hw.HWError) as e:
        hw.hw_coined_evolve(G, 0, [64], hw.HW_C128, 1, 4, x, x)        # mark out of range
    assert e.value.status == hw.HW_EINVAL
    with pytest.raises(hw.HWError) as e:
        hw.hw_coined_evolve(G, 0, [1, 1], hw.HW_C128, 1, 4, x, x)      # repeated mark
    assert e.value.status == hw.HW_EINVAL
    with pytest.raises(hw.HWError) as e:
        hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 4, x[:-1], x[1:])  # overlapping buffers
    assert e.value.status == hw.HW_EINVAL
    G.free()


@pytest.mark.parametrize("tile", [1, 6, 7, 12, 13, 14])
@pytest.mark.parametrize("dt,B", [(1, 8), (2, 4), (1, 64)])
def test_batched_every_launch_shape(hw, tile, dt, B):
    # every register-row shape and both TMA-ring shapes, with a record; degrees
    # up to 20 exercise the rows that do not fit the register/ring capacity
    import torch
    g = synth.erdos_renyi(3000, 10 / 2999, seed=17)
    ar = oracle.Arcs(*g)
    n, steps = ar.n, 9
    psi0 = synth.gaussian_states(ar.num_arcs, B, seed=5)
    marked = [4, n - 2]
    row_ptr, col = synth.adjacency_csr(*g)
    G = hw.hw_graph_csr(n, row_ptr, col)
    cdt = torch.complex128 if dt == 2 else torch.complex64
    x = torch.from_numpy(psi0).to("cuda", cdt).reshape(-1)
    out = torch.empty_like(x)
    rec = torch.empty(steps * B, dtype=torch.float64, device="cuda")
    hw.hw_coined_evolve(G, 0, marked, dt, B, steps, x, out, rec, opts={"tile": tile})
    torch.cuda.synchronize()
    psi = out.cpu().numpy().astype(np.complex128).reshape(-1, B)
    recs = rec.cpu().numpy().reshape(steps, B)
    for b in (0, B - 1):
        ref, rr = oracle.coined_evolve(ar, psi0[:, b], steps, 0, marked, record=True)
        tol = TOL128 if dt == 2 else 1e-5
        assert np.max(np.abs(psi[:, b] - ref)) <= tol
        assert np.max(np.abs(recs[:, b] - rr)) <= tol
    G.free()
