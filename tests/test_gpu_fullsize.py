"""Parity at the benchmarked sizes, in the launch configuration bench.py times.

Configuration 2 (1024 x 1024 torus search, 3000 steps): the whole run is
compared with the oracle (amplitudes, per-vertex probabilities and the marked
probability after every step).  Configuration 4 (Erdos-Renyi, n = 2^20, 64
states drawn on the device as the benchmark draws them, 500 steps): batch
columns 0, 1, 31 and 63 are compared with the oracle over the whole run
(amplitudes and per-vertex probabilities), and every column's norm.  The
degree-20 hypercube record (2^20 vertices, complex128): 12 steps of the same
walk against the oracle.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torus_search():
    L, steps = 1024, 3000
    g = synth.torus(L)
    m = synth.seeded_vertex(2, L * L)
    ar = oracle.Arcs(*g)
    psi0 = synth.uniform_state(ar.num_arcs)
    ref, rec = oracle.coined_evolve(ar, psi0, steps, marked=[m], record=True)
    return g, m, ar, psi0, ref, rec, oracle.prob_coined(ar, ref)


def _run(hw, g, m, psi0, steps, dt):
    import torch
    n = g[0]
    row_ptr, col = synth.adjacency_csr(*g)
    G = hw.hw_graph_csr(n, row_ptr, col)
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    x = torch.from_numpy(psi0).to("cuda", cdt)
    out = torch.empty_like(x)
    rec = torch.empty(steps, dtype=torch.float64, device="cuda")
    prob = torch.empty(n, dtype=torch.float64, device="cuda")
    norm = torch.empty(1, dtype=torch.float64, device="cuda")
    hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [m], dt, 1, steps, x, out, rec)
    hw.hw_probability(G, n, dt, 1, out, prob, norm)
    torch.cuda.synchronize()
    res = out.cpu().numpy().astype(np.complex128), rec.cpu().numpy(), prob.cpu().numpy(), float(norm.item())
    G.free()
    return res


def test_config2_complex128_full_run(hw, torus_search):
    g, m, ar, psi0, ref, rec_ref, p_ref = torus_search
    psi, rec, prob, norm = _run(hw, g, m, psi0, 3000, hw.HW_C128)
    assert np.max(np.abs(psi - ref)) <= 1e-12
    assert np.max(np.abs(rec - rec_ref)) <= 1e-12
    assert np.max(np.abs(prob - p_ref)) <= 1e-12
    assert abs(norm - 1.0) <= 1e-12
    assert abs(rec[-1] - prob[m]) <= 1e-15


def test_config2_complex64_full_run(hw, torus_search):
    g, m, ar, psi0, ref, rec_ref, p_ref = torus_search
    psi, rec, prob, norm = _run(hw, g, m, psi0, 3000, hw.HW_C64)
    assert np.sum(np.abs(prob - p_ref)) <= 1e-3
    assert np.max(np.abs(rec - rec_ref)) <= 1e-4
    assert abs(norm - 1.0) <= 1e-4


def test_config4_batched_full_run_columns(hw):
    # the benchmark's input: 64 Gaussian states drawn on the device by the
    # seeded recipe (synth.gaussian_states_device, seed 4), rounded to complex64
    import torch
    n0 = 1 << 20
    g = synth.erdos_renyi(n0, 8.0 / (n0 - 1), seed=5)
    n = g[0]
    ar = oracle.Arcs(*g)
    A2, B, steps = ar.num_arcs, 64, 500
    cols = [0, 1, 31, 63]
    x = synth.gaussian_states_device(A2, B, seed=4, dtype=torch.complex64)
    # the device draws agree with the host recipe up to the complex64 rounding
    # of values that differ in their last float64 bits
    for b in (0, 63):
        z = synth.complex_gaussian(4, A2, b * A2)      # column b of synth.gaussian_states
        host = z / np.sqrt(np.sum(np.abs(z) ** 2))
        dev = x[:, b].cpu().numpy()
        assert np.max(np.abs(dev - host.astype(np.complex64))) <= 2.0 ** -23 * np.max(np.abs(host))
    row_ptr, col = synth.adjacency_csr(*g)
    G = hw.hw_graph_csr(n, row_ptr, col)
    out = torch.empty_like(x)
    hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [], hw.HW_C64, B, steps, x, out)
    prob = torch.empty(n * B, dtype=torch.float64, device="cuda")
    norm = torch.empty(B, dtype=torch.float64, device="cuda")
    hw.hw_probability(G, n, hw.HW_C64, B, out, prob, norm)
    probs = prob.reshape(n, B).cpu().numpy()
    got_all = out.cpu().numpy()
    for b in cols:
        start = x[:, b].cpu().numpy().astype(np.complex128)   # the complex64-rounded start
        ref = oracle.coined_evolve(ar, start, steps)
        got = got_all[:, b].astype(np.complex128)
        # complex64 rounding, 2^-24 relative per operation, a few operations per
        # amplitude and step, accumulated at worst linearly over the run
        tol = steps * 4 * 2.0 ** -24 * np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) <= tol, b
        assert np.sum(np.abs(probs[:, b] - oracle.prob_coined(ar, ref))) <= 1e-3, b
    assert np.max(np.abs(norm.cpu().numpy() - 1.0)) <= 1e-4
    G.free()


def test_hypercube20_complex128_against_oracle(hw):
    # the bench's degree-20 record: the 2^20-vertex hypercube, uniform start,
    # one seeded mark, complex128 in the two-pass kernel (index-free), here for
    # 12 steps with the marked probability after every step, against the oracle
    import torch
    k, steps = 20, 12
    g = synth.hypercube(k)
    n = g[0]
    m = synth.seeded_vertex(3, n)
    ar = oracle.Arcs(*g)
    psi0 = synth.uniform_state(ar.num_arcs)
    ref, rr = oracle.coined_evolve(ar, psi0, steps, marked=[m], record=True)
    row_ptr, col = synth.adjacency_csr(*g)
    G = hw.hw_graph_csr(n, row_ptr, col)
    x = torch.from_numpy(psi0).cuda()
    y = torch.empty_like(x)
    rec = torch.empty(steps, dtype=torch.float64, device="cuda")
    hw.hw_coined_evolve(G, 0, [m], 2, 1, steps, x, y, rec)
    torch.cuda.synchronize()
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12
    assert np.max(np.abs(rec.cpu().numpy() - rr)) <= 1e-12
    G.free()
