"""Parity at the benchmarked sizes, in the launch configuration bench.py times.

Configuration 2 (1024 x 1024 torus search, 3000 steps): the whole run is
compared with the oracle (amplitudes, per-vertex probabilities and the marked
probability after every step).  Configuration 4 (Erdos-Renyi, n = 2^20, 64
states, 500 steps): sampled batch columns are compared with the oracle over a
prefix of the run, and every column's norm over the whole run.
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


def test_config4_batched_sampled_columns(hw):
    import torch
    n0 = 1 << 20
    g = synth.erdos_renyi(n0, 8.0 / (n0 - 1), seed=5)
    n = g[0]
    ar = oracle.Arcs(*g)
    A2, B = ar.num_arcs, 64
    cols = [0, 63]
    gen = torch.Generator(device="cuda").manual_seed(4)
    x = torch.randn((A2, B), dtype=torch.complex64, device="cuda", generator=gen)
    x /= torch.linalg.vector_norm(x, dim=0, keepdim=True)
    seeded = {}
    for b in cols:
        z = synth.complex_gaussian(4, A2, b * A2)
        z /= math.sqrt(np.sum(np.abs(z) ** 2))
        seeded[b] = z
        x[:, b] = torch.from_numpy(z).to("cuda", torch.complex64)
    row_ptr, col = synth.adjacency_csr(*g)
    G = hw.hw_graph_csr(n, row_ptr, col)
    out = torch.empty_like(x)
    prefix = 100
    hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [], hw.HW_C64, B, prefix, x, out)
    prob = torch.empty(n * B, dtype=torch.float64, device="cuda")
    hw.hw_probability(G, n, hw.HW_C64, B, out, prob)
    probs = prob.reshape(n, B).cpu().numpy()
    for b in cols:
        start = x[:, b].cpu().numpy().astype(np.complex128)   # the complex64-rounded start
        ref = oracle.coined_evolve(ar, start, prefix)
        assert np.sum(np.abs(probs[:, b] - oracle.prob_coined(ar, ref))) <= 1e-3
    norm = torch.empty(B, dtype=torch.float64, device="cuda")
    hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [], hw.HW_C64, B, 500, x, out)
    hw.hw_probability(G, n, hw.HW_C64, B, out, None, norm)
    assert np.max(np.abs(norm.cpu().numpy() - 1.0)) <= 1e-4
    G.free()
