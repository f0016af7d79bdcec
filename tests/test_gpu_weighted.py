"""GPU parity of the continuous-time walk with a weighted adjacency,
H = -gamma W - sum_m |m><m| (Sec. 3.1 with A generalised to a Hermitian W),
against the FP64 oracle: the sparse-action series (real and complex W, one and
several columns, records), the dense U (real symmetric W, complex128 and the
complex64 tensor-core path; complex W through the sparse series on the
identity's columns), the flux ring's closed form, and the calls that a
weighted graph does not take.

Tolerances: complex128 max-abs <= 1e-12; complex64 probability L1 <= 1e-3
(sparse series) and entry-wise 2e-6 (dense U, as the unweighted tests).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL128 = 1e-12


def _torch():
    import torch
    return torch


def _wgraph(hw, g, we):
    n, eu, ev = g
    rp, col, w = synth.weighted_csr(n, eu, ev, we)
    return hw.hw_graph_csr_weighted(n, rp, col, w)


def _sparse(hw, G, gamma, marked, tau, dt, steps, psi0, batch=1):
    torch = _torch()
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    x = torch.from_numpy(np.ascontiguousarray(psi0)).to("cuda", cdt)
    y = torch.empty_like(x)
    rec = torch.empty(steps * batch, dtype=torch.float64, device="cuda") if marked else None
    hw.hw_ctqw_evolve_sparse(G, gamma, list(marked), tau, dt, batch, steps, x, y, rec)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128), None if rec is None else rec.cpu().numpy()


GRAPHS = [
    ("er2k", synth.erdos_renyi(2000, 8 / 1999, seed=5)),
    ("torus37x53", synth.torus_rect(37, 53)),
    ("star", synth.star(300)),
]


@pytest.mark.parametrize("name,g", GRAPHS)
@pytest.mark.parametrize("cplx", [False, True])
def test_sparse_c128_matches_oracle(hw, name, g, cplx):
    n, eu, ev = g
    we = synth.edge_weights(eu.size, seed=3, complex_phase=cplx)
    G = _wgraph(hw, g, we)
    ar = oracle.Arcs(n, eu, ev)
    w = ar.weights(eu, ev, we)
    marked = [0, n - 1]
    gamma, tau, steps = 0.35, 0.2, 9
    psi0 = synth.random_state(n, seed=12)
    got, rec = _sparse(hw, G, gamma, marked, tau, hw.HW_C128, steps, psi0)
    ref, rr = oracle.ctqw_evolve(ar, gamma, psi0, tau, steps, marked, record=True, weights=w)
    assert np.max(np.abs(got - ref)) <= TOL128
    assert np.max(np.abs(rec - rr)) <= TOL128
    G.free()


@pytest.mark.parametrize("cplx", [False, True])
def test_sparse_c64_and_batch(hw, cplx):
    g = synth.erdos_renyi(3000, 6 / 2999, seed=7)
    n, eu, ev = g
    we = synth.edge_weights(eu.size, seed=4, complex_phase=cplx)
    G = _wgraph(hw, g, we)
    ar = oracle.Arcs(n, eu, ev)
    w = ar.weights(eu, ev, we)
    gamma, tau = 0.25, 0.1
    psi0 = synth.random_state(n, seed=1)
    ref = oracle.ctqw_evolve(ar, gamma, psi0, tau, 1000, [7], weights=w)
    got, _ = _sparse(hw, G, gamma, [7], tau, hw.HW_C64, 1000, psi0)
    assert np.sum(np.abs(np.abs(got) ** 2 - np.abs(ref) ** 2)) <= 1e-3
    # three columns at once, complex128
    B = 3
    cols = synth.gaussian_states(n, B, seed=6)
    gotb, recb = _sparse(hw, G, gamma, [7, 100], tau, hw.HW_C128, 5, cols.reshape(-1), batch=B)
    gotb = gotb.reshape(n, B)
    recb = recb.reshape(5, B)
    for b in range(B):
        rb, rrb = oracle.ctqw_evolve(ar, gamma, cols[:, b], tau, 5, [7, 100], record=True, weights=w)
        assert np.max(np.abs(gotb[:, b] - rb)) <= TOL128
        assert np.max(np.abs(recb[:, b] - rrb)) <= TOL128
    G.free()


def test_flux_ring_closed_form(hw):
    N, gamma, tau, phi = 101, 0.5, 0.7, 0.3
    n, eu, ev = synth.cycle(N)
    G = _wgraph(hw, (n, eu, ev), np.full(eu.size, np.exp(1j * phi)))
    psi0 = synth.random_state(N, seed=8)
    E = -2 * gamma * np.cos(2 * np.pi * np.arange(N) / N + phi)
    got, _ = _sparse(hw, G, gamma, [], tau, hw.HW_C128, 40, psi0)
    want = np.fft.ifft(np.exp(-1j * E * tau * 40) * np.fft.fft(psi0))
    assert np.max(np.abs(got - want)) <= TOL128
    G.free()


@pytest.mark.parametrize("name,g,gamma,marked,t", [
    ("Q6", synth.hypercube(6), 1 / 6, [5], 1.0),
    ("er300", synth.erdos_renyi(300, 0.03, seed=4), 0.3, [0, 17], 0.5),
    ("reg3_778", synth.random_regular(778, 3, seed=4), 1 / 3, [5, 700], 0.4),
])
def test_dense_expm_real_weights(hw, name, g, gamma, marked, t):
    torch = _torch()
    n, eu, ev = g
    we = synth.edge_weights(eu.size, seed=9)
    G = _wgraph(hw, g, we)
    ar = oracle.Arcs(n, eu, ev)
    w = ar.weights(eu, ev, we)
    cols = np.unique(np.array([0, 1, 130, 257, n // 2, n - 2, n - 1]) % n)
    ref = oracle.ctqw_columns(ar, gamma, t, cols, marked=marked, weights=w)
    for powers in (2, 1):   # sparse x dense products with W, dense GEMMs
        for dt, tol in ((hw.HW_C128, TOL128), (hw.HW_C64, 2e-6)):
            cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
            U = torch.empty((n, n), dtype=cdt, device="cuda")
            hw.hw_ctqw_expm(G, gamma, marked, t, dt, U, opts={"taylor_powers": powers})
            Uh = U.cpu().numpy()
            assert np.max(np.abs(Uh[:, cols] - ref)) <= tol, (dt, powers)
            assert np.max(np.abs(Uh - Uh.T)) <= tol      # H real symmetric: U symmetric
    G.free()


@pytest.mark.parametrize("name,g,gamma,marked,t", [
    ("Q6", synth.hypercube(6), 1 / 6, [5], 1.0),
    ("er300", synth.erdos_renyi(300, 0.03, seed=4), 0.3, [0, 17], 0.5),
    ("torus37x53", synth.torus_rect(37, 53), 0.25, [100], 0.7),
])
def test_dense_expm_complex_weights(hw, name, g, gamma, marked, t):
    # a complex Hermitian W: the dense U (formed by the sparse series on the
    # identity's columns) against the oracle's columns, U unitary
    # (U^dagger U = I), and the dense application of U against the sparse series
    torch = _torch()
    n, eu, ev = g
    we = synth.edge_weights(eu.size, seed=9, complex_phase=True)
    G = _wgraph(hw, g, we)
    ar = oracle.Arcs(n, eu, ev)
    w = ar.weights(eu, ev, we)
    cols = np.unique(np.array([0, 1, 130, 257, n // 2, n - 2, n - 1]) % n)
    ref = oracle.ctqw_columns(ar, gamma, t, cols, marked=marked, weights=w)
    psi0 = synth.random_state(n, seed=4)
    for dt, tol in ((hw.HW_C128, TOL128), (hw.HW_C64, 2e-6)):
        cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
        U = torch.empty((n, n), dtype=cdt, device="cuda")
        hw.hw_ctqw_expm(G, gamma, marked, t, dt, U)
        Uh = U.cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(Uh[:, cols] - ref)) <= tol, dt
        assert np.max(np.abs(Uh.conj().T @ Uh - np.eye(n))) <= 50 * tol
        x = torch.from_numpy(psi0).to("cuda", cdt)
        y = torch.empty_like(x)
        hw.hw_ctqw_evolve(U, n, dt, 1, 3, x, y, [], None)
        sp, _ = _sparse(hw, G, gamma, marked, t, dt, 3, psi0)
        assert np.max(np.abs(y.cpu().numpy().astype(np.complex128) - sp)) <= 10 * tol
    G.free()


def test_plan_uses_the_weights(hw):
    g = synth.erdos_renyi(500, 0.02, seed=3)
    n, eu, ev = g
    we = 3.0 * synth.edge_weights(eu.size, seed=2)
    G = _wgraph(hw, g, we)
    rowabs = np.zeros(n)
    np.add.at(rowabs, eu, np.abs(we))
    np.add.at(rowabs, ev, np.abs(we))
    gamma, t, marked = 0.4, 0.3, [11]
    norm1 = max(gamma * rowabs.max(), gamma * rowabs[11] + 1.0) * t
    s = 0
    while norm1 / 2 ** s > 0.5:
        s += 1
    deg, sq = hw.hw_ctqw_plan(G, gamma, marked, t)
    assert sq == s
    G.free()


def test_weighted_graph_refusals(hw):
    torch = _torch()
    g = synth.torus_rect(5, 6)
    n, eu, ev = g
    G = _wgraph(hw, g, synth.edge_weights(eu.size, seed=1, complex_phase=True))
    x = torch.zeros(G.num_arcs, dtype=torch.complex128, device="cuda")
    with pytest.raises(hw.HWError) as e:
        hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 3, x, torch.empty_like(x))
    assert e.value.status == hw.HW_EINVAL
    G.free()
