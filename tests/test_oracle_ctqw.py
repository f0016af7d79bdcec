"""Pins for the CTQW oracle (Sec. 3.1, H = -gamma A - sum_m |m><m|, U = e^{-iHt}).

Closed forms: complete graph, hypercube (tensor product of 2x2 rotations), cycle
(Fourier diagonalisation), the marked hypercube reduced to Hamming-weight
classes, and scipy's expm (Al-Mohy & Higham) on small graphs.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth


def test_complete_graph_closed_form():
    # A = J - I, H = -gamma A: e^{-iHt} = e^{-i gamma t} (I + (e^{i gamma N t} - 1)/N J)
    N, gamma, t = 9, 0.3, 0.7
    ar = oracle.Arcs(*synth.complete(N))
    U = oracle.ctqw_columns(ar, gamma, t, np.arange(N))
    ref = np.exp(-1j * gamma * t) * (np.eye(N) + (np.exp(1j * gamma * N * t) - 1) / N * np.ones((N, N)))
    assert np.max(np.abs(U - ref)) < 1e-14


@pytest.mark.parametrize("k,gamma,t", [(6, 0.4, 1.3), (4, 1.0, 7.5)])
def test_hypercube_closed_form(k, gamma, t):
    # A = sum_j X_j, so e^{i gamma t A} = prod_j (cos(gamma t) I + i sin(gamma t) X_j):
    # U[u, v] = cos^(k - h) (i sin)^h with h = Hamming distance(u, v).
    N = 1 << k
    ar = oracle.Arcs(*synth.hypercube(k))
    U = oracle.ctqw_columns(ar, gamma, t, np.arange(N))
    u = np.arange(N)
    h = np.array([[bin(a ^ b).count("1") for b in u] for a in u])
    c, s = math.cos(gamma * t), math.sin(gamma * t)
    ref = c ** (k - h) * (1j * s) ** h
    assert np.max(np.abs(U - ref)) < 1e-13


def test_hypercube_search_hamming_reduction():
    # One marked vertex m, uniform start.  By symmetry the state lives on the
    # Hamming-weight classes |r> around m (r = 0..k), where
    #   A|r> = sqrt(r (k - r + 1)) |r-1> + sqrt((r + 1)(k - r)) |r+1>,
    # and the marked projector is |0><0|.  Diagonalise the (k+1)x(k+1) matrix.
    k, gamma, dt, steps = 10, 1.0 / 10, 0.1, 300
    N = 1 << k
    ar = oracle.Arcs(*synth.hypercube(k))
    m = synth.seeded_vertex(3, N)
    psi0 = synth.uniform_state(N)
    psi, rec = oracle.ctqw_evolve(ar, gamma, psi0, dt, steps, marked=[m], record=True)
    A = np.zeros((k + 1, k + 1))
    for r in range(k):
        A[r, r + 1] = A[r + 1, r] = math.sqrt((r + 1) * (k - r))
    H = -gamma * A
    H[0, 0] -= 1.0
    w, V = np.linalg.eigh(H)
    x0 = np.array([math.sqrt(math.comb(k, r) / N) for r in range(k + 1)])
    times = dt * np.arange(1, steps + 1)
    amp0 = (V[0, :][None, :] * np.exp(-1j * np.outer(times, w))) @ (V.T @ x0)
    assert np.max(np.abs(rec - np.abs(amp0) ** 2)) < 1e-12
    # the final state is constant on each Hamming class
    xr = V @ (np.exp(-1j * w * times[-1]) * (V.T @ x0))
    hd = np.array([bin(v ^ m).count("1") for v in range(N)])
    ref = xr[hd] / np.sqrt([math.comb(k, r) for r in hd])
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_cycle_fourier_closed_form():
    # C_N: A = sum_q 2 cos(2 pi q / N) |f_q><f_q|, f_q(v) = e^{2 pi i q v / N}/sqrt(N).
    # Paper's cycle example: 101 vertices, walker departing from vertex 50, t = 50.
    N, gamma, t = 101, 0.5, 50.0
    ar = oracle.Arcs(*synth.cycle(N))
    psi0 = np.zeros(N, complex)
    psi0[50] = 1.0
    q = np.arange(N)
    lam = 2 * np.cos(2 * np.pi * q / N)
    v = np.arange(N)
    F = np.exp(2j * np.pi * np.outer(v, q) / N) / math.sqrt(N)
    ref = F @ (np.exp(1j * gamma * t * lam) * (F.conj().T @ psi0))
    got_one = oracle.ctqw_evolve(ar, gamma, psi0, t, 1)          # one application, split inside
    got_many = oracle.ctqw_evolve(ar, gamma, psi0, t / 100, 100)  # 100 applications
    assert np.max(np.abs(got_one - ref)) < 1e-12
    assert np.max(np.abs(got_many - ref)) < 1e-12


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_small_graphs_against_scipy_expm(seed):
    n, eu, ev = synth.erdos_renyi(14, 0.35, seed=seed, drop_isolated=False)
    ar = oracle.Arcs(n, eu, ev)
    A = np.zeros((n, n))
    A[eu, ev] = A[ev, eu] = 1.0
    marked = [0, 5]
    gamma, dt = 0.7, 2.0
    H = -gamma * A
    for m in marked:
        H[m, m] -= 1.0
    U = scipy.linalg.expm(-1j * H * dt)
    got = oracle.ctqw_columns(ar, gamma, dt, np.arange(n), marked=marked)
    assert np.max(np.abs(got - U)) < 1e-13
    psi0 = synth.random_state(n, seed=seed + 10)
    got = oracle.ctqw_evolve(ar, gamma, psi0, dt, 5, marked=marked)
    assert np.max(np.abs(got - np.linalg.matrix_power(U, 5) @ psi0)) < 1e-12
    p = oracle.prob_vertex(got)
    assert abs(p.sum() - 1.0) < 1e-13


def test_single_vector_action_and_vertex_probability():
    n, eu, ev = synth.erdos_renyi(12, 0.4, seed=6, drop_isolated=False)
    ar = oracle.Arcs(n, eu, ev)
    A = np.zeros((n, n))
    A[eu, ev] = A[ev, eu] = 1.0
    H = -0.9 * A
    H[3, 3] -= 1.0
    x = synth.random_state(n, seed=8)
    ref = scipy.linalg.expm(-1j * H * 0.7) @ x
    assert np.max(np.abs(oracle.ctqw_action(ar, 0.9, 0.7, x, marked=[3]) - ref)) < 1e-13
    p = oracle.prob_vertex(np.array([3 + 4j, 1j, 0.0]))
    assert np.array_equal(p, np.array([25.0, 1.0, 0.0]))
