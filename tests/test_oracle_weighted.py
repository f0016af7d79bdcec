"""Pins for the oracle's weighted Hamiltonian H = -gamma W - sum_m |m><m|
(Sec. 3.1 with the adjacency A generalised to a weighted, Hermitian W).

Against scipy's expm of the dense H built from the edge list (real and
complex weights, with marks); the magnetic-flux ring, whose plane waves
diagonalise H with energies -2 gamma cos(2 pi k / N + phi) (this fixes which
arc carries the weight and which its conjugate); the hypercube with one
weight per dimension, a tensor product of 2 x 2 rotations; and W = c A, which
is the unweighted walk at gamma c.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth


def _dense_h(n, eu, ev, we, gamma, marked):
    H = np.zeros((n, n), dtype=np.complex128)
    for u, v, w in zip(eu, ev, we):
        H[u, v] += -gamma * w
        H[v, u] += -gamma * np.conj(w)
    for m in marked:
        H[m, m] -= 1.0
    return H


def _small():
    yield "K5", synth.complete(5)
    yield "Q3", synth.hypercube(3)
    yield "C8", synth.cycle(8)
    yield "er12", synth.erdos_renyi(12, 0.4, seed=11, drop_isolated=False)
    yield "torus3x4", synth.torus_rect(3, 4)


@pytest.mark.parametrize("name,g", list(_small()))
@pytest.mark.parametrize("cplx", [False, True])
def test_weighted_matches_scipy_expm(name, g, cplx):
    n, eu, ev = g
    we = synth.edge_weights(eu.size, seed=21, complex_phase=cplx)
    ar = oracle.Arcs(n, eu, ev)
    w = ar.weights(eu, ev, we)
    gamma, dt, marked = 0.7, 0.9, [0, n - 1]
    U = scipy.linalg.expm(-1j * dt * _dense_h(n, eu, ev, we, gamma, marked))
    cols = oracle.ctqw_columns(ar, gamma, dt, list(range(n)), marked, weights=w)
    assert np.max(np.abs(cols - U)) < 1e-13
    psi0 = synth.random_state(n, seed=5)
    got = oracle.ctqw_evolve(ar, gamma, psi0, dt, 7, marked, weights=w)
    want = np.linalg.matrix_power(U, 7) @ psi0
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("phi", [0.3, -1.1, np.pi / 5])
def test_flux_ring_closed_form(phi):
    N, gamma, dt = 101, 0.5, 0.7
    n, eu, ev = synth.cycle(N)     # edges (v, v + 1 mod N)
    we = np.full(eu.size, np.exp(1j * phi))
    ar = oracle.Arcs(n, eu, ev)
    w = ar.weights(eu, ev, we)
    psi0 = synth.random_state(N, seed=8)
    # arc (v, v+1) carries e^{i phi}: the plane wave e^{i theta v} has energy
    # -2 gamma cos(theta + phi)
    theta = 2 * np.pi * np.arange(N) / N
    E = -2 * gamma * np.cos(theta + phi)
    for steps in (1, 5, 40):
        want = np.fft.ifft(np.exp(-1j * E * dt * steps) * np.fft.fft(psi0))
        got = oracle.ctqw_evolve(ar, gamma, psi0, dt, steps, weights=w)
        assert np.max(np.abs(got - want)) < 1e-12, steps


def test_hypercube_with_one_weight_per_dimension():
    k, gamma, t = 8, 0.3, 1.3
    n, eu, ev = synth.hypercube(k)
    c = synth.edge_weights(k, seed=33)
    dim = np.array([int(np.log2(u ^ v)) for u, v in zip(eu, ev)])
    ar = oracle.Arcs(n, eu, ev)
    w = ar.weights(eu, ev, c[dim])
    # H = -gamma sum_j c_j X_j, so U = prod_j (cos(gamma c_j t) + i sin(gamma c_j t) X_j)
    cols = [0, 5, 77, 255]
    got = oracle.ctqw_columns(ar, gamma, t, cols, weights=w)
    for ci, v in enumerate(cols):
        x = np.arange(n) ^ v
        want = np.ones(n, dtype=np.complex128)
        for j in range(k):
            bit = (x >> j) & 1
            want *= np.where(bit == 1, 1j * np.sin(gamma * c[j] * t), np.cos(gamma * c[j] * t))
        assert np.max(np.abs(got[:, ci] - want)) < 1e-13


def test_uniform_weight_is_a_scaled_gamma():
    n, eu, ev = synth.erdos_renyi(300, 0.03, seed=4)
    ar = oracle.Arcs(n, eu, ev)
    w = ar.weights(eu, ev, np.full(eu.size, 2.5))
    psi0 = synth.random_state(n, seed=2)
    a = oracle.ctqw_evolve(ar, 0.2, psi0, 0.4, 6, [3], weights=w)
    b = oracle.ctqw_evolve(ar, 0.5, psi0, 0.4, 6, [3])
    assert np.max(np.abs(a - b)) < 1e-13
