"""Pins for the oracle's persistent shift on the torus (Sec. 3.2, the Grid
class's persistent shift: the walker keeps its direction of motion).

The torus walk without marked vertices commutes with translations, so in the
momentum basis it is a 4 x 4 matrix per wave vector k: the shift multiplies the
amplitude of direction d by e^{-i k.delta_d} (persistent) or also sends it to
the opposite direction (flip-flop), and the Grover coin is the same matrix
everywhere.  The tests evolve seeded states that way, with numpy FFTs and
matrix powers, and compare with the oracle's per-arc evolution in the sorted
arc basis.  Further pins: the persistent shift is a permutation of order
lcm(L1, L2) (each direction cycles around its axis), the flip-flop shift an
involution, and the uniform state is stationary under both.
"""
import math

import numpy as np
import pytest

import oracle
import synth

# directions: up (x-1), left (y-1), right (y+1), down (x+1)
DELTA = [(-1, 0), (0, -1), (0, 1), (1, 0)]
OPP = [3, 2, 1, 0]


def _positions(L1, L2, ar):
    """pos[d][x, y] = index in the arc basis of the arc leaving (x, y) in direction d,
    found by sorting the four neighbour labels (and checked against the oracle's heads)."""
    pos = np.zeros((4, L1, L2), dtype=np.int64)
    for x in range(L1):
        for y in range(L2):
            v = x * L2 + y
            lab = [((x + dx) % L1) * L2 + (y + dy) % L2 for dx, dy in DELTA]
            order = np.argsort(lab)
            for rank, d in enumerate(order):
                a = ar.row_ptr[v] + rank
                assert ar.head[a] == lab[d]
                pos[d, x, y] = a
    return pos


def _momentum_evolve(L1, L2, psi_dir, steps, persistent):
    """psi_dir[d, x, y] evolved by U(k)^steps in the Fourier basis."""
    G = 0.5 * np.ones((4, 4)) - np.eye(4)
    F = np.fft.fft2(psi_dir, axes=(1, 2))
    kx = 2 * np.pi * np.fft.fftfreq(L1)
    ky = 2 * np.pi * np.fft.fftfreq(L2)
    out = np.empty_like(F)
    P = np.zeros((4, 4))
    for d in range(4):
        P[OPP[d] if not persistent else d, d] = 1.0
    for i in range(L1):
        for j in range(L2):
            # a translation by delta multiplies the transform by e^{-i k.delta}
            ph = np.array([np.exp(-1j * (kx[i] * dx + ky[j] * dy)) for dx, dy in DELTA])
            U = P @ np.diag(ph) @ G
            out[:, i, j] = np.linalg.matrix_power(U, steps) @ F[:, i, j]
    return np.fft.ifft2(out, axes=(1, 2))


@pytest.mark.parametrize("L1,L2", [(3, 5), (4, 7), (6, 6), (5, 3), (8, 4)])
@pytest.mark.parametrize("persistent", [True, False])
def test_shift_matches_momentum_space(L1, L2, persistent):
    n, eu, ev = synth.torus_rect(L1, L2)
    ar = oracle.Arcs(n, eu, ev)
    pos = _positions(L1, L2, ar)
    psi0 = synth.random_state(ar.num_arcs, seed=41 + L1 * 10 + L2)
    for steps in (1, 2, 7, 19):
        got = oracle.coined_evolve(ar, psi0, steps, oracle.GROVER,
                                   persistent_torus=(L1, L2) if persistent else None)
        want = _momentum_evolve(L1, L2, psi0[pos], steps, persistent)
        assert np.max(np.abs(got[pos] - want)) < 1e-12, (L1, L2, steps)


@pytest.mark.parametrize("L1,L2", [(3, 4), (5, 7), (6, 9)])
def test_persistent_shift_order(L1, L2):
    n, eu, ev = synth.torus_rect(L1, L2)
    ar = oracle.Arcs(n, eu, ev)
    pos = _positions(L1, L2, ar)
    idx = np.arange(ar.num_arcs, dtype=np.complex128)   # labels travel with the amplitudes
    cur = idx.copy()
    lcm = L1 * L2 // math.gcd(L1, L2)
    for t in range(1, lcm + 1):
        cur = oracle.shift_persistent_torus(ar, L1, L2, cur)
        # an arc along the rows (left/right) is back after L2 shifts, along the columns after L1
        if t % L2 == 0:
            assert np.array_equal(cur[pos[1]], idx[pos[1]]) and np.array_equal(cur[pos[2]], idx[pos[2]])
        else:
            assert not np.array_equal(cur[pos[2]], idx[pos[2]])
        if t % L1 == 0:
            assert np.array_equal(cur[pos[0]], idx[pos[0]]) and np.array_equal(cur[pos[3]], idx[pos[3]])
    assert np.array_equal(cur, idx)
    # one shift moves the arc leaving (x, y) rightwards to the arc leaving (x, y+1) rightwards
    one = oracle.shift_persistent_torus(ar, L1, L2, idx)
    assert np.array_equal(one[pos[2]], np.roll(idx[pos[2]], 1, axis=1))
    assert np.array_equal(one[pos[3]], np.roll(idx[pos[3]], 1, axis=0))
    # the flip-flop shift is an involution and differs from the persistent one
    ff = oracle.shift(ar, idx)
    assert np.array_equal(oracle.shift(ar, ff), idx)
    assert not np.array_equal(ff, one)


def test_uniform_state_stationary_under_persistent_shift():
    L1, L2 = 7, 5
    n, eu, ev = synth.torus_rect(L1, L2)
    ar = oracle.Arcs(n, eu, ev)
    psi0 = np.full(ar.num_arcs, 1 / math.sqrt(ar.num_arcs), dtype=np.complex128)
    psi = oracle.coined_evolve(ar, psi0, 50, oracle.GROVER, persistent_torus=(L1, L2))
    assert np.max(np.abs(psi - psi0)) < 1e-15


def test_persistent_evolution_composes_coin_and_shift():
    L1, L2 = 6, 5
    n, eu, ev = synth.torus_rect(L1, L2)
    ar = oracle.Arcs(n, eu, ev)
    psi = synth.random_state(ar.num_arcs, seed=5)
    marked = [4, 17]
    want = psi.copy()
    for _ in range(9):
        want = oracle.shift_persistent_torus(ar, L1, L2, oracle.coin(ar, want, oracle.FOURIER, marked))
    got, rec = oracle.coined_evolve(ar, psi, 9, oracle.FOURIER, marked=marked, record=True,
                                    persistent_torus=(L1, L2))
    assert np.array_equal(got, want)
    p = oracle.prob_coined(ar, got)
    assert rec[-1] == pytest.approx(p[marked].sum(), abs=1e-15)
