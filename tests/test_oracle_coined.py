"""Pins for the coined-walk oracle (Sec. 3.2): brute force, closed forms, invariants.

Each test checks the oracle against something other than itself: explicit dense
S and C matrices built from the definitions by enumeration, a 3-dimensional
reduced walk on the complete graph, exact permutation dynamics on the cycle,
symmetry, parity and light-cone zeros on the torus.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _graphs():
    yield "er12", synth.erdos_renyi(12, 0.4, seed=11, drop_isolated=False)
    yield "K5", synth.complete(5)
    yield "Q3", synth.hypercube(3)
    yield "C8", synth.cycle(8)
    yield "star6", synth.star(6)
    yield "path5", synth.path(5)
    yield "torus3", synth.torus(3)
    # two components plus an isolated vertex (degree 0)
    yield "mixed", (9, np.array([0, 1, 2, 4, 5, 5], np.int64), np.array([1, 2, 0, 5, 6, 7], np.int64))


def _brute_arcs(n, eu, ev):
    A = np.zeros((n, n), dtype=int)
    A[eu, ev] = 1
    A[ev, eu] = 1
    arcs = [(v, w) for v in range(n) for w in range(n) if A[v, w]]
    return A, arcs


def _dense_walk(n, arcs, coin_kind, marked):
    """Explicit matrices: S|v,w> = |w,v>; C block per vertex (Grover / Fourier / -I)."""
    idx = {a: i for i, a in enumerate(arcs)}
    dim = len(arcs)
    S = np.zeros((dim, dim))
    for (v, w), i in idx.items():
        S[idx[(w, v)], i] = 1.0
    C = np.zeros((dim, dim), dtype=complex)
    for v in range(n):
        block = [idx[a] for a in arcs if a[0] == v]
        d = len(block)
        for j, rj in enumerate(block):
            for k, ck in enumerate(block):
                if v in marked:
                    C[rj, ck] = -1.0 if j == k else 0.0
                elif coin_kind == oracle.GROVER:
                    C[rj, ck] = 2.0 / d - (1.0 if j == k else 0.0)
                else:
                    C[rj, ck] = np.exp(2j * np.pi * j * k / d) / np.sqrt(d)
    return S, C


@pytest.mark.parametrize("name,g", list(_graphs()))
def test_arcs_match_enumeration(name, g):
    n, eu, ev = g
    A, arcs = _brute_arcs(n, eu, ev)
    ar = oracle.Arcs(n, eu, ev)
    assert ar.num_arcs == len(arcs) == 2 * len(eu)
    assert np.array_equal(ar.head, np.array([w for _, w in arcs], dtype=np.int32))
    assert np.array_equal(ar.row_ptr, np.concatenate([[0], np.cumsum(A.sum(1))]))
    pos = {a: i for i, a in enumerate(arcs)}
    assert np.array_equal(ar.rev, np.array([pos[(w, v)] for v, w in arcs]))
    tail = ar.tail()
    assert np.array_equal(ar.rev[ar.rev], np.arange(ar.num_arcs))
    assert np.array_equal(tail[ar.rev], ar.head)


def test_arcs_reject_invalid():
    with pytest.raises(ValueError):
        oracle.Arcs(3, np.array([0, 1]), np.array([1, 1]))        # self-loop
    with pytest.raises(ValueError):
        oracle.Arcs(3, np.array([0, 1]), np.array([1, 0]))        # same edge twice
    with pytest.raises(ValueError):
        oracle.Arcs(3, np.array([0]), np.array([3]))              # out of range


@pytest.mark.parametrize("coin_kind", [oracle.GROVER, oracle.FOURIER])
@pytest.mark.parametrize("name,g", list(_graphs()))
def test_evolution_matches_dense_matrix_power(name, g, coin_kind):
    n, eu, ev = g
    _, arcs = _brute_arcs(n, eu, ev)
    marked = [1] if name in ("er12", "K5", "Q3", "mixed") else []
    S, C = _dense_walk(n, arcs, coin_kind, set(marked))
    U = S @ C
    assert np.allclose(U.conj().T @ U, np.eye(len(arcs)), atol=1e-13)
    ar = oracle.Arcs(n, eu, ev)
    psi0 = synth.random_state(ar.num_arcs, seed=21)
    for t in (1, 2, 7):
        ref = np.linalg.matrix_power(U, t) @ psi0
        got = oracle.coined_evolve(ar, psi0, t, coin_kind, marked)
        assert np.max(np.abs(got - ref)) < 1e-13, (name, t)
    # coin and shift separately
    assert np.max(np.abs(oracle.coin(ar, psi0, coin_kind, marked) - C @ psi0)) < 1e-14
    assert np.array_equal(oracle.shift(ar, psi0), S @ psi0)


def test_uniform_state_is_stationary_without_marks():
    # Grover coin fixes a constant block; the flip-flop shift permutes equal values.
    n, eu, ev = synth.erdos_renyi(300, 0.02, seed=5)
    ar = oracle.Arcs(n, eu, ev)
    psi0 = synth.uniform_state(ar.num_arcs)
    psi = oracle.coined_evolve(ar, psi0, 37)
    assert np.max(np.abs(psi - psi0)) < 1e-15


def test_cycle_grover_is_exact_translation():
    # d = 2: the Grover coin is the swap, so S C moves arc (v, v+1) to (v-1, v)
    # and arc (v, v-1) to (v+1, v): a permutation, exact in floating point.
    N = 11
    n, eu, ev = synth.cycle(N)
    ar = oracle.Arcs(n, eu, ev)
    _, arcs = _brute_arcs(n, eu, ev)
    pos = {a: i for i, a in enumerate(arcs)}
    R = np.array([pos[(v, (v + 1) % N)] for v in range(N)])
    L = np.array([pos[(v, (v - 1) % N)] for v in range(N)])
    psi0 = synth.random_state(ar.num_arcs, seed=3)
    for t in (1, 5, 23):
        psi = oracle.coined_evolve(ar, psi0, t)
        assert np.array_equal(psi[R], psi0[R][(np.arange(N) + t) % N])
        assert np.array_equal(psi[L], psi0[L][(np.arange(N) - t) % N])


def test_complete_graph_search_reduced_walk():
    # K_N, marked m, uniform start: amplitudes stay constant on the arc classes
    # (m,u), (u,m), (u,u').  One step of S C on the class amplitudes (al, be, ga):
    #   coin at u (d = N-1): mean mu = (be + (N-2) ga)/(N-1); coin at m: -I
    #   shift: al' = 2mu - be,  be' = -al,  ga' = 2mu - ga.
    N, steps = 24, 60
    n, eu, ev = synth.complete(N)
    ar = oracle.Arcs(n, eu, ev)
    m = 5
    psi0 = synth.uniform_state(ar.num_arcs)
    psi, rec = oracle.coined_evolve(ar, psi0, steps, marked=[m], record=True)
    al = be = ga = 1.0 / math.sqrt(N * (N - 1))
    curve = []
    for _ in range(steps):
        mu = (be + (N - 2) * ga) / (N - 1)
        al, be, ga = 2 * mu - be, -al, 2 * mu - ga
        curve.append((N - 1) * abs(al) ** 2)
    assert np.max(np.abs(rec - np.array(curve))) < 1e-14
    tail = ar.tail()
    assert np.allclose(psi[(tail == m)], al, atol=1e-14, rtol=0)
    assert np.allclose(psi[(ar.head == m)], be, atol=1e-14, rtol=0)
    other = (tail != m) & (ar.head != m)
    assert np.allclose(psi[other], ga, atol=1e-14, rtol=0)
    assert max(curve) > 0.4   # the search amplifies the marked vertex


def test_coin_powers():
    n, eu, ev = synth.erdos_renyi(40, 0.2, seed=9)
    ar = oracle.Arcs(n, eu, ev)
    x = synth.random_state(ar.num_arcs, seed=4)
    g2 = oracle.coin(ar, oracle.coin(ar, x))
    assert np.max(np.abs(g2 - x)) < 1e-14                     # Grover is a reflection
    f = x
    for _ in range(4):
        f = oracle.coin(ar, f, oracle.FOURIER)
    assert np.max(np.abs(f - x)) < 1e-13                      # F_d^4 = I
    assert np.array_equal(oracle.coin(ar, x, marked=np.arange(n)), -x)   # -I everywhere
    assert np.array_equal(oracle.shift(ar, oracle.shift(ar, x)), x)       # S^2 = I


@pytest.mark.parametrize("coin_kind", [oracle.GROVER, oracle.FOURIER])
def test_norm_is_conserved(coin_kind):
    n, eu, ev = synth.erdos_renyi(500, 0.015, seed=12)
    ar = oracle.Arcs(n, eu, ev)
    psi0 = synth.random_state(ar.num_arcs, seed=13)
    psi = oracle.coined_evolve(ar, psi0, 200, coin_kind, marked=[3, 77])
    assert abs(np.sum(np.abs(psi) ** 2) - 1.0) < 1e-13
    assert abs(oracle.prob_coined(ar, psi).sum() - 1.0) < 1e-13


def test_torus_symmetry_parity_and_light_cone():
    # 64 x 64 torus, start on the 4 arcs of (32, 32), 100 Grover steps.
    L, T = 64, 100
    n, eu, ev = synth.torus(L)
    ar = oracle.Arcs(n, eu, ev)
    c = 32 * L + 32
    psi0 = synth.state_on_vertex_arcs(synth.arc_offsets(n, eu, ev), c)
    p = oracle.prob_coined(ar, oracle.coined_evolve(ar, psi0, T)).reshape(L, L)
    x = np.arange(L)
    refl = (2 * 32 - x) % L
    assert np.max(np.abs(p - p[refl, :])) < 1e-14
    assert np.max(np.abs(p - p[:, refl])) < 1e-14
    assert np.max(np.abs(p - p.T)) < 1e-14
    X, Y = np.meshgrid(x, x, indexing="ij")
    dist = np.minimum(abs(X - 32), L - abs(X - 32)) + np.minimum(abs(Y - 32), L - abs(Y - 32))
    assert np.all(p[(X + Y) % 2 == 1] == 0.0)      # bipartite: even steps stay on even sites
    assert abs(p.sum() - 1.0) < 1e-13
    p20 = oracle.prob_coined(ar, oracle.coined_evolve(ar, psi0, 20)).reshape(L, L)
    assert np.all(p20[dist > 20] == 0.0)           # light cone: one edge per step
    assert np.all(p20[dist == 20] > 0.0)
