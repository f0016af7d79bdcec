"""Host helpers of the sampling API: sample counts of range(start, end, stride)
and the search success curve, pinned to the closed-form reduced walk of the
coined search on the complete graph (the oracle supplies the states)."""
import math

import numpy as np

import oracle
import paper_2406_08186_b300 as hw
import synth


def test_sample_count_matches_range():
    for start, end, stride in ((0, 50, 5), (3, 40, 7), (5, 5, 1), (0, 21, 1), (2, 3, 10)):
        assert hw.sample_count(start, end, stride) == len(range(start, end, stride))


def test_success_curve_on_complete_graph():
    N, steps, m = 24, 40, 3
    n, eu, ev = synth.complete(N)
    ar = oracle.Arcs(n, eu, ev)
    psi = synth.uniform_state(ar.num_arcs)
    probs = []
    for _ in range(steps):
        psi = oracle.coined_evolve(ar, psi, 1, marked=[m])
        probs.append(oracle.prob_coined(ar, psi))
    curve, k, pmax = hw.success_curve(np.array(probs), [m])
    al = be = ga = 1.0 / math.sqrt(N * (N - 1))
    ref = []
    for _ in range(steps):
        mu = (be + (N - 2) * ga) / (N - 1)
        al, be, ga = 2 * mu - be, -al, 2 * mu - ga
        ref.append((N - 1) * al * al)
    assert np.max(np.abs(curve - np.array(ref))) < 1e-13
    assert k == int(np.argmax(ref))
    assert abs(pmax - max(ref)) < 1e-13
    # two marks: the curve is the sum of their probabilities
    c2, _, _ = hw.success_curve(np.array(probs), [m, 0])
    assert np.allclose(c2, np.array(probs)[:, m] + np.array(probs)[:, 0])
