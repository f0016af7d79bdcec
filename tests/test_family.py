"""Graph families recognised from the adjacency (torus, hypercube) and the
label arithmetic that replaces the head and reversal tables for them.

The arithmetic (family.cuh) compiles as host C++ and is compared with brute
force (sorted neighbour lists searched for each reversed / continued arc) on
every torus 3..12 x 3..12 and hypercube Q_1..Q_16; the detection is checked on
the families, on relabelled copies and on other graphs.  CPU only."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_2406_08186_b300 as hw
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_label_arithmetic_matches_brute_force(tmp_path):
    exe = tmp_path / "family_check"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2406_08186_b300", "csrc"),
                           "-o", str(exe), os.path.join(ROOT, "tests", "family_check.cpp")])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok ")
    assert int(out.stdout.split()[1]) > 1_000_000


def _kind(n, eu, ev, scramble=7):
    rp, col = synth.adjacency_csr(n, eu, ev, scramble_seed=scramble)
    return hw.hw_graph_structure_host(n, rp, col)


@pytest.mark.parametrize("L1,L2", [(3, 3), (3, 4), (4, 3), (5, 9), (64, 64), (7, 100)])
def test_torus_detected(L1, L2):
    kind, dims = _kind(*synth.torus_rect(L1, L2))
    assert kind == hw.HW_GRAPH_TORUS and dims == (L1, L2)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 10, 12])
def test_hypercube_detected(k):
    kind, dims = _kind(*synth.hypercube(k))
    assert kind == hw.HW_GRAPH_HYPERCUBE and dims == (k, 0)


def test_relabelled_and_other_graphs_are_generic():
    n, eu, ev = synth.torus_rect(6, 7)
    perm = np.random.default_rng(3).permutation(n)
    assert _kind(n, perm[eu], perm[ev])[0] == hw.HW_GRAPH_GENERIC
    n, eu, ev = synth.hypercube(6)
    perm = np.random.default_rng(4).permutation(n)
    assert _kind(n, perm[eu], perm[ev])[0] == hw.HW_GRAPH_GENERIC
    for g in (synth.cycle(9), synth.complete(6), synth.random_regular(64, 4, seed=5), synth.star(7),
              synth.erdos_renyi(50, 0.1, seed=2, drop_isolated=False)):
        assert _kind(*g)[0] == hw.HW_GRAPH_GENERIC
    # a torus with one edge moved (still 4-regular) is not a torus
    n, eu, ev = synth.torus_rect(5, 5)
    eu, ev = eu.copy(), ev.copy()
    assert _kind(n, eu, ev)[0] == hw.HW_GRAPH_TORUS
    # swap the endpoints of two disjoint edges: (a,b),(c,d) -> (a,d),(c,b)
    i, j = 0, 12
    a, b, c, d = eu[i], ev[i], eu[j], ev[j]
    assert len({a, b, c, d}) == 4
    ev[i], ev[j] = d, b
    assert _kind(n, eu, ev)[0] == hw.HW_GRAPH_GENERIC
