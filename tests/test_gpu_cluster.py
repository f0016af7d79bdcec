"""Whole coined walks of small regular graphs in one launch (one thread-block
cluster holding the state in distributed shared memory, Sec. 3.2): against the
FP64 oracle (complex128 1e-12), bit-identical to the one-launch-per-step path
(hw_opts.launch_mode 2 against 1, and the default's measured choice), with
marks, a strided record, in place, the persistent shift, ragged vertex
ranges, fewer vertices than CTAs, more vertices per CTA than thread pairs,
degrees 2..8 and sizes up to 49152 arcs."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CASES = [
    ("torus64", synth.torus(64)),                       # configuration 1's graph
    ("torus7x9", synth.torus_rect(7, 9)),               # 63 vertices: ragged CTA ranges
    ("cycle5", synth.cycle(5)),                         # degree 2, fewer vertices than CTAs
    ("Q7", synth.hypercube(7)),                         # degree 7
    ("reg3", synth.random_regular(1002, 3, seed=4)),
    ("reg5", synth.random_regular(600, 5, seed=8)),
    ("reg8", synth.random_regular(2048, 8, seed=6)),    # 16384 arcs, almost all exchanged between CTAs
    ("torus64x96", synth.torus_rect(64, 96)),           # 24576 arcs
    # 24000 arcs (complex64 in one launch): 750 vertices per CTA against 512
    # thread pairs, so threads take a second vertex in a step
    ("cycle12000", synth.cycle(12000)),
    ("torus96x128", synth.torus_rect(96, 128)),         # 49152 arcs: fits the cluster in both precisions
]


def _graph(hw, g):
    row_ptr, col = synth.adjacency_csr(*g)
    return hw.hw_graph_csr(g[0], row_ptr, col)


@pytest.mark.parametrize("name,g", CASES)
@pytest.mark.parametrize("dt", [2, 1])
def test_cluster_walk_matches_oracle_and_per_step_path(hw, name, g, dt):
    import torch
    n = g[0]
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    marked = sorted({1, n // 2, n - 1}) if n > 2 else [1]
    steps, stride = 37, 3
    psi0 = synth.random_state(ar.num_arcs, seed=13)
    cdt = torch.complex128 if dt == 2 else torch.complex64
    x = torch.from_numpy(psi0).to("cuda", cdt)
    slots = steps // stride
    outs, recs = [], []
    # one launch, one launch per step, and the default's measured choice
    for mode in (2, 1, 0):
        y = torch.empty_like(x)
        rec = torch.empty(slots, dtype=torch.float64, device="cuda")
        hw.hw_coined_evolve(G, 0, marked, dt, 1, steps, x, y, rec, opts={"record_stride": stride, "launch_mode": mode})
        outs.append(y)
        recs.append(rec)
    torch.cuda.synchronize()
    for k in (1, 2):
        assert torch.equal(outs[0], outs[k])
        assert torch.equal(recs[0], recs[k])
    ref, rr = oracle.coined_evolve(ar, psi0, steps, marked=marked, record=True)
    got = outs[0].cpu().numpy().astype(np.complex128)
    if dt == 2:
        assert np.max(np.abs(got - ref)) <= 1e-12
        assert np.max(np.abs(recs[0].cpu().numpy() - rr[stride - 1::stride][:slots])) <= 1e-12
    else:
        assert np.max(np.abs(got - ref)) <= 1e-5
        assert np.max(np.abs(recs[0].cpu().numpy() - rr[stride - 1::stride][:slots])) <= 1e-5
    G.free()


def test_cluster_walk_in_place_and_persistent_shift(hw):
    import torch
    L1, L2 = 12, 10
    g = synth.torus_rect(L1, L2)
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    psi0 = synth.random_state(ar.num_arcs, seed=3)
    for shift in (0, 1):
        x = torch.from_numpy(psi0).cuda()
        hw.hw_coined_evolve(G, 0, [17], 2, 1, 21, x, x, opts={"shift": shift, "launch_mode": 2})   # in place, odd steps
        ref = oracle.coined_evolve(ar, psi0, 21, marked=[17], persistent_torus=(L1, L2) if shift else None)
        torch.cuda.synchronize()
        assert np.max(np.abs(x.cpu().numpy() - ref)) <= 1e-12
        y = torch.from_numpy(psi0).cuda()
        hw.hw_coined_evolve(G, 0, [17], 2, 1, 21, y, y, opts={"shift": shift, "launch_mode": 1})
        torch.cuda.synchronize()
        assert torch.equal(x, y)
    G.free()


def test_configuration1_in_one_launch_dihedral_symmetry(hw):
    # configuration 1: the 64 x 64 torus from the four arcs of (32, 32), 100
    # steps; besides the oracle, the probabilities are symmetric under the
    # reflections x -> 64 - x, y -> 64 - y and the swap x <-> y about (32, 32)
    import torch
    n, eu, ev = synth.torus(64)
    G = _graph(hw, (n, eu, ev))
    psi0 = synth.state_on_vertex_arcs(synth.arc_offsets(n, eu, ev), 32 * 64 + 32)
    x = torch.from_numpy(psi0).cuda()
    y = torch.empty_like(x)
    prob = torch.empty(n, dtype=torch.float64, device="cuda")
    hw.hw_coined_evolve(G, 0, [], 2, 1, 100, x, y, opts={"launch_mode": 2})
    hw.hw_probability(G, n, 2, 1, y, prob)
    ar = oracle.Arcs(n, eu, ev)
    ref = oracle.prob_coined(ar, oracle.coined_evolve(ar, psi0, 100))
    p = prob.cpu().numpy()
    assert np.max(np.abs(p - ref)) <= 1e-12
    P = p.reshape(64, 64)
    idx = (64 - np.arange(64)) % 64
    assert np.max(np.abs(P - P[idx, :])) <= 1e-13
    assert np.max(np.abs(P - P[:, idx])) <= 1e-13
    assert np.max(np.abs(P - P.T)) <= 1e-13
    G.free()


def test_cluster_walk_record_single_mark_and_one_step(hw):
    import torch
    g = synth.torus(64)
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    psi0 = synth.uniform_state(ar.num_arcs)
    x = torch.from_numpy(psi0).cuda()
    for steps in (1, 100):
        y = torch.empty_like(x)
        rec = torch.empty(steps, dtype=torch.float64, device="cuda")
        hw.hw_coined_evolve(G, 0, [2080], 2, 1, steps, x, y, rec, opts={"launch_mode": 2})
        ref, rr = oracle.coined_evolve(ar, psi0, steps, marked=[2080], record=True)
        torch.cuda.synchronize()
        assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12
        assert np.max(np.abs(rec.cpu().numpy() - rr)) <= 1e-12
    with pytest.raises(hw.HWError):
        hw.hw_coined_evolve(G, 0, [], 2, 1, 3, x, x, opts={"launch_mode": 3})
    G.free()


def test_cluster_walk_long_marked_list(hw):
    # more marked vertices than travel with the launch (> 16): the list is
    # searched in device memory; records of every marked vertex summed
    import torch
    g = synth.torus(32)
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    marked = list(range(3, 1024, 47))            # 22 vertices
    psi0 = synth.random_state(ar.num_arcs, seed=21)
    x = torch.from_numpy(psi0).cuda()
    outs = []
    for mode in (2, 1):
        y = torch.empty_like(x)
        rec = torch.empty(30, dtype=torch.float64, device="cuda")
        hw.hw_coined_evolve(G, 0, marked, 2, 1, 30, x, y, rec, opts={"launch_mode": mode})
        outs.append((y, rec))
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    ref, rr = oracle.coined_evolve(ar, psi0, 30, marked=marked, record=True)
    assert np.max(np.abs(outs[0][0].cpu().numpy() - ref)) <= 1e-12
    assert np.max(np.abs(outs[0][1].cpu().numpy() - rr)) <= 1e-12
    G.free()
