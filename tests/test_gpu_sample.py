"""Sampled evolution (simulate(range=(start, end, stride)), Sec. 3.1-3.2, 4.1-4.2):
each sampled state against the FP64 oracle and against hw_coined_evolve /
hw_ctqw_evolve for the same step counts (bit-identical), probabilities per
sample, the search curve of the complete graph against its closed form, and
the argument checks."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _graph(hw, g):
    row_ptr, col = synth.adjacency_csr(*g)
    return hw.hw_graph_csr(g[0], row_ptr, col)


@pytest.mark.parametrize("name,g,dt", [
    ("torus32_c128", synth.torus(32), 2),          # edge-major path
    ("torus32_c64", synth.torus(32), 1),
    ("er_c128", synth.erdos_renyi(1500, 6 / 1499, seed=3), 2),   # arc-major path
])
@pytest.mark.parametrize("start,end,stride", [(3, 40, 7), (0, 21, 5), (5, 6, 1)])
def test_coined_samples(hw, name, g, dt, start, end, stride):
    import torch
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    n = g[0]
    psi0 = synth.random_state(ar.num_arcs, seed=9)
    cdt = torch.complex128 if dt == 2 else torch.complex64
    x = torch.from_numpy(psi0).to("cuda", cdt)
    R = hw.sample_count(start, end, stride)
    states = torch.empty((R, ar.num_arcs), dtype=cdt, device="cuda")
    prob = torch.empty((R, n), dtype=torch.float64, device="cuda")
    marked = [7]
    hw.hw_coined_sample(G, 0, marked, dt, 1, start, end, stride, x, states, prob)
    torch.cuda.synchronize()
    for r in range(R):
        t = start + r * stride
        ref = oracle.coined_evolve(ar, psi0, t, marked=marked)
        got = states[r].cpu().numpy().astype(np.complex128)
        if dt == 2:
            assert np.max(np.abs(got - ref)) <= 1e-12
        else:
            assert np.max(np.abs(got - ref)) < 1e-5
        assert np.max(np.abs(prob[r].cpu().numpy() - oracle.prob_coined(ar, got))) < 1e-12
        # the same as one evolve of t steps
        y = torch.empty_like(x)
        hw.hw_coined_evolve(G, 0, marked, dt, 1, t, x, y)
        torch.cuda.synchronize()
        assert torch.equal(y, states[r])
    G.free()


def test_coined_samples_batched_and_probabilities_only(hw):
    import torch
    g = synth.torus(24)
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    B = 3
    psi0 = np.stack([synth.random_state(ar.num_arcs, seed=s) for s in (1, 2, 3)], axis=1)
    x = torch.from_numpy(np.ascontiguousarray(psi0)).to("cuda", torch.complex128)
    R = hw.sample_count(2, 30, 9)
    prob = torch.empty((R, g[0], B), dtype=torch.float64, device="cuda")
    hw.hw_coined_sample(G, 0, [4], 2, B, 2, 30, 9, x, None, prob)
    torch.cuda.synchronize()
    for r in range(R):
        for b in range(B):
            ref = oracle.coined_evolve(ar, psi0[:, b], 2 + 9 * r, marked=[4])
            assert np.max(np.abs(prob[r, :, b].cpu().numpy() - oracle.prob_coined(ar, ref))) < 1e-12
    G.free()


def _search_curve_kn(N, steps):
    # K_N with one mark from the uniform state: the class amplitudes (al, be, ga)
    # of arcs (m,u), (u,m), (u,u') follow a 3-term recursion; p_m = (N-1) |al|^2
    al = be = ga = 1.0 / math.sqrt(N * (N - 1))
    ref = []
    for _ in range(steps):
        mu = (be + (N - 2) * ga) / (N - 1)
        al, be, ga = 2 * mu - be, -al, 2 * mu - ga
        ref.append((N - 1) * al * al)
    return np.array(ref)


def test_complete_graph_search_curve(hw):
    # the success curve and its peak from the device, against the closed form
    import torch
    N, steps = 40, 50
    g = synth.complete(N)
    G = _graph(hw, g)
    m = 11
    ar_arcs = N * (N - 1)
    x = torch.full((ar_arcs,), 1 / math.sqrt(ar_arcs), dtype=torch.complex128, device="cuda")
    prob = torch.empty((steps, N), dtype=torch.float64, device="cuda")
    hw.hw_coined_sample(G, 0, [m], 2, 1, 1, steps + 1, 1, x, None, prob)
    curve, k, pmax = hw.success_curve(prob, [m])
    ref = _search_curve_kn(N, steps)
    assert np.max(np.abs(curve.cpu().numpy() - ref)) < 1e-12
    assert k == int(np.argmax(ref)) and abs(pmax - ref.max()) < 1e-12
    G.free()


def test_success_curve_matches_oracle_record(hw):
    # two marks, two states per sample: the curve of every column against the
    # marked-probability record of the oracle's walk, and the peak against
    # the record's (unique) maximum
    import torch
    g = synth.torus(16)
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    marked = [37, 200]
    B, start, end, stride = 2, 3, 90, 3
    psi0 = np.stack([synth.random_state(ar.num_arcs, seed=s) for s in (11, 12)], axis=1)
    x = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
    R = hw.sample_count(start, end, stride)
    prob = torch.empty((R, g[0], B), dtype=torch.float64, device="cuda")
    hw.hw_coined_sample(G, 0, marked, 2, B, start, end, stride, x, None, prob)
    curve = torch.empty((R, B), dtype=torch.float64, device="cuda")
    kmax = torch.empty(B, dtype=torch.int64, device="cuda")
    vmax = torch.empty(B, dtype=torch.float64, device="cuda")
    hw.hw_success_curve(prob, marked, curve, kmax, vmax)
    torch.cuda.synchronize()
    for b in range(B):
        _, rec = oracle.coined_evolve(ar, psi0[:, b], end, marked=marked, record=True)
        ref = rec[start - 1:end - 1:stride]       # rec[t-1] = marked probability after step t
        got = curve[:, b].cpu().numpy()
        assert np.max(np.abs(got - ref)) < 1e-12
        assert int(kmax[b]) == int(np.argmax(ref))
        assert abs(float(vmax[b]) - ref.max()) < 1e-12
    G.free()


def test_success_curve_edge_cases(hw):
    import torch
    dev = "cuda"
    # ties go to the earliest sample; NaN entries never win (sums of dyadic
    # values, so every sum below is exact)
    prob = torch.tensor([[[0.25], [0.125]], [[0.375], [0.0]], [[float("nan")], [0.5]], [[0.125], [0.25]]],
                        dtype=torch.float64, device=dev)            # [R=4][n=2][batch=1]
    curve = torch.empty((4, 1), dtype=torch.float64, device=dev)
    k = torch.empty(1, dtype=torch.int64, device=dev)
    v = torch.empty(1, dtype=torch.float64, device=dev)
    hw.hw_success_curve(prob, [0, 1], curve, k, v)
    c = curve[:, 0].cpu().numpy()
    assert c[0] == 0.375 and c[1] == 0.375 and math.isnan(c[2]) and c[3] == 0.375
    assert int(k) == 0 and float(v) == 0.375
    # only NaN: no maximum
    hw.hw_success_curve(prob[2:3], [0], curve[:1], k, v)
    assert int(k) == -1 and math.isnan(float(v))
    # no samples: argmax -1, maximum NaN
    empty = torch.empty((0, 2), dtype=torch.float64, device=dev)
    hw.hw_success_curve(empty, [1], torch.empty(0, dtype=torch.float64, device=dev), k, v)
    assert int(k) == -1 and math.isnan(float(v))
    # more marks than travel with the launch (> 16): the list goes to the device
    R, n = 7, 300
    p = torch.rand((R, n), dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(3))
    marks = list(range(5, 300, 9))
    cv = torch.empty(R, dtype=torch.float64, device=dev)
    hw.hw_success_curve(p, marks, cv, k, v)
    pn = p.cpu().numpy()
    ref = pn[:, marks].sum(axis=1)
    assert np.max(np.abs(cv.cpu().numpy() - ref)) < 1e-13
    assert int(k) == int(np.argmax(ref))
    # argument checks
    for bad in ([], [n], [3, 3]):
        with pytest.raises(hw.HWError) as e:
            hw.hw_success_curve(p, bad, cv, k, v)
        assert e.value.status == hw.HW_EINVAL
    with pytest.raises(hw.HWError):
        hw.hw_success_curve(p, [1], p.view(-1)[:R])      # curve inside prob


def test_ctqw_samples(hw):
    import torch
    k, gamma, dt_, = 7, 1 / 7, 0.2
    g = synth.hypercube(k)
    n = g[0]
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    marked = [5]
    for dt in (2, 1):
        cdt = torch.complex128 if dt == 2 else torch.complex64
        U = torch.empty((n, n), dtype=cdt, device="cuda")
        hw.hw_ctqw_expm(G, gamma, marked, dt_, dt, U)
        psi0 = synth.random_state(n, seed=5)
        x = torch.from_numpy(psi0).to("cuda", cdt)
        R = hw.sample_count(2, 30, 4)
        states = torch.empty((R, n), dtype=cdt, device="cuda")
        prob = torch.empty((R, n), dtype=torch.float64, device="cuda")
        hw.hw_ctqw_sample(U, n, dt, 1, 2, 30, 4, x, states, prob)
        torch.cuda.synchronize()
        for r in range(R):
            t = 2 + 4 * r
            ref = oracle.ctqw_evolve(ar, gamma, psi0, dt_, t, marked=marked)
            got = states[r].cpu().numpy().astype(np.complex128)
            assert np.max(np.abs(got - ref)) <= (1e-12 if dt == 2 else 2e-5)
            assert np.max(np.abs(prob[r].cpu().numpy() - np.abs(got) ** 2)) < 1e-12
            y = torch.empty_like(x)
            hw.hw_ctqw_evolve(U, n, dt, 1, t, x, y)
            torch.cuda.synchronize()
            assert torch.equal(y, states[r])
    G.free()


def test_sample_arguments(hw):
    import torch
    g = synth.torus(8)
    G = _graph(hw, g)
    x = torch.zeros(G.num_arcs, dtype=torch.complex128, device="cuda")
    hw.hw_coined_sample(G, 0, [], 2, 1, 5, 5, 1, x, None, None)        # no samples: nothing to do
    for start, end, stride in ((0, 10, 0), (4, 3, 1), (-1, 3, 1)):
        with pytest.raises(hw.HWError) as e:
            hw.hw_coined_sample(G, 0, [], 2, 1, start, end, stride, x, None, None)
        assert e.value.status == hw.HW_EINVAL
    out = torch.empty((2, G.num_arcs), dtype=torch.complex128, device="cuda")
    with pytest.raises(hw.HWError):
        hw.hw_coined_sample(G, 0, [], 2, 1, 0, 2, 1, out[0], out, None)  # input inside the output
    G.free()
