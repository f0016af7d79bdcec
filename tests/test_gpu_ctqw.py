"""GPU parity of the continuous-time walk (Sec. 3.1) against the FP64 oracle.

U = e^{-iH dt} from hw_ctqw_expm, with its Taylor powers formed both ways
(sparse x dense products with the graph, the default, and dense n^3 GEMMs:
FP64 for complex128, tensor cores for complex64), is compared column by
column with the oracle's sparse series action, and the evolved states / marked-vertex curves
from hw_ctqw_evolve with the oracle's evolution.  complex128: max-abs <= 1e-12;
complex64: probability L1 <= 1e-3 after 1000+ applications.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL128 = 1e-12


def _graph(hw, g):
    n, eu, ev = g
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    return hw.hw_graph_csr(n, row_ptr, col)


POWERS = [2, 1]   # hw_opts.taylor_powers: sparse x dense products, dense GEMMs


def gpu_expm(hw, g, gamma, marked, t, dt=2, opts=None, powers=2):
    import torch
    opts = dict(opts or {})
    opts["taylor_powers"] = powers
    G = _graph(hw, g)
    n = g[0]
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    U = torch.empty((n, n), dtype=cdt, device="cuda")
    hw.hw_ctqw_expm(G, gamma, list(marked), t, dt, U, opts=opts)
    torch.cuda.synchronize()
    return G, U


def gpu_evolve(hw, U, psi0, steps, marked, dt=2, batch=1, record=True, opts=None):
    import torch
    n = U.shape[0]
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    x = torch.from_numpy(np.ascontiguousarray(psi0)).to("cuda", cdt)
    out = torch.empty_like(x)
    rec = torch.empty(steps * batch, dtype=torch.float64, device="cuda") if record else None
    hw.hw_ctqw_evolve(U, n, dt, batch, steps, x, out, list(marked), rec, opts=opts)
    prob = torch.empty(n * batch, dtype=torch.float64, device="cuda")
    norm = torch.empty(batch, dtype=torch.float64, device="cuda")
    hw.hw_probability(None, n, dt, batch, out, prob, norm)
    torch.cuda.synchronize()
    return (out.cpu().numpy().astype(np.complex128), None if rec is None else rec.cpu().numpy(),
            prob.cpu().numpy(), norm.cpu().numpy())


CASES = [
    ("Q6", synth.hypercube(6), 1 / 6, [5]),
    ("er300", synth.erdos_renyi(300, 0.03, seed=4), 0.3, [0, 17, 299 - 40]),
    ("C101", synth.cycle(101), 0.5, []),
    ("K33", synth.complete(33), 1 / 33, [32]),
    ("star", synth.star(130), 0.2, [0]),
]


@pytest.mark.parametrize("powers", POWERS)
@pytest.mark.parametrize("t", [0.1, 1.0, 10.0])
@pytest.mark.parametrize("name,g,gamma,marked", CASES)
def test_expm_c128_matches_oracle_columns(hw, name, g, gamma, marked, t, powers):
    marked = [m for m in marked if m < g[0]]
    G, U = gpu_expm(hw, g, gamma, marked, t, powers=powers)
    ar = oracle.Arcs(*g)
    ref = oracle.ctqw_columns(ar, gamma, t, np.arange(g[0]), marked=marked)
    # Each squaring roughly doubles the rounding error already in U, so the
    # 1e-12 bar (the configured workloads need s <= 2) widens as 2^s / 64 for
    # the stress cases with many squarings (the star at t = 10 needs s = 10).
    s = hw.hw_ctqw_plan(G, gamma, marked, t)[1]
    tol = TOL128 * max(1.0, 2.0 ** s / 64)
    assert np.max(np.abs(U.cpu().numpy() - ref)) <= tol
    G.free()


@pytest.mark.parametrize("powers", POWERS)
def test_expm_c64_close(hw, powers):
    g = synth.hypercube(7)
    G, U = gpu_expm(hw, g, 1 / 7, [3], 0.1, dt=1, powers=powers)
    ar = oracle.Arcs(*g)
    ref = oracle.ctqw_columns(ar, 1 / 7, 0.1, np.arange(128), marked=[3])
    assert np.max(np.abs(U.cpu().numpy() - ref)) < 2e-6
    G.free()


@pytest.mark.parametrize("name,g,gamma,marked,t", [
    # 1/gamma = 3 is exact in one fp16 slice: Y keeps one slice (two products)
    ("reg3_exact", synth.random_regular(778, 3, seed=4), 1 / 3, [5, 700], 0.4),
    # gamma = 0.3: Y needs two slices (three products)
    ("er_two_slices", synth.erdos_renyi(1000, 0.006, seed=6), 0.3, [990], 0.25),
])
@pytest.mark.parametrize("powers", POWERS)
def test_expm_c64_ragged_multi_tile(hw, name, g, gamma, marked, t, powers):
    # n not a multiple of the 128 x 256 tiles (or of the sparse kernel's
    # 8 x 256 blocks), several cluster tiles and mirrored blocks; columns
    # checked against the oracle's action
    n = g[0]
    G, U = gpu_expm(hw, g, gamma, marked, t, dt=1, powers=powers)
    ar = oracle.Arcs(*g)
    cols = np.array([0, 1, 130, 257, n // 2, n - 2, n - 1])
    ref = oracle.ctqw_columns(ar, gamma, t, cols, marked=marked)
    got = U.cpu().numpy()[:, cols]
    assert np.max(np.abs(got - ref)) < 2e-6
    # rows equal columns: U is symmetric because H is
    Uh = U.cpu().numpy()
    assert np.max(np.abs(Uh - Uh.T)) < 2e-6
    G.free()


@pytest.mark.parametrize("name,g,gamma,marked,t", [
    ("reg3_exact", synth.random_regular(778, 3, seed=4), 1 / 3, [5, 700], 0.4),   # n not a multiple of 256
    ("er_two_slices", synth.erdos_renyi(1000, 0.006, seed=6), 0.3, [990], 0.25),
    ("Q12", synth.hypercube(12), 1 / 12, [1234], 0.1),                           # configuration 3's graph
])
@pytest.mark.parametrize("mode", [0, 2, 3])
def test_expm_c64_pair_tiles_match_single_tiles(hw, name, g, gamma, marked, t, mode):
    # the tensor-core powers on CTA pairs (256 x 256 tiles, hw_opts.gemm_tiles
    # = 2) and on single CTAs (128 x 256, = 1) run the same MMAs in the same
    # order per output element: U agrees bit for bit, in every precision mode
    # (fp16 x 2; bf16 x 2; bf16 x 3), and matches the oracle's columns
    n = g[0]
    Us = []
    for tiles in (1, 2):
        G, U = gpu_expm(hw, g, gamma, marked, t, dt=1, powers=1, opts={"gemm_tiles": tiles, "gemm_mode": mode})
        Us.append(U)
        G.free()
    import torch
    assert torch.equal(Us[0], Us[1])
    ar = oracle.Arcs(*g)
    cols = np.array([0, 1, 255, 256, n // 2, n - 1])
    ref = oracle.ctqw_columns(ar, gamma, t, cols, marked=marked)
    tol = 2e-6 if mode != 2 else 2e-3   # bf16 x 2 keeps about 16 bits
    assert np.max(np.abs(Us[1].cpu().numpy()[:, cols] - ref)) < tol


@pytest.mark.parametrize("powers", POWERS)
def test_expm_hypercube_closed_form(hw, powers):
    # no marks: U[u, v] = cos(gamma t)^(k-h) (i sin(gamma t))^h, h = Hamming distance
    k, gamma, t = 8, 0.25, 3.0
    G, U = gpu_expm(hw, synth.hypercube(k), gamma, [], t, powers=powers)
    u = np.arange(1 << k)
    h = np.array([bin(x).count("1") for x in range(1 << k)])
    H = h[u[:, None] ^ u[None, :]]
    ref = math.cos(gamma * t) ** (k - H) * (1j * math.sin(gamma * t)) ** H
    assert np.max(np.abs(U.cpu().numpy() - ref)) <= TOL128
    G.free()


def test_plan_matches_stated_rule(hw):
    g = synth.hypercube(12)
    G = _graph(hw, g)
    m = synth.seeded_vertex(3, 4096)
    assert hw.hw_ctqw_plan(G, 1 / 12, [m], 0.1) == (12, 0)   # ||H dt|| = 0.2
    assert hw.hw_ctqw_plan(G, 1 / 12, [m], 1.0)[1] == 2
    assert hw.hw_ctqw_plan(G, 1 / 12, [m], 10.0)[1] == 6
    G.free()


def test_evolve_matches_oracle_and_hamming_reduction(hw):
    k, gamma, dt, steps = 10, 1 / 10, 0.1, 300
    g = synth.hypercube(k)
    N = 1 << k
    m = synth.seeded_vertex(3, N)
    G, U = gpu_expm(hw, g, gamma, [m], dt)
    psi0 = synth.uniform_state(N)
    psi, rec, prob, norm = gpu_evolve(hw, U, psi0, steps, [m])
    ar = oracle.Arcs(*g)
    ref, rec_ref = oracle.ctqw_evolve(ar, gamma, psi0, dt, steps, marked=[m], record=True)
    assert np.max(np.abs(psi - ref)) <= TOL128
    assert np.max(np.abs(rec - rec_ref)) <= TOL128
    assert np.max(np.abs(prob - oracle.prob_vertex(ref))) <= TOL128
    assert abs(norm[0] - 1) < 1e-12
    # independent closed form: Hamming-weight classes around m
    A = np.zeros((k + 1, k + 1))
    for r in range(k):
        A[r, r + 1] = A[r + 1, r] = math.sqrt((r + 1) * (k - r))
    Hr = -gamma * A
    Hr[0, 0] -= 1.0
    w, V = np.linalg.eigh(Hr)
    x0 = np.array([math.sqrt(math.comb(k, r) / N) for r in range(k + 1)])
    times = dt * np.arange(1, steps + 1)
    amp0 = (V[0, :][None, :] * np.exp(-1j * np.outer(times, w))) @ (V.T @ x0)
    assert np.max(np.abs(rec - np.abs(amp0) ** 2)) <= TOL128
    G.free()


@pytest.mark.parametrize("name,g,marked", [
    # one state, complex128: the three-product application; n past one and two
    # 1024-column chunks and off the 4-row CTA grid, and tiny graphs
    ("reg3_1500", synth.random_regular(1500, 3, seed=8), [3, 1499]),
    ("er_2047", synth.erdos_renyi(2051, 0.003, seed=5), [-1]),   # isolated vertices dropped: n = 2047
    ("path3", synth.path(3), [1]),
    ("K2", synth.complete(2), []),
])
def test_evolve_three_product_sizes(hw, name, g, marked):
    n = g[0]
    marked = [m % n for m in marked]
    G, U = gpu_expm(hw, g, 0.35, marked, 0.2)
    psi0 = synth.random_state(n, seed=n)
    steps = 25
    psi, rec, prob, norm = gpu_evolve(hw, U, psi0, steps, marked, record=bool(marked))
    ar = oracle.Arcs(*g)
    if marked:
        ref, rr = oracle.ctqw_evolve(ar, 0.35, psi0, 0.2, steps, marked=marked, record=True)
        assert np.max(np.abs(rec - rr)) <= TOL128
    else:
        ref = oracle.ctqw_evolve(ar, 0.35, psi0, 0.2, steps, marked=marked)
    assert np.max(np.abs(psi - ref)) <= TOL128
    assert abs(norm[0] - np.sum(np.abs(psi0) ** 2)) < 1e-12
    G.free()


def test_evolve_batched_and_in_place(hw):
    import torch
    g = synth.erdos_renyi(200, 0.05, seed=2)
    n = g[0]
    marked = [1, 150]
    G, U = gpu_expm(hw, g, 0.4, marked, 0.3)
    ar = oracle.Arcs(*g)
    B, steps = 3, 40
    psi0 = synth.gaussian_states(n, B, seed=9)
    psi, rec, prob, norm = gpu_evolve(hw, U, psi0, steps, marked, batch=B)
    psi = psi.reshape(n, B)
    rec = rec.reshape(steps, B)
    for b in range(B):
        ref, rr = oracle.ctqw_evolve(ar, 0.4, psi0[:, b], 0.3, steps, marked=marked, record=True)
        assert np.max(np.abs(psi[:, b] - ref)) <= TOL128
        assert np.max(np.abs(rec[:, b] - rr)) <= TOL128
    # in place, odd step count
    x = torch.from_numpy(psi0[:, 0].copy()).cuda()
    hw.hw_ctqw_evolve(U, n, hw.HW_C128, 1, 7, x, x)
    ref = oracle.ctqw_evolve(ar, 0.4, psi0[:, 0], 0.3, 7, marked=marked)
    assert np.max(np.abs(x.cpu().numpy() - ref)) <= TOL128
    G.free()


@pytest.mark.parametrize("powers,sym", [(p, 0) for p in POWERS] + [(0, 1)])
@pytest.mark.parametrize("dt", [2, 1])
def test_config3_hypercube12_search_full_size(hw, dt, powers, sym):
    # Q_12, gamma = 1/12, one seeded mark, dt = 0.1, uniform start, 2000
    # applications; sym = 1: the applications read one triangle of U (packed),
    # as the benchmark's complex64 evolve does (complex128 keeps the dense form)
    k, gamma, tstep, steps = 12, 1 / 12, 0.1, 2000
    g = synth.hypercube(k)
    N = 1 << k
    m = synth.seeded_vertex(3, N)
    G, U = gpu_expm(hw, g, gamma, [m], tstep, dt=dt, powers=powers)
    ar = oracle.Arcs(*g)
    cols = np.array([0, m, 1, 2047, 4095, 1234, 3000, 77])
    refU = oracle.ctqw_columns(ar, gamma, tstep, cols, marked=[m])
    Uc = U[:, torch_index(cols)].cpu().numpy()
    psi0 = synth.uniform_state(N)
    psi, rec, prob, norm = gpu_evolve(hw, U, psi0, steps, [m], dt=dt, opts={"u_symmetric": sym})
    ref, rec_ref = oracle.ctqw_evolve(ar, gamma, psi0, tstep, steps, marked=[m], record=True)
    if dt == 2:
        assert np.max(np.abs(Uc - refU)) <= TOL128
        assert np.max(np.abs(psi - ref)) <= TOL128
        assert np.max(np.abs(rec - rec_ref)) <= TOL128
    else:
        assert np.max(np.abs(Uc - refU)) < 2e-6
        assert np.sum(np.abs(prob - oracle.prob_vertex(ref))) <= 1e-3
        assert np.max(np.abs(rec - rec_ref)) < 1e-4
    G.free()


@pytest.mark.parametrize("dt,powers", [(2, 0), (2, 1), (1, 0), (1, 2)])
def test_expm_whole_matrix_probes(hw, dt, powers):
    # U of configuration 3 (Q_12, gamma = 1/12, one mark, dt = 0.1) checked as
    # a whole matrix, not column by column: U x for two seeded random states
    # against the oracle's sparse series applied to x (Freivalds-style
    # probes), and unitarity on the same probes, U^dagger (U x) = x with
    # |U x| = |x|; the products are taken on the host in double
    k, gamma, tstep = 12, 1 / 12, 0.1
    g = synth.hypercube(k)
    N = 1 << k
    m = synth.seeded_vertex(3, N)
    G, U = gpu_expm(hw, g, gamma, [m], tstep, dt=dt, powers=powers)
    Uh = U.cpu().numpy().astype(np.complex128)
    G.free()
    ar = oracle.Arcs(*g)
    tol = TOL128 if dt == 2 else 1e-5
    for seed in (21, 22):
        x = synth.random_state(N, seed=seed)
        y = Uh @ x
        ref = oracle.ctqw_action(ar, gamma, tstep, x, marked=[m])
        assert np.max(np.abs(y - ref)) <= tol
        assert np.max(np.abs(Uh.conj().T @ y - x)) <= tol
        assert abs(np.linalg.norm(y) - np.linalg.norm(x)) <= tol


@pytest.mark.parametrize("powers", [1, 2])
def test_expm_rejects_bad_tile_form(hw, powers):
    # hw_opts.gemm_tiles is 0..2 whatever form the powers take
    with pytest.raises(hw.HWError):
        gpu_expm(hw, synth.hypercube(6), 1 / 6, [5], 0.1, dt=1, powers=powers, opts={"gemm_tiles": 3})


def _hamming_reduction(k, gamma, m_steps, tstep, m):
    # one marked vertex, uniform start: the state stays on the Hamming-weight
    # classes |r> around the mark, A|r> = sqrt(r (k-r+1))|r-1> + sqrt((r+1)(k-r))|r+1>,
    # and H = -gamma A - |0><0| is (k+1) x (k+1): exact p_m(t) for every step,
    # and the final probabilities (constant on each class)
    import math
    N = 1 << k
    A = np.zeros((k + 1, k + 1))
    for r in range(k):
        A[r, r + 1] = A[r + 1, r] = math.sqrt((r + 1) * (k - r))
    H = -gamma * A
    H[0, 0] -= 1.0
    w, V = np.linalg.eigh(H)
    x0 = np.array([math.sqrt(math.comb(k, r) / N) for r in range(k + 1)])
    times = tstep * np.arange(1, m_steps + 1)
    amp0 = (V[0, :][None, :] * np.exp(-1j * np.outer(times, w))) @ (V.T @ x0)
    xr = V @ (np.exp(-1j * w * times[-1]) * (V.T @ x0))
    hd = np.array([bin(v ^ m).count("1") for v in range(N)])
    prob = np.abs(xr[hd]) ** 2 / np.array([math.comb(k, r) for r in hd])
    return np.abs(amp0) ** 2, prob


@pytest.mark.parametrize("dt,sym", [(2, 0), (1, 0), (1, 1)])
def test_config3_critical_gamma_against_hamming_reduction(hw, dt, sym):
    # configuration 3 at the critical gamma_c = sum_r C(k, r)/r / (2N) of Q_12
    # (0.09298...; 1/12 is off-critical): the marked probability rises to about
    # 0.84 near t = 108 instead of peaking at 0.078; the recorded curve of all
    # 2000 applications against the exact Hamming-weight reduction
    import math
    k, tstep, steps = 12, 0.1, 2000
    N = 1 << k
    gamma = sum(math.comb(k, r) / r for r in range(1, k + 1)) / (2 * N)
    g = synth.hypercube(k)
    m = synth.seeded_vertex(3, N)
    G, U = gpu_expm(hw, g, gamma, [m], tstep, dt=dt, powers=0)
    _, rec, prob, norm = gpu_evolve(hw, U, synth.uniform_state(N), steps, [m], dt=dt, opts={"u_symmetric": sym})
    ref, prob_ref = _hamming_reduction(k, gamma, steps, tstep, m)
    if dt == 2:
        assert np.max(np.abs(rec - ref)) <= TOL128
        assert np.max(np.abs(prob - prob_ref)) <= TOL128
    else:
        # complex64: L1 of the probabilities <= 1e-3 (the stated bound), which
        # also bounds the error of any one of them, p_m(t) included (here p_m
        # reaches 0.84, so its absolute error is larger than at gamma = 1/12)
        assert np.sum(np.abs(prob - prob_ref)) <= 1e-3
        assert np.max(np.abs(rec - ref)) <= 1e-3
    assert 0.8 < rec.max() < 0.9 and 100.0 < tstep * (1 + int(np.argmax(rec))) < 115.0
    G.free()


def torch_index(cols):
    import torch
    return torch.from_numpy(np.asarray(cols)).cuda()


@pytest.mark.parametrize("dt", [2, 1])
@pytest.mark.parametrize("n_bits,steps", [(7, 40), (12, 300)])
def test_symmetric_apply_matches_dense_apply_and_oracle(hw, dt, n_bits, steps):
    # U from hw_ctqw_expm is complex symmetric; reading one triangle of blocks
    # must give the dense application's result (n = 128 spans two 64-blocks,
    # n = 4096 is the benchmarked size)
    import torch
    k = n_bits
    g = synth.hypercube(k)
    N = 1 << k
    m = synth.seeded_vertex(3, N)
    G, U = gpu_expm(hw, g, 1.0 / k, [m], 0.1, dt=dt)
    cdt = torch.complex128 if dt == 2 else torch.complex64
    x = torch.full((N,), 1.0 / np.sqrt(N), dtype=cdt, device="cuda")
    outs = []
    for sym in (0, 1):
        y = torch.empty_like(x)
        rec = torch.empty(steps, dtype=torch.float64, device="cuda")
        hw.hw_ctqw_evolve(U, N, dt, 1, steps, x, y, [m], rec, opts={"u_symmetric": sym})
        outs.append((y.cpu().numpy().astype(np.complex128), rec.cpu().numpy()))
    ar = oracle.Arcs(*g)
    ref, rr = oracle.ctqw_evolve(ar, 1.0 / k, synth.uniform_state(N), 0.1, steps, marked=[m], record=True)
    if dt == 2:
        assert np.max(np.abs(outs[1][0] - outs[0][0])) <= TOL128
        assert np.max(np.abs(outs[1][0] - ref)) <= TOL128
        assert np.max(np.abs(outs[1][1] - rr)) <= TOL128
    else:
        assert np.sum(np.abs(np.abs(outs[1][0]) ** 2 - np.abs(ref) ** 2)) <= 1e-3
        assert np.max(np.abs(outs[1][1] - rr)) <= 1e-4
    G.free()


@pytest.mark.parametrize("name,g,gamma,marked", [
    # even n, not a multiple of the 64-vertex blocks: edge blocks packed with zeros past n
    ("reg3_778", synth.random_regular(778, 3, seed=4), 1 / 3, [5, 700]),
    # uneven degrees, isolated vertices dropped (n = 998)
    ("er_998", synth.erdos_renyi(1000, 0.006, seed=6), 0.3, [10]),
    # odd n: a lane's two columns straddle n in the last block
    ("reg4_999", synth.random_regular(999, 4, seed=5), 0.25, [998]),
    # one block, smaller than the 64 x 64 block (a single diagonal block)
    ("cycle_10", synth.cycle(10), 0.5, [3]),
    # two block rows, the second one vertex high
    ("cycle_65", synth.cycle(65), 0.5, [64]),
])
def test_symmetric_apply_ragged_sizes(hw, name, g, gamma, marked):
    import torch
    n = g[0]
    marked = [m for m in marked if m < n]
    G, U = gpu_expm(hw, g, gamma, marked, 0.25, dt=1)
    x = torch.from_numpy(synth.random_state(n, seed=3)).to("cuda", torch.complex64)
    outs = []
    for sym in (0, 1):
        y = torch.empty_like(x)
        rec = torch.empty(60, dtype=torch.float64, device="cuda")
        hw.hw_ctqw_evolve(U, n, hw.HW_C64, 1, 60, x, y, marked, rec, opts={"u_symmetric": sym})
        outs.append((y.cpu().numpy().astype(np.complex128), rec.cpu().numpy()))
    ar = oracle.Arcs(*g)
    ref, rr = oracle.ctqw_evolve(ar, gamma, synth.random_state(n, seed=3), 0.25, 60, marked=marked, record=True)
    for y, rec in outs:
        assert np.sum(np.abs(np.abs(y) ** 2 - np.abs(ref) ** 2)) <= 1e-3
        assert np.max(np.abs(rec - rr)) <= 1e-4
    assert np.max(np.abs(outs[1][0] - outs[0][0])) <= 1e-5
    G.free()
