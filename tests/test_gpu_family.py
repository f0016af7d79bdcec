"""GPU parity on the recognised graph families (torus, hypercube): the
index-free kernels (positions computed from labels) against the table-driven
kernels, bit for bit, and the persistent shift of the torus (Sec. 3.2)
against the FP64 oracle.

Tolerances: complex128 amplitudes max-abs <= 1e-12; complex64 probability
vectors L1 <= 1e-3.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL128 = 1e-12
TOL64_L1 = 1e-3


def _torch():
    import torch
    return torch


def _graph(hw, g):
    n, eu, ev = g
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    return hw.hw_graph_csr(n, row_ptr, col)


def _evolve(hw, G, psi0, steps, dt, coin=0, marked=(), addressing=0, shift=0, record=False, batch=1):
    torch = _torch()
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    x = torch.from_numpy(np.ascontiguousarray(psi0)).to("cuda", cdt)
    out = torch.empty_like(x)
    rec = torch.full((steps * batch,), -1.0, dtype=torch.float64, device="cuda") if record else None
    hw.hw_coined_evolve(G, coin, list(marked), dt, batch, steps, x, out, rec,
                        opts={"addressing": addressing, "shift": shift})
    prob = torch.empty(G.n * batch, dtype=torch.float64, device="cuda")
    norm = torch.empty(batch, dtype=torch.float64, device="cuda")
    hw.hw_probability(G, G.n, dt, batch, out, prob, norm)
    torch.cuda.synchronize()
    return out.cpu(), prob.cpu().numpy(), None if rec is None else rec.cpu()


TORI = [(3, 3), (3, 5), (7, 4), (33, 65), (130, 257), (37, 300), (1024, 1024)]


@pytest.mark.parametrize("L1,L2", TORI)
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("coin", [0, 1])
@pytest.mark.parametrize("dt", [1, 2])
def test_torus_index_free_bit_identical_to_tables(hw, L1, L2, shift, coin, dt):
    g = synth.torus_rect(L1, L2)
    G = _graph(hw, g)
    assert hw.hw_graph_structure(G) == (hw.HW_GRAPH_TORUS, (L1, L2))
    psi0 = synth.random_state(G.num_arcs, seed=L1 + 7 * L2)
    marked = [0, G.n - 1, G.n // 3]
    steps = 9 if G.n > 100000 else 31
    a = _evolve(hw, G, psi0, steps, dt, coin, marked, addressing=0, shift=shift, record=True)
    b = _evolve(hw, G, psi0, steps, dt, coin, marked, addressing=1, shift=shift, record=True)
    torch = _torch()
    assert torch.equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert torch.equal(a[2], b[2])
    G.free()


@pytest.mark.parametrize("L1,L2", [(3, 5), (7, 4), (33, 65), (130, 257)])
@pytest.mark.parametrize("coin", [0, 1])
def test_persistent_shift_c128_matches_oracle(hw, L1, L2, coin):
    g = synth.torus_rect(L1, L2)
    ar = oracle.Arcs(*g)
    G = _graph(hw, g)
    psi0 = synth.random_state(ar.num_arcs, seed=3 + L1)
    marked = [0, G.n - 1, G.n // 2]
    steps = 23
    ref, rec_ref = oracle.coined_evolve(ar, psi0, steps, coin, marked, record=True, persistent_torus=(L1, L2))
    for addressing in (0, 1):
        psi, prob, rec = _evolve(hw, G, psi0, steps, hw.HW_C128, coin, marked, addressing, shift=1, record=True)
        assert np.max(np.abs(psi.numpy() - ref)) <= TOL128
        assert np.max(np.abs(prob - oracle.prob_coined(ar, ref))) <= TOL128
        assert np.max(np.abs(rec.numpy() - rec_ref)) <= TOL128
    G.free()


def test_persistent_shift_c64_1000_steps(hw):
    # the figure's setting: Grover coin, persistent shift, walker leaving the
    # centre of a grid; here a 41 x 41 torus, 1000 steps
    L = 41
    g = synth.torus_rect(L, L)
    ar = oracle.Arcs(*g)
    G = _graph(hw, g)
    c = (L // 2) * L + L // 2
    psi0 = synth.state_on_vertex_arcs(synth.arc_offsets(*g), c)
    ref = oracle.coined_evolve(ar, psi0, 1000, 0, persistent_torus=(L, L))
    p_ref = oracle.prob_coined(ar, ref)
    _, p, _ = _evolve(hw, G, psi0, 1000, hw.HW_C64, 0, (), 0, shift=1)
    assert np.sum(np.abs(p - p_ref)) <= TOL64_L1
    G.free()


def test_persistent_shift_batched_and_arc_major_paths(hw):
    # batch > 1 runs the arc-major batched kernels with the persistent table
    L1, L2, B = 9, 14, 3
    g = synth.torus_rect(L1, L2)
    ar = oracle.Arcs(*g)
    G = _graph(hw, g)
    cols = [synth.random_state(ar.num_arcs, seed=50 + b) for b in range(B)]
    psi0 = np.stack(cols, axis=1).reshape(-1)
    for coin in (0, 1):
        psi, _, _ = _evolve(hw, G, psi0, 17, hw.HW_C128, coin, [5], shift=1, batch=B)
        got = psi.numpy().reshape(ar.num_arcs, B)
        for b in range(B):
            ref = oracle.coined_evolve(ar, cols[b], 17, coin, [5], persistent_torus=(L1, L2))
            assert np.max(np.abs(got[:, b] - ref)) <= TOL128
    G.free()


def test_persistent_shift_sampled_matches_evolve(hw):
    torch = _torch()
    L1, L2 = 12, 10
    g = synth.torus_rect(L1, L2)
    G = _graph(hw, g)
    psi0 = torch.from_numpy(synth.random_state(G.num_arcs, seed=9)).cuda()
    R = 5
    states = torch.empty((R, G.num_arcs), dtype=torch.complex128, device="cuda")
    hw.hw_coined_sample(G, 0, [3], hw.HW_C128, 1, 2, 2 + 3 * R, 3, psi0, states, None, opts={"shift": 1})
    for r in range(R):
        out = torch.empty_like(psi0)
        hw.hw_coined_evolve(G, 0, [3], hw.HW_C128, 1, 2 + 3 * r, psi0, out, opts={"shift": 1})
        assert torch.equal(out, states[r])
    G.free()


def test_persistent_shift_needs_a_torus(hw):
    torch = _torch()
    for g in (synth.hypercube(5), synth.cycle(10)):
        G = _graph(hw, g)
        x = torch.zeros(G.num_arcs, dtype=torch.complex128, device="cuda")
        with pytest.raises(hw.HWError) as e:
            hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 3, x, torch.empty_like(x), opts={"shift": 1})
        assert e.value.status == hw.HW_EINVAL
        with pytest.raises(hw.HWError):
            hw.hw_coined_evolve(G, 0, [], hw.HW_C128, 1, 3, x, torch.empty_like(x), opts={"addressing": 2})
        G.free()


# degrees 9..16 complex128 and 16..20 complex64 take the register-resident
# hypercube kernel with index-free addressing and the two-pass kernel through
# the table; other (degree, precision) pairs the two-pass or arc-major kernels
@pytest.mark.parametrize("k", [9, 12, 16, 17])
@pytest.mark.parametrize("dt", [1, 2])
def test_hypercube_index_free_bit_identical_and_matches_oracle(hw, k, dt):
    g = synth.hypercube(k)
    G = _graph(hw, g)
    assert hw.hw_graph_structure(G) == (hw.HW_GRAPH_HYPERCUBE, (k, 0))
    psi0 = synth.random_state(G.num_arcs, seed=k)
    marked = [0, G.n - 1, 77]
    steps = 15
    a = _evolve(hw, G, psi0, steps, dt, 0, marked, addressing=0, record=True)
    b = _evolve(hw, G, psi0, steps, dt, 0, marked, addressing=1, record=True)
    torch = _torch()
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[2])
    if (dt == hw.HW_C128 and k <= 12) or k >= 16:
        ar = oracle.Arcs(*g)
        ref, rec_ref = oracle.coined_evolve(ar, psi0, steps, 0, marked, record=True)
        if dt == hw.HW_C128:
            assert np.max(np.abs(a[0].numpy() - ref)) <= TOL128
            assert np.max(np.abs(a[2].numpy() - rec_ref)) <= TOL128
        else:
            assert np.sum(np.abs(a[1] - oracle.prob_coined(ar, ref))) <= TOL64_L1
            assert np.max(np.abs(a[2].numpy() - rec_ref)) <= 1e-5
    G.free()


@pytest.mark.parametrize("name,g", [("torus", synth.torus_rect(37, 53)), ("torus_sq", synth.torus(256)),
                                    ("Q11", synth.hypercube(11)), ("Q16", synth.hypercube(16))])
@pytest.mark.parametrize("dt", [1, 2])
def test_sparse_ctqw_index_free(hw, name, g, dt):
    torch = _torch()
    G = _graph(hw, g)
    n = G.n
    marked = [1, n - 2]
    gamma, tau, steps = 0.25, 0.1, 12
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    psi0 = synth.random_state(n, seed=4)
    x = torch.from_numpy(psi0).to("cuda", cdt)
    outs = []
    for addressing in (0, 1):
        y = torch.empty_like(x)
        rec = torch.empty(steps, dtype=torch.float64, device="cuda")
        hw.hw_ctqw_evolve_sparse(G, gamma, marked, tau, dt, 1, steps, x, y, rec, opts={"addressing": addressing})
        outs.append((y.cpu(), rec.cpu()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    if n <= 70000:
        ar = oracle.Arcs(*g)
        ref = oracle.ctqw_evolve(ar, gamma, psi0, tau, steps, marked)
        got = outs[0][0].numpy().astype(np.complex128)
        if dt == hw.HW_C128:
            assert np.max(np.abs(got - ref)) <= TOL128
        else:
            assert np.sum(np.abs(np.abs(got) ** 2 - np.abs(ref) ** 2)) <= TOL64_L1
    G.free()


def test_complex128_sums_on_every_path_of_the_integer_sum(hw):
    # amplitudes spanning many binades inside one vertex (the sequential
    # fallback), subnormals, exact zeros and cancelling pairs, next to
    # ordinary ones (the integer path): the degree-4 coin against the oracle,
    # and the index-free and table kernels bit for bit
    L1, L2 = 24, 40
    g = synth.torus_rect(L1, L2)
    ar = oracle.Arcs(*g)
    G = _graph(hw, g)
    psi0 = synth.random_state(ar.num_arcs, seed=17)
    rng = np.random.default_rng(5)
    scale = 10.0 ** rng.integers(-40, 3, size=ar.num_arcs)
    psi0 = psi0 * scale
    psi0[::7] = 0.0
    psi0[1::11] = 5e-320 + 0j                          # subnormal real parts
    psi0[3::13] = -psi0[2::13][: psi0[3::13].size]     # cancelling neighbours in a block
    psi0 = psi0 / np.sqrt(np.sum(np.abs(psi0) ** 2))
    ref = oracle.coined_evolve(ar, psi0, 9, 0, [3, 500])
    a = _evolve(hw, G, psi0, 9, hw.HW_C128, 0, [3, 500], addressing=0)
    b = _evolve(hw, G, psi0, 9, hw.HW_C128, 0, [3, 500], addressing=1)
    torch = _torch()
    assert torch.equal(a[0], b[0])
    assert np.max(np.abs(a[0].numpy() - ref)) <= TOL128
    G.free()


@pytest.mark.parametrize("name,g", [("reg18_1000", synth.random_regular(1000, 18, seed=3)),   # 1000 = 31 x 32 + 8
                                    ("reg24_777", synth.random_regular(778, 24, seed=5)),
                                    ("Q18", synth.hypercube(18))])
def test_complex128_high_degree_two_pass_matches_oracle(hw, name, g):
    # complex128 Grover of degree 17..24 takes the two-pass kernel (sums, then
    # the rows again last-first); regular graphs through the table, the
    # hypercube from its labels
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    psi0 = synth.random_state(ar.num_arcs, seed=8)
    marked = [2, G.n // 3, G.n - 1]
    steps = 11
    a = _evolve(hw, G, psi0, steps, hw.HW_C128, 0, marked, addressing=0, record=True)
    ref, rec_ref = oracle.coined_evolve(ar, psi0, steps, 0, marked, record=True)
    assert np.max(np.abs(a[0].numpy() - ref)) <= TOL128
    assert np.max(np.abs(a[2].numpy() - rec_ref)) <= TOL128
    G.free()
