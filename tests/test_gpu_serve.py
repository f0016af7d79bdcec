"""Serving (continuous batching of walk jobs) and the sparse-action CTQW path.

The sparse action e^{-iH dt} psi is compared with the FP64 oracle.  Served
jobs are compared with the plain one-job-at-a-time calls, a job's result must
be identical alone and in a mix, admission must respect the memory arena,
and unsupported or oversized jobs must be rejected at submit.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _graph(hw, g):
    row_ptr, col = synth.adjacency_csr(*g)
    return hw.hw_graph_csr(g[0], row_ptr, col)


@pytest.mark.parametrize("name,g,gamma,marked,t", [
    ("Q10", synth.hypercube(10), 0.1, [700], 0.1),
    ("er", synth.erdos_renyi(600, 0.01, seed=3), 0.4, [2, 100], 0.3),
    ("cycle", synth.cycle(101), 0.5, [], 5.0),           # ||H dt|| = 5: split into 16 parts
])
def test_sparse_ctqw_matches_oracle(hw, name, g, gamma, marked, t):
    import torch
    n = g[0]
    marked = [m for m in marked if m < n]
    G = _graph(hw, g)
    ar = oracle.Arcs(*g)
    psi0 = synth.random_state(n, seed=4)
    steps = 40
    for dt in (2, 1):
        cdt = torch.complex128 if dt == 2 else torch.complex64
        x = torch.from_numpy(psi0).to("cuda", cdt)
        y = torch.empty_like(x)
        rec = torch.empty(steps, dtype=torch.float64, device="cuda") if marked else None
        hw.hw_ctqw_evolve_sparse(G, gamma, marked, t, dt, 1, steps, x, y, rec)
        ref, rr = oracle.ctqw_evolve(ar, gamma, psi0, t, steps, marked=marked, record=True)
        got = y.cpu().numpy().astype(np.complex128)
        if dt == 2:
            assert np.max(np.abs(got - ref)) <= 1e-12
            if marked:
                assert np.max(np.abs(rec.cpu().numpy() - rr)) <= 1e-12
        else:
            assert np.sum(np.abs(np.abs(got) ** 2 - np.abs(ref) ** 2)) <= 1e-4
    G.free()


def _plain(hw, G, kind, dt, steps, marked, gamma=0.0, t=0.0):
    """The one-job-at-a-time path: uniform start, evolve, probabilities, record."""
    import torch
    cdt = torch.complex128 if dt == 2 else torch.complex64
    dim = G.num_arcs if kind == hw.HW_JOB_COINED else G.n
    x = torch.full((dim,), 1.0 / np.sqrt(dim), dtype=cdt, device="cuda")
    y = torch.empty_like(x)
    rec = torch.empty(steps, dtype=torch.float64, device="cuda") if marked else None
    if kind == hw.HW_JOB_COINED:
        hw.hw_coined_evolve(G, 0, marked, dt, 1, steps, x, y, rec)
    else:
        hw.hw_ctqw_evolve_sparse(G, gamma, marked, t, dt, 1, steps, x, y, rec)
    prob = torch.empty(G.n, dtype=torch.float64, device="cuda")
    hw.hw_probability(G if kind == hw.HW_JOB_COINED else None, G.n, dt, 1, y, prob)
    torch.cuda.synchronize()
    return prob.cpu().numpy(), None if rec is None else rec.cpu().numpy()


DEGREE = {"torus": 4, "Q9": 9, "reg3": 3, "reg8": 8, "t": 4, "torus72": 4, "Q12": 12, "reg8k": 8, "torus96": 4}


def _mix(hw):
    graphs = {
        "torus": _graph(hw, synth.torus(48)),
        "Q9": _graph(hw, synth.hypercube(9)),
        "reg3": _graph(hw, synth.random_regular(2000, 3, seed=1)),
        "reg8": _graph(hw, synth.random_regular(1500, 8, seed=2)),
        # 5184 vertices: too many for a complex128 job in one CTA's shared
        # memory, so this CTQW job takes the tiled path (one launch per term)
        "torus72": _graph(hw, synth.torus(72)),
    }
    jobs = [
        ("torus", hw.HW_JOB_COINED, 2, 37, [5, 600]),
        ("torus", hw.HW_JOB_COINED, 1, 120, [17]),
        ("Q9", hw.HW_JOB_COINED, 2, 25, []),
        ("reg3", hw.HW_JOB_COINED, 1, 64, [0, 1, 2, 1999]),
        ("reg8", hw.HW_JOB_COINED, 2, 10, [7]),
        ("Q9", hw.HW_JOB_CTQW, 2, 30, [3]),
        ("reg3", hw.HW_JOB_CTQW, 1, 12, [10, 20]),
        ("torus", hw.HW_JOB_CTQW, 2, 8, []),
        ("reg8", hw.HW_JOB_CTQW, 1, 50, [1499]),
        ("torus72", hw.HW_JOB_CTQW, 2, 6, [100, 5000]),
    ]
    return graphs, jobs


def _serve(hw, graphs, jobs, arena=1 << 30, substeps=8):
    """Submit every job at once, run rounds until all are collectable, return results in order."""
    srv = hw.Server(arena, max_jobs=64, substeps=substeps)
    ids = [srv.submit(graphs[gname], kind, dt, steps, marked, gamma=1.0 / DEGREE[gname], time=0.1)
           for gname, kind, dt, steps, marked in jobs]
    done = srv.drain()
    assert sorted(done) == sorted(ids)
    out = [srv.result(i) for i in ids]
    srv.close()
    return out


def test_served_jobs_match_plain_calls_and_are_mix_independent(hw):
    graphs, jobs = _mix(hw)
    mixed = _serve(hw, graphs, jobs)
    for (gname, kind, dt, steps, marked), (prob, rec, lat) in zip(jobs, mixed):
        G = graphs[gname]
        p_ref, r_ref = _plain(hw, G, kind, dt, steps, marked, 1.0 / DEGREE[gname], 0.1)
        tol = 1e-12 if dt == 2 else 1e-5
        assert np.max(np.abs(prob - p_ref)) <= tol, (gname, kind, dt)
        if marked:
            assert np.max(np.abs(rec - r_ref)) <= tol
        assert abs(prob.sum() - 1.0) < (1e-12 if dt == 2 else 1e-4)
        assert lat > 0
    # each job alone gives bit-identical results to the same job in the mix
    for k in (0, 3, 5, 6, 9):
        alone = _serve(hw, graphs, [jobs[k]])[0]
        assert np.array_equal(alone[0], mixed[k][0])
        if jobs[k][4]:
            assert np.array_equal(alone[1], mixed[k][1])
    for G in graphs.values():
        G.free()


def test_served_coined_matches_oracle(hw):
    g = synth.torus(40)
    G = _graph(hw, g)
    (prob, rec, _), = _serve(hw, {"t": G}, [("t", hw.HW_JOB_COINED, 2, 55, [33, 800])])
    ar = oracle.Arcs(*g)
    ref, rr = oracle.coined_evolve(ar, synth.uniform_state(ar.num_arcs), 55, marked=[33, 800], record=True)
    assert np.max(np.abs(prob - oracle.prob_coined(ar, ref))) <= 1e-12
    assert np.max(np.abs(rec - rr)) <= 1e-12
    G.free()


def test_served_ctqw_matches_oracle(hw):
    # both CTQW branches of the server against the FP64 oracle, with marks and
    # the marked-probability record: shared-memory ("local") jobs, complex128
    # on 4096 vertices and complex64 on 8192; tiled jobs (one launch per
    # series term), complex128 on 5184 vertices and complex64 on 9216
    gs = {"Q12": synth.hypercube(12), "reg8k": synth.random_regular(8192, 8, seed=5),
          "torus72": synth.torus(72), "torus96": synth.torus(96)}
    graphs = {k: _graph(hw, g) for k, g in gs.items()}
    jobs = [("Q12", hw.HW_JOB_CTQW, 2, 25, [4077, 9]),
            ("reg8k", hw.HW_JOB_CTQW, 1, 40, [3]),
            ("torus72", hw.HW_JOB_CTQW, 2, 15, [100, 5000]),
            ("torus96", hw.HW_JOB_CTQW, 1, 20, [1, 4000, 9000])]
    served = _serve(hw, graphs, jobs)
    for (gname, kind, dt, steps, marked), (prob, rec, _) in zip(jobs, served):
        ar = oracle.Arcs(*gs[gname])
        n = gs[gname][0]
        ref, rr = oracle.ctqw_evolve(ar, 1.0 / DEGREE[gname], np.full(n, 1 / np.sqrt(n), dtype=np.complex128),
                                     0.1, steps, marked=marked, record=True)
        p_ref = np.abs(ref) ** 2
        if dt == 2:
            assert np.max(np.abs(prob - p_ref)) <= 1e-12, gname
            assert np.max(np.abs(rec - rr)) <= 1e-12, gname
        else:
            assert np.sum(np.abs(prob - p_ref)) <= 1e-3, gname
            assert np.max(np.abs(rec - rr)) <= 1e-4, gname
    for G in graphs.values():
        G.free()


def test_admission_waits_for_arena_memory(hw):
    # each job needs ~2 x 2|E| x 16 B; the arena fits about two at a time
    g = synth.torus(128)
    G = _graph(hw, g)
    per_job = 2 * G.num_arcs * 16 + G.n * 8 + 2 * 400 * 8 + 4096
    srv = hw.Server(int(2.5 * per_job), max_jobs=16, substeps=4)
    ids = [srv.submit(G, hw.HW_JOB_COINED, 2, 40 + i, [i]) for i in range(6)]
    peak = 0
    done = []
    while len(done) < len(ids):
        srv.run()
        done += srv.poll()
        st = srv.stats()
        peak = max(peak, st["resident"])
        assert st["arena_used"] <= int(2.5 * per_job)
    assert peak == 2
    for i, jid in enumerate(ids):
        prob, rec, _ = srv.result(jid)
        p_ref, r_ref = _plain(hw, G, hw.HW_JOB_COINED, 2, 40 + i, [i])
        assert np.max(np.abs(prob - p_ref)) <= 1e-12
    srv.close()
    G.free()


def test_submit_rejections(hw):
    G = _graph(hw, synth.torus(256))      # one state alone is 4 MiB
    irregular = _graph(hw, synth.erdos_renyi(300, 0.02, seed=1))
    srv = hw.Server(1 << 20, max_jobs=4, substeps=2)
    with pytest.raises(hw.HWError) as e:
        srv.submit(G, hw.HW_JOB_COINED, 2, 10)          # needs more than the 1 MiB arena
    assert e.value.status == hw.HW_ENOMEM
    with pytest.raises(hw.HWError) as e:
        srv.submit(irregular, hw.HW_JOB_COINED, 2, 10)  # coined serving needs a regular graph
    assert e.value.status == hw.HW_EUNSUPPORTED
    with pytest.raises(hw.HWError) as e:
        srv.submit(G, hw.HW_JOB_COINED, 2, 10, [1, 2, 3, 4, 5])
    assert e.value.status == hw.HW_EINVAL
    srv.close()
    G.free()
    irregular.free()
