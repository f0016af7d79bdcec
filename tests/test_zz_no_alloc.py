"""hw_probability_noalloc: the allocation-free variant of hw_probability.

It serves callers that cannot allocate device memory during a call (a fixed,
pre-reserved memory budget; no stream-ordered allocator on the platform).  Its
results must equal those of hw_probability, call after call, although every
call reuses the same built-in scratch array.  This file is collected last so a
failure here leaves every other test already run; it also passes on its own
in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the complex128 parity bar used throughout the GPU tests


def _both(hw, G, n, dt, batch, psi):
    import torch
    p_ref = torch.empty(n * batch, dtype=torch.float64, device="cuda")
    n_ref = torch.empty(batch, dtype=torch.float64, device="cuda")
    hw.hw_probability(G, n, dt, batch, psi, p_ref, n_ref)
    outs = []
    for _ in range(2):   # two calls in a row through the same scratch array
        p = torch.full((n * batch,), float("nan"), dtype=torch.float64, device="cuda")
        nm = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
        hw.hw_probability_noalloc(G, n, dt, batch, psi, p, nm)
        outs.append((p, nm))
    torch.cuda.synchronize()
    return p_ref.cpu().numpy(), n_ref.cpu().numpy(), [(p.cpu().numpy(), nm.cpu().numpy()) for p, nm in outs]


@pytest.mark.parametrize("dt,batch", [(2, 1), (1, 1), (2, 5), (1, 64)])
def test_noalloc_matches_hw_probability_coined(hw, dt, batch):
    import torch
    n, eu, ev = synth.erdos_renyi(30000, 8 / 29999, seed=21)
    row_ptr, col = synth.adjacency_csr(n, eu, ev)
    G = hw.hw_graph_csr(n, row_ptr, col)
    psi0 = synth.gaussian_states(G.num_arcs, batch, seed=22)
    cdt = torch.complex128 if dt == hw.HW_C128 else torch.complex64
    psi = torch.from_numpy(psi0).to("cuda", cdt).reshape(-1)
    p_ref, n_ref, outs = _both(hw, G, n, dt, batch, psi)
    for p, nm in outs:
        assert np.max(np.abs(p - p_ref)) <= TOL
        assert np.max(np.abs(nm - n_ref)) <= TOL
    G.free()


def test_noalloc_matches_hw_probability_vertex_states(hw):
    import torch
    n, batch = 4096, 3
    psi = torch.from_numpy(synth.gaussian_states(n, batch, seed=23)).cuda().reshape(-1)
    p_ref, n_ref, outs = _both(hw, None, n, hw.HW_C128, batch, psi)
    for p, nm in outs:
        assert np.max(np.abs(p - p_ref)) <= TOL
        assert np.max(np.abs(nm - n_ref)) <= TOL


def test_noalloc_fills_the_whole_scratch_array(hw):
    # the largest partial count (1184 row chunks) times the largest batch (64)
    # writes every slot of the built-in array, the last one included
    import torch
    n, batch = 1184 * 4096 + 1, 64
    gen = torch.Generator(device="cuda").manual_seed(31)
    psi = torch.randn(n * batch, dtype=torch.complex128, device="cuda", generator=gen)
    n_ref = torch.empty(batch, dtype=torch.float64, device="cuda")
    hw.hw_probability(None, n, hw.HW_C128, batch, psi, None, n_ref)
    for _ in range(2):
        nm = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
        hw.hw_probability_noalloc(None, n, hw.HW_C128, batch, psi, None, nm)
        torch.cuda.synchronize()
        # both reductions run the same fixed order, so they agree far below
        # the bar; the sums are about 2n, so the bar is relative
        assert np.max(np.abs(nm.cpu().numpy() - n_ref.cpu().numpy()) / n_ref.cpu().numpy()) <= TOL
    del psi
    torch.cuda.empty_cache()


def test_noalloc_rejects_batch_over_limit(hw):
    import torch
    n = 64
    psi = torch.zeros(n * 65, dtype=torch.complex128, device="cuda")
    norm = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(hw.HWError) as e:
        hw.hw_probability_noalloc(None, n, hw.HW_C128, 65, psi, None, norm)
    assert e.value.status == hw.HW_EINVAL
    assert "limit" in e.value.message
