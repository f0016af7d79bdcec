"""The failure path of the device-side waits: every wait on the device has a
time budget, so no call blocks without limit.  The one-launch walk's bounded
mbarrier wait is made to run out on a barrier that no copy completes (nothing
faults, nothing waits without a limit); the next call on the graph reports
HW_ETIMEDOUT, and the call after it runs normally and matches the oracle, so
the context stays usable."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_device_wait_runs_out_and_is_reported(hw):
    import torch
    n, eu, ev = synth.torus(8)
    G = hw.hw_graph_csr(n, *synth.adjacency_csr(n, eu, ev))
    psi0 = synth.random_state(G.num_arcs, seed=11)
    x = torch.from_numpy(psi0).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    t0 = time.time()
    hw.hw_check_device_wait(G)
    torch.cuda.synchronize()
    waited = time.time() - t0
    # the wait's 2 s budget, after which the kernel ends by itself
    assert 1.5 < waited < 30
    with pytest.raises(hw.HWError) as e:
        hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [], hw.HW_C128, 1, 5, x, y)
    assert e.value.status == hw.HW_ETIMEDOUT
    # the error word is cleared and the device still works
    hw.hw_coined_evolve(G, hw.HW_COIN_GROVER, [], hw.HW_C128, 1, 5, x, y)
    torch.cuda.synchronize()
    ref = oracle.coined_evolve(oracle.Arcs(n, eu, ev), psi0, 5, oracle.GROVER)
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12
    G.free()
