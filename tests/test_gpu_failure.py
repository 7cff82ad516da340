"""Failure detection without a GPU fault: a bounded device wait that runs out (GB300).

The persistent two-sweep kernel waits on a grid barrier between sweeps and on the
mbarrier of each tile prefetch.  Every such wait polls at most a set number of times,
then writes LSP_ERR_TIMEOUT into the plan's sticky error word and returns (after the
copy in flight has landed).  Here the limit is set to one poll so that the barriers run
out; the call must come back, report the timeout, refuse further steps, and recover
after lsp_set_state.
"""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["persistent", "tma"])
def test_bounded_wait_expires_and_plan_recovers(lib, which):
    """persistent: the grid barrier and prefetch waits of the two-sweep persistent kernel (2^16);
    tma: the tile-copy waits of the TMA-fed two-sweep kernels (2^20)."""
    import torch
    inst = w.c2(16 if which == "persistent" else 20)
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64")
    plan.set_path(lib.PATH_MULTIPASS if which == "persistent" else lib.PATH_RANK1_TMA)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.set_wait_limit(1)
    plan.strang_steps(inst.dt, 200)
    assert plan.status() == -7                          # LSP_ERR_TIMEOUT, no fault
    with pytest.raises(lib.LspError) as e:
        plan.strang_steps(inst.dt, 1)
    assert e.value.code == -7
    torch.cuda.synchronize()
    plan.set_wait_limit(0)
    plan.set_state(torch.from_numpy(u0).cuda())
    assert plan.status() == 0
    plan.strang_steps(inst.dt, 20)
    assert plan.status() == 0
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 20)
    got = plan.get_state(prec="c128").cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 5e-5
    plan.destroy()
