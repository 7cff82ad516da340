"""The allocation-free entry point lsp_strang_steps_noalloc against the plan-based one.

Some callers cannot allocate device memory (an allocator that must own every
device byte, a real-time loop that may not allocate once running); they use
lsp_strang_steps_noalloc, whose scratch lives in a fixed device array.  This
file runs last so that a failure here leaves every other test already run.
"""

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 5e-5}


def _inputs(inst):
    from oracle import lattice as L
    P = L.lattice_points(inst.Z, inst.n)
    return inst.v(P), inst.u0(P)


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("which", ["c1", "n8192"])
def test_noalloc_matches_plan_on_two_calls(lib, prec, which):
    import torch
    if which == "c1":
        inst = w.c1()
        plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec, aa="explicit", index_set=inst.index_set)
    else:
        if prec == "c128":
            pytest.skip("complex128 allocation-free path holds at most 6400 points")
        inst = w.c2(13)
        plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
    v, u0 = _inputs(inst)
    dt = np.complex64 if prec == "c64" else np.complex128
    tdt = torch.complex64 if prec == "c64" else torch.complex128
    vd = torch.from_numpy(v).cuda()
    norm2 = torch.from_numpy(plan.index_norms().astype(np.int32)).cuda()
    u = torch.from_numpy(u0.astype(dt)).cuda()
    plan.set_potential(vd)
    plan.set_state(torch.from_numpy(u0.astype(dt)).cuda())
    for call in range(2):                     # two calls in a row share the fixed scratch
        lib.strang_steps_noalloc(u, vd, norm2, inst.gamma, inst.dt, 25)
        plan.strang_steps(inst.dt, 25)
        ref = plan.get_state(prec="c128").cpu().numpy()
        got = u.to(torch.complex128).cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < TOL[prec], (call, err)
    assert u.dtype == tdt


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    import torch
    u = torch.zeros(8193, dtype=torch.complex64, device="cuda")
    v = torch.zeros(8193, dtype=torch.float64, device="cuda")
    nrm = torch.zeros(8193, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.LspError) as e:
        lib.strang_steps_noalloc(u, v, nrm, 0.1, 1e-3, 1)
    assert e.value.code == -4
