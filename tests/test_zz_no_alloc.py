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


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_noalloc_c1_1000_steps_against_oracle(lib, prec):
    """The allocation-free loop directly against the FP64 oracle on the d = 2, n = 961
    workload (box |h_j| <= 15, z = (1, 31)): 1000 steps of dt = 1e-3, two calls of 500."""
    import torch
    from oracle import lattice as L
    from oracle import strang as S
    inst = w.c1()
    v, u0 = _inputs(inst)
    norms = L.explicit_norms(inst.index_set, inst.Z, inst.n)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 1000)
    dt = np.complex64 if prec == "c64" else np.complex128
    u = torch.from_numpy(u0.astype(dt)).cuda()
    vd = torch.from_numpy(v).cuda()
    nd = torch.from_numpy(norms.astype(np.int32)).cuda()
    for _ in range(2):
        lib.strang_steps_noalloc(u, vd, nd, inst.gamma, inst.dt, 500)
    got = u.to(torch.complex128).cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < TOL[prec], err


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_noalloc_odd_prime_factors(lib, prec):
    """n = 3465 = 3^2 5 7 11: radix-3, -5, -7 and -11 passes, against the plan path and the oracle."""
    import torch
    from oracle import lattice as L
    from oracle import strang as S
    Z, n, gamma, dts = np.array([1, 1021, 2311]), 3465, 0.2, 2e-3
    P = L.lattice_points(Z, n)
    rng = np.random.default_rng(5)
    v = 1.0 + np.cos(2 * np.pi * P[:, 0]) * np.cos(2 * np.pi * (P[:, 1] - P[:, 2]))
    u0 = np.exp(-np.sum((P - 0.5) ** 2, axis=1) / 0.02) * np.exp(2j * np.pi * 2 * P[:, 1])
    u0 = u0 + 0.01 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    norms, _ = L.minl2_norms_dp(Z, n)
    ref = S.strang(u0, v, norms, n, gamma, dts, 60)
    dt = np.complex64 if prec == "c64" else np.complex128
    plan = lib.Plan(Z.reshape(-1, 1), n, gamma, prec=prec)
    assert np.array_equal(plan.index_norms(), norms)
    vd = torch.from_numpy(v).cuda()
    plan.set_potential(vd)
    plan.set_state(torch.from_numpy(u0.astype(dt)).cuda())
    plan.strang_steps(dts, 60)
    via_plan = plan.get_state(prec="c128").cpu().numpy()
    u = torch.from_numpy(u0.astype(dt)).cuda()
    lib.strang_steps_noalloc(u, vd, torch.from_numpy(norms.astype(np.int32)).cuda(), gamma, dts, 60)
    got = u.to(torch.complex128).cpu().numpy()
    for name, x in (("noalloc", got), ("plan", via_plan)):
        err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
        assert err < TOL[prec], (name, err)
    plan.destroy()


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    import torch
    u = torch.zeros(8193, dtype=torch.complex64, device="cuda")
    v = torch.zeros(8193, dtype=torch.float64, device="cuda")
    nrm = torch.zeros(8193, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.LspError) as e:
        lib.strang_steps_noalloc(u, v, nrm, 0.1, 1e-3, 1)
    assert e.value.code == -4
