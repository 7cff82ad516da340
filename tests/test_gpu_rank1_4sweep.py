"""Rank-1 four-sweep path (rows of 4096 points, columns split in two sweeps), path selection and
autotuning, against the FP64 oracle (GB300)."""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 5e-5}


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(lib, inst, prec, nsteps, path=None, dt=None):
    import torch
    dt = inst.dt if dt is None else dt
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
    if path is not None:
        plan.set_path(path)
        assert plan.info()["path"] == path
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.strang_steps(dt, nsteps)
    assert plan.status() == 0
    got = plan.get_state(prec="c128").cpu().numpy()
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, dt, nsteps)
    return got, ref, plan, (P, norms, v, u0)


@pytest.mark.parametrize("m", [20, 22])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_four_sweep_parity(lib, m, prec):
    inst = w.c2(m)
    got, ref, plan, _ = _run(lib, inst, prec, 50, path=lib.PATH_RANK1_4SWEEP)
    assert plan.info()["N1"] == 4096 and plan.info()["N2"] == inst.npoints // 4096
    assert rel_l2(got, ref) < TOL[prec]


def test_four_sweep_default_beyond_two_sweep_sizes(lib):
    """n = 2^24 (c128) and 2^23 (c128) exceed the complex128 two-sweep kernels: the plan takes the
    four-sweep path on its own; in complex64 the TMA two-sweep path is the default at 2^24 and the
    four-sweep path is taken on request."""
    import torch
    inst = w.c2(24)
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    del P
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 10)
    for prec in ("c128", "c64"):
        plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
        if prec == "c64":
            assert plan.info()["path"] == lib.PATH_RANK1_TMA
            plan.set_path(lib.PATH_RANK1_4SWEEP)
        assert plan.info()["path"] == lib.PATH_RANK1_4SWEEP
        plan.set_potential(torch.from_numpy(v).cuda())
        plan.set_state(torch.from_numpy(u0).cuda())
        plan.strang_steps(inst.dt, 10)
        assert plan.status() == 0
        assert rel_l2(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL[prec]
        del plan
    p23 = lib.Plan(w.c2(23).Zmat, (1 << 23,), 0.05, prec="c128")
    assert p23.info()["path"] == lib.PATH_RANK1_4SWEEP


def test_four_sweep_spectral(lib):
    import torch
    inst = w.c2(22)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(inst.npoints) + 1j * rng.standard_normal(inst.npoints)
    for prec, tol in (("c128", 1e-13), ("c64", 2e-6)):
        plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
        plan.set_path(lib.PATH_RANK1_4SWEEP)
        plan.set_state(torch.from_numpy(u).cuda())
        got = plan.get_state(space="spectral", prec="c128").cpu().numpy()
        assert rel_l2(got, S.coeffs(u, inst.n)) < tol


def test_paths_set_path_and_errors(lib):
    inst = w.c2(20)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64")
    assert plan.info()["path"] == lib.PATH_RANK1_TMA            # complex64 default from 2^20 to 2^23
    assert lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128").info()["path"] == lib.PATH_MULTIPASS
    assert set(plan.paths()) == {lib.PATH_MULTIPASS, lib.PATH_RANK1_4SWEEP, lib.PATH_RANK1_TMA}
    c128 = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128")
    assert set(c128.paths()) == {lib.PATH_MULTIPASS, lib.PATH_RANK1_4SWEEP}    # the TMA path is complex64 only
    with pytest.raises(lib.LspError) as e:
        c128.set_path(lib.PATH_RANK1_TMA)
    assert e.value.code == -8
    with pytest.raises(lib.LspError) as e:
        plan.set_path(lib.PATH_RANK2)
    assert e.value.code == -8
    with pytest.raises(lib.LspError) as e:
        plan.set_path(7)
    assert e.value.code == -1
    small = lib.Plan(np.array([1, 5]), (64,), 0.1, prec="c64")
    assert small.paths() == [lib.PATH_SMALL]


def test_autotune_keeps_results_and_state(lib):
    """autotune times both rank-1 paths on a scratch copy, keeps the faster, and the plan's
    state and later steps are unchanged by it."""
    import torch
    inst = w.c2(22)
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128")
    assert plan.info()["path"] == lib.PATH_MULTIPASS           # complex128 default at 2^22
    assert lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64").info()["path"] == lib.PATH_RANK1_TMA
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    chosen, ms = plan.autotune(inst.dt, 10)
    assert set(ms) == {lib.PATH_MULTIPASS, lib.PATH_RANK1_4SWEEP} and all(t > 0 for t in ms.values())  # c128
    assert chosen == min(ms, key=ms.get) and plan.info()["path"] == chosen
    assert rel_l2(plan.get_state().cpu().numpy(), u0) == 0.0
    plan.strang_steps(inst.dt, 20)
    assert rel_l2(plan.get_state().cpu().numpy(), S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 20)) < 1e-10


def test_four_sweep_batch_and_adjoint(lib):
    import torch
    inst = w.c4(20)
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plans = [lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128") for _ in range(2)]
    plans[1].set_path(lib.PATH_RANK1_4SWEEP)
    for p in plans:
        p.set_potential(torch.from_numpy(v).cuda())
        p.set_state(torch.from_numpy(u0).cuda())
    b = lib.Batch(plans)
    b.steps([1e-3, 2e-3], 15)
    assert b.status() == 0
    for p, dt in zip(plans, (1e-3, 2e-3)):
        assert rel_l2(p.get_state().cpu().numpy(), S.strang(u0, v, norms, inst.n, inst.gamma, dt, 15)) < 1e-10
    plans[0].set_path(lib.PATH_RANK1_4SWEEP)        # a batch member may not change path
    with pytest.raises(lib.LspError) as e:
        b.steps([1e-3, 1e-3], 1)
    assert e.value.code == -1
    b.destroy()
    phi = inst.phi(P)
    J, gv_ref, gu_ref, uN = S.strang_adjoint(u0, v, norms, inst.n, inst.gamma, inst.dt, 10, phi)
    p = plans[1]
    p.set_state(torch.from_numpy(u0).cuda())
    lam = torch.from_numpy(2.0 * S.inner(phi, uN) * phi / phi.size).cuda()
    gv = torch.empty(inst.npoints, dtype=torch.float64, device="cuda")
    gu = torch.empty(inst.npoints, dtype=torch.complex128, device="cuda")
    lib.adjoint(p, inst.dt, 10, lam, gv, gu, 3)
    assert p.status() == 0
    assert rel_l2(gv.cpu().numpy(), gv_ref) < 1e-9
    assert rel_l2(gu.cpu().numpy(), gu_ref) < 1e-9


def test_c2_1000_steps_complex64_against_complex128(lib):
    """The bench workload (d = 6, n = 2^22, 1000 steps): the complex64 four-sweep path against
    the complex128 two-sweep path (itself pinned to the oracle), and the complex64 norm drift."""
    import torch
    inst = w.c2(22)
    pts = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64").lattice_points()
    v, u0 = torch.from_numpy(inst.v(pts)).cuda(), torch.from_numpy(inst.u0(pts)).cuda()
    out = {}
    for prec, path in (("c64", lib.PATH_RANK1_4SWEEP), ("c128", lib.PATH_MULTIPASS)):
        plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
        plan.set_path(path)
        plan.set_potential(v)
        plan.set_state(u0)
        n0, _ = plan.observables()
        plan.strang_steps(inst.dt, 1000)
        n1, _ = plan.observables()
        out[prec] = (plan.get_state(prec="c128"), abs(n1 / n0 - 1))
    err = float(torch.linalg.norm(out["c64"][0] - out["c128"][0]) / torch.linalg.norm(out["c128"][0]))
    print(f"C2 1000 steps: complex64 four-sweep rel-L2 {err:.3e}, norm drift {out['c64'][1]:.3e}")
    assert err < 5e-5 and out["c64"][1] < 5e-5 and out["c128"][1] < 1e-12


def test_sweep_times_leave_the_state(lib):
    """lsp_sweep_times: positive per-sweep durations on the four-sweep paths, the plan's state
    untouched, UNSUPPORTED on the two-sweep path."""
    import torch
    inst = w.c2(20)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64")
    plan.set_path(lib.PATH_RANK1_4SWEEP)
    u0 = torch.randn(inst.npoints, dtype=torch.complex64, device="cuda")
    plan.set_state(u0)
    t = plan.sweep_times(inst.dt, 8)
    assert set(t) == {"P", "A", "K", "A_inv"} and all(x > 0 for x in t.values())
    assert torch.equal(plan.get_state(), u0)
    plan.set_path(lib.PATH_MULTIPASS)
    with pytest.raises(lib.LspError) as e:
        plan.sweep_times(inst.dt, 8)
    assert e.value.code == -8
