"""Rank-2 multipass path (row sweep + two column sweeps per half step) against the FP64 oracle (GB300).

Element-by-element parity on lattices up to 2^22 points; on the full 2^14 x 2^12 lattice
(2^26 points, d = 16) spot checks the oracle computes one value at a time (spectral
coefficients by direct sums, the closed-form constant-potential evolution of plane
waves) and properties that hold at any size (norm, time reversal, FP32 against FP64).
"""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 5e-5}
SHAPES = [((10, 8), 6), ((11, 9), 8), ((12, 10), 10)]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _inst(shape, bound):
    return w.c5(*shape, 16, bound)


def _plan(lib, inst, prec):
    return lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)


def test_rank2_plan_path_points_and_norms(lib):
    inst = _inst(*SHAPES[0])
    plan = _plan(lib, inst, "c64")
    info = plan.info()
    assert info["path"] == lib.PATH_RANK2
    assert (info["N1"], info["N2"]) == (inst.n[1], inst.n[0])
    assert np.array_equal(plan.lattice_points(), L.lattice_points(inst.Z, inst.n))
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    assert np.array_equal(plan.index_norms(), norms)


@pytest.mark.parametrize("shape,bound", SHAPES, ids=[f"{s[0]}x{s[1]}" for s, _ in SHAPES])
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_rank2_spectral_coefficients(lib, shape, bound, prec):
    import torch
    inst = _inst(shape, bound)
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(inst.npoints) + 1j * rng.standard_normal(inst.npoints)
    plan = _plan(lib, inst, prec)
    plan.set_state(torch.from_numpy(u).cuda())
    got = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    assert rel_l2(got, S.coeffs(u, inst.n)) < (1e-13 if prec == "c128" else 2e-6)
    assert rel_l2(plan.get_state(prec="c128").cpu().numpy(), u) < (1e-15 if prec == "c128" else 1e-7)


def _run(lib, inst, prec, nsteps, dt=None):
    import torch
    dt = inst.dt if dt is None else dt
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plan = _plan(lib, inst, prec)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.strang_steps(dt, nsteps)
    assert plan.status() == 0
    got = plan.get_state(prec="c128").cpu().numpy()
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, dt, nsteps)
    return got, ref, u0


@pytest.mark.parametrize("shape,bound,nsteps", [(SHAPES[0][0], SHAPES[0][1], 50), (SHAPES[1][0], SHAPES[1][1], 50),
                                                 (SHAPES[2][0], SHAPES[2][1], 20)],
                         ids=["1024x256", "2048x512", "4096x1024"])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_rank2_strang_parity(lib, shape, bound, nsteps, prec):
    got, ref, _ = _run(lib, _inst(shape, bound), prec, nsteps)
    assert rel_l2(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_rank2_1000_steps(lib, prec):
    """Tolerances of the 1000-step runs on a 2^18-point rank-2 lattice, large dt; the norm
    drift bound for complex64 is the relative-L2 bound."""
    got, ref, u0 = _run(lib, _inst(*SHAPES[0]), prec, 1000, dt=1e-2)
    err = rel_l2(got, ref)
    drift = abs(S.norm2(got) / S.norm2(u0) - 1.0)
    print(f"rank-2 2^10 x 2^8, 1000 steps, {prec}: rel-L2 {err:.3e}, norm drift {drift:.3e}")
    assert err < TOL[prec]
    assert drift < (1e-12 if prec == "c128" else TOL["c64"])


def test_rank2_batch_and_adjoint(lib):
    """Rank-2 plans inside a batch (own dt each) and the adjoint of a rank-2 plan."""
    import torch
    inst = _inst(*SHAPES[0])
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plans = [_plan(lib, inst, "c128") for _ in range(2)]
    dts = [1e-3, 3e-3]
    for p in plans:
        p.set_potential(torch.from_numpy(v).cuda())
        p.set_state(torch.from_numpy(u0).cuda())
    b = lib.Batch(plans)
    b.steps(dts, 30)
    assert b.status() == 0
    for p, dt in zip(plans, dts):
        ref = S.strang(u0, v, norms, inst.n, inst.gamma, dt, 30)
        assert rel_l2(p.get_state().cpu().numpy(), ref) < 1e-10
    b.destroy()
    phi = w.gaussian_packet(P, 0.1, [0.6] + [0.5] * (inst.d - 1))
    J, gv_ref, gu_ref, uN = S.strang_adjoint(u0, v, norms, inst.n, inst.gamma, inst.dt, 12, phi)
    p = plans[0]
    p.set_state(torch.from_numpy(u0).cuda())
    lam = torch.from_numpy(2.0 * S.inner(phi, uN) * phi / phi.size).cuda()
    gv = torch.empty(inst.npoints, dtype=torch.float64, device="cuda")
    gu = torch.empty(inst.npoints, dtype=torch.complex128, device="cuda")
    lib.adjoint(p, inst.dt, 12, lam, gv, gu, 4)
    assert p.status() == 0
    assert rel_l2(gv.cpu().numpy(), gv_ref) < 1e-9
    assert rel_l2(gu.cpu().numpy(), gu_ref) < 1e-9


# ---------------------------------------------------------------------------
# Full size: 2^14 x 2^12, d = 16
# ---------------------------------------------------------------------------
def _full_plane_waves():
    """Five plane waves with ||h||^2 <= 4: each is the unique minimal-norm vector of its bin
    for the C5 lattice (every vector of norm^2 <= 4 lies in the hyperbolic cross, on which
    the lattice is injective)."""
    inst = w.c5()
    H = np.zeros((5, 16), dtype=np.int64)
    H[1, 0] = 1
    H[2, 3], H[2, 9] = 1, -1
    H[3, 5] = 2
    H[4, 1], H[4, 6], H[4, 11], H[4, 15] = 1, -1, 1, 1
    xi = L.residues(H, inst.Z, inst.n)
    norms = (H ** 2).sum(1)
    c = np.array([0.3, 1.0, 0.5j, -0.4 + 0.2j, 0.25])
    return inst, xi, norms, c


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_rank2_full_size_plane_waves(lib, prec):
    """200 steps on the full lattice with a constant potential: sampled values against the
    closed-form evolution, and the minimal norms of the five bins."""
    import torch
    inst, xi, norms, c = _full_plane_waves()
    plan = _plan(lib, inst, prec)
    chi = xi[:, 0] * inst.n[1] + xi[:, 1]
    assert np.array_equal(plan.index_norms()[chi], norms)
    u0 = w.plane_waves(xi, c, inst.n)
    vc = 0.37
    plan.set_potential(torch.full((inst.npoints,), vc, dtype=torch.float64, device="cuda"))
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.strang_steps(inst.dt, inst.nsteps)
    assert plan.status() == 0
    got = plan.get_state(prec="c128").cpu().numpy()
    rng = np.random.default_rng(11)
    idx = np.concatenate([np.arange(4096), rng.choice(inst.npoints, size=8192, replace=False)])
    kappa = np.stack(np.unravel_index(idx, inst.n), axis=1)
    ref = S.plane_wave_evolution(xi, norms, c, inst.n, inst.gamma, inst.dt, inst.nsteps, vc, kappa)
    assert rel_l2(got[idx], ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_rank2_full_size_sampled_spectral(lib, prec):
    import torch
    inst = w.c5()
    rng = np.random.default_rng(12)
    u = (rng.standard_normal(inst.npoints) + 1j * rng.standard_normal(inst.npoints))
    plan = _plan(lib, inst, prec)
    plan.set_state(torch.from_numpy(u).cuda())
    got = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    chi = np.concatenate([[0, 1, inst.n[1], inst.npoints - 1], rng.choice(inst.npoints, size=12, replace=False)])
    xi = np.stack(np.unravel_index(chi, inst.n), axis=1)
    ref = S.coeff_at(u, inst.n, xi)
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(got[chi] - ref)) < (1e-11 if prec == "c128" else 2e-5) * scale


def test_rank2_full_size_c5_workload(lib):
    """C5 (v = pair cosines, product Gaussian, 200 steps): FP32 against FP64, norm
    conservation, and time reversal of the FP64 run."""
    import torch
    inst = w.c5()
    v, u0 = w.c5_fields(inst)
    vt, ut = torch.from_numpy(v).cuda(), torch.from_numpy(u0).cuda()
    outs = {}
    for prec in ("c128", "c64"):
        plan = _plan(lib, inst, prec)
        plan.set_potential(vt)
        plan.set_state(ut)
        plan.strang_steps(inst.dt, inst.nsteps)
        assert plan.status() == 0
        outs[prec] = plan.get_state(prec="c128")
        n0 = float(torch.mean(torch.abs(ut) ** 2))
        drift = abs(float(torch.mean(torch.abs(outs[prec]) ** 2)) / n0 - 1.0)
        assert drift < (1e-12 if prec == "c128" else 1e-5)
        if prec == "c128":
            plan.strang_steps(-inst.dt, inst.nsteps)
            back = plan.get_state()
            assert float(torch.linalg.norm(back - ut) / torch.linalg.norm(ut)) < 1e-10
        del plan
    r = float(torch.linalg.norm(outs["c64"] - outs["c128"]) / torch.linalg.norm(outs["c128"]))
    assert r < TOL["c64"]
