"""Adjoint (lsp_adjoint, torch.autograd) against the FP64 oracle gradient and finite differences (GB300)."""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu


def _case(which):
    if which == "small":
        inst = w.c1()
        return inst, dict(aa="explicit", index_set=inst.index_set), L.explicit_norms(inst.index_set, inst.Z, inst.n)
    inst = w.c4(14)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    return inst, {}, norms


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("which", ["small", "multipass"])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_adjoint_matches_oracle(lib, which, prec):
    import torch
    inst, kw, norms = _case(which)
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    phi = w.gaussian_packet(P, 0.1, [0.6] + [0.5] * (inst.d - 1))
    nsteps, dt = 20, inst.dt
    J, gv_ref, gu_ref, uN_ref = S.strang_adjoint(u0, v, norms, inst.n, inst.gamma, dt, nsteps, phi, ckpt=6)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec, **kw)
    cdt = torch.complex64 if prec == "c64" else torch.complex128
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    # lambda_N = 2 <phi, u_N> phi / n  (J = |<u_N, phi>|^2), from the oracle's u_N
    c = S.inner(phi, uN_ref)
    lamT = torch.from_numpy(2.0 * c * phi / phi.size).to(cdt).cuda()
    gv = torch.empty(inst.npoints, dtype=torch.float64, device="cuda")
    gu = torch.empty(inst.npoints, dtype=cdt, device="cuda")
    lib.adjoint(plan, dt, nsteps, lamT, gv, gu, 6)
    assert plan.status() == 0
    tol = 1e-9 if prec == "c128" else 2e-4
    assert _rel(gv.cpu().numpy(), gv_ref) < tol
    assert _rel(gu.cpu().numpy(), gu_ref) < tol
    # the plan's state is left at u_N
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), uN_ref) < (1e-10 if prec == "c128" else 5e-5)


def test_adjoint_checkpoint_stride_invariance(lib):
    import torch
    inst, kw, norms = _case("multipass")
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128", **kw)
    rng = np.random.default_rng(0)
    lam = torch.from_numpy(rng.standard_normal(inst.npoints) + 1j * rng.standard_normal(inst.npoints)).cuda()
    outs = []
    for ck in (1, 5, 0):
        plan.set_potential(torch.from_numpy(v).cuda())
        plan.set_state(torch.from_numpy(u0).cuda())
        gv = torch.empty(inst.npoints, dtype=torch.float64, device="cuda")
        gu = torch.empty(inst.npoints, dtype=torch.complex128, device="cuda")
        lib.adjoint(plan, inst.dt, 17, lam, gv, gu, ck)
        outs.append((gv.cpu().numpy(), gu.cpu().numpy()))
    for gv, gu in outs[1:]:
        assert np.allclose(gv, outs[0][0], rtol=0, atol=1e-12 * np.abs(outs[0][0]).max())
        assert np.allclose(gu, outs[0][1], rtol=0, atol=1e-12 * np.abs(outs[0][1]).max())


def test_autograd_function_matches_oracle(lib):
    import torch
    from paper_1808_06357_gb300.autograd import strang_evolve
    inst, kw, norms = _case("multipass")
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    phi = w.gaussian_packet(P, 0.1, [0.6] + [0.5] * (inst.d - 1))
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128", **kw)
    vt = torch.from_numpy(v).cuda().requires_grad_(True)
    ut = torch.from_numpy(u0).cuda().requires_grad_(True)
    pt = torch.from_numpy(phi).cuda()
    uN = strang_evolve(plan, vt, ut, inst.dt, 12)
    J = torch.abs(torch.mean(torch.conj(uN) * pt)) ** 2
    J.backward()
    Jr, gv_ref, gu_ref, _ = S.strang_adjoint(u0, v, norms, inst.n, inst.gamma, inst.dt, 12, phi)
    assert abs(J.item() - Jr) < 1e-12 * abs(Jr)
    assert _rel(vt.grad.cpu().numpy(), gv_ref) < 1e-9
    assert _rel(ut.grad.cpu().numpy(), gu_ref) < 1e-9


def test_adjoint_full_size_directional_derivative(lib):
    """n = 2^20, d = 4, 500 steps: <dJ/dv, dv> from the complex64 adjoint against a central
    difference of J computed with complex128 forward runs."""
    import torch
    inst = w.c4(20)
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    phi = inst.phi(P)
    pt = torch.from_numpy(phi).cuda()
    N = inst.nsteps
    f64 = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128")

    def J_of(vv):
        f64.set_potential(torch.from_numpy(vv).cuda())
        f64.set_state(torch.from_numpy(u0).cuda())
        f64.strang_steps(inst.dt, N)
        uN = f64.get_state()
        c = torch.mean(torch.conj(pt) * uN)
        return float(torch.abs(c) ** 2), uN

    J0, uN = J_of(v)
    f32 = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64")
    f32.set_potential(torch.from_numpy(v).cuda())
    f32.set_state(torch.from_numpy(u0).cuda())
    c = torch.mean(torch.conj(pt) * uN)
    lamT = (2.0 * c * pt / inst.npoints).to(torch.complex64)
    gv = torch.empty(inst.npoints, dtype=torch.float64, device="cuda")
    gu = torch.empty(inst.npoints, dtype=torch.complex64, device="cuda")
    lib.adjoint(f32, inst.dt, N, lamT, gv, gu, 0)
    assert f32.status() == 0
    rng = np.random.default_rng(1)
    dv = rng.standard_normal(inst.npoints)
    eps = 1e-3
    fd = (J_of(v + eps * dv)[0] - J_of(v - eps * dv)[0]) / (2 * eps)
    an = float(gv.cpu().numpy() @ dv)
    assert abs(fd - an) < 2e-3 * abs(fd), (fd, an)
