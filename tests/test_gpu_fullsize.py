"""Full-length runs of the configurations against the FP64 oracle (GB300).

Spec tolerances after the configuration's whole run: relative L2 error
<= 5e-5 (complex64) and <= 1e-10 (complex128), norm drift reported.  The oracle's
runs take minutes (tests/_oracle_refs.py) and start in the background when these
tests are collected.
"""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 5e-5}


def _rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.oracle_job("c2_1000")
def test_c2_1000_steps_every_path_against_oracle(lib):
    """C2 (d = 6, n = 2^22, gamma = 0.05, dt = 1e-3): 1000 steps on every execution path of
    both precisions, element by element against the oracle's 1000 FP64 steps (eq. StrangTDSE,
    Algorithm 1)."""
    import torch
    import _oracle_refs as R
    inst = w.c2(22)
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = torch.from_numpy(inst.v(P)).cuda(), torch.from_numpy(inst.u0(P)).cuda()
    del P
    results = []
    for prec in ("c64", "c128"):
        plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
        for path in plan.paths():
            plan.set_path(path)
            plan.set_potential(v)
            plan.set_state(u0)
            n0, _ = plan.observables()
            plan.strang_steps(inst.dt, 1000)
            assert plan.status() == 0
            n1, _ = plan.observables()
            results.append((prec, path, plan.get_state(prec="c128").cpu().numpy(), abs(n1 / n0 - 1)))
        plan.destroy()
    ref, n_start, n_end = R.get("c2_1000")
    assert abs(n_end / n_start - 1) < 1e-12
    for prec, path, got, drift in results:
        err = _rel(got, ref)
        print(f"C2 1000 steps {prec} path {path}: rel-L2 vs oracle {err:.3e}, norm drift {drift:.3e}")
        assert err < TOL[prec], (prec, path, err)
        assert drift < TOL[prec], (prec, path, drift)


@pytest.mark.oracle_job("c3_500")
def test_c3_batch_500_steps_sample_against_oracle(lib):
    """C3 (256 instances, n = 2^12..2^20, d = 3..8, per-instance dt, complex64): the whole batch
    advanced 500 steps in batched calls; one instance of every lattice size against the oracle."""
    import torch
    import _oracle_refs as R
    insts = w.c3()
    plans = []
    for inst in insts:
        P = L.lattice_points(inst.Z, inst.n)
        p = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64")
        p.set_potential(torch.from_numpy(inst.v(P)).cuda())
        p.set_state(torch.from_numpy(inst.u0(P)).cuda())
        plans.append(p)
    batch = lib.Batch(plans)
    dts = [inst.dt for inst in insts]
    batch.steps(dts, 250)
    batch.steps(dts, 250)
    assert batch.status() == 0
    ids, finals = R.get("c3_500")
    assert len(ids) == 9
    for i in ids:
        err = _rel(plans[i].get_state(prec="c128").cpu().numpy(), finals[i])
        print(f"C3 {insts[i].name} path {plans[i].info()['path']} 500 steps: rel-L2 vs oracle {err:.3e}")
        assert err < TOL["c64"], (insts[i].name, err)
    batch.destroy()


@pytest.mark.oracle_job("c4_500")
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_c4_adjoint_500_steps_against_oracle_gradient(lib, prec):
    """C4 (d = 4, n = 2^20, 500 steps, ceil(sqrt(500)) checkpoints): dJ/dv and dJ/du0 of
    J = |<u_N, phi>|^2 from lsp_adjoint against the oracle's reverse-mode gradient, and the
    forward state u_N the call leaves behind against the oracle's."""
    import torch
    import _oracle_refs as R
    inst = w.c4(20)
    P = L.lattice_points(inst.Z, inst.n)
    v, u0, phi = inst.v(P), inst.u0(P), inst.phi(P)
    del P
    J, gv_ref, gu_ref, uN_ref = R.get("c4_500")
    cdt = torch.complex64 if prec == "c64" else torch.complex128
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    lamT = torch.from_numpy(2.0 * S.inner(phi, uN_ref) * phi / phi.size).to(cdt).cuda()
    gv = torch.empty(inst.npoints, dtype=torch.float64, device="cuda")
    gu = torch.empty(inst.npoints, dtype=cdt, device="cuda")
    lib.adjoint(plan, inst.dt, inst.nsteps, lamT, gv, gu, 0)
    assert plan.status() == 0
    e_v = _rel(gv.cpu().numpy(), gv_ref)
    e_u = _rel(gu.cpu().numpy(), gu_ref)
    e_f = _rel(plan.get_state(prec="c128").cpu().numpy(), uN_ref)
    print(f"C4 adjoint {prec} path {plan.info()['path']}: rel-L2 dJ/dv {e_v:.3e}, dJ/du0 {e_u:.3e}, u_N {e_f:.3e}")
    tol_g = 1e-9 if prec == "c128" else 5e-4
    assert e_v < tol_g and e_u < tol_g
    assert e_f < TOL[prec]
    plan.destroy()
