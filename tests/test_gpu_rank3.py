"""Rank-3 and rank-4 lattices against the FP64 oracle (GB300).

A rank-r lattice (Sec. 2.5) has N = n_1 ... n_r points p_kappa = frac(sum_i z_i kappa_i / n_i),
kappa lexicographic, and bins xi = (h.z_1 mod n_1, ..., h.z_r mod n_r) in lexicographic (chi)
order; the Strang step's transform is the r-D DFT over Z_{n_1} x ... x Z_{n_r}.  These run on the
SMEM-resident path (one CTA per instance, every step in one launch).  Checked: lattice points,
minimal-l2 norms and the index table; 50 Strang steps element by element in complex64 and
complex128 with the spectral output; observables; the adjoint; a batch mixing ranks 1, 3 and 4.
The lattices are seeded, with distinct points (Def. 1); one has moduli 12, 6, 3 (radix 3).
"""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 5e-5}

LATTICES = {
    "r3_d4_16x8x4": (np.array([[1, 0, 0], [9, 2, 11], [12, 15, 12], [4, 5, 10]]), (16, 8, 4)),
    "r3_d5_32x16x8": (np.array([[1, 0, 0], [31, 3, 3], [11, 4, 0], [14, 5, 7], [8, 11, 4]]), (32, 16, 8)),
    "r3_grid_16x16x8": (np.eye(3, dtype=np.int64), (16, 16, 8)),
    "r3_d4_12x6x3": (np.array([[1, 0, 0], [2, 1, 0], [10, 4, 2], [1, 3, 2]]), (12, 6, 3)),
    "r4_d5_8x4x4x2": (np.array([[1, 0, 0, 0], [3, 0, 3, 0], [6, 0, 3, 1], [1, 1, 2, 0], [6, 3, 3, 0]]),
                      (8, 4, 4, 2)),
}
GAMMA, DT = 0.1, 2e-3


def _rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _inputs(Z, n):
    P = L.lattice_points(Z, n)
    d = P.shape[1]
    v = w.v_cos_sum_prod(P)
    u0 = w.gaussian_packet(P, 0.15, [0.5] * d, k0=1)
    return P, v, u0


def _plan(lib, Z, n, prec, v, u0):
    import torch
    plan = lib.Plan(Z, n, GAMMA, prec=prec)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    return plan


@pytest.mark.parametrize("name", list(LATTICES))
def test_points_norms_and_index_table(lib, name):
    Z, n = LATTICES[name]
    plan = lib.Plan(Z, n, GAMMA, prec="c64")
    info = plan.info()
    assert info["path"] == lib.PATH_SMALL
    assert info["n"] == int(np.prod(n))
    assert np.array_equal(plan.lattice_points(), L.lattice_points(Z, n))
    norms, _ = L.minl2_norms_dp(Z, n)
    assert np.array_equal(plan.index_norms(), norms)
    H = plan.index_table()
    assert np.array_equal(L.chi_index(H, Z, n), np.arange(int(np.prod(n))))   # h_chi lies in bin chi
    assert np.array_equal((H.astype(np.int64) ** 2).sum(axis=1), norms)      # with the minimal norm
    plan.destroy()


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("name", list(LATTICES))
def test_strang_50_steps_matches_oracle(lib, name, prec):
    Z, n = LATTICES[name]
    P, v, u0 = _inputs(Z, n)
    plan = _plan(lib, Z, n, prec, v, u0)
    plan.strang_steps(DT, 50)
    assert plan.status() == 0
    norms, _ = L.minl2_norms_dp(Z, n)
    ref = S.strang(u0, v, norms, n, GAMMA, DT, 50)
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL[prec]
    spec = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    assert _rel(spec, S.coeffs(ref, n)) < TOL[prec]
    nn, e = plan.observables()
    # complex64: 50 steps of FP32 rounding move the norm by a few 1e-6 (the state is held to 5e-5
    # above, which bounds the norm's relative error by 1e-4)
    tol_n, tol_e = (1e-12, 1e-10) if prec == "c128" else (1e-5, 1e-4)
    assert abs(nn - S.norm2(ref)) < tol_n * S.norm2(ref)
    e_ref = S.energy(ref, v, norms, n, GAMMA)
    assert abs(e - e_ref) < tol_e * abs(e_ref)
    plan.destroy()


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_rank3_adjoint_matches_oracle(lib, prec):
    import torch
    Z, n = LATTICES["r3_d4_16x8x4"]
    P, v, u0 = _inputs(Z, n)
    norms, _ = L.minl2_norms_dp(Z, n)
    phi = w.gaussian_packet(P, 0.12, [0.6, 0.5, 0.5, 0.5])
    nsteps = 20
    J, gv_ref, gu_ref, uN_ref = S.strang_adjoint(u0, v, norms, n, GAMMA, DT, nsteps, phi, ckpt=5)
    plan = _plan(lib, Z, n, prec, v, u0)
    cdt = torch.complex64 if prec == "c64" else torch.complex128
    c = S.inner(phi, uN_ref)
    lamT = torch.from_numpy(2.0 * c * phi / phi.size).to(cdt).cuda()
    gv = torch.empty(P.shape[0], dtype=torch.float64, device="cuda")
    gu = torch.empty(P.shape[0], dtype=cdt, device="cuda")
    lib.adjoint(plan, DT, nsteps, lamT, gv, gu, 5)
    assert plan.status() == 0
    tol = 1e-9 if prec == "c128" else 2e-4
    assert _rel(gv.cpu().numpy(), gv_ref) < tol
    assert _rel(gu.cpu().numpy(), gu_ref) < tol
    plan.destroy()


def test_batch_mixing_ranks(lib):
    """Instances of rank 1, 3 and 4 (uneven sizes, their own step sizes) in one batch, each against
    the oracle after 30 steps."""
    cases = [
        (np.array([1, 34]), (55,), 1e-3),
        LATTICES["r3_d5_32x16x8"] + (2e-3,),
        LATTICES["r4_d5_8x4x4x2"] + (3e-3,),
        LATTICES["r3_d4_12x6x3"] + (1.5e-3,),
    ]
    plans, refs = [], []
    for Z, n, dt in cases:
        P, v, u0 = _inputs(Z, n)
        plans.append(_plan(lib, Z, n, "c64", v, u0))
        norms, _ = L.minl2_norms_dp(Z, n)
        refs.append(S.strang(u0, v, norms, n, GAMMA, dt, 30))
    batch = lib.Batch(plans)
    batch.steps([c[2] for c in cases], 30)
    assert batch.status() == 0
    for p, ref in zip(plans, refs):
        assert _rel(p.get_state(prec="c128").cpu().numpy(), ref) < TOL["c64"]
