"""The mixed-radix two-sweep path (execution path 5) against the FP64 oracle (GB300).

Rank-1 lattices whose n is not a power of two and exceeds the SMEM-resident size: n = N1 N2
(N2 <= N1 <= 4096), rows of N1 points and columns of N2 points, line transforms with any radix
(3, 5, 7, 11 ... as well as 2..16).  The column tiles hold C = 4096 / N2 columns and the row tiles
4096 / N1 rows, so most sizes have a ragged last tile.  Checked: 50 Strang steps element by
element in complex64 and complex128 with the spectral output, a power-of-two size on request,
the adjoint, a batch, and the sizes the path cannot take.
"""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 5e-5}
GAMMA, DT = 0.1, 2e-3
# n: 3 5^5 7 (N1 375, N2 175), 2^10 3^3, 3 5 7 2^10, 3^6 5^3 11 (about 10^6 points)
SIZES = [(65625, 3), (27648, 4), (107520, 3), (1002375, 3)]


def _rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _lattice(n, d, seed=7):
    rng = np.random.default_rng(seed + n)
    while True:                                      # components prime to n: n distinct points
        z = np.concatenate([[1], rng.integers(1, n, d - 1)])
        if all(np.gcd(int(c), n) == 1 for c in z):
            return z


def _inputs(z, n):
    P = L.lattice_points(z, (n,))
    d = P.shape[1]
    return P, w.v_cos_sum_prod(P), w.gaussian_packet(P, 0.15, [0.5] * d, k0=1)


def _plan(lib, z, n, prec, v, u0):
    import torch
    plan = lib.Plan(z, (n,), GAMMA, prec=prec)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    return plan


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n,d", SIZES)
def test_mixed_radix_50_steps_matches_oracle(lib, n, d, prec):
    z = _lattice(n, d)
    P, v, u0 = _inputs(z, n)
    plan = _plan(lib, z, n, prec, v, u0)
    info = plan.info()
    assert info["path"] == lib.PATH_MIXED
    assert info["N1"] * info["N2"] == n and info["N2"] <= info["N1"] <= 4096
    plan.strang_steps(DT, 50)
    assert plan.status() == 0
    norms, _ = L.minl2_norms_dp(z, (n,))
    ref = S.strang(u0, v, norms, (n,), GAMMA, DT, 50)
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL[prec]
    spec = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    assert _rel(spec, S.coeffs(ref, (n,))) < TOL[prec]
    plan.destroy()


def test_mixed_radix_on_request_where_the_smem_path_applies(lib):
    """n = 2^12 3 fits the SMEM-resident path (the default there); the mixed-radix path runs it
    on request; power-of-two sizes, which have the butterfly paths, are not offered to it."""
    n = 12288
    z = _lattice(n, 3)
    P, v, u0 = _inputs(z, n)
    plan = _plan(lib, z, n, "c64", v, u0)
    assert plan.info()["path"] == lib.PATH_SMALL and lib.PATH_MIXED in plan.paths()
    assert lib.PATH_MIXED not in lib.Plan(_lattice(1 << 16, 3), (1 << 16,), GAMMA, prec="c64").paths()
    plan.set_path(lib.PATH_MIXED)
    plan.strang_steps(DT, 20)
    assert plan.status() == 0
    norms, _ = L.minl2_norms_dp(z, (n,))
    ref = S.strang(u0, v, norms, (n,), GAMMA, DT, 20)
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL["c64"]
    plan.destroy()


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_mixed_radix_adjoint_matches_oracle(lib, prec):
    import torch
    n, d = 27648, 4
    z = _lattice(n, d)
    P, v, u0 = _inputs(z, n)
    norms, _ = L.minl2_norms_dp(z, (n,))
    phi = w.gaussian_packet(P, 0.12, [0.6] + [0.5] * (d - 1))
    nsteps = 16
    J, gv_ref, gu_ref, uN_ref = S.strang_adjoint(u0, v, norms, (n,), GAMMA, DT, nsteps, phi, ckpt=4)
    plan = _plan(lib, z, n, prec, v, u0)
    assert plan.info()["path"] == lib.PATH_MIXED
    cdt = torch.complex64 if prec == "c64" else torch.complex128
    c = S.inner(phi, uN_ref)
    lamT = torch.from_numpy(2.0 * c * phi / phi.size).to(cdt).cuda()
    gv = torch.empty(n, dtype=torch.float64, device="cuda")
    gu = torch.empty(n, dtype=cdt, device="cuda")
    lib.adjoint(plan, DT, nsteps, lamT, gv, gu, 4)
    assert plan.status() == 0
    tol = 1e-9 if prec == "c128" else 2e-4
    assert _rel(gv.cpu().numpy(), gv_ref) < tol
    assert _rel(gu.cpu().numpy(), gu_ref) < tol
    plan.destroy()


def test_mixed_radix_in_a_batch(lib):
    """Mixed-radix instances stepped with others in one batch, each against the oracle."""
    cases = [(65625, 3, 2e-3), (27648, 4, 1e-3), (961, 2, 3e-3)]
    plans, refs = [], []
    for n, d, dt in cases:
        z = _lattice(n, d)
        P, v, u0 = _inputs(z, n)
        plans.append(_plan(lib, z, n, "c64", v, u0))
        norms, _ = L.minl2_norms_dp(z, (n,))
        refs.append(S.strang(u0, v, norms, (n,), GAMMA, dt, 25))
    batch = lib.Batch(plans)
    batch.steps([c[2] for c in cases], 25)
    assert batch.status() == 0
    for p, ref in zip(plans, refs):
        assert _rel(p.get_state(prec="c128").cpu().numpy(), ref) < TOL["c64"]


def test_sizes_no_path_takes_are_rejected(lib):
    """n = 4 * 8191 (a prime factor above 4096, beyond the SMEM-resident size): TOO_LARGE."""
    n = 4 * 8191
    with pytest.raises(lib.LspError) as e:
        lib.Plan(_lattice(n, 3), (n,), GAMMA, prec="c64")
    assert e.value.code == -4
