"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300)."""

import math

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 5e-5}        # relative L2 after the run (spec bounds)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_plan(lib, inst, prec, aa="minl2"):
    kw = {}
    if aa == "explicit":
        kw["index_set"] = inst.index_set
    return lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec, aa=aa, **kw)


def host_state(plan):
    import torch
    return plan.get_state(prec="c128").cpu().numpy()


def run_both(lib, inst, prec, nsteps, aa="minl2", dt=None, path=None):
    import torch
    dt = inst.dt if dt is None else dt
    P = L.lattice_points(inst.Z, inst.n)
    if aa == "explicit":
        norms = L.explicit_norms(inst.index_set, inst.Z, inst.n)
    else:
        norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plan = make_plan(lib, inst, prec, aa)
    if path is not None:
        plan.set_path(path)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.strang_steps(dt, nsteps)
    assert plan.status() == 0
    got = host_state(plan)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, dt, nsteps)
    return got, ref, u0, plan


# ---------------------------------------------------------------------------
# plan-time quantities
# ---------------------------------------------------------------------------
PLAN_CASES = [
    (w.c1(), "small"),
    (w.c2(13), "small"),
    (w.c2(16), "multipass"),
    (w.Instance("rank2", 3, (12, 6), np.array([[1, 0], [3, 1], [5, 5]]), 0.1, 1e-3, 10,
                w.v_smooth, lambda p: w.gaussian_packet(p, 0.2, [0.5] * 3)), "small"),
]


@pytest.mark.parametrize("inst,path", PLAN_CASES, ids=[c[0].name for c in PLAN_CASES])
def test_lattice_points_and_minl2_norms_bit_exact(lib, inst, path):
    plan = make_plan(lib, inst, "c64")
    info = plan.info()
    assert info["path"] == (lib.PATH_SMALL if path == "small" else lib.PATH_MULTIPASS)
    assert np.array_equal(plan.lattice_points(), L.lattice_points(inst.Z, inst.n))
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    assert np.array_equal(plan.index_norms(), norms)
    H = plan.index_table()
    assert np.array_equal(L.chi_index(H, inst.Z, inst.n), np.arange(inst.npoints))
    assert np.array_equal((H.astype(np.int64) ** 2).sum(1), norms)


def test_minl2_norms_c2_full_size(lib):
    inst = w.c2(22)
    plan = make_plan(lib, inst, "c64")
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    assert np.array_equal(plan.index_norms(), norms)


def test_explicit_index_set(lib):
    inst = w.c1()
    plan = make_plan(lib, inst, "c128", aa="explicit")
    assert np.array_equal(plan.index_norms(), L.explicit_norms(inst.index_set, inst.Z, inst.n))


# ---------------------------------------------------------------------------
# spectral coefficients (eq. approx_uhat)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("m", [13, 14, 15, 16, 17, 18, 19, 20])
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_spectral_coefficients(lib, m, prec):
    import torch
    inst = w.c2(m)
    P = L.lattice_points(inst.Z, inst.n)
    rng = np.random.default_rng(m)
    u = rng.standard_normal(inst.npoints) + 1j * rng.standard_normal(inst.npoints)
    plan = make_plan(lib, inst, prec)
    plan.set_state(torch.from_numpy(u).cuda())
    got = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    ref = S.coeffs(u, inst.n)
    assert rel_l2(got, ref) < (1e-13 if prec == "c128" else 2e-6)
    # the state itself is untouched
    assert rel_l2(host_state(plan), u) < (1e-15 if prec == "c128" else 1e-7)


def test_spectral_small_path_rank2(lib):
    import torch
    inst = PLAN_CASES[3][0]
    rng = np.random.default_rng(3)
    u = rng.standard_normal(inst.npoints) + 1j * rng.standard_normal(inst.npoints)
    plan = make_plan(lib, inst, "c128")
    plan.set_state(torch.from_numpy(u).cuda())
    got = plan.get_state(space="spectral").cpu().numpy()
    assert rel_l2(got, S.coeffs(u, inst.n)) < 1e-13


# ---------------------------------------------------------------------------
# Strang steps against the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_c1_full_run(lib, prec):
    """C1: d=2, n=961 = 31^2 (SMEM-resident path, radix-31 passes), 1000 steps."""
    inst = w.c1()
    got, ref, u0, _ = run_both(lib, inst, prec, inst.nsteps, aa="explicit")
    assert rel_l2(got, ref) < TOL[prec]


# radix plans: m=13 (64 x 128), 14 (128x128), 15 (128x256), 16, 17 (256x512), 18, 19, 20 (1024^2)
@pytest.mark.parametrize("m", [13, 14, 15, 16, 17, 18, 19, 20])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_multipass_parity(lib, m, prec):
    inst = w.c2(m)
    nsteps = 50
    got, ref, u0, plan = run_both(lib, inst, prec, nsteps, path=lib.PATH_MULTIPASS)
    assert plan.info()["path"] == lib.PATH_MULTIPASS
    assert rel_l2(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_multipass_1000_steps(lib, prec):
    inst = w.c2(16)
    got, ref, u0, _ = run_both(lib, inst, prec, 1000)
    err = rel_l2(got, ref)
    drift = abs(np.linalg.norm(got) / np.linalg.norm(u0) - 1)
    print(f"n=2^16 {prec}: rel-L2 {err:.3e}, norm drift {drift:.3e}")
    assert err < TOL[prec]


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_c2_full_size_short_run(lib, prec):
    """C2 at n = 2^22, 20 steps against the oracle, on both rank-1 paths: the two-sweep kernel
    (4096 x 1024 four-step split) and the four-sweep kernels (4096 x 32 x 32)."""
    import torch
    inst = w.c2(22)
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 20)
    for path in (lib.PATH_MULTIPASS, lib.PATH_RANK1_4SWEEP):
        plan = make_plan(lib, inst, prec)
        plan.set_path(path)
        plan.set_potential(torch.from_numpy(v).cuda())
        plan.set_state(torch.from_numpy(u0).cuda())
        plan.strang_steps(inst.dt, 20)
        assert plan.status() == 0
        assert rel_l2(host_state(plan), ref) < TOL[prec]


def test_free_evolution_closed_form(lib):
    """v = 0: bin-wise exact phase exp(-i gamma 2 pi^2 |h|^2 t) (eq. Fourier-ODE), n = 2^20."""
    import torch
    inst = w.c2(20)
    plan = make_plan(lib, inst, "c64")
    P = L.lattice_points(inst.Z, inst.n)
    u0 = inst.u0(P)
    plan.set_potential(torch.zeros(inst.npoints, dtype=torch.float64, device="cuda"))
    plan.set_state(torch.from_numpy(u0).cuda())
    N, dt = 300, 1e-3
    plan.strang_steps(dt, N)
    got = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    norms = plan.index_norms()
    c0 = S.coeffs(u0, inst.n)
    exact = c0 * np.exp(-1j * inst.gamma * 2 * np.pi ** 2 * norms * N * dt)
    assert rel_l2(got, exact) < 2e-5


def test_constant_potential_phase(lib):
    import torch
    inst = w.c2(16)
    P = L.lattice_points(inst.Z, inst.n)
    u0 = inst.u0(P)
    plan = make_plan(lib, inst, "c128")
    plan.set_potential(torch.full((inst.npoints,), 1.7, dtype=torch.float64, device="cuda"))
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.strang_steps(1e-3, 100)
    got = host_state(plan)
    norms = plan.index_norms()
    ref = S.samples(S.coeffs(u0, inst.n) * np.exp(-1j * inst.gamma * 2 * np.pi ** 2 * norms * 0.1), inst.n)
    ref *= np.exp(-1j * 1.7 * 0.1 / inst.gamma)
    assert rel_l2(got, ref) < 1e-11


def test_time_reversal(lib):
    import torch
    inst = w.c2(18)
    P = L.lattice_points(inst.Z, inst.n)
    u0 = inst.u0(P)
    plan = make_plan(lib, inst, "c128")
    plan.set_potential(torch.from_numpy(inst.v(P)).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.strang_steps(2e-3, 50)
    plan.strang_steps(-2e-3, 50)
    assert rel_l2(host_state(plan), u0) < 1e-12


def test_zero_steps_is_noop_and_precision_conversions(lib):
    import torch
    inst = w.c2(14)
    P = L.lattice_points(inst.Z, inst.n)
    u0 = inst.u0(P)
    plan = make_plan(lib, inst, "c64")
    plan.set_state(torch.from_numpy(u0).cuda())              # complex128 into a c64 plan
    plan.strang_steps(1e-3, 0)
    a = plan.get_state(prec="c64").cpu().numpy()
    b = plan.get_state(prec="c128").cpu().numpy()
    assert np.array_equal(a.astype(np.complex128), b)
    assert rel_l2(b, u0) < 1e-7
    host = np.empty(inst.npoints, dtype=np.complex128)
    plan.get_state(out=host)
    assert np.array_equal(host, b)


def test_error_codes(lib):
    with pytest.raises(lib.LspError) as e:
        lib.Plan(np.array([[1, 1], [1, 1]]), (6, 4), 0.1)        # 4 does not divide 6
    assert e.value.code == -2
    inst = w.c1()
    bad = inst.index_set.copy()
    bad[1] = bad[0]
    with pytest.raises(lib.LspError) as e:
        lib.Plan(inst.Zmat, inst.n, 0.1, prec="c128", aa="explicit", index_set=bad)
    assert e.value.code == -3
    plan = make_plan(lib, w.c2(13), "c64")
    with pytest.raises(lib.LspError) as e:
        plan.strang_steps(1e-3, -1)
    assert e.value.code == -1
    with pytest.raises(lib.LspError) as e:
        lib.Plan(np.array([1, 3]), (1 << 26,), 0.1, prec="c128")   # beyond every rank-1 path
    assert e.value.code == -4
