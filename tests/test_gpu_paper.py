"""The paper's own workloads on the GPU (Table 1 lattices; g1, g2, v1, v2 of Sec. 3.2),
the observables of Sec. 3.3, and the convergence and conservation experiments, against the
FP64 oracle (GB300)."""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_setup(inst):
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    return P, norms, inst.v(P), inst.u0(P)


OBS_CASES = [
    ("smem rank-1", lambda: w.c1(), "explicit", None),
    ("two-sweep", lambda: w.c2(16), "minl2", None),
    ("four-sweep rank-1", lambda: w.c2(20), "minl2", 3),
    ("rank-2", lambda: w.c5(10, 8, 16, 6), "minl2", None),
]


@pytest.mark.parametrize("name,make,aa,path", OBS_CASES, ids=[c[0] for c in OBS_CASES])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_observables_match_oracle(lib, name, make, aa, path, prec):
    import torch
    inst = make()
    P = L.lattice_points(inst.Z, inst.n)
    norms = L.explicit_norms(inst.index_set, inst.Z, inst.n) if aa == "explicit" else L.minl2_norms_dp(inst.Z, inst.n)[0]
    v, u0 = inst.v(P), inst.u0(P)
    kw = {"index_set": inst.index_set} if aa == "explicit" else {}
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec, aa=aa, **kw)
    if path is not None:
        plan.set_path(path)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    tol_n, tol_e = (1e-12, 1e-10) if prec == "c128" else (2e-6, 1e-4)
    for k in range(2):
        u = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 10 * k)
        nn, e = plan.observables()
        e_ref = S.energy(u, v, norms, inst.n, inst.gamma)
        assert abs(nn - S.norm2(u)) < tol_n * S.norm2(u)
        assert abs(e - e_ref) < tol_e * abs(e_ref)
        plan.strang_steps(inst.dt, 10)


@pytest.mark.parametrize("d,m,init,pot,gamma,nsteps", [(2, 18, "g1", "v1", 0.1, 50), (2, 20, "g2", "v2", 0.5, 20),
                                                      (3, 22, "g1", "v2", 0.01, 10)])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_table1_lattices_parity(lib, d, m, init, pot, gamma, nsteps, prec):
    import torch
    inst = w.paper_instance(d, m, init=init, pot=pot, gamma=gamma, dt=1e-2)
    P, norms, v, u0 = _oracle_setup(inst)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.strang_steps(inst.dt, nsteps)
    assert plan.status() == 0
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, nsteps)
    assert rel_l2(plan.get_state(prec="c128").cpu().numpy(), ref) < (1e-10 if prec == "c128" else 5e-5)


def test_convergence_protocol_matches_oracle(lib):
    """Sec. 3.2 protocol at reduced size (T = 0.2, M = 1000), smooth potential v1: the GPU's errors
    equal the oracle's and fall with the second power of the step.  (With the harmonic v2, whose
    periodic extension has a kink at x_j = 0, the oracle shows orders 1.6-1.7 and then a plateau
    in this range.)"""
    from paper_1808_06357_gb300 import experiments as X
    ms = (10, 20, 40, 80)
    inst = w.paper_instance(2, 18, init="g1", pot="v1", gamma=0.5)
    r = X.convergence(inst, ms=ms, M=1000, T=0.2, prec="c128")
    P, norms, v, u0 = _oracle_setup(inst)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, 0.2 / 1000, 1000)
    for m in ms:
        um = S.strang(u0, v, norms, inst.n, inst.gamma, 0.2 / m, m)
        e = float(np.sqrt(np.mean(np.abs(um - ref) ** 2)))
        assert abs(r["errors"][m] - e) < 1e-6 * e
    for k, q in r["orders"].items():
        assert 1.9 < q < 2.1, (k, q)


def test_conservation_matches_oracle(lib):
    """Sec. 3.3 observables along a run (d = 2, n = 2^18, g1, v2, gamma = 0.5): the GPU's norm and
    energy at every sample equal the oracle's; the norm varies at round-off only."""
    from paper_1808_06357_gb300 import experiments as X
    inst = w.paper_instance(2, 18, init="g1", pot="v2", gamma=0.5)
    r = X.conservation(inst, dt=1e-2, T=0.5, every=5, prec="c128")
    P, norms, v, u0 = _oracle_setup(inst)
    Ph = S.potential_half_phase(v, inst.gamma, 1e-2)
    K = S.kinetic_phase(norms, inst.gamma, 1e-2)
    u = u0.copy()
    for k in range(r["samples"]):
        assert abs(r["norm"][k] - S.norm2(u)) < 1e-12
        e = S.energy(u, v, norms, inst.n, inst.gamma)
        assert abs(r["energy"][k] - e) < 1e-10 * abs(e)
        for _ in range(5):
            u = S.strang_step(u, Ph, K, inst.n)
    assert r["delta_norm"] < 1e-12
    assert 0 < r["delta_energy"] < 0.05


def test_table1_high_dimension_full_size(lib):
    """d = 12, n = 2^25 (Table 1), g1, v2, gamma = 0.5: 20 steps in complex64 and complex128 agree,
    and both keep the norm."""
    import torch
    inst = w.paper_instance(12, 25, init="g1", pot="v2", gamma=0.5, dt=1e-2)
    p64 = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64")
    assert p64.info()["path"] == lib.PATH_RANK1_4SWEEP
    pts = p64.lattice_points()
    v = torch.from_numpy(inst.v(pts)).cuda()
    u0 = torch.from_numpy(inst.u0(pts)).cuda()
    del pts
    outs = {}
    for prec in ("c64", "c128"):
        plan = p64 if prec == "c64" else lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128")
        plan.set_potential(v)
        plan.set_state(u0)
        n0, _ = plan.observables()
        plan.strang_steps(inst.dt, 20)
        n1, _ = plan.observables()
        assert abs(n1 / n0 - 1) < (1e-12 if prec == "c128" else 1e-5)
        outs[prec] = plan.get_state(prec="c128")
        del plan
    r = float(torch.linalg.norm(outs["c64"] - outs["c128"]) / torch.linalg.norm(outs["c128"]))
    assert r < 5e-5


def test_initial_error_matches_oracle_coefficients(lib):
    """Sec. 3.4 e_total of g1 (gamma = 1) on the d = 2 Table 1 lattices: the library's lattice-rule
    coefficients equal the oracle's, so both give the same e_total against the exact coefficients,
    and e_total falls from n = 2^18 to 2^20."""
    from oracle import initial_error as G
    from paper_1808_06357_gb300 import experiments as X
    es = {}
    for lg in (18, 20):
        z = w.table1_z(2, lg)
        ga, H = X.lattice_rule_coefficients(z, lg, lambda p: G.g1_samples(p, 1.0), gamma=1.0)
        n = (1 << lg,)
        assert np.array_equal(L.chi_index(H, z, n), np.arange(n[0]))
        g = G.g1_coefficients(H, 1.0)
        es[lg] = G.e_total(g, ga)
        if lg == 18:
            P = L.lattice_points(z, n)
            ref = S.coeffs(G.g1_samples(P, 1.0), n)
            assert np.max(np.abs(ga - ref)) < 1e-12
            assert abs(es[lg] - G.e_total(g, ref)) < 1e-9 * es[lg]
    assert es[20] < es[18]


@pytest.mark.parametrize("which", ["smem", "two-sweep", "four-sweep", "rank-2"])
def test_composed_steps_match_oracle(lib, which):
    """lsp_strang_composed (fourth-order triple of Strang steps) on every path against the oracle's
    composition, complex128."""
    import torch
    inst, kw, path = {"smem": (w.c1(), {"aa": "explicit"}, None), "two-sweep": (w.c2(16), {}, None),
                      "four-sweep": (w.c2(20), {}, 3), "rank-2": (w.c5(10, 8, 16, 6), {}, None)}[which]
    if kw.get("aa") == "explicit":
        kw = {"aa": "explicit", "index_set": inst.index_set}
        norms = L.explicit_norms(inst.index_set, inst.Z, inst.n)
    else:
        norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128", **kw)
    if path is not None:
        plan.set_path(path)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    wts = lib.yoshida4()
    plan.strang_composed(5e-3, 6, wts)
    assert plan.status() == 0
    ref = S.strang_composed(u0, v, norms, inst.n, inst.gamma, 5e-3, 6, wts)
    assert rel_l2(plan.get_state().cpu().numpy(), ref) < 1e-10
    plan.strang_steps(5e-3, 3)                       # the plan's own tables are intact afterwards
    ref = S.strang(ref, v, norms, inst.n, inst.gamma, 5e-3, 3)
    assert rel_l2(plan.get_state().cpu().numpy(), ref) < 1e-10


def test_composed_fourth_order_small_lattice(lib):
    """On the n = 55 lattice where the oracle's composed step is pinned to fourth order against the
    exact semi-discrete propagator, the GPU composition equals the oracle's at every step size."""
    import torch
    Z, n = np.array([1, 34]), (55,)
    P = L.lattice_points(Z, n)
    norms, _ = L.minl2_norms_dp(Z, n)
    v, u0 = w.v_smooth(P), w.gaussian_packet(P, 0.2, [0.5, 0.5], k0=1)
    plan = lib.Plan(Z, n, 0.5, prec="c128")
    plan.set_potential(torch.from_numpy(v).cuda())
    for m in (80, 160, 320):
        plan.set_state(torch.from_numpy(u0).cuda())
        plan.strang_composed(1.0 / m, m, lib.yoshida4())
        ref = S.strang_composed(u0, v, norms, n, 0.5, 1.0 / m, m, lib.yoshida4())
        assert rel_l2(plan.get_state().cpu().numpy(), ref) < 1e-11


def test_time_dependent_potential_by_steps(lib):
    """A time-dependent potential v(x, t) = v1(x) (1 + 0.5 sin 2 pi t) (extension named in Sec. 5):
    one lsp_strang_steps call per step with the potential at the step's midpoint, against the
    oracle doing the same."""
    import torch
    inst = w.c2(16)
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v1, u0 = w.v_smooth(P), inst.u0(P)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128")
    plan.set_state(torch.from_numpy(u0).cuda())
    dt, u = 1e-2, u0.copy()
    for k in range(20):
        vk = v1 * (1 + 0.5 * np.sin(2 * np.pi * (k + 0.5) * dt))
        plan.set_potential(torch.from_numpy(vk).cuda())
        plan.strang_steps(dt, 1)
        u = S.strang(u, vk, norms, inst.n, inst.gamma, dt, 1)
    assert rel_l2(plan.get_state().cpu().numpy(), u) < 1e-11
