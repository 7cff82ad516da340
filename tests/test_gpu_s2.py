"""The TMA-fed two-sweep rank-1 path (execution path 4) against the FP64 oracle (GB300).

Rows of 4096 points and columns of n / 4096 points: n = 2^20 .. 2^23 covers column
tiles of 16, 8, 4 and 2 columns (tensor boxes of 128, 64, 32 and 16 bytes per row); n = 2^24
runs tiles of 8192 points on 512-thread CTAs (two rows, each transformed by one half of the
CTA, or two 4096-point columns).
"""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu

TOL64 = 5e-5


def _rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(lib, inst, prec="c64"):
    import torch
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    plan = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
    plan.set_path(lib.PATH_RANK1_TMA)
    plan.set_potential(torch.from_numpy(v).cuda())
    plan.set_state(torch.from_numpy(u0).cuda())
    return plan, v, u0


@pytest.mark.parametrize("m,nsteps", [(16, 20), (17, 5), (18, 17), (19, 4), (20, 20), (21, 7), (22, 17), (23, 3),
                                      (24, 2)])
def test_tma_two_sweep_matches_oracle(lib, m, nsteps):
    """Every sweep kind of the path (head, row with the byte-index K, mid, tail), plain launches
    below 16 steps and the replayed graph from 16 on, against the oracle's steps."""
    inst = w.c2(m)
    plan, v, u0 = _plan(lib, inst)
    assert plan.info()["path"] == lib.PATH_RANK1_TMA
    assert plan.info()["N1"] == 4096 and plan.info()["N2"] == (1 << m) // 4096
    plan.strang_steps(inst.dt, nsteps)
    assert plan.status() == 0
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, nsteps)
    err = _rel(plan.get_state(prec="c128").cpu().numpy(), ref)
    assert err < TOL64, err
    # spectral output (column forward sweep, row forward sweep with 1/n) against the oracle
    spec = plan.get_state(space="spectral", prec="c128").cpu().numpy()
    assert _rel(spec, S.coeffs(ref, inst.n)) < TOL64
    plan.destroy()


def test_wide_tiles_every_schedule_graph_replay(lib):
    """n = 2^24 (8192-point tiles, 512 threads): 16 steps replayed from the captured graph under
    each schedule, against one oracle run; spectral output under the default schedule."""
    inst = w.c2(24)
    plan, v, u0 = _plan(lib, inst)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 16)
    import torch
    for sched in (0, 1, 2):
        plan.set_schedule(sched)
        plan.set_state(torch.from_numpy(u0).cuda())
        plan.strang_steps(inst.dt, 16)
        assert plan.status() == 0
        err = _rel(plan.get_state(prec="c128").cpu().numpy(), ref)
        assert err < TOL64, (sched, err)
    plan.set_schedule(1)
    plan.set_state(torch.from_numpy(u0).cuda())
    plan.strang_steps(inst.dt, 16)
    assert _rel(plan.get_state(space="spectral", prec="c128").cpu().numpy(), S.coeffs(ref, inst.n)) < TOL64
    plan.destroy()


@pytest.mark.parametrize("sched", [0, 1, 2])
@pytest.mark.parametrize("m", [20, 22])
def test_every_schedule_matches_oracle(lib, m, sched):
    """The three kernel schedules (exchange buffers, CTAs per SM, P by TMA or direct loads) give
    the oracle's result: 19 steps (graph replay), spectral output included."""
    inst = w.c2(m)
    plan, v, u0 = _plan(lib, inst)
    plan.set_schedule(sched)
    assert plan.schedule() == (lib.PATH_RANK1_TMA, sched)
    plan.strang_steps(inst.dt, 19)
    assert plan.status() == 0
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 19)
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL64
    assert _rel(plan.get_state(space="spectral", prec="c128").cpu().numpy(), S.coeffs(ref, inst.n)) < TOL64
    with pytest.raises(lib.LspError):
        plan.set_schedule(3)
    plan.destroy()


def test_autotune_decision_is_cached_across_plans(lib):
    """The first plan of a geometry is timed on every path and schedule; a second plan of the same
    geometry takes the stored decision (same path, schedule and times) without timing."""
    import torch
    lib.autotune_cache(clear=True)
    inst = w.c2(20)
    a, v, u0 = _plan(lib, inst)
    pa, ms_a = a.autotune(inst.dt, 20)
    assert lib.autotune_cache() == 1
    assert lib.PATH_RANK1_TMA in ms_a and all(t > 0 for t in ms_a.values())
    b = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64")
    b.set_potential(torch.from_numpy(v).cuda())
    b.set_state(torch.from_numpy(u0).cuda())
    pb, ms_b = b.autotune(inst.dt, 20)
    assert lib.autotune_cache() == 1
    assert (pb, ms_b) == (pa, ms_a) and b.schedule() == a.schedule()
    b.strang_steps(inst.dt, 5)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    assert _rel(b.get_state(prec="c128").cpu().numpy(), S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 5)) < TOL64
    a.destroy()
    b.destroy()


def test_tma_two_sweep_k_table_without_byte_index(lib):
    """max ||h||^2 >= 256 (d = 4, n = 2^20, the adjoint workload's lattice): K is read from the
    8-byte table in the row sweep instead of the byte index."""
    inst = w.c4(20)
    plan, v, u0 = _plan(lib, inst)
    assert plan.info()["max_norm2"] >= 256
    plan.strang_steps(inst.dt, 18)
    assert plan.status() == 0
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 18)
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL64
    plan.destroy()


def test_tma_two_sweep_graph_replay_and_repeated_calls(lib):
    """Calls of 16 and more steps replay the captured launches; two calls of 20 and one of 3
    equal 43 oracle steps; a changed step size rebuilds the tables."""
    inst = w.c2(20)
    plan, v, u0 = _plan(lib, inst)
    plan.strang_steps(inst.dt, 20)
    plan.strang_steps(inst.dt, 20)
    plan.strang_steps(inst.dt, 3)
    plan.strang_steps(2 * inst.dt, 16)
    assert plan.status() == 0
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 43)
    ref = S.strang(ref, v, norms, inst.n, inst.gamma, 2 * inst.dt, 16)
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL64
    plan.destroy()


def test_tma_two_sweep_adjoint_autotune_and_batch(lib):
    """The path's steps on other state buffers (adjoint checkpoints, autotune scratch) and inside
    a batch give the same results as the plan's own calls."""
    import torch
    inst = w.c2(20)
    plan, v, u0 = _plan(lib, inst)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    P = L.lattice_points(inst.Z, inst.n)
    phi = w.gaussian_packet(P, 0.1, [0.6] + [0.5] * (inst.d - 1))
    J, gv_ref, gu_ref, uN = S.strang_adjoint(u0, v, norms, inst.n, inst.gamma, inst.dt, 12, phi, ckpt=4)
    lam = torch.from_numpy(2.0 * S.inner(phi, uN) * phi / phi.size).to(torch.complex64).cuda()
    gv = torch.empty(inst.npoints, dtype=torch.float64, device="cuda")
    gu = torch.empty(inst.npoints, dtype=torch.complex64, device="cuda")
    lib.adjoint(plan, inst.dt, 12, lam, gv, gu, 4)
    assert plan.status() == 0
    assert _rel(gv.cpu().numpy(), gv_ref) < 2e-4 and _rel(gu.cpu().numpy(), gu_ref) < 2e-4
    # sweep times: the column and row sweeps of this path, the state untouched
    before = plan.get_state().clone()
    t = plan.sweep_times(inst.dt, 8)
    assert t["P"] > 0 and t["K"] > 0 and t["A"] < 0 and t["A_inv"] < 0
    assert torch.equal(plan.get_state(), before)
    # batch: the instance steps through its own path
    plan.set_state(torch.from_numpy(u0).cuda())
    b = lib.Batch([plan])
    b.steps([inst.dt], 25)
    assert b.status() == 0
    ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 25)
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL64
    b.destroy()
    # autotune sees the path and leaves the state alone
    path, ms = plan.autotune(inst.dt, 20)
    assert lib.PATH_RANK1_TMA in ms and path in ms
    assert _rel(plan.get_state(prec="c128").cpu().numpy(), ref) < TOL64
    plan.destroy()


def test_batch_of_uneven_sizes_in_one_launch_per_sweep(lib):
    """Path-4 instances of 2^16 .. 2^20 points (d = 3..8, each with its own lattice, potential and
    step size) advance together: one launch per sweep over all their tiles, graph-replayed for
    20-step calls and launched directly for 5; every instance ends where it ends when stepped
    alone (same arithmetic), and one instance of every size is checked against the oracle."""
    import torch
    pool = w.c3()
    insts = []
    for m in range(16, 21):
        insts += [i for i in pool if i.npoints == 1 << m][:2]
    plans, singles, refs = [], [], []
    for inst in insts:
        for lst in (plans, singles):
            p, v, u0 = _plan(lib, inst)
            lst.append(p)
        refs.append((v, u0))
    kidx = [p.info()["max_norm2"] < 256 for p in plans]
    assert any(kidx) and not all(kidx), kidx                  # K by byte index and from the table
    batch = lib.Batch(plans)
    dts = [inst.dt for inst in insts]
    for n in (20, 5, 20):
        batch.steps(dts, n)
        for q, dt in zip(singles, dts):
            q.strang_steps(dt, n)
    assert batch.status() == 0
    for p, q, inst in zip(plans, singles, insts):
        assert torch.equal(p.get_state(), q.get_state()), inst.name
    for k in range(0, len(insts), 2):
        inst, (v, u0) = insts[k], refs[k]
        norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
        ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 45)
        assert _rel(plans[k].get_state(prec="c128").cpu().numpy(), ref) < TOL64, inst.name
    batch.destroy()
