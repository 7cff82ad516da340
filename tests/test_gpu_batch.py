"""Batched stepping (lsp_batch_*) against the oracle and against single-plan runs (GB300)."""

import numpy as np
import pytest

from oracle import lattice as L
from oracle import strang as S
import workloads as w

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 5e-5}


def _setup(lib, insts, prec):
    import torch
    plans, ref_in = [], []
    for inst in insts:
        P = L.lattice_points(inst.Z, inst.n)
        v, u0 = inst.v(P), inst.u0(P)
        p = lib.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec)
        p.set_potential(torch.from_numpy(v).cuda())
        p.set_state(torch.from_numpy(u0).cuda())
        plans.append(p)
        ref_in.append((v, u0))
    return plans, ref_in


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_batch_matches_oracle_and_single_runs(lib, prec):
    insts = w.c3(count=12, seed=7, min_log2=12, max_log2=16)
    nsteps = 30
    plans, ref_in = _setup(lib, insts, prec)
    paths = {p.info()["path"] for p in plans}
    assert paths == {lib.PATH_SMALL, lib.PATH_MULTIPASS}        # both groups exercised
    batch = lib.Batch(plans)
    batch.steps([inst.dt for inst in insts], nsteps)
    assert batch.status() == 0
    got = [p.get_state(prec="c128").cpu().numpy() for p in plans]
    # same instances run singly
    singles, _ = _setup(lib, insts, prec)
    for p, inst in zip(singles, insts):
        p.strang_steps(inst.dt, nsteps)
    for g, p, inst, (v, u0) in zip(got, singles, insts, ref_in):
        s = p.get_state(prec="c128").cpu().numpy()
        assert np.array_equal(g, s), inst.name
        norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
        ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, nsteps)
        err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        assert err < TOL[prec], (inst.name, err)
    batch.destroy()


def test_batch_repeated_calls_and_zero_steps(lib):
    insts = w.c3(count=5, seed=3, min_log2=13, max_log2=15)
    plans, ref_in = _setup(lib, insts, "c64")
    batch = lib.Batch(plans)
    dts = [inst.dt for inst in insts]
    batch.steps(dts, 0)
    batch.steps(dts, 7)
    batch.steps(dts, 8)
    assert batch.status() == 0
    for p, inst, (v, u0) in zip(plans, insts, ref_in):
        norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
        ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 15)
        g = p.get_state(prec="c128").cpu().numpy()
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < TOL["c64"]


def test_batch_rejects_mixed_precision(lib):
    insts = w.c3(count=2, seed=1, min_log2=12, max_log2=13)
    a = lib.Plan(insts[0].Zmat, insts[0].n, 0.1, prec="c64")
    b = lib.Plan(insts[1].Zmat, insts[1].n, 0.1, prec="c128")
    with pytest.raises(lib.LspError) as e:
        lib.Batch([a, b])
    assert e.value.code == -8


def test_batch_of_four_sweep_instances(lib):
    """Rank-1 four-sweep instances of 2^20 points (d = 3..8, each with its own z, v and dt;
    K read from the table or through the byte index, two groups) advance together, one launch
    per sweep, beside a two-sweep and an SMEM-resident instance.  A 20-step call replays a
    captured graph, a 5-step call launches directly; each instance ends where it ends when
    stepped alone, and two of them are checked against the oracle."""
    import torch
    pool = w.c3()
    big = [i for i in pool if i.npoints == 1 << 20]
    ds = sorted({i.d for i in big})
    four = [next(i for i in big if i.d == d) for d in (ds[0], ds[-1])] + [i for i in big if i.d not in (ds[0], ds[-1])][:2]
    others = [next(i for i in pool if i.npoints == 1 << 16), next(i for i in pool if i.npoints == 1 << 12)]
    insts = four + others
    plans, ref_in = _setup(lib, insts, "c64")
    singles, _ = _setup(lib, insts, "c64")
    for p, q in zip(plans[:4], singles[:4]):
        p.set_path(lib.PATH_RANK1_4SWEEP)
        q.set_path(lib.PATH_RANK1_4SWEEP)
    kidx = [p.info()["max_norm2"] < 256 for p in plans[:4]]
    assert any(kidx) and not all(kidx), kidx                  # both K forms
    batch = lib.Batch(plans)
    dts = [inst.dt for inst in insts]
    for n in (20, 5, 20):
        batch.steps(dts, n)
        for q, dt in zip(singles, dts):
            q.strang_steps(dt, n)
    assert batch.status() == 0
    for k, (p, q, inst) in enumerate(zip(plans, singles, insts)):
        g = p.get_state(prec="c128").cpu().numpy()
        s = q.get_state(prec="c128").cpu().numpy()
        assert np.linalg.norm(g - s) / np.linalg.norm(s) < 1e-6, inst.name
    for k in (0, 1):
        inst, (v, u0) = insts[k], ref_in[k]
        norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
        ref = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 45)
        g = plans[k].get_state(prec="c128").cpu().numpy()
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < TOL["c64"], inst.name
    batch.destroy()


@pytest.mark.parametrize("m,prec", [(11, "c64"), (12, "c64"), (13, "c64"), (11, "c128"), (12, "c128")])
def test_small_line_kernel_parity(lib, m, prec):
    """Rank-1 lattices of 2^11 .. 2^13 points run the SMEM-resident one-line kernel (state in
    registers across steps): 40 steps against the oracle, alone and in a batch beside a
    mixed-radix SMEM instance (n = 961) of the same call."""
    inst = w.Instance(f"line 2^{m}", 5, (1 << m,), w.random_rank1(5, 1 << m, w.Rng(m, 9)), 0.1, 2e-3, 40,
                      w.v_smooth, lambda p: w.gaussian_packet(p, 0.1, [0.5] * 5))
    other = w.Instance("n=961", 2, (961,), np.array([1, 31]), 0.1, 1e-3, 40, w.v_smooth,
                       lambda p: w.gaussian_packet(p, 0.1, [0.5] * 2))
    plans, ref_in = _setup(lib, [inst, other], prec)
    single, _ = _setup(lib, [inst], prec)
    for p in (plans[0], single[0]):
        if m >= 13:                                # two-sweep by default from 2^13
            p.set_path(lib.PATH_SMALL)
        assert p.info()["path"] == lib.PATH_SMALL
    single[0].strang_steps(inst.dt, 25)
    single[0].strang_steps(inst.dt, 15)
    batch = lib.Batch(plans)
    batch.steps([inst.dt, other.dt], 25)
    batch.steps([inst.dt, other.dt], 15)
    assert batch.status() == 0 and single[0].status() == 0
    for k, it in enumerate((inst, other)):
        v, u0 = ref_in[k]
        norms, _ = L.minl2_norms_dp(it.Z, it.n)
        ref = S.strang(u0, v, norms, it.n, it.gamma, it.dt, 40)
        g = plans[k].get_state(prec="c128").cpu().numpy()
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < TOL[prec], it.name
    s = single[0].get_state(prec="c128").cpu().numpy()
    assert np.array_equal(s, plans[0].get_state(prec="c128").cpu().numpy())
    batch.destroy()
