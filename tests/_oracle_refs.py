"""Long FP64 oracle runs behind the full-length parity tests (test infrastructure).

The oracle needs minutes for the full configurations (n = 2^22 for 1000 steps, the
n = 2^20 adjoint over 500 steps), so these runs start in spawned worker processes as
soon as pytest has collected the tests that need them (tests/conftest.py), and the GPU
tests that compare against them run meanwhile.  Spawned workers touch no GPU: only
numpy and the oracle.  A test run alone starts its own job on first use.
"""

from __future__ import annotations

import multiprocessing as mp

import numpy as np

C3_SAMPLE_STEPS = 500


def c2_final(nsteps: int):
    """C2 (d = 6, n = 2^22, HC(64) reconstructing lattice): u after nsteps oracle steps, and its norm."""
    from oracle import lattice as L
    from oracle import strang as S
    import workloads as w
    inst = w.c2(22)
    P = L.lattice_points(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    del P
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    u = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, nsteps)
    return u, S.norm2(u0), S.norm2(u)


def c3_sample_ids(insts):
    """One instance per lattice size of the 256-instance batch (the first of each size)."""
    seen, ids = set(), []
    for i, inst in enumerate(insts):
        if inst.npoints not in seen:
            seen.add(inst.npoints)
            ids.append(i)
    return ids


def c3_sample_finals(nsteps: int):
    """C3: u after nsteps oracle steps for one instance of every lattice size (ids, finals)."""
    from oracle import lattice as L
    from oracle import strang as S
    import workloads as w
    insts = w.c3()
    ids = c3_sample_ids(insts)
    out = {}
    for i in ids:
        inst = insts[i]
        P = L.lattice_points(inst.Z, inst.n)
        v, u0 = inst.v(P), inst.u0(P)
        norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
        out[i] = S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, nsteps)
    return ids, out


def c4_adjoint(nsteps: int):
    """C4 (d = 4, n = 2^20): J = |<u_N, phi>|^2, dJ/dv, dJ/du0 and u_N from the oracle's
    reverse-mode Strang loop with ceil(sqrt(N)) checkpoints."""
    from oracle import lattice as L
    from oracle import strang as S
    import workloads as w
    inst = w.c4(20)
    P = L.lattice_points(inst.Z, inst.n)
    v, u0, phi = inst.v(P), inst.u0(P), inst.phi(P)
    del P
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    return S.strang_adjoint(u0, v, norms, inst.n, inst.gamma, inst.dt, nsteps, phi)


JOBS = {
    "c2_1000": (c2_final, (1000,)),
    "c3_500": (c3_sample_finals, (C3_SAMPLE_STEPS,)),
    "c4_500": (c4_adjoint, (500,)),
}

_pool = None
_results = {}


def start(names):
    """Submit the named jobs (once each) to a pool of spawned workers."""
    global _pool
    todo = [n for n in names if n not in _results]
    if not todo:
        return
    if _pool is None:
        _pool = mp.get_context("spawn").Pool(processes=max(1, min(len(JOBS), mp.cpu_count() - 1)))
    for n in todo:
        fn, args = JOBS[n]
        _results[n] = _pool.apply_async(fn, args)


def get(name: str, timeout: float = 1800.0):
    start([name])
    return _results[name].get(timeout)


def stop():
    global _pool
    if _pool is not None:
        _pool.terminate()
        _pool.join()
        _pool = None
    _results.clear()
