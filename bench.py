"""Benchmark: lattice-point Strang steps per second on the n = 2^22, d = 6 rank-1 workload.

One bench step = one lsp_strang_steps(dt, 1000) call on the d = 6, n = 2^22
reconstructing rank-1 lattice (hyperbolic cross prod(1+|h_j|) <= 64,
minimal-l2 anti-aliasing set, gamma = 0.05, dt = 1e-3): every row of the hot
path (phase-table build, potential phase, forward FFT, kinetic phase, inverse
FFT, merged potential phase, 1000-step driver) runs inside the timed region.
The state (32 MiB c64) and phase tables fit in L2, so L2 is flushed (a 512 MiB
write) before every timed step; each step is timed alone with CUDA events.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (weak scaling).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lattice-point Strang steps/s (n·steps/s), FP32 vs FP64 at stated error; HBM %"
STEPS_PER_CALL = 1000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-c128", action="store_true", help="skip the complex128 side measurement")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plan", action="store_true", help="skip the plan-time (DP, CBC) side measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-instance batched measurement")
    ap.add_argument("--no-rank2", action="store_true", help="skip the rank-2 2^14 x 2^12 batch measurement")
    ap.add_argument("--no-side", action="store_true", help="skip the C1, C4 and rank-1 2^24 side measurements")
    ap.add_argument("--log2n", type=int, default=22, help="lattice size 2^m of the d=6 workload (profiling)")
    ap.add_argument("--inner", type=int, default=STEPS_PER_CALL, help="Strang steps per bench step")
    ap.add_argument("--workload", default="c2", choices=["c2", "c5"],
                    help="c2: the headline run (with its side measurements); c5: only the rank-2 "
                         "2^14 x 2^12 batch (profiling; --inner steps per call, --batch instances)")
    ap.add_argument("--batch", type=int, default=4, help="instances of the c5 workload")
    ap.add_argument("--path", type=int, default=-1,
                    help="execution path of the headline plan (default: autotuned); 0 two-sweep, 3 four-sweep")
    return ap.parse_args()


# CUDA sources each profiled kernel family is built from
KERNEL_SOURCES = {
    "mp_persistent": ["lsp_internal.cuh", "lsp_tile.cuh", "lsp_mp.cuh", "lsp_mp_c64_hi.cu"],
    "sweep4_rank2": ["lsp_internal.cuh", "lsp_tile.cuh", "lsp_sweep4.cuh", "lsp_sweep4_r2.cu"],
    "sweep4_rank1": ["lsp_internal.cuh", "lsp_tile.cuh", "lsp_sweep4.cuh", "lsp_sweep4_r1.cu"],
    "s2": ["lsp_internal.cuh", "lsp_tile.cuh", "lsp_async.cuh", "lsp_s2.cuh", "lsp_s2.cu"],
}


def csrc_digest(family: str) -> str:
    """Checksum of the sources of one kernel family (identifies the kernels an ncu record belongs to)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, "paper_1808_06357_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record(name: str, family: str):
    """DRAM bytes per launch from a committed ncu record, if it was taken on the current sources."""
    prof = os.path.join(ROOT, "profiles", f"traffic_{name}.json")
    try:
        rec = json.load(open(prof))
        if rec.get("csrc_sha256_16") == csrc_digest(family):
            return rec
    except Exception:
        pass
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("LSP_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(items, rank: int, world: int):
    """Independent instances of a batch, dealt round-robin to the ranks (no collective needed)."""
    return list(items)[rank::world]


def c2_inputs(m: int = 22):
    import workloads as w
    return w.c2(m)


def host_description():
    """CPU model and core count of this host (recorded with every oracle timing)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"cpu": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def _oracle_worker(args):
    """One oracle replica (spawned process): FP64 Strang steps on the full state for ~budget_s."""
    m, budget_s = args
    import workloads as w
    from oracle import lattice as L
    from oracle import strang as S
    inst = w.c2(m)
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    del P
    S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 1)            # warm
    steps, t0, u = 0, time.perf_counter(), u0
    while time.perf_counter() - t0 < budget_s:
        u = S.strang(u, v, norms, inst.n, inst.gamma, inst.dt, 1)
        steps += 1
    return steps, time.perf_counter() - t0


def cpu_oracle_rate(inst, budget_s: float = 15.0):
    """The FP64 oracle (as it stands) on a bounded sample: Strang steps on the full state, first on
    one core, then as independent replicas on every host core (spawned processes; numpy's FFT
    is single-threaded, so replicas are how the oracle uses all cores)."""
    import numpy as np
    from oracle import lattice as L
    from oracle import strang as S
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    del P
    S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 1)          # warm
    steps, t0 = 0, time.perf_counter()
    u = u0
    while time.perf_counter() - t0 < budget_s / 2:
        u = S.strang(u, v, norms, inst.n, inst.gamma, inst.dt, 1)
        steps += 1
    el = time.perf_counter() - t0
    one = {"value": inst.npoints * steps / el, "steps": steps, "seconds": el}
    del u, v, u0
    cores = os.cpu_count() or 1
    m = int(round(math.log2(inst.npoints)))
    import multiprocessing as mp
    try:
        with mp.get_context("spawn").Pool(processes=cores) as pool:
            res = pool.map(_oracle_worker, [(m, budget_s / 2)] * cores)
        tot = sum(inst.npoints * st / sec for st, sec in res)
        allc = {"value": tot, "replicas": cores, "steps_per_replica": [st for st, _ in res]}
    except Exception as e:                                           # e.g. not enough host memory
        allc = {"value": None, "error": str(e)[:200]}
    return one, allc


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    inst = c2_inputs()
    import numpy as np
    from oracle import lattice as L
    from oracle import strang as S
    P = L.lattice_points(inst.Z, inst.n)
    norms, _ = L.minl2_norms_dp(inst.Z, inst.n)
    v, u0 = inst.v(P), inst.u0(P)
    per_step = 3                                                    # oracle Strang steps per bench step
    for _ in range(args.warmup):
        S.strang(u0, v, norms, inst.n, inst.gamma, inst.dt, 1)
    times = []
    u = u0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u = S.strang(u, v, norms, inst.n, inst.gamma, inst.dt, per_step)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = inst.npoints * per_step * args.steps / tot
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "lattice-point steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "rank-1 lattice d=6 n=2^22 HC(64) reconstructing, MINL2, gamma=0.05, dt=1e-3",
                   "strang_steps_per_bench_step": per_step, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "lattice-point steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} Strang steps of the full n=2^22 state per bench step",
                         "host": host_description()},
        "e2e": {"value": value, "unit": "lattice-point steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_c5(args):
    """Only the rank-2 batch (complex64): a profiling entry with a short, configurable run."""
    import torch

    import paper_1808_06357_gb300 as lsp
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clk = Clocks(local)
    clk.start()
    r = measure_rank2(args, lsp, torch, dev, local, flush, stream, world, precs=("c64",), nsteps=args.inner,
                      count=args.batch, calls64=args.steps)
    clocks = clk.stop()
    if rank == 0:
        c = r["c64"]
        print(json.dumps({"metric": METRIC, "value": c["value"], "unit": c["unit"], "n_gpus": world,
                          "steps": args.steps, "warmup": 1, "ms_per_step": c["ms_per_call"],
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                          "data": "synthetic", "config": {"workload": r["workload"]}, "roofline": c["roofline"],
                          "clocks": clocks}))


def run_ours(args):
    import numpy as np
    import torch

    import paper_1808_06357_gb300 as lsp

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    global STEPS_PER_CALL
    STEPS_PER_CALL = args.inner
    inst = c2_inputs(args.log2n)
    n = inst.npoints

    # inputs: lattice points from the library, input functions from the workload module
    plan = lsp.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64", device=local)
    pts = plan.lattice_points()
    v_h = inst.v(pts)
    u0_h = inst.u0(pts)
    v_d = torch.from_numpy(v_h).to(dev)
    u0_d = torch.from_numpy(u0_h.astype(np.complex64)).to(dev)
    plan.set_potential(v_d)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # schedule choice (untimed): time up to 100 steps on every available path, keep the fastest
    plan.set_state(u0_d)
    if args.path < 0:
        path, tune_ms = plan.autotune(inst.dt, min(100, STEPS_PER_CALL))
    else:
        plan.set_path(args.path)
        path, tune_ms = args.path, {}

    def one_call(p):
        p.strang_steps(inst.dt, STEPS_PER_CALL)

    def timed(p, k, w):
        p.set_state(u0_d)
        for _ in range(w):
            one_call(p)
        torch.cuda.synchronize()
        ms = []
        for _ in range(k):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_call(p)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        if p.status() != 0:
            raise RuntimeError("device status " + lsp.strerror(p.status()))
        return ms

    clk = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    ms = timed(plan, args.steps, args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    tot_ms = max_over_ranks(sum(ms), world)
    value = world * n * STEPS_PER_CALL * args.steps / (tot_ms / 1e3)

    # roofline of the whole step: the method's algorithmic bytes of all the call's steps over the
    # whole call (phase-table build and every sweep inside)
    hbm, src = peaks()
    alg_bytes = 48.0 * n * STEPS_PER_CALL                # 6 s per point-step, s = 8 B (c64)
    kern_s = statistics.mean(ms) / 1e3
    step_achieved = alg_bytes / kern_s / 1e9
    step_traffic = None
    rec = None
    if args.log2n == 22 and STEPS_PER_CALL == 1000:
        # DRAM bytes of one call from committed ncu records (None once the kernel sources changed)
        if path == lsp.PATH_MULTIPASS:
            rec = traffic_record("c64_n2p22", "mp_persistent")
            step_traffic = rec.get("bytes_per_launch") if rec else None
        elif path == lsp.PATH_RANK1_4SWEEP:
            rec = traffic_record("c64_n2p22_4sweep", "sweep4_rank1")
            step_traffic = rec.get("bytes_per_call_1000_steps") if rec else None
    # roofline of the dominant kernel.  Two-sweep path: the persistent kernel is the call (one
    # launch runs all its sweeps).  Four-sweep path: the K sweep (DFT_4096, K, IDFT_4096; 31 % of
    # the step), algorithmic bytes 24 per point (state read and written, the K table), its mean
    # launch time taken live by lsp_sweep_times (CUDA events on the launching stream, 64 steps).
    if path == lsp.PATH_RANK1_4SWEEP:
        sw = plan.sweep_times(inst.dt, 64, stream=stream)
        k_bytes = 24.0 * n
        k_traffic = None
        if rec:
            z = rec.get("per_kind_mid_step", {}).get("14")
            k_traffic = z["dram_read"] + z["dram_write"] if z else None
        kernel = {"name": "sweep4 K sweep (Z: DFT_4096, K by byte index, IDFT_4096)", "ms_per_launch": sw["K"],
                  "alg_bytes_per_launch": k_bytes, "sweep_ms": sw}
        achieved = k_bytes / (sw["K"] / 1e3) / 1e9
        traffic = k_traffic
    elif path == lsp.PATH_RANK1_TMA:
        # two sweeps per step, each 24 algorithmic bytes per point (state read and written, one
        # phase table: P in the column sweep, K in the row sweep); the slower one is reported
        sw = plan.sweep_times(inst.dt, 64, stream=stream)
        k_bytes = 24.0 * n
        which = "P" if sw["P"] >= sw["K"] else "K"
        name = ("s2 column sweep (IDFT_N2, 1/n, P, DFT_N2; TMA tensor tiles)" if which == "P" else
                "s2 row sweep (W_n, DFT_4096, K by byte index, IDFT_4096, conj W_n; TMA bulk tiles)")
        rec = traffic_record(f"c64_n2p{args.log2n}_tma", "s2") if STEPS_PER_CALL == 1000 else None
        k_traffic = rec.get("per_launch", {}).get(which) if rec else None
        step_traffic = rec.get("bytes_per_call_1000_steps") if rec else None
        kernel = {"name": name, "ms_per_launch": sw[which], "alg_bytes_per_launch": k_bytes,
                  "sweep_ms": {"column": sw["P"], "row": sw["K"]}}
        achieved = k_bytes / (sw[which] / 1e3) / 1e9
        traffic = k_traffic
    else:
        kernel = {"name": "mp_persistent (all 2N-1 sweeps of a call in one launch)",
                  "ms_per_launch": statistics.mean(ms), "alg_bytes_per_launch": alg_bytes}
        achieved, traffic = step_achieved, step_traffic
    launches = {lsp.PATH_MULTIPASS: 5, lsp.PATH_RANK1_4SWEEP: 3 + 4 * STEPS_PER_CALL,
                lsp.PATH_RANK1_TMA: 3 + 2 * STEPS_PER_CALL}.get(path, 0)

    # complex128 side measurement on the same workload
    c128 = None
    if not args.no_c128:
        p2 = lsp.Plan(inst.Zmat, inst.n, inst.gamma, prec="c128", device=local)
        p2.set_potential(v_d)
        u0_d2 = torch.from_numpy(u0_h).to(dev)
        p2.set_state(u0_d2)
        p2.strang_steps(inst.dt, 10)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps2 = 100
        flush.fill_(1.0)
        e0.record(stream)
        p2.strang_steps(inst.dt, steps2)
        e1.record(stream)
        e1.synchronize()
        t2 = e0.elapsed_time(e1) / 1e3
        fp64 = lsp.fma_rate("c128", device=local)
        flops = 10.0 * math.log2(n) + 12.0                 # algorithmic flops per point-step (two FFTs, two phases)
        tf = flops * n * steps2 / t2 / 1e12
        c128 = {"value": n * steps2 / t2, "unit": "lattice-point steps/s", "steps_timed": steps2,
                "path": p2.info()["path"], "achieved_GBps": 96.0 * n * steps2 / t2 / 1e9,
                "roofline": {"bound": "alu", "achieved": tf, "peak": fp64, "unit": "TFLOP/s", "frac": tf / fp64,
                             "peak_source": "measured: lsp_fma_rate (FP64 FMA chains on every SM, CUDA events)",
                             "flops_per_point_step": flops,
                             "hbm_frac": 96.0 * n * steps2 / t2 / 1e9 / peaks()[0]}}
        p2.destroy()

    # end-to-end through the public API with host buffers (pinned), per bench step:
    # set_potential (n f64) + set_state (n c64) H2D, 1000 steps, get_state (n c64) D2H
    e2e = None
    if not args.no_e2e:
        v_pin = torch.from_numpy(v_h).pin_memory()
        u_pin = torch.from_numpy(u0_h.astype(np.complex64)).pin_memory()
        out_pin = torch.empty(n, dtype=torch.complex64).pin_memory()
        plan.set_potential(v_pin.numpy())
        plan.set_state(u_pin.numpy())
        one_call(plan)
        plan.get_state(out=out_pin.numpy())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.set_potential(v_pin.numpy())
            plan.set_state(u_pin.numpy())
            one_call(plan)
            plan.get_state(out=out_pin.numpy())          # synchronises
        el = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": world * n * STEPS_PER_CALL * args.steps / el, "unit": "lattice-point steps/s",
               "h2d_bytes_per_step": n * 8 + n * 8, "d2h_bytes_per_step": n * 8}

    batched = None
    if not args.no_batched and args.log2n == 22:
        batched = measure_batched(args, lsp, torch, dev, local, flush, stream, world, rank)
    rank2 = None
    if not args.no_rank2:
        rank2 = measure_rank2(args, lsp, torch, dev, local, flush, stream, world)

    plan_time = None
    if rank == 0 and not args.no_plan:
        plan_time = measure_plan_time(lsp, inst, local)
    side = None
    if not args.no_side and args.log2n == 22:
        side = {"c1": measure_c1(lsp, torch, dev, local, stream, world),
                "c4_adjoint": measure_c4(lsp, torch, dev, local, flush, stream, world),
                "rank1_2p24": measure_large(lsp, torch, dev, local, flush, stream, world, 24)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        one, allc = cpu_oracle_rate(inst)
        host = host_description()
        if allc.get("value"):
            cpu = {"value": allc["value"], "unit": "lattice-point steps/s", "cores": allc["replicas"], "kind": "oracle",
                   "sample": f"FP64 Strang steps of the full n=2^22 state for ~7.5 s in each of {allc['replicas']} "
                             f"independent replicas (spawned processes, numpy FFT, 1 thread each)",
                   "single_core": {"value": one["value"], "sample": f"{one['steps']} steps in {one['seconds']:.1f} s"},
                   "host": host}
        else:
            cpu = {"value": one["value"], "unit": "lattice-point steps/s", "cores": 1, "kind": "oracle",
                   "sample": f"{one['steps']} FP64 Strang steps of the full n=2^22 state ({one['seconds']:.1f} s, "
                             f"numpy FFT, 1 thread)", "all_cores_error": allc.get("error"), "host": host}
        if plan_time is not None:
            cpu["plan_time"] = cbc_oracle_time(plan_time)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "lattice-point steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"rank-1 lattice d=6 n=2^{args.log2n}, HC(64) reconstructing z, "
                                   f"MINL2 anti-aliasing set, gamma=0.05, dt=1e-3, {STEPS_PER_CALL} Strang steps per "
                                   "bench step, complex64 state", "l2": "flushed (512 MiB write) before every timed step",
                       "parallelism": f"replicas x{world}",
                       "path": {0: "two-sweep persistent",
                                3: "four-sweep",
                                4: f"two-sweep, TMA-fed tiles (4096 x {n >> 12})"}.get(path, str(path)),
                       "schedule": plan.schedule()[1],
                       "autotune_ms": {str(k): round(v, 3) for k, v in tune_ms.items()},
                       "autotune_steps": min(100, STEPS_PER_CALL)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "peak_source": src, "kernel": kernel,
                         "step": {"achieved": step_achieved, "frac": step_achieved / hbm, "traffic": step_traffic,
                                  "alg_bytes_per_point_step": 48,
                                  "what": "the method's 48 B per point-step over the whole timed call"}},
            "complex128": c128,
            "batched": batched,
            "rank2": rank2,
            "plan_time": plan_time,
            "side": side,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches * args.steps,     # build_klut, build_tables, then the path's sweeps
        }
        print(json.dumps(out))
    plan.destroy()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _event_ms(torch, stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def measure_c1(lsp, torch, dev, local, stream, world):
    """C1: d = 2, n = 961 = 31^2, z = (1, 31), box |h_j| <= 15 (explicit set), gamma = 0.1, dt = 1e-3,
    1000 steps per call on the SMEM-resident path (one CTA runs every step), complex128 and complex64."""
    import numpy as np
    import workloads as w
    inst = w.c1()
    out = {"workload": "rank-1 lattice d=2 n=961 z=(1,31), explicit box |h_j|<=15, gamma=0.1, dt=1e-3, "
                       "1000 steps per call; the 15 KB state stays in one SM's shared memory"}
    for prec in ("c128", "c64"):
        p = lsp.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec, aa="explicit", index_set=inst.index_set, device=local)
        pts = p.lattice_points()
        p.set_potential(torch.from_numpy(inst.v(pts)).to(dev))
        u0 = torch.from_numpy(inst.u0(pts)).to(dev)
        p.set_state(u0)
        p.strang_steps(inst.dt, 1000)
        torch.cuda.synchronize()
        ms = [_event_ms(torch, stream, lambda: p.strang_steps(inst.dt, 1000)) for _ in range(3)]
        t = max_over_ranks(sum(ms), world) / 1e3
        out[prec] = {"value": world * inst.npoints * 1000 * len(ms) / t, "unit": "lattice-point steps/s",
                     "ms_per_call": 1e3 * t / len(ms), "path": p.info()["path"]}
        p.destroy()
    return out


def measure_c4(lsp, torch, dev, local, flush, stream, world):
    """C4: the adjoint call (d = 4, n = 2^20, 500 steps, ceil(sqrt(500)) checkpoints, complex64):
    forward run with checkpoints, recomputation per segment, backward run and gradient
    accumulation; reported as gradients per second and as lattice-point steps per second of
    the forward run they cover."""
    import numpy as np
    import workloads as w
    inst = w.c4(20)
    p = lsp.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64", device=local)
    pts = p.lattice_points()
    v = torch.from_numpy(inst.v(pts)).to(dev)
    u0 = torch.from_numpy(inst.u0(pts).astype(np.complex64)).to(dev)
    phi = torch.from_numpy(inst.phi(pts)).to(dev)
    del pts
    p.set_potential(v)
    lam = (2.0 * phi / inst.npoints).to(torch.complex64)
    gv = torch.empty(inst.npoints, dtype=torch.float64, device=dev)
    gu = torch.empty(inst.npoints, dtype=torch.complex64, device=dev)

    def call():
        p.set_state(u0)
        lsp.adjoint(p, inst.dt, inst.nsteps, lam, gv, gu, 0)
    call()
    torch.cuda.synchronize()
    ms = []
    for _ in range(2):
        flush.fill_(1.0)
        ms.append(_event_ms(torch, stream, call))
    if p.status() != 0:
        raise RuntimeError("adjoint status " + lsp.strerror(p.status()))
    t = max_over_ranks(sum(ms), world) / 1e3
    out = {"value": world * len(ms) / t, "unit": "gradients/s", "ms_per_gradient": 1e3 * t / len(ms),
           "forward_equivalent": world * inst.npoints * inst.nsteps * len(ms) / t, "path": p.info()["path"],
           "workload": "d=4 n=2^20 random-unit rank-1 lattice, MINL2 set, gamma=0.1, dt=1e-3, 500 steps, grad of "
                       "|<u_T, phi>|^2 wrt v and u0, ceil(sqrt(500)) checkpoints, complex64"}
    p.destroy()
    return out


def measure_large(lsp, torch, dev, local, flush, stream, world, m):
    """Rank-1 n = 2^m beyond L2 (2^24 complex64: 128 MiB state, 128 MiB of each phase table), d = 6,
    100 steps per call on every available path (after one untimed call each); the fastest path's
    rate against the method's 48 B per point-step."""
    import numpy as np
    import workloads as w
    inst = w.c2(m)
    p = lsp.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64", device=local)
    pts = p.lattice_points()
    p.set_potential(torch.from_numpy(inst.v(pts)).to(dev))
    u0 = torch.from_numpy(inst.u0(pts).astype(np.complex64)).to(dev)
    del pts
    hbm, _ = peaks()
    per_path = {}
    for path in p.paths():
        p.set_path(path)
        p.set_state(u0)
        p.strang_steps(inst.dt, 100)
        torch.cuda.synchronize()
        flush.fill_(1.0)
        t = _event_ms(torch, stream, lambda: p.strang_steps(inst.dt, 100)) / 1e3
        per_path[path] = inst.npoints * 100 / t
    if p.status() != 0:
        raise RuntimeError("status " + lsp.strerror(p.status()))
    best = max(per_path, key=per_path.get)
    rate = per_path[best]
    p.destroy()
    # cold-L2 DRAM bytes per point-step of the kernels that ran, from the committed ncu record
    rec = traffic_record(f"c64_n2p{m}_tma", "s2") if best == lsp.PATH_RANK1_TMA else None
    return {"value": world * rate, "unit": "lattice-point steps/s", "path": best,
            "per_path": {str(k): v for k, v in per_path.items()},
            "roofline": {"bound": "hbm", "achieved": 48.0 * rate / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": 48.0 * rate / 1e9 / hbm, "alg_bytes_per_point_step": 48,
                         "dram_bytes_per_point_step": rec.get("per_point_step") if rec else None},
            "workload": f"rank-1 lattice d=6 n=2^{m} random units, MINL2 set, gamma=0.05, dt=1e-3, 100 steps per call"}


def measure_plan_time(lsp, inst, local):
    """Plan-time work on the GPU: plan creation (minimal-l2 norms by the min-plus DP, tables) and the
    component-by-component reconstructing lattice for C2's index set (HC(64), d=6, n=2^22, 400 seeded
    candidates per component); the oracle's search on the same candidates is timed in the CPU-baseline leg."""
    import workloads as w
    t0 = time.perf_counter()
    p = lsp.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64", device=local)
    t_plan = time.perf_counter() - t0
    p.destroy()
    I = w.hyperbolic_cross(6, 64)
    n = 1 << 22
    cand = w.cbc_candidates(6, n, 400, w.Rng(0, 21))
    lsp.cbc_reconstructing(I, n, cand, device=local)           # warm-up (context, module load)
    t0 = time.perf_counter()
    Zg, fixed = lsp.cbc_reconstructing(I, n, cand, device=local)
    t_gpu = time.perf_counter() - t0
    out = {"plan_create_ms": 1e3 * t_plan,
           "cbc": {"workload": "reconstructing rank-1 lattice for HC(64), d=6 (51,233 vectors), n=2^22, "
                               "400 seeded candidates per component",
                   "gpu_ms": 1e3 * t_gpu, "components_fixed": fixed, "z": [int(x) for x in Zg[:, 0]]}}
    return out


def cbc_oracle_time(plan_time):
    """CPU-baseline leg of the plan-time measurement: the oracle's component-by-component search on
    the same index set and candidates, timed on one host core."""
    import workloads as w
    from oracle import lattice as L
    I = w.hyperbolic_cross(6, 64)
    cand = w.cbc_candidates(6, 1 << 22, 400, w.Rng(0, 21))
    t0 = time.perf_counter()
    Zo, fo = L.cbc_reconstructing(I, 1 << 22, cand)
    el = time.perf_counter() - t0
    same = plan_time is not None and fo == plan_time["cbc"]["components_fixed"] and \
        [int(x) for x in Zo[:, 0]] == plan_time["cbc"]["z"]
    return {"cbc_oracle_ms": 1e3 * el, "cbc_same_lattice": bool(same)}


def measure_batched(args, lsp, torch, dev, local, flush, stream, world, rank=0):
    """256 independent instances (d in 3..8, n = 2^12..2^20, per-instance dt, 500 steps,
    complex64) advanced by lsp_batch_steps; the working set (~1.4 GB) exceeds L2.  With
    several ranks the instances are dealt round-robin to them (no collective).  Two batch
    layouts are timed: every instance on its default path, and every instance of 2^16 points
    or more on the TMA two-sweep path (all sizes together, one launch per sweep); the
    faster is reported, the other beside it."""
    runs = {layout: _batched_once(args, lsp, torch, dev, local, flush, stream, world, rank, layout)
            for layout in ("default", "tma")}
    best = max(runs, key=lambda k: runs[k]["value"])
    out = dict(runs[best])
    out["layout"] = best
    out["layouts"] = {k: {"value": v["value"], "ms_per_call": v["ms_per_call"]} for k, v in runs.items()}
    return out


def _batched_once(args, lsp, torch, dev, local, flush, stream, world, rank, layout):
    import numpy as np
    import workloads as w
    all_insts = w.c3()
    insts = shard(all_insts, rank, world)
    plans, u0s = [], []
    for inst in insts:
        p = lsp.Plan(inst.Zmat, inst.n, inst.gamma, prec="c64", device=local)
        if layout == "tma" and lsp.PATH_RANK1_TMA in p.paths():
            p.set_path(lsp.PATH_RANK1_TMA)
        pts = p.lattice_points()
        p.set_potential(torch.from_numpy(inst.v(pts)).to(dev))
        u0s.append(torch.from_numpy(inst.u0(pts).astype(np.complex64)).to(dev))
        plans.append(p)
    batch = lsp.Batch(plans)
    dts = [inst.dt for inst in insts]
    nsteps = insts[0].nsteps
    for p, u in zip(plans, u0s):
        p.set_state(u)
    for _ in range(3):
        batch.steps(dts, nsteps)
    torch.cuda.synchronize()
    ms = []
    for _ in range(min(args.steps, 3)):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.steps(dts, nsteps)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    if batch.status() != 0:
        raise RuntimeError("batch status " + lsp.strerror(batch.status()))
    npts = sum(inst.npoints for inst in insts)
    npts_all = sum(inst.npoints for inst in all_insts)
    t = max_over_ranks(sum(ms), world) / 1e3
    hbm, _ = peaks()
    mean_s = statistics.mean(ms) / 1e3
    achieved = 48.0 * npts * nsteps / mean_s / 1e9
    out = {"value": npts_all * nsteps * len(ms) / t, "unit": "lattice-point steps/s",
           "instances": len(all_insts), "points": npts_all, "steps": nsteps, "timed_calls": len(ms),
           "sharding": f"instances dealt round-robin to {world} rank(s)",
           "ms_per_call": 1e3 * t / len(ms),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm},
           "workload": "256 instances, d in 3..8, n=2^m m in 12..20, per-instance dt in [1e-4,1e-2], "
                       "gamma=0.1, cosine-series v, complex64, 500 steps per call"}
    batch.destroy()
    for p in plans:
        p.destroy()
    return out


def measure_rank2(args, lsp, torch, dev, local, flush, stream, world, precs=("c64", "c128"), nsteps=None,
                  count=None, calls64=2):
    """Rank-2 lattice 2^14 x 2^12 (2^26 points), d = 16, batch of 4 instances advanced
    200 steps per call through lsp_batch_steps, complex64 and complex128.  Each
    instance's state (0.5 / 1 GiB) exceeds L2."""
    import workloads as w
    inst = w.c5()
    v_h, u_h = w.c5_fields(inst)
    v_d = torch.from_numpy(v_h).to(dev)
    n = inst.npoints
    nsteps = inst.nsteps if nsteps is None else nsteps
    count = inst.extra["batch"] if count is None else count
    hbm, _ = peaks()
    out = {"workload": "rank-2 lattice d=16, n1 x n2 = 2^14 x 2^12 (2^26 points), HC(16) reconstructing Z, "
                       "MINL2 set, v = sum_{j<k} 0.1 cos 2 pi (x_j - x_k), product Gaussian, gamma=0.1, "
                       f"dt=1e-3, batch of {count}, {nsteps} steps per call"}
    for prec, cb, calls in (("c64", 8, calls64), ("c128", 16, 1)):
        if prec not in precs:
            continue
        cdt = torch.complex64 if prec == "c64" else torch.complex128
        u_d = torch.from_numpy(u_h).to(dev).to(cdt)
        plans = [lsp.Plan(inst.Zmat, inst.n, inst.gamma, prec=prec, device=local) for _ in range(count)]
        for p in plans:
            p.set_potential(v_d)
            p.set_state(u_d)
        batch = lsp.Batch(plans)
        dts = [inst.dt] * count
        batch.steps(dts, 5)                                 # warm-up
        torch.cuda.synchronize()
        ms = []
        for _ in range(calls):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.steps(dts, nsteps)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        if batch.status() != 0:
            raise RuntimeError("rank-2 batch status " + lsp.strerror(batch.status()))
        t = max_over_ranks(sum(ms), world) / 1e3
        mean_s = statistics.mean(ms) / 1e3
        achieved = 6 * cb * n * count * nsteps / mean_s / 1e9
        out[prec] = {"value": world * n * count * nsteps * calls / t, "unit": "lattice-point steps/s",
                     "timed_calls": calls, "ms_per_call": 1e3 * t / calls,
                     "roofline": {"bound": "hbm" if prec == "c64" else "alu", "achieved": achieved, "peak": hbm,
                                  "unit": "GB/s", "frac": achieved / hbm,
                                  "alg_bytes_per_point_step": 6 * cb, "sweep_bytes_per_point_step": 10 * cb}}
        batch.destroy()
        for p in plans:
            p.destroy()
        del u_d
        torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c5":
        run_c5(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
