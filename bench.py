"""Benchmark of the Lagrangian Gauss-Newton-Krylov hot path on GB300.

One step = one Gauss-Newton Hessian matvec H dv (Sec. 3.2) on the 3D
intensity-preserving workload: 128^3 template, stationary velocity on 64^3 x 3
(786,432 unknowns), N = 8 RK4 steps, trilinear interpolation, diffusion
regularizer.  The matvec runs through the library's public call (``hessvec``):
velocity/template/direction packing, the fused J^T h^d J kernel, the gradient
unpack and the regularizer stencil.  Inputs are seeded synthetic data shaped
like the paper's 3D problems.

Printed (one JSON line, rank 0):
  value     Hessian matvecs/s over all ranks (inputs resident in HBM; L2 flushed
            between timed matvecs by a 512 MiB write, flush not timed)
  e2e       the same metric with the inputs copied from pinned host memory and
            the result copied back inside every timed step
  roofline  the fused matvec kernel: algorithmic bytes / its CUDA-event time,
            against the measured HBM copy bandwidth
  cpu_baseline  the FP64 oracle's matvec on a sample of voxels, host cores
  extra     forward voxel-steps/s and the time-to-solution of one zero-start
            Gauss-Newton solve to a 1e-3 gradient-norm drop (outside the timed
            region)

``--impl reference`` times the FP64 CPU oracle on the same workload instead
(bounded sample per step).  Multi-GPU runs (torchrun) are replicas: every rank
solves its own seeded problem, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "3d_transport_128"
METRIC = "Hessian matvecs/s (3D 128^3 transport, v 64^3x3 stationary, N=8 RK4, trilinear)"
UNIT = "matvec/s"
L2_FLUSH_BYTES = 512 << 20


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of the ranks' values (the slowest rank sets the job time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(step_ms: float, world: int) -> float:
    """Whole-job matvecs/s: every rank finishes one matvec per step (replicas)."""
    return world * 1000.0 / step_ms


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(1.0)   # let nvidia-smi start before the timed region opens
        except Exception:
            self.proc = None
        return self

    def mark(self, start: bool):
        """Open (start=True) or close the timed window; only samples inside it count."""
        now = time.time()
        if start:
            self.window = [now, None]
        elif self.window:
            self.window[1] = now

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo, hi = (self.window or [0.0, None])
        hi = (hi or time.time()) + 0.06
        for ts, ln in self.lines:
            if not (lo <= ts <= hi):
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- inputs --

def make_problem(seed):
    from paper_1703_04446_gb300 import synth
    ins = synth.make_inputs(WORKLOAD, seed=seed)
    wl = ins["workload"]
    dv = synth.random_velocity(wl.velocity, wl.time_nodes, 0.5 * max(wl.image.h) * 8, seed + 11)
    ins["dv"] = np.ascontiguousarray(dv, dtype=np.float32)
    return ins


def algorithmic_bytes_hess(wl):
    """Compulsory HBM bytes of one fused J^T h^d J launch: read v and dv (n floats
    each), read T (M floats), write the gradient accumulator (n floats)."""
    n = wl.time_nodes * wl.image.d * int(np.prod(wl.velocity.m))
    M = int(np.prod(wl.image.m))
    return 4 * (3 * n + M)


# FP32 FLOPs (FMA = 2) of one voxel-step of the fused matvec in 3D for a
# stationary velocity, counted from the kernel's formulation (the cell's
# multilinear interpolant held as polynomial coefficients):
#   tangent step: 4 stages x (locate 3 FFMA + 3 FADD, q / h 3 FMUL, per
#     component value and gradient 11 FFMA, J q 1 FMUL + 2 FFMA, dv value
#     7 FFMA) = 4 x 135, plus the RK4 state updates 18 FADD + 36 FFMA = 90 -> 630;
#   adjoint step: 4 stages x (the stage's cell and offsets read from the
#     tangent sweep's record, no locate; coefficients of v . mu 7 FMUL +
#     14 FFMA, its gradient 8 FFMA, nu 3 FMUL, the pending block in moment
#     form: offset products 4 FMUL, 3 FADD + 21 FFMA) = 4 x 103, plus
#     bookkeeping 12 FMUL + 9 FFMA + 12 FADD = 42 -> 454.
# The coefficients themselves (13 FADD per component when a stage enters a
# new cell) and the block's conversion from moments to corners (12 FADD per
# component when the cell changes) depend on the data and are not counted;
# ncu's executed counts are in the committed profile.
HESS_FLOPS_PER_VOXEL_STEP = 1084


def algorithmic_flops_hess(wl):
    return HESS_FLOPS_PER_VOXEL_STEP * int(np.prod(wl.image.m)) * wl.rk4_steps


def fp32_peak_tflops(sms):
    """FP32 peak from unit counts and the maximum SM clock: the device's SMs x
    128 FP32 lanes x 2 FLOPs (FMA) x clock."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return sms * 128 * 2 * mhz * 1e6 / 1e12, mhz


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in ("trace_impl.cuh", "fsum.cuh", "trace3d.cu", "lgnk_internal.h"):
        with open(os.path.join(ROOT, "paper_1703_04446_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_counters():
    """Counters of the fused kernel from the committed ncu summary (DRAM bytes
    and warp instructions per launch), or {} when the kernel source has changed
    since that capture."""
    path = os.path.join(ROOT, "profiles", "hess_transport_128.txt")
    vals = {}
    try:
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    except OSError:
        return {}
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return {}
    out = {}
    for key, name in (("traffic", "traffic_bytes_per_launch"), ("warp_inst", "smsp__inst_executed.sum")):
        try:
            out[key] = int(float(vals[name].split()[0]))
        except (KeyError, ValueError, IndexError):
            pass
    return out


def assembled_matvec(ctx, v, T, dv, stream, reps=50):
    """The assembled-J variant on the benchmark workload (outside the timed
    region): assembly time, blocks per voxel, the Hessian matvec through the
    stored rows (whole call and its ELL kernel), and the bytes one ELL HESS
    launch must read at least (counts, keys and blocks of every row, once)."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(2):
        blocks = ctx.assemble(v, T)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(5):
        ctx.assemble(v, T)
    ev[1].record(stream)
    torch.cuda.synchronize()
    asm_ms = ev[0].elapsed_time(ev[1]) / 5
    out = torch.empty_like(dv)
    for _ in range(5):
        ctx.hessvec_assembled(dv, out=out)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        ctx.hessvec_assembled(dv, out=out)
    ev[1].record(stream)
    torch.cuda.synchronize()
    hv_ms = ev[0].elapsed_time(ev[1]) / reps
    ctx.profile(True)
    for _ in range(reps):
        ctx.hessvec_assembled(dv, out=out)
    ell_ms, n_ell, _ = ctx.profile_read()
    ctx.profile(False)
    M = T.numel()
    d = T.dim()
    row_bytes = 4 * M + blocks * (8 + 4 * (2 ** d) * d)
    return {"assemble_ms": asm_ms, "blocks_per_voxel": blocks / M, "hessvec_ms": hv_ms,
            "matvecs_per_s": 1e3 / hv_ms, "ell_kernel_ms": ell_ms / max(n_ell, 1),
            "ell_min_bytes": row_bytes, "ell_min_bytes_gbs": row_bytes / (ell_ms / max(n_ell, 1) * 1e-3) / 1e9}


def other_workloads(dev, names=("2d_continuity_256", "3d_continuity_brain")):
    """Matvec and forward times of the mass-preserving workloads (the continuity
    push-forward and its derivatives), measured outside the timed region."""
    import torch
    from paper_1703_04446_gb300 import lgnk, synth
    out = {}
    stream = torch.cuda.current_stream(dev)
    for name in names:
        ins = synth.make_inputs(name, seed=0)
        wl = ins["workload"]
        ctx = lgnk.Context(lgnk.Problem.from_workload(wl), device=dev)
        dv = synth.random_velocity(wl.velocity, wl.time_nodes, 2 * min(wl.image.h), 5).astype(np.float32)
        tv, tT, tdv = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (ins["v0"], ins["T"], dv))
        res = torch.empty_like(tv)

        def avg_ms(fn, n):
            for _ in range(2):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1) / n

        h_ms = avg_ms(lambda: ctx.hessvec(tv, tT, tdv, res), 10)
        f_ms = avg_ms(lambda: ctx.forward(tv, tT), 10)
        out[name] = {"unknowns": int(tv.numel()), "voxels": int(tT.numel()), "time_nodes": wl.time_nodes,
                     "rk4_steps": wl.rk4_steps, "hessvec_ms": h_ms, "matvecs_per_s": 1000.0 / h_ms,
                     "forward_ms": f_ms,
                     "forward_voxel_steps_per_s": int(tT.numel()) * wl.rk4_steps / (f_ms * 1e-3)}
        ctx.close()
        del tv, tT, tdv, res
    return out


def other_solves(dev, max_gn):
    """Zero-start Gauss-Newton solves of the other workloads to a 1e-3
    gradient-norm drop (outside the timed region; wall time around the call,
    the second of two identical solves so that CUDA-graph capture is not
    counted; the first is reported too).  The 2D intensity-preserving workload
    uses its configured 10 outer / 20 inner iterations; the brain-scale one is
    capped at 5 GN iterations (labelled: a capped solve, not a time to
    solution unless its status is ok)."""
    import torch
    from paper_1703_04446_gb300 import lgnk, synth
    plans = {"2d_transport_64": dict(max_gn=10, max_pcg=20), "2d_continuity_256": dict(max_gn=max_gn, max_pcg=50),
             "3d_continuity_brain": dict(max_gn=5, max_pcg=20)}
    out = {}
    for name, plan in plans.items():
        ins = synth.make_inputs(name, seed=0)
        wl = ins["workload"]
        ctx = lgnk.Context(lgnk.Problem.from_workload(wl), device=dev)
        tT, tR = (torch.from_numpy(ins[k]).to(dev) for k in ("T", "R"))
        times = []
        for _ in range(2):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            _, rep = ctx.solve(tT, tR, None, gn_grad_rtol=1e-3, pcg_rtol=0.1, **plan)
            torch.cuda.synchronize(dev)
            times.append(time.perf_counter() - t0)
        out[name] = {"seconds": times[1], "first_call_seconds": times[0], "gn_iters": rep["gn_iters"],
                     "pcg_iters": rep["pcg_iters"], "grad_ratio": rep["g"] / rep["g0"], "J0": rep["J0"],
                     "J": rep["J"], "status": rep["status_name"], **plan,
                     "kind": "time to solution" if rep["status_name"] == "ok" else "capped solve"}
        ctx.close()
        del tT, tR
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------- CPU oracle --

def _oracle_setup(ins):
    from oracle import lagrangian as L
    from oracle.objective import Problem as OP
    wl = ins["workload"]
    ig = L.Grid(wl.image.m, wl.image.lo, wl.image.hi)
    vg = L.Grid(wl.velocity.m, wl.velocity.lo, wl.velocity.hi)
    op = OP(ig, vg, K=wl.time_nodes, N=wl.rk4_steps, model=wl.model, reg=wl.regularizer, alpha=wl.alpha,
            gamma=wl.gamma)
    return wl, ig, vg, op


def oracle_voxel_terms(ins, idx):
    """The per-voxel terms J_i^T h^d J_i dv of the oracle's Gauss-Newton matvec
    (Sec. 3.2; independent per voxel) for the voxels idx, summed."""
    from oracle import lagrangian as L
    wl, ig, vg, _ = _oracle_setup(ins)
    v = ins["v0"].astype(np.float64)
    dv = ins["dv"].astype(np.float64)
    T = ins["T"].astype(np.float64)
    xc = L.cell_centres(ig)[:, idx]
    y, dy, hist = L.characteristics(v, vg, xc, wl.rk4_steps, -1, dv=dv, keep=True)
    _, gT = L.interpolate(T, ig, y, gradient=True)
    du = np.sum(gT * dy, axis=0)
    return L.characteristics_adjoint(v, vg, hist, wl.rk4_steps, -1, ig.cell_volume * du * gT)


def oracle_regularizer_seconds(ins):
    from oracle.objective import reg_operator
    _, _, _, op = _oracle_setup(ins)
    dv = ins["dv"].astype(np.float64)
    t0 = time.perf_counter()
    op.alpha * reg_operator(op, dv) + op.gamma * dv
    return time.perf_counter() - t0


def _sample(ins, frac, seed):
    M = int(np.prod(ins["workload"].image.m))
    return np.random.default_rng(seed).choice(M, size=max(1, int(frac * M)), replace=False), M


# worker side of the all-cores oracle (a spawn pool: each worker imports numpy
# and the oracle itself and holds the inputs)
_POOL_INS = {}


def _pool_init(ins):
    _POOL_INS["ins"] = ins


def _pool_terms(idx):
    t0 = time.perf_counter()
    oracle_voxel_terms(_POOL_INS["ins"], idx)
    return time.perf_counter() - t0


class OraclePool:
    """The oracle's per-voxel matvec terms spread over `cores` host processes
    (spawned, one numpy thread each), chunks of the voxel sample per process."""

    def __init__(self, ins, cores):
        import multiprocessing as mp
        self.cores = cores
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        self.pool = mp.get_context("spawn").Pool(cores, initializer=_pool_init, initargs=(ins,))
        self.pool.map(_pool_terms, [np.arange(8) for _ in range(cores)])    # imports, warm-up

    def run(self, idx):
        """Wall seconds to compute the terms of voxels idx on all processes."""
        chunks = np.array_split(idx, self.cores * 4)
        t0 = time.perf_counter()
        self.pool.map(_pool_terms, chunks)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_rate(frac, t_char, t_reg):
    """Full matvecs/s: the sampled characteristic work scaled to all voxels plus
    one regularizer."""
    return 1.0 / (t_char / frac + t_reg)


def cpu_baseline(ins, target_s=12.0):
    """The oracle's matvec rate on one host core and on all of them (a bounded
    voxel sample of about target_s seconds each)."""
    idx, M = _sample(ins, 1.0 / 512, 0)
    t0 = time.perf_counter()
    oracle_voxel_terms(ins, idx)
    tc = time.perf_counter() - t0
    frac = len(idx) / M
    if tc < target_s / 4:
        idx, M = _sample(ins, min(1.0, frac * target_s / max(tc, 1e-3)), 1)
        t0 = time.perf_counter()
        oracle_voxel_terms(ins, idx)
        tc = time.perf_counter() - t0
        frac = len(idx) / M
    tr = oracle_regularizer_seconds(ins)
    one = oracle_rate(frac, tc, tr)
    cores = os.cpu_count() or 1
    pool = OraclePool(ins, cores)
    try:
        idx_all, _ = _sample(ins, min(1.0, frac * cores), 2)
        frac_all = len(idx_all) / M
        tc_all = pool.run(idx_all)
    finally:
        pool.close()
    value = oracle_rate(frac_all, tc_all, tr)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 numpy oracle matvec: per-voxel terms of {frac_all * 100:.2f}% of the 128^3 voxels "
                      f"({len(idx_all)} characteristics, N=8) split over {cores} spawned processes "
                      f"(one numpy thread each), {tc_all:.1f} s wall, plus the full-grid regularizer "
                      f"({tr:.2f} s, one core); value = 1 / (sample time / fraction + regularizer time)",
            "one_core": {"value": one, "cores": 1,
                         "sample": f"{frac * 100:.2f}% of the voxels ({int(round(frac * M))} characteristics) "
                                   f"in {tc:.1f} s on one core, plus the regularizer"},
            "nproc": cores}


# ------------------------------------------------------------------- main --

def run_reference(args):
    """The oracle (FP64 numpy, the paper ships no code) on the host cores: each
    step is the per-voxel work of a bounded voxel sample spread over all cores,
    scaled to a full matvec, plus the full-grid regularizer."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    ins = make_problem(seed=0)
    cores = os.cpu_count() or 1
    M = int(np.prod(ins["workload"].image.m))
    frac = min(1.0, cores / 256.0)   # 8192 characteristics per core and step: about 1-2 s of wall time
    tr = oracle_regularizer_seconds(ins)
    pool = OraclePool(ins, cores)
    try:
        for k in range(min(args.warmup, 1)):
            pool.run(_sample(ins, frac / 4, 1000 + k)[0])
        tot_f, tot_c = 0.0, 0.0
        for k in range(args.steps):
            idx, _ = _sample(ins, frac, k)
            tot_c += pool.run(idx)
            tot_f += len(idx) / M
    finally:
        pool.close()
    val = oracle_rate(tot_f, tot_c, tr)
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * (tot_c + args.steps * tr) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "image": [128, 128, 128], "velocity": [64, 64, 64, 3],
                       "rk4_steps": 8, "l2": "n/a (host)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "nproc": cores,
                             "sample": f"{frac * 100:.3f}% of the voxels per step (per-voxel terms of the "
                                       f"Gauss-Newton matvec) over {cores} spawned processes, plus the full-grid "
                                       "regularizer on one core; value = 1 / (sampled time / sampled fraction + "
                                       "regularizer time)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1703_04446_gb300 import lgnk

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ins = make_problem(seed=rank)
    wl = ins["workload"]
    prob = lgnk.Problem.from_workload(wl)
    ctx = lgnk.Context(prob, device=dev)
    tv, tT, tR, tdv = (torch.from_numpy(ins[k]).to(dev) for k in ("v0", "T", "R", "dv"))
    out = torch.empty_like(tv)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        ctx.hessvec(tv, tT, tdv, out)
    barrier()

    # timed region: K matvecs, each between CUDA events; L2 flushed between them
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ctx.profile(True)
    with ClockSampler(local) as clk:
        barrier()
        clk.mark(True)
        for k in range(args.steps):
            flush.fill_(float(k))
            starts[k].record(stream)
            ctx.hessvec(tv, tT, tdv, out)
            ends[k].record(stream)
        barrier()
        clk.mark(False)
    kern_ms, kern_n, launches = ctx.profile_read()
    ctx.profile(False)
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    step_ms = max_over_ranks(step_ms, world, dev)
    value = job_throughput(step_ms, world)

    # end to end through the public call: every step copies its inputs (v, T, dv)
    # from pinned host memory and reads its result back.  The inputs are
    # double-buffered on the device, so step i+1's uploads (one stream) and
    # step i-1's read-back (another) run under step i's matvec.
    hin = [torch.from_numpy(ins[k]).pin_memory() for k in ("v0", "T", "dv")]
    hout = [torch.empty(tv.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    din = [[torch.empty(h.shape, dtype=h.dtype, device=dev) for h in hin] for _ in range(2)]
    dout = [torch.empty(tv.shape, dtype=torch.float32, device=dev) for _ in range(2)]
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    loaded, computed, fetched = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))

    def upload(i):
        b = i % 2
        with torch.cuda.stream(up):
            if i >= 2:
                up.wait_event(computed[b])          # step i - 2 is done with these buffers
            for d, h in zip(din[b], hin):
                d.copy_(h, non_blocking=True)
            loaded[b].record(up)

    def step(i):
        b = i % 2
        stream.wait_event(loaded[b])
        if i >= 2:
            stream.wait_event(fetched[b])           # step i - 2's result has been read back
        ctx.hessvec(din[b][0], din[b][1], din[b][2], dout[b])
        computed[b].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(computed[b])
            hout[b].copy_(dout[b], non_blocking=True)
            fetched[b].record(down)

    def e2e_run(steps):
        up.wait_stream(stream)                      # the first upload starts after what precedes it
        upload(0)
        for i in range(steps):
            if i + 1 < steps:
                upload(i + 1)
            step(i)
        stream.wait_stream(down)

    e2e_run(3)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)

    # extras outside the timed region: forward throughput, time-to-solution
    fwd_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(3):
        ctx.forward(tv, tT)
    fwd_ev[0].record(stream)
    for _ in range(10):
        ctx.forward(tv, tT)
    fwd_ev[1].record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = fwd_ev[0].elapsed_time(fwd_ev[1]) / 10
    voxel_steps = int(np.prod(wl.image.m)) * wl.rk4_steps
    # objective + gradient (SSD, J^T of the residual, regularizer) on the same problem
    og_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(2):
        ctx.objective(tv, tT, tR, grad=True)
    og_ev[0].record(stream)
    for _ in range(10):
        ctx.objective(tv, tT, tR, grad=True)
    og_ev[1].record(stream)
    torch.cuda.synchronize(dev)
    objgrad_ms = og_ev[0].elapsed_time(og_ev[1]) / 10
    asm = assembled_matvec(ctx, tv, tT, tdv, stream)
    others = {} if args.no_other_workloads else other_workloads(dev)
    warm = None
    if args.warm_start:
        # learned warm start: 2048 solver-generated 128^2 training pairs, 256
        # held-out pairs (under a minute with the tensor-core convolutions)
        from paper_1703_04446_gb300 import warmstart
        warm = warmstart.run()
        warm["conv_peak_tflops"] = {"bf16": _bf16_peak(), "kind": "measured cuBLAS bf16 (burst)"}
    tts = None
    if not args.no_solve:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, rep = ctx.solve(tT, tR, None, max_gn=args.max_gn, gn_grad_rtol=1e-3, max_pcg=50, pcg_rtol=0.1)
        torch.cuda.synchronize(dev)
        rep_g0 = rep["g0"]
        tts = {"seconds": time.perf_counter() - t0, "gn_iters": rep["gn_iters"], "pcg_iters": rep["pcg_iters"],
               "hessvecs": rep["hessvecs"], "grad_ratio": rep["g"] / rep["g0"], "J0": rep["J0"], "J": rep["J"],
               "status": rep["status_name"], "max_gn": args.max_gn, "matvec": "assembled",
               "assembled_gn": rep["assembled_gn"]}
        # the same solve with the matrix-free products in every PCG iteration
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, rep = ctx.solve(tT, tR, None, max_gn=args.max_gn, gn_grad_rtol=1e-3, max_pcg=50, pcg_rtol=0.1, matvec=0)
        torch.cuda.synchronize(dev)
        tts["matrix_free"] = {"seconds": time.perf_counter() - t0, "gn_iters": rep["gn_iters"],
                              "pcg_iters": rep["pcg_iters"], "grad_ratio": rep["g"] / rep["g0"], "J": rep["J"],
                              "status": rep["status_name"]}
        # the paper's setting: multilevel continuation (3 levels, 32^3 / 64^3 / 128^3 images), stopped on
        # the finest level at the same gradient norm as the solve above, 1e-3 |g(v = 0)| (a level also stops
        # at 1e-3 of its own starting gradient, which ends the coarse levels)
        g_zero = rep_g0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        # (twice the single-level cap: from the coarse levels' minimum the finest level needs about 40 steps)
        _, reps = lgnk.lgnk_solve_multilevel(prob, tT, tR, 3, max_gn=2 * args.max_gn, gn_grad_rtol=1e-3, max_pcg=50,
                                             pcg_rtol=0.1, gn_grad_atol=1e-3 * g_zero)
        torch.cuda.synchronize(dev)
        tts["multilevel_3"] = {"seconds": time.perf_counter() - t0,
                               "level_seconds": [r["seconds"] for r in reps],
                               "gn_iters": [r["gn_iters"] for r in reps], "pcg_iters": [r["pcg_iters"] for r in reps],
                               "finest_grad_ratio": reps[-1]["g"] / reps[-1]["g0"],
                               "grad_over_zero_start_grad": reps[-1]["g"] / g_zero, "J": reps[-1]["J"],
                               "status": reps[-1]["status_name"]}
        tts["other_workloads"] = other_solves(dev, args.max_gn)

    if rank != 0:
        return
    hbm_peak, peak_kind = _peaks()
    kern_avg_ms = kern_ms / max(kern_n, 1)
    alg = algorithmic_bytes_hess(wl)
    flops = algorithmic_flops_hess(wl)
    achieved = flops / (kern_avg_ms * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_mhz = fp32_peak_tflops(sms)
    prof = profiled_counters()
    traffic = prof.get("traffic")
    n = int(tv.numel())
    M = int(tT.numel())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "image": list(wl.image.m), "velocity": list(wl.velocity.m) + [3],
                   "time_nodes": wl.time_nodes, "rk4_steps": wl.rk4_steps, "unknowns": n,
                   "regularizer": wl.regularizer, "l2": "flushed between timed steps (512 MiB write, untimed)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": job_throughput(e2e_ms, world), "unit": UNIT, "h2d_bytes_per_step": 4 * (2 * n + M),
                "d2h_bytes_per_step": 4 * n},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "trace_kernel<3,stat,transport,HESS>",
                     "kernel_ms": kern_avg_ms, "flops_per_launch": flops,
                     "peak_kind": f"FP32 from {sms} SMs (device count) x 128 lanes x 2 x max SM clock "
                                  f"{peak_mhz:.0f} MHz", "sms": sms,
                     "hbm": {"algorithmic_bytes": alg, "achieved_gbs": alg / (kern_avg_ms * 1e-3) / 1e9,
                             "peak_gbs": hbm_peak, "frac": alg / (kern_avg_ms * 1e-3) / 1e9 / hbm_peak,
                             "peak_kind": peak_kind},
                     # the kernel is bound by instruction issue: warp instructions (one ncu capture)
                     # per launch over its live time, against 4 issue slots per SM and clock
                     "issue": None if "warp_inst" not in prof else {
                         "warp_inst_per_launch": prof["warp_inst"],
                         "achieved_ginst_s": prof["warp_inst"] / (kern_avg_ms * 1e-3) / 1e9,
                         "peak_ginst_s": sms * 4 * peak_mhz * 1e6 / 1e9,
                         "frac": prof["warp_inst"] / (kern_avg_ms * 1e-3) / (sms * 4 * peak_mhz * 1e6)}},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "extra": {"forward_voxel_steps_per_s": voxel_steps / (fwd_ms * 1e-3), "forward_ms": fwd_ms,
                  "objective_gradient_ms": objgrad_ms, "time_to_solution": tts, "assembled": asm, "other_workloads": others,
                  **({"warm_start": warm} if warm is not None else {})},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ins)
    print(json.dumps(line), flush=True)


def profile_case(args):
    """A short fixed invocation of one kernel for ncu captures: an S^3
    transport image (the benchmark's ellipsoid phantom), an (S/2)^3
    stationary velocity, N = 8, alpha = 1e-2.  'hess' launches the fused
    matrix-free matvec `launches` times; 'ell' assembles J once and then
    launches the assembled matvec `launches` times; 'solve' runs `launches`
    Gauss-Newton iterations (every kernel of the solver); 'cont' launches the
    mass-preserving matvec (9 time nodes, N = 16, as the brain-scale workload)
    `launches` times."""
    import torch
    from paper_1703_04446_gb300 import lgnk, synth
    if args.profile_case == "ws":
        # the warm-start network (c = 32) on a batch of 32 pairs of S^2 images: `launches`
        # predictions (each 7 convolution GEMMs), then `launches` training steps
        S, c, B = args.size, 32, 32
        net = lgnk.WarmStart(S, c, B, 0.05)
        net.set_params(torch.from_numpy(synth.warmstart_init(c, 0)))
        rng = np.random.default_rng(0)
        T, R = (torch.from_numpy(rng.uniform(size=(B, S, S)).astype(np.float32)).cuda() for _ in range(2))
        vt = torch.from_numpy((0.05 * rng.normal(size=(B, 2, S // 2, S // 2))).astype(np.float32)).cuda()
        for _ in range(args.launches):
            v = net.predict(T, R)
        for _ in range(args.launches):
            net.train_step(T, R, vt, 1e-4, return_loss=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "ws", "size": S, "launches": args.launches,
                          "checksum": float(v.double().abs().sum())}))
        return
    S = args.size
    lo, hi = (0.0,) * 3, (1.0,) * 3
    ig = synth.GridSpec((S,) * 3, lo, hi)
    vg = synth.GridSpec((S // 2,) * 3, lo, hi)
    T = synth.ellipsoid_phantom(synth.centres(ig), np.random.default_rng(0), lo, hi).astype(np.float32)
    h = 1.0 / S
    v = synth.random_velocity(vg, 1, 8 * h, 7).astype(np.float32)
    dv = synth.random_velocity(vg, 1, 2 * h, 5).astype(np.float32)
    prob = lgnk.Problem(image_m=(S,) * 3, velocity_m=(S // 2,) * 3, time_nodes=1, rk4_steps=8, alpha=1e-2)
    ctx = lgnk.Context(prob)
    tv, tT, tdv = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (v, T, dv))
    out = torch.empty_like(tdv)
    if args.profile_case == "ell":
        ctx.assemble(tv, tT)
        for _ in range(args.launches):
            ctx.hessvec_assembled(tdv, out=out)
    elif args.profile_case == "cont":
        # the mass-preserving matvec on the shape of the brain-scale workload's grids (9 time nodes, N = 16)
        cprob = lgnk.Problem(image_m=(S,) * 3, velocity_m=(S // 2,) * 3, time_nodes=9, rk4_steps=16,
                             model="continuity", alpha=1e-3)
        cctx = lgnk.Context(cprob)
        cv = torch.from_numpy(synth.random_velocity(vg, 9, 6 * h, 7).astype(np.float32)).cuda()
        cdv = torch.from_numpy(synth.random_velocity(vg, 9, 2 * h, 5).astype(np.float32)).cuda()
        rho = (tT / tT.sum()).contiguous()
        cout = torch.empty_like(cdv)
        for _ in range(args.launches):
            cctx.hessvec(cv, rho, cdv, cout)
        out = cout
    elif args.profile_case == "solve":
        # `launches` Gauss-Newton iterations from v = 0 towards the phantom moved by v, with
        # direct launches (profiling mode: no CUDA graphs) so that a profiler sees every PCG kernel
        R = ctx.forward(tv, tT)
        ctx.profile(True)
        _, rep = ctx.solve(tT, R, None, max_gn=args.launches, gn_grad_rtol=1e-3, max_pcg=50, pcg_rtol=0.1)
        out.copy_(tdv)
        print(json.dumps({k: rep[k] for k in ("gn_iters", "pcg_iters", "hessvecs", "seconds")}))
    else:
        for _ in range(args.launches):
            ctx.hessvec(tv, tT, tdv, out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "size": S, "launches": args.launches,
                      "checksum": float(out.double().abs().sum())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lgnk", choices=["lgnk", "reference"])
    ap.add_argument("--max-gn", type=int, default=30)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true")
    ap.add_argument("--profile-case", choices=["hess", "ell", "solve", "cont", "ws"], default=None,
                    help="run only a short fixed invocation of one kernel (for ncu captures)")
    ap.add_argument("--size", type=int, default=128, help="image cells per axis of --profile-case")
    ap.add_argument("--launches", type=int, default=3, help="kernel launches of --profile-case")
    ap.add_argument("--no-warm-start", dest="warm_start", action="store_false",
                    help="skip training and evaluating the learned warm start (2D 128^2 pairs, under a minute)")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
