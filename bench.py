"""Benchmark of BRMerge SpGEMM on one GB300 (or N, one independent product per GPU).

Headline workload: C = A*A, A the R-MAT graph of scale 20 (n = 2^20, edge
factor 16, quadrant probabilities (0.57, 0.19, 0.19, 0.05), duplicates
removed), FP64 values U[-1,1), seeded (synthetic: the paper's SuiteSparse
matrices are not used).  It is the largest configuration that runs on one
GPU: ~20.9e9 intermediate products, nnz(C) ~9.7e9, C ~116 GB.  One step is one
whole BRMerge-Precise call (product counts + binning, symbolic pass, prefix
sum, allocation of C, numeric pass) on inputs already resident in HBM.  The
output (116 GB) is far larger than the 129 MB L2, so no explicit L2 flush is
needed between steps.

Metric (the paper's, Section IV-A): GFLOP/s = 2 * intermediate products / s.

Printed: one JSON line with the value (device-timed, all ranks), e2e (the
same call with host buffers: A copied in from pinned host memory and all of
C copied back every step), the roofline of the dominant kernel (the column
tiles of the long rows' numeric pass, k_long_tile, timed live with CUDA events
that the library records on its launch stream), clocks sampled with nvidia-smi during the timed
region, a cpu_baseline (the CPU oracle on a bounded sample of rows, on all
host cores and on one), and under "also" the other configurations measured in
the same run: the Erdos-Renyi product, the FP32 and FP32+TwoSum paths of the
R-MAT product with their error against the FP64 oracle, the 512-product batch
against 512 single calls, and the differentiable form's forward and backward.

``--impl reference`` times the CPU oracle itself (the only reference that
exists for this method) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2206_06611_gb300 import inputs as I  # noqa: E402

METRIC = "SpGEMM GFLOP/s (2*products/s)"
UNIT = "GFLOP/s"

# Row bins of the default options (include/brm.h): rows with more than this
# many products, or more lists, are the long rows.
BLOCK_MAX_NPROD = 4096
BLOCK_MAX_L = 1024

# DRAM bytes (read + write) of one launch of the dominant kernel, from an ncu
# capture of the current source of that kernel (dram__bytes_read.sum +
# dram__bytes_write.sum), or None when the kernel changed after the capture:
# numeric_tile -- k_long_tile<PF64> on the R-MAT scale 20 workload itself (a
# one-pass capture of those two counters); numeric_reg -- k_rows_perm<PF64,
# 32, 8> on the ER workload itself.
TRAFFIC = {"numeric_tile": 47356340736 + 66491058944, "numeric_reg": 3.900762e9 + 3.183467e9}

# Long rows that take the column tiles by default (include/brm.h, option
# long_window): at most this many lists and at least this many products.
TILE_MAX_L = 2048
TILE_MIN_NPROD = 65536


def workload_name(scale: int) -> str:
    return f"R-MAT scale {scale} ef16 (0.57,0.19,0.19,0.05) dedup, C=A*A, FP64, BRMerge-Precise"


ER_WORKLOAD = "ER n=2^20, 16 nnz/row, C=A*A, FP64, BRMerge-Precise"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def reduce_max(x: float, dist, device) -> float:
    """x maximised over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(products_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job GFLOP/s: every rank does its own product (weak scaling); the
    slowest rank's time counts."""
    return world * 2.0 * products_per_rank * steps / (ms_max * 1e-3) / 1e9


def rank_seed(rank: int) -> int:
    """Each rank multiplies its own independent matrix (no data-path collective)."""
    return I.DEFAULT_SEED + rank


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def check_world(args, world: int):
    """--gpus must agree with the launch: N > 1 runs under torchrun with N ranks."""
    if args.gpus != world:
        raise SystemExit(f"--gpus {args.gpus} but {world} rank(s) were launched; run N > 1 as "
                         f"python -m torch.distributed.run --nproc-per-node {args.gpus} bench.py --gpus {args.gpus}")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index: int):
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(dev_index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes (compulsory traffic) of the numeric pass over some rows
# ---------------------------------------------------------------------------
def numeric_bytes(A, B, rows_mask, row_nnz_c, vbytes):
    """A's rows once (row_ptr entries, columns, values), the B rows they name
    once (two row_ptr entries, columns, values), C's row_ptr entries read and
    its columns and values written once -- for the rows in rows_mask."""
    alen = np.diff(A.rp.astype(np.int64))
    blen = np.diff(B.rp.astype(np.int64))
    rows = np.nonzero(rows_mask)[0]
    ents = np.repeat(rows_mask, alen)
    touched = np.zeros(B.rows, dtype=bool)
    touched[A.col[ents]] = True
    a_bytes = len(rows) * 4 + int(alen[rows].sum()) * (4 + vbytes)
    b_bytes = int(touched.sum()) * 2 * 4 + int(blen[touched].sum()) * (4 + vbytes)
    c_bytes = len(rows) * 8 + int(row_nnz_c[rows].sum()) * (4 + vbytes)
    return a_bytes + b_bytes + c_bytes


def long_rows_mask(A, nprod):
    L = np.diff(A.rp.astype(np.int64))
    return (nprod > 0) & ((nprod > BLOCK_MAX_NPROD) | (L > BLOCK_MAX_L))


def tile_rows_mask(A, nprod):
    """The long rows of the column tiles under the default options."""
    L = np.diff(A.rp.astype(np.int64))
    return long_rows_mask(A, nprod) & (L <= TILE_MAX_L) & (nprod >= TILE_MIN_NPROD)


def roofline(trace, phase, alg_bytes, traffic_key):
    k_ms, k_launch = trace.get(phase, (0.0, 0))
    if not k_launch:
        return None
    per_launch_ms = k_ms / k_launch
    peak, peak_kind = peaks()
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": phase, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "traffic": TRAFFIC.get(traffic_key),
            "algorithmic_bytes": alg_bytes, "kernel_ms": per_launch_ms, "launches_per_step": k_launch}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def sample_rows(nprod, budget_products: int, seed: int):
    """Seeded random rows (without replacement, in increasing order) whose
    products add up to about budget_products."""
    order = np.argsort(I.rand_u64(seed, 77, np.arange(len(nprod))), kind="stable")
    cum = np.cumsum(nprod[order])
    k = int(np.searchsorted(cum, budget_products)) + 1
    return np.sort(order[:max(1, min(k, len(order)))]).astype(np.int64)


def oracle_rate(A, nprod, target_s: float, threads: int, seed: int):
    """GFLOP/s of the oracle's Gustavson (row-parallel over nprod-balanced
    groups) on a seeded row sample sized for about target_s seconds."""
    import oracle
    oracle.build()
    rows = sample_rows(nprod, int(2e6) * threads, seed)
    t0 = time.perf_counter()
    oracle.gustavson_parallel(A, A, threads, rows)
    dt = max(time.perf_counter() - t0, 1e-6)
    rate = nprod[rows].sum() / dt
    rows = sample_rows(nprod, int(rate * target_s), seed + 1)
    t0 = time.perf_counter()
    oracle.gustavson_parallel(A, A, threads, rows)
    dt = time.perf_counter() - t0
    return 2.0 * float(nprod[rows].sum()) / dt / 1e9, dt, len(rows), int(nprod[rows].sum())


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    A = I.rmat(args.scale, 16)
    nprod = oracle.row_nprod(A, A)
    threads = os.cpu_count() or 1
    for w in range(args.warmup):
        oracle_rate(A, nprod, 1.0, threads, 1000 + w)
    vals, secs, info = [], [], None
    for s in range(args.steps):
        v, dt, nrows, npr = oracle_rate(A, nprod, 6.0, threads, 2000 + s)
        vals.append(v)
        secs.append(dt)
        info = (nrows, npr)
    value = float(np.mean(vals))
    sample = (f"per step ~{info[0]} seeded random rows of {A.rows} ({info[1]:.3g} of {int(nprod.sum()):.3g} "
              f"products) of A*A, Gustavson FP64 on {threads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.scale), "n": A.rows, "nnz_A": A.nnz, "nprod": int(nprod.sum()),
                   "global_batch": 1, "parallelism": "cpu oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# timing helpers
# ---------------------------------------------------------------------------
def _timed(fn, steps, warmup):
    """Milliseconds per call of fn (CUDA events on the current stream)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _traced(fn, steps, warmup):
    """(ms per call, {phase: (ms per call, launches per call)})."""
    from paper_2206_06611_gb300 import brm
    for _ in range(warmup):
        fn()
    brm.brm_trace_reset()
    brm.brm_trace_enable(True)
    ms = _timed(fn, steps, 0)
    t = brm.brm_trace_read()
    brm.brm_trace_enable(False)
    return ms, {k: (v[0] / steps, v[1] / steps) for k, v in t.items() if v[1]}


def _rows_to_host(C, rows):
    """(row_ptr, col, val) of the given rows of a device result."""
    import torch
    rp = C.rp.cpu().numpy()
    starts, ends = rp[rows], rp[rows + 1]
    idx = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)]) if len(rows) else np.zeros(0, np.int64)
    it = torch.from_numpy(idx).to(C.col.device)
    crp = np.zeros(len(rows) + 1, dtype=np.int64)
    crp[1:] = np.cumsum(ends - starts)
    return crp, C.col[it].cpu().numpy(), C.val[it].cpu().numpy().astype(np.float64)


def _row_err(crp, val, ref):
    d = (val - ref.val) ** 2
    cs, ca = np.concatenate(([0.0], np.cumsum(d))), np.concatenate(([0.0], np.cumsum(ref.abs ** 2)))
    num = np.sqrt(np.maximum(cs[crp[1:]] - cs[crp[:-1]], 0))
    den = np.sqrt(np.maximum(ca[crp[1:]] - ca[crp[:-1]], 0))
    return np.where(den > 0, num / np.where(den > 0, den, 1), 0)


# ---------------------------------------------------------------------------
# GPU arm: the headline line
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    from paper_2206_06611_gb300 import brm
    import oracle

    rank, world, local = dist_env()
    check_world(args, world)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    brm.load()

    def barrier():
        if dist is not None:
            dist.barrier()

    # every rank multiplies its own independent matrix (weak scaling), or
    # with --shard the ranks share one product by the static row split
    # (strong scaling: each rank its rows of C, B whole on every rank, one
    # all-gather of the ranks' nnz per step)
    shard = args.shard and world > 1
    seed = I.DEFAULT_SEED if shard else rank_seed(rank)
    if args.workload == "er":
        A = I.erdos_renyi(1 << 20, 16, seed=seed)
        wname = ER_WORKLOAD
        phase = "numeric_reg"
    else:
        A = I.rmat(args.scale, 16, seed=seed)
        wname = workload_name(args.scale)
        phase = "numeric_tile"
    vbytes = 8
    nprod = oracle.row_nprod(A, A)
    nprod_total = int(nprod.sum())
    dA = brm.to_device(A, device=f"cuda:{dev}")
    st = torch.cuda.current_stream()
    if shard:
        bounds = brm.brm_row_split(dA, dA, world)
        r0, r1 = bounds[rank], bounds[rank + 1]
        dL = brm.row_slice(dA, r0, r1)
    else:
        r0, r1 = 0, A.rows
        dL = dA

    def step(left):
        Cx = brm.brm_spgemm_precise(left, dA if shard else left)
        if shard:
            brm.global_row_offset(Cx.nnz, None, Cx.rp.device)
        return Cx

    def value_of(ms_total, nsteps):
        # whole-job GFLOP/s: weak -- every rank its own product; strong -- one product
        return job_gflops(nprod_total, 1 if shard else world, nsteps, ms_total)

    # warm-up (also gives the result's row lengths)
    C = None
    for _ in range(args.warmup):
        C = step(dL)
    torch.cuda.synchronize()
    row_nnz = np.zeros(A.rows, dtype=np.int64)
    row_nnz[r0:r1] = np.diff(C.rp.cpu().numpy())
    nnz_c = C.nnz
    del C
    torch.cuda.empty_cache()

    # ---- device-resident timed region --------------------------------------
    clocks = Clocks(dev) if rank == 0 else None
    brm.brm_trace_reset()
    brm.brm_trace_enable(True)
    launches0 = brm.brm_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        C = step(dL)
        del C
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = (brm.brm_kernel_launches() - launches0) / args.steps
    trace = brm.brm_trace_read()
    brm.brm_trace_enable(False)
    clk = clocks.stop() if clocks else None
    ms_max = reduce_max(ms, dist, f"cuda:{dev}")
    value = value_of(ms_max, args.steps)

    # ---- end to end: host buffers, copies inside the timed region ----------
    # the step's inputs come in from pinned host memory every step (A, or
    # this rank's rows of A and the whole B); all of the step's C goes back
    # to the host every step, through two pinned staging buffers used in
    # turn (C is larger than is sensible to pin at once)
    s0, s1 = int(A.rp[r0]), int(A.rp[r1])
    host_in = [("rp", (A.rp[r0:r1 + 1].astype(np.int64) - s0).astype(np.int32)), ("col", A.col[s0:s1]),
               ("val", A.val[s0:s1])]
    if shard:
        host_in += [("brp", A.rp.astype(np.int32)), ("bcol", A.col.astype(np.int32)), ("bval", A.val)]
    hA = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in host_in}
    dIn = {k: torch.empty_like(v, device=f"cuda:{dev}") for k, v in hA.items()}
    h2d = sum(t.numel() * t.element_size() for t in hA.values())
    stage_bytes = 1 << 30
    stages = [torch.empty(stage_bytes, dtype=torch.uint8).pin_memory() for _ in range(2)]
    d2h = (r1 - r0 + 1) * 8 + nnz_c * (4 + vbytes)
    dL2 = brm.DeviceCSR(r1 - r0, A.cols, dIn["rp"], dIn["col"], dIn["val"])
    dB2 = brm.DeviceCSR(A.rows, A.cols, dIn["brp"], dIn["bcol"], dIn["bval"]) if shard else dL2

    def copy_out(t, k):
        b = t.view(torch.uint8).reshape(-1)
        for o in range(0, b.numel(), stage_bytes):
            n = min(stage_bytes, b.numel() - o)
            stages[k % 2][:n].copy_(b[o:o + n], non_blocking=True)
            k += 1
        return k

    e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(st)
    for _ in range(e_steps):
        for k in hA:
            dIn[k].copy_(hA[k], non_blocking=True)
        C = brm.brm_spgemm_precise(dL2, dB2)
        if shard:
            brm.global_row_offset(C.nnz, None, C.rp.device)
        k = copy_out(C.rp, 0)
        k = copy_out(C.col, k)
        copy_out(C.val, k)
        del C
    f1.record(st)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    barrier()
    e2e_ms = reduce_max(e2e_ms, dist, f"cuda:{dev}")
    e2e_value = value_of(e2e_ms, e_steps)
    del stages, hA, dIn, dL2, dB2
    torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ------------------------------------
    if phase == "numeric_tile":
        mask = tile_rows_mask(A, nprod)
    else:
        L = np.diff(A.rp.astype(np.int64))
        mask = (nprod > 0) & (nprod <= 1024) & (L <= 256)
    mask[:r0] = False        # this rank's rows (all of them without --shard)
    mask[r1:] = False
    per_step = {k: (v[0] / args.steps, v[1] / args.steps) for k, v in trace.items() if v[1]}
    # the traffic figures are for the workloads the captures scaled to
    tkey = phase if not shard and (args.workload == "er" or args.scale == 20) else None
    roof = roofline(per_step, phase, numeric_bytes(A, A, mask, row_nnz, vbytes), tkey)
    phases = {k: round(v[0], 4) for k, v in per_step.items()}

    # ---- CPU oracle on bounded samples ---------------------------------------
    cpu = None
    if not args.no_cpu and world == 1:
        threads = os.cpu_count() or 1
        v, dt, nrows, npr = oracle_rate(A, nprod, args.cpu_seconds, threads, 11)
        v1, dt1, nrows1, npr1 = oracle_rate(A, nprod, args.cpu_seconds / 3, 1, 12)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{nrows} seeded random rows of {A.rows} ({npr:.3g} products) of A*A, Gustavson FP64, "
                         f"{dt:.1f} s on {threads} threads",
               "value_1core": v1,
               "sample_1core": f"{nrows1} seeded random rows ({npr1:.3g} products), {dt1:.1f} s on 1 thread",
               "cpu_model": cpu_model()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "n": A.rows, "nnz_A": A.nnz, "nprod": nprod_total, "nnz_C": nnz_c,
                   "global_batch": 1 if shard else world,
                   "parallelism": (f"row split of one product over {world} GPUs" if shard
                                   else f"independent products x{world}"),
                   "l2": "output larger than L2 every step; no flush"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e_steps},
        "gpu_launches": launches,
        "roofline": roof,
        "phases_ms_per_step": phases,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    if world == 1 and not args.headline_only:
        also = {}
        if args.workload != "er":
            also["er"] = _guard(extra_er, args)
            also["rmat_precision"] = _guard(extra_rmat_precision, args, A, nprod, ms_max / args.steps)
            also["rmat_symbolic"] = _guard(extra_symbolic, args, A)
        also["batched"] = _guard(extra_batched, args)
        also["differentiable"] = _guard(extra_diff, args)
        line["also"] = also
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _guard(fn, *a):
    import torch
    try:
        return fn(*a)
    except Exception as e:  # a failing extra must not hide the headline
        return {"error": f"{type(e).__name__}: {e}"}
    finally:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# the other configurations (the "also" block)
# ---------------------------------------------------------------------------
def extra_er(args):
    """Erdos-Renyi n = 2^20, 16 per row: GFLOP/s and the numeric register
    kernel's roofline."""
    from paper_2206_06611_gb300 import brm
    import oracle
    A = I.erdos_renyi(1 << 20, 16)
    nprod = oracle.row_nprod(A, A)
    dA = brm.to_device(A)
    C = brm.brm_spgemm_precise(dA, dA)
    row_nnz = np.diff(C.rp.cpu().numpy())
    del C
    ms, tr = _traced(lambda: brm.brm_spgemm_precise(dA, dA), max(args.steps, 20), 3)
    L = np.diff(A.rp.astype(np.int64))
    mask = (nprod > 0) & (nprod <= 1024) & (L <= 256)
    return {"workload": ER_WORKLOAD, "ms_per_step": ms, "gflops": 2.0 * nprod.sum() / (ms * 1e-3) / 1e9,
            "roofline": roofline(tr, "numeric_reg", numeric_bytes(A, A, mask, row_nnz, 8), "numeric_reg"),
            "phases_ms": {k: round(v[0], 4) for k, v in tr.items()}}


def extra_rmat_precision(args, A, nprod, ms_f64):
    """The same R-MAT product with FP32 values, plain and TwoSum-compensated:
    time, speedup over the FP64 headline, and per-row error (normwise, scaled
    by |A||B|) against the FP64 oracle on 400 sampled rows, the 100 longest
    among them."""
    import torch
    from paper_2206_06611_gb300 import brm
    import oracle
    top = np.argsort(-nprod, kind="stable")[:100]
    rows = np.unique(np.concatenate([top, I.rand_below(17, 30, np.arange(300), A.rows)]))
    Af = A.astype(np.float32)
    A64 = I.CSR(A.rows, A.cols, A.rp, A.col, Af.val.astype(np.float64))
    ref = oracle.gustavson_parallel(A64, A64, os.cpu_count() or 1, rows, with_abs=True)
    out = {}
    for name, comp in (("f32", False), ("f32_twosum", True)):
        dA = brm.to_device(Af)
        C = brm.brm_spgemm_precise(dA, dA, compensated=comp)
        crp, col, val = _rows_to_host(C, rows)
        assert np.array_equal(col, ref.col), "structure differs from the oracle"
        err = _row_err(crp, val, ref)
        del C
        torch.cuda.empty_cache()
        steps = max(2, min(args.steps, 5))
        ms, tr = _traced(lambda: brm.brm_spgemm_precise(dA, dA, compensated=comp), steps, 1)
        out[name] = {"ms_per_step": ms, "gflops": 2.0 * nprod.sum() / (ms * 1e-3) / 1e9,
                     "speedup_vs_f64": ms_f64 / ms,
                     "row_err_vs_f64_oracle": {"max": float(err.max()), "median": float(np.median(err)),
                                               "rows": int(len(rows))},
                     "phases_ms": {k: round(v[0], 3) for k, v in tr.items()}}
        del dA
        torch.cuda.empty_cache()
    return out


def extra_symbolic(args, A):
    """The symbolic pass of the same R-MAT product by sorting (default) and by
    the paper's hashing (option symbolic_hash): per-phase device times."""
    from paper_2206_06611_gb300 import brm
    dA = brm.to_device(A)
    out = {}
    for name, h in (("sort", False), ("hash", True)):
        ms, tr = _traced(lambda: brm.brm_spgemm_symbolic(dA, dA, symbolic_hash=h), max(2, min(args.steps, 5)), 1)
        out[name] = {"ms_per_call": ms, "phases_ms": {k: round(v[0], 3) for k, v in tr.items()}}
    return out


def extra_batched(args):
    """512 uneven products: one batched call vs 512 single calls, the numeric
    pass replayed from a CUDA graph, autotuned bins; FP64 and FP32."""
    import torch
    from paper_2206_06611_gb300 import brm
    import oracle
    out = {"workload": "batched: 512 products A_i*A_i, n_i log-uniform in [1e3, 2e5], half 3-D Laplacian, "
                       "half ER with 4..32 per row"}
    mats64 = I.batched_mix(512)
    total = int(sum(oracle.row_nprod(M, M).sum() for M in mats64))
    for name, dtype in (("f64", np.float64), ("f32", np.float32)):
        dev = [brm.to_device(M.astype(dtype)) for M in mats64]
        gf = lambda ms: 2.0 * total / (ms * 1e-3) / 1e9  # noqa: E731

        def batched():
            C, _ = brm.brm_spgemm_batched(dev, dev)
            del C

        def separate():
            for d in dev:
                C = brm.brm_spgemm_precise(d, d)
                del C

        r = {"nprod": total}
        r["separate_ms"] = _timed(separate, 3, 1)
        r["batched_ms"] = _timed(batched, 5, 2)
        opts, tune_ms = brm.brm_autotune(dev, dev)
        r["autotuned"] = {k: opts[k] for k in ("reg_keys", "reg_warps", "warp_max_nprod", "block_max_nprod",
                                                "reg_max_nprod")}
        r["autotune_best_ms"] = tune_ms

        def batched_tuned():
            C, _ = brm.brm_spgemm_batched(dev, dev, **opts)
            del C

        r["batched_tuned_ms"] = _timed(batched_tuned, 5, 2)
        b = brm.Batch(dev, dev, **opts)
        r["numeric_graph_ms"] = _timed(b.graph_launch, 5, 2)
        r["numeric_launch_ms"] = _timed(b.numeric, 5, 2)
        b.check()
        b.close()
        for k in ("separate_ms", "batched_ms", "batched_tuned_ms"):
            r[k.replace("_ms", "_gflops")] = gf(r[k])
        r["speedup_batched_vs_separate"] = r["separate_ms"] / r["batched_tuned_ms"]
        out[name] = r
        del dev
        torch.cuda.empty_cache()
    return out


def extra_diff(args):
    """Differentiable C = A*B (A R-MAT scale 18 ef16, B ER 2^18 with 8 per row,
    FP32 N(0,1)): forward, hand-written backward, and the FP64 plain forward."""
    import torch
    from paper_2206_06611_gb300 import brm
    import oracle
    A = I.normal_values(I.rmat(18, 16), 101)
    B = I.normal_values(I.erdos_renyi(1 << 18, 8), 102)
    total = int(oracle.row_nprod(A, B).sum())
    dA, dB = brm.to_device(A), brm.to_device(B)
    a_val = dA.val.clone().requires_grad_(True)
    b_val = dB.val.clone().requires_grad_(True)
    Aq = brm.DeviceCSR(A.rows, A.cols, dA.rp, dA.col, a_val)
    Bq = brm.DeviceCSR(B.rows, B.cols, dB.rp, dB.col, b_val)
    C = brm.spgemm(Aq, Bq)
    G = torch.from_numpy(I.rand_normal(103, I.S_GRAD, np.arange(C.nnz)).astype(np.float32)).cuda()
    Cd = brm.DeviceCSR(C.rows, C.cols, C.rp, C.col, None)
    del C

    def fwd():
        Cx = brm.spgemm(Aq, Bq)
        del Cx

    def fwd_bwd():
        Cx = brm.spgemm(Aq, Bq)
        (Cx.val * G).sum().backward()
        a_val.grad = None
        b_val.grad = None

    def bwd_only():
        brm.brm_spgemm_backward(dA, dB, Cd, G)

    d64A, d64B = brm.to_device(A.astype(np.float64)), brm.to_device(B.astype(np.float64))

    def fwd64():
        Cx = brm.brm_spgemm_precise(d64A, d64B)
        del Cx

    steps = max(args.steps, 10)
    out = {"workload": "differentiable C=A*B, A R-MAT scale 18 ef16, B ER 2^18 8/row, FP32 N(0,1)", "nprod": total}
    out["fwd_f32_ms"] = _timed(fwd, steps, 3)
    out["bwd_f32_ms"] = _timed(bwd_only, steps, 3)
    out["fwd_bwd_f32_ms"] = _timed(fwd_bwd, steps, 3)
    out["fwd_f64_plain_ms"] = _timed(fwd64, steps, 3)
    out["speedup_f32_fwd_vs_f64_plain"] = out["fwd_f64_plain_ms"] / out["fwd_f32_ms"]
    out["fwd_f32_gflops"] = 2.0 * total / (out["fwd_f32_ms"] * 1e-3) / 1e9
    return out


# ---------------------------------------------------------------------------
# fixed call sequences for ncu captures (no timing)
# ---------------------------------------------------------------------------
def run_profile(args):
    """er       two BRMerge-Precise calls on the ER workload (n = --profile-n);
    rmat     two BRMerge-Precise calls on R-MAT of scale --scale;
    batched  a prepared batch of the product mix (--batch-count products),
             its numeric pass twice, then one brm_spgemm_batched call;
    diff     the differentiable workload's forward and backward once each."""
    import torch
    from paper_2206_06611_gb300 import brm
    torch.cuda.set_device(0)
    if args.workload == "batched":
        mats = I.batched_mix(args.batch_count)
        dev = [brm.to_device(M) for M in mats]
        b = brm.Batch(dev, dev)
        for _ in range(2):
            b.numeric()
            torch.cuda.synchronize()
        C, _ = brm.brm_spgemm_batched(dev, dev)
        torch.cuda.synchronize()
        info = {"profile": "batched", "nnz_C": C.nnz}
    elif args.workload == "diff":
        A = I.normal_values(I.rmat(18, 16), 101)
        B = I.normal_values(I.erdos_renyi(1 << 18, 8), 102)
        dA, dB = brm.to_device(A), brm.to_device(B)
        a_val = dA.val.clone().requires_grad_(True)
        C = brm.spgemm(brm.DeviceCSR(A.rows, A.cols, dA.rp, dA.col, a_val), dB)
        G = torch.from_numpy(I.rand_normal(103, I.S_GRAD, np.arange(C.nnz)).astype(np.float32)).cuda()
        (C.val * G).sum().backward()
        torch.cuda.synchronize()
        info = {"profile": "diff", "nnz_C": C.nnz}
    else:
        A = I.rmat(args.scale, 16) if args.workload == "rmat" else I.erdos_renyi(args.profile_n, 16)
        dA = brm.to_device(A, device="cuda:0")
        for _ in range(2):
            lw = {} if args.long_window is None else {"long_window": args.long_window}   # else the library's default
            C = brm.brm_spgemm_precise(dA, dA, long_bucket=args.long_bucket, **lw)
            torch.cuda.synchronize()
            del C
        info = {"profile": args.workload, "n": A.rows, "long_bucket": args.long_bucket,
                "long_window": args.long_window}
    info["launches"] = brm.brm_kernel_launches()
    print(json.dumps(info), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="brm", choices=["brm", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--headline-only", action="store_true", help="skip the 'also' block")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: split one product's rows over the ranks (strong scaling) instead of one "
                         "independent product per rank")
    ap.add_argument("--profile", action="store_true", help="two calls only (for ncu captures)")
    ap.add_argument("--profile-n", type=int, default=1 << 20)
    ap.add_argument("--workload", default="rmat", choices=["rmat", "er", "batched", "diff"],
                    help="rmat (default) or er: the headline line; batched / diff: --profile only")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="--profile --workload batched: products of the mix (the first of the 512)")
    ap.add_argument("--long-bucket", action="store_true",
                    help="--profile: long rows' numeric pass by column buckets (option long_bucket)")
    ap.add_argument("--long-window", type=int, choices=[0, 1, 2], default=None,
                    help="--profile: option long_window (0 merge rounds only, 1 the default split, 2 column tiles "
                         "for every long row of at most 65535 lists)")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload in ("batched", "diff"):
        raise SystemExit("--workload batched/diff only with --profile (their numbers are in the 'also' block)")
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
