"""Benchmark of BRMerge SpGEMM on one GB300 (or N, one independent product per GPU).

Workload: C = A*A, A Erdos-Renyi with n = 2^20 rows and exactly 16 distinct
uniform columns per row, FP64 values U[-1,1), seeded (synthetic; the paper's
SuiteSparse matrices are not used).  One step = one whole BRMerge-Precise call
(product counts + binning, symbolic pass, prefix sum, allocation of C,
numeric pass) on inputs already resident in HBM.  The inputs (A: 205 MB) and
the output (C: 3.2 GB) are both larger than the 129 MB L2, so no explicit L2
flush is needed between steps.

Metric (the paper's, Section IV-A): GFLOP/s = 2 * intermediate products / s.

Printed: one JSON line with value (device-timed, all ranks), e2e (through the
same C-ABI call with host buffers: A copied in from pinned host memory and C
copied back every step), the roofline of the dominant kernel (the numeric
kernel of the busiest bin -- for this workload the register bin of 8 threads
per row -- timed live with CUDA events recorded by the library on its launch
stream), clocks sampled with nvidia-smi during the timed region, and a
cpu_baseline (the CPU oracle on a bounded sample of rows).

``--impl reference`` times the CPU oracle itself (the only reference that
exists for this method) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
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
WORKLOAD = "ER n=2^20, 16 nnz/row, C=A*A, FP64, BRMerge-Precise"

# DRAM bytes (read + write) of one launch of the dominant kernel (the numeric
# register-bin kernel on this workload), from an ncu capture of the current
# kernel source (dram__bytes_read.sum + dram__bytes_write.sum); set to None
# whenever that kernel changes until it is captured again.
NUMERIC_REG_TRAFFIC = 3.898992e9 + 3.184545e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


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
                                          "-lms", "200", "-i", str(dev_index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
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
# algorithmic bytes of the numeric pass (compulsory traffic, per launch)
# ---------------------------------------------------------------------------
def numeric_bytes(A, B, nnz_c, vbytes):
    """A once (row_ptr, col, val), the B rows A touches once, C.row_ptr read
    once and C's columns and values written once."""
    touched = np.zeros(B.rows, dtype=bool)
    touched[A.col] = True
    blen = np.diff(B.rp.astype(np.int64))
    b_bytes = int(touched.sum()) * 2 * 4 + int(blen[touched].sum()) * (4 + vbytes)
    a_bytes = (A.rows + 1) * 4 + A.nnz * (4 + vbytes)
    c_bytes = (A.rows + 1) * 8 + nnz_c * (4 + vbytes)
    return a_bytes + b_bytes + c_bytes


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(A, target_s: float, threads: int):
    """Time the oracle's Gustavson (row-parallel over nprod-balanced groups)
    on the first rows of A*A, enough for about target_s seconds."""
    import oracle
    oracle.build()
    nprod = oracle.row_nprod(A, A)
    # calibrate on a small slice
    rows = np.arange(min(A.rows, 20000), dtype=np.int64)
    t0 = time.perf_counter()
    oracle.gustavson_parallel(A, A, threads, rows)
    dt = time.perf_counter() - t0
    rate = nprod[rows].sum() / max(dt, 1e-6)
    want = int(min(A.rows, max(len(rows), rate * target_s / max(nprod.mean(), 1))))
    rows = np.arange(want, dtype=np.int64)
    t0 = time.perf_counter()
    oracle.gustavson_parallel(A, A, threads, rows)
    dt = time.perf_counter() - t0
    flops = 2.0 * float(nprod[rows].sum())
    return flops / dt / 1e9, dt, want


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    A = I.erdos_renyi(1 << 20, 16)
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(A, 2.0, threads)
    vals, secs, rows = [], [], 0
    for _ in range(args.steps):
        v, dt, rows = oracle_sample(A, 8.0, threads)
        vals.append(v)
        secs.append(dt)
    value = float(np.mean(vals))
    sample = f"first {rows} of {A.rows} rows of A*A per step (Gustavson, FP64)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": 1, "parallelism": "cpu oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    from paper_2206_06611_gb300 import brm

    rank, world, local = dist_env()
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

    # every rank multiplies its own independent matrix (weak scaling)
    A = I.erdos_renyi(1 << 20, 16, seed=rank_seed(rank))
    vbytes = 8
    dA = brm.to_device(A, device=f"cuda:{dev}")
    st = torch.cuda.current_stream()

    # warm-up (also gives the result size)
    C = None
    for _ in range(args.warmup):
        C = brm.brm_spgemm_precise(dA, dA)
    torch.cuda.synchronize()
    nnz_c = C.nnz
    del C
    nprod_total = brm.brm_row_nprod(dA, dA)[1]

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
        C = brm.brm_spgemm_precise(dA, dA)
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
    value = job_gflops(nprod_total, world, args.steps, ms_max)

    # ---- end to end: host buffers, copies inside the timed region ----------
    hA = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
          for k, v in (("rp", A.rp.astype(np.int32)), ("col", A.col.astype(np.int32)), ("val", A.val))}
    h2d = sum(t.numel() * t.element_size() for t in hA.values())
    out_rp = torch.empty(A.rows + 1, dtype=torch.int64).pin_memory()
    out_col = torch.empty(nnz_c, dtype=torch.int32).pin_memory()
    out_val = torch.empty(nnz_c, dtype=torch.float64).pin_memory()
    d2h = out_rp.numel() * 8 + nnz_c * (4 + vbytes)
    dA2 = brm.DeviceCSR(A.rows, A.cols, torch.empty_like(dA.rp), torch.empty_like(dA.col), torch.empty_like(dA.val))
    e_steps = max(1, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(st)
    for _ in range(e_steps):
        dA2.rp.copy_(hA["rp"], non_blocking=True)
        dA2.col.copy_(hA["col"], non_blocking=True)
        dA2.val.copy_(hA["val"], non_blocking=True)
        C = brm.brm_spgemm_precise(dA2, dA2)
        out_rp.copy_(C.rp, non_blocking=True)
        out_col.copy_(C.col, non_blocking=True)
        out_val.copy_(C.val, non_blocking=True)
        del C
    f1.record(st)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    barrier()
    e2e_ms = reduce_max(e2e_ms, dist, f"cuda:{dev}")
    e2e_value = job_gflops(nprod_total, world, e_steps, e2e_ms)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel ------------------------------------
    kern = max(("numeric_reg", "numeric_warp", "numeric_block", "numeric_long"), key=lambda k: trace[k][0])
    k_ms, k_launch = trace[kern]
    per_launch_ms = k_ms / max(k_launch, 1)
    alg_bytes = numeric_bytes(A, A, nnz_c, vbytes) if kern.startswith("numeric") else None
    peak, peak_kind = peaks()
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9 if alg_bytes else None
    roofline = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "peak_source": peak_kind,
                "traffic": NUMERIC_REG_TRAFFIC if kern == "numeric_reg" else None,
                "algorithmic_bytes": alg_bytes, "kernel_ms": per_launch_ms}
    phases = {k: round(v[0] / args.steps, 4) for k, v in trace.items() if v[1]}

    # ---- CPU oracle on a bounded sample --------------------------------------
    cpu = None
    if not args.no_cpu and world == 1:
        threads = os.cpu_count() or 1
        v, dt, rows = oracle_sample(A, args.cpu_seconds, threads)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {rows} of {A.rows} rows of A*A (Gustavson FP64, {dt:.1f} s)"}

    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": A.rows, "nnz_A": A.nnz, "nprod": nprod_total, "nnz_C": nnz_c,
                   "global_batch": world, "parallelism": f"independent products x{world}",
                   "l2": "inputs (205 MB) and output (3.2 GB) exceed L2; no flush"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e_steps},
        "gpu_launches": launches,
        "roofline": roofline,
        "phases_ms_per_step": phases,
        "clocks": clk,
        "cpu_baseline": cpu,
    }), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_profile(args):
    """A short fixed sequence of calls for ncu to capture (no timing):
    er       two BRMerge-Precise calls on the ER workload (n = --profile-n);
    rmat     two BRMerge-Precise calls on R-MAT of scale --scale;
             er and rmat take the long rows' numeric pass by column buckets
             with --long-bucket;
    batched  a prepared batch of the product mix (--batch-count products,
             512 by default), its numeric pass twice, then one
             brm_spgemm_batched call;
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
            C = brm.brm_spgemm_precise(dA, dA, long_bucket=args.long_bucket)
            torch.cuda.synchronize()
            del C
        info = {"profile": args.workload, "n": A.rows, "long_bucket": args.long_bucket}
    info["launches"] = brm.brm_kernel_launches()
    print(json.dumps(info), flush=True)


# ---------------------------------------------------------------------------
# the other configurations (reported beside the headline line)
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


def _sample_rows(nprod, count, seed):
    top = np.argsort(-nprod, kind="stable")[: count // 4]
    rnd = I.rand_below(seed, 30, np.arange(count), len(nprod))
    return np.unique(np.concatenate([top, rnd]))


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


def run_rmat(args):
    """R-MAT A*A: FP64 plain, FP32 plain and FP32 with TwoSum; GFLOP/s and the
    FP32 error against the FP64 oracle on sampled rows."""
    import torch
    import oracle
    from paper_2206_06611_gb300 import brm
    torch.cuda.set_device(0)
    A = I.rmat(args.scale, 16)
    nprod = oracle.row_nprod(A, A)
    total = int(nprod.sum())
    rows = _sample_rows(nprod, 400, 17)
    ref = oracle.gustavson(A, A, rows, with_abs=True)
    out = {"workload": f"R-MAT scale {args.scale} ef16 dedup, C=A*A, BRMerge-Precise", "n": A.rows, "nnz_A": A.nnz,
           "nprod": total}
    for mode, dtype, comp in (("f64", np.float64, False), ("f32", np.float32, False), ("f32_twosum", np.float32, True)):
        dA = brm.to_device(A, dtype=dtype)
        C = brm.brm_spgemm_precise(dA, dA, compensated=comp)
        torch.cuda.synchronize()
        crp, col, val = _rows_to_host(C, rows)
        assert np.array_equal(col, ref.col), "structure differs from the oracle"
        d = (val - ref.val) ** 2
        cs, ca = np.concatenate(([0.0], np.cumsum(d))), np.concatenate(([0.0], np.cumsum(ref.abs ** 2)))
        num = np.sqrt(np.maximum(cs[crp[1:]] - cs[crp[:-1]], 0))
        den = np.sqrt(np.maximum(ca[crp[1:]] - ca[crp[:-1]], 0))
        err = np.where(den > 0, num / np.where(den > 0, den, 1), 0)
        nnz_c = C.nnz
        del C
        torch.cuda.empty_cache()

        def step():
            Cx = brm.brm_spgemm_precise(dA, dA, compensated=comp)
            del Cx

        brm.brm_trace_reset()
        brm.brm_trace_enable(True)
        ms = _timed(step, args.steps, max(1, min(args.warmup, 2)))
        t = brm.brm_trace_read()
        brm.brm_trace_enable(False)
        n_calls = args.steps + max(1, min(args.warmup, 2))
        out[mode] = {"ms_per_step": ms, "gflops": 2.0 * total / (ms * 1e-3) / 1e9, "nnz_C": nnz_c,
                     "phases_ms": {k: round(v[0] / n_calls, 3) for k, v in t.items() if v[1]},
                     "row_err_vs_f64_oracle": {"max": float(err.max()), "median": float(np.median(err)),
                                               "rows": int(len(rows))}}
        del dA
        torch.cuda.empty_cache()
    # the long rows' numeric pass by column buckets instead of merge rounds
    # (option long_bucket; the same bits), FP64
    dA = brm.to_device(A)

    def bucket_step():
        Cx = brm.brm_spgemm_precise(dA, dA, long_bucket=True)
        del Cx

    brm.brm_trace_reset()
    brm.brm_trace_enable(True)
    ms = _timed(bucket_step, args.steps, max(1, min(args.warmup, 2)))
    t = brm.brm_trace_read()
    brm.brm_trace_enable(False)
    n_calls = args.steps + max(1, min(args.warmup, 2))
    out["f64_long_bucket"] = {"ms_per_step": ms, "gflops": 2.0 * total / (ms * 1e-3) / 1e9,
                              "phases_ms": {k: round(v[0] / n_calls, 3) for k, v in t.items() if v[1]}}
    del dA
    torch.cuda.empty_cache()
    # BRMerge-Upper: C_bar of every product (about 251 GB here) does not fit
    # beside C, so it runs in row chunks
    dA = brm.to_device(A)
    try:
        def upper_step():
            Cx = brm.brm_spgemm_upper(dA, dA, upper_chunk_bytes=16 << 30)
            del Cx

        ms = _timed(upper_step, 1, 1)
        out["f64_upper_chunked"] = {"ms_per_step": ms, "gflops": 2.0 * total / (ms * 1e-3) / 1e9,
                                    "chunk_bytes": 16 << 30}
    except brm.BrmError as e:
        out["f64_upper_chunked"] = {"error": str(e)}
    del dA
    torch.cuda.empty_cache()
    out["speedup_f32_vs_f64"] = out["f64"]["ms_per_step"] / out["f32"]["ms_per_step"]
    out["speedup_f32_twosum_vs_f64"] = out["f64"]["ms_per_step"] / out["f32_twosum"]["ms_per_step"]
    print(json.dumps(out), flush=True)


def run_batched(args):
    """512 uneven products: one batched call vs 512 single calls, the numeric
    pass replayed from a CUDA graph, autotuned bins; FP64 and FP32."""
    import torch
    import oracle
    from paper_2206_06611_gb300 import brm
    torch.cuda.set_device(0)
    out = {"workload": "batched: 512 products A_i*A_i, n_i log-uniform in [1e3, 2e5], half 3-D Laplacian, "
                       "half ER with 4..32 per row"}
    mats64 = I.batched_mix(512)
    total = int(sum(oracle.row_nprod(M, M).sum() for M in mats64))
    for name, dtype in (("f64", np.float64), ("f32", np.float32)):
        mats = [M.astype(dtype) for M in mats64]
        dev = [brm.to_device(M) for M in mats]
        gf = lambda ms: 2.0 * total / (ms * 1e-3) / 1e9  # noqa: E731

        def batched():
            C, _ = brm.brm_spgemm_batched(dev, dev)
            del C

        def separate():
            for d in dev:
                C = brm.brm_spgemm_precise(d, d)
                del C

        r = {"nprod": total, "rows": int(sum(M.rows for M in mats))}
        r["separate_ms"] = _timed(separate, max(1, args.steps // 2), 1)
        r["batched_ms"] = _timed(batched, args.steps, 2)
        opts, tune_ms = brm.brm_autotune(dev, dev)
        r["autotuned"] = {"reg_keys": opts["reg_keys"], "reg_warps": opts["reg_warps"], "tune_call_ms": tune_ms}

        def batched_tuned():
            C, _ = brm.brm_spgemm_batched(dev, dev, **opts)
            del C

        r["batched_tuned_ms"] = _timed(batched_tuned, args.steps, 2)
        b = brm.Batch(dev, dev, **opts)
        r["numeric_graph_ms"] = _timed(b.graph_launch, args.steps, 2)
        r["numeric_launch_ms"] = _timed(b.numeric, args.steps, 2)
        b.check()
        b.close()
        for k in ("separate_ms", "batched_ms", "batched_tuned_ms"):
            r[k.replace("_ms", "_gflops")] = gf(r[k])
        r["speedup_batched_vs_separate"] = r["separate_ms"] / r["batched_tuned_ms"]
        out[name] = r
        del dev
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def run_diff(args):
    """Differentiable C = A*B (A R-MAT scale 18 ef16, B ER 2^18 with 8 per row,
    FP32 N(0,1)): forward + hand-written backward, and the FP64 plain forward."""
    import torch
    import oracle
    from paper_2206_06611_gb300 import brm
    torch.cuda.set_device(0)
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
    del C

    def fwd():
        Cx = brm.spgemm(Aq, Bq)
        del Cx

    def fwd_bwd():
        Cx = brm.spgemm(Aq, Bq)
        (Cx.val * G).sum().backward()
        a_val.grad = None
        b_val.grad = None

    C = brm.spgemm(Aq, Bq)
    Cd = brm.DeviceCSR(C.rows, C.cols, C.rp, C.col, None)
    del C

    def bwd_only():
        brm.brm_spgemm_backward(dA, dB, Cd, G)

    d64A, d64B = brm.to_device(A.astype(np.float64)), brm.to_device(B.astype(np.float64))

    def fwd64():
        Cx = brm.brm_spgemm_precise(d64A, d64B)
        del Cx

    out = {"workload": "differentiable C=A*B, A R-MAT scale 18 ef16, B ER 2^18 8/row, FP32 N(0,1)",
           "nprod": total}
    out["fwd_f32_ms"] = _timed(fwd, args.steps, 3)
    out["bwd_f32_ms"] = _timed(bwd_only, args.steps, 3)
    out["fwd_bwd_f32_ms"] = _timed(fwd_bwd, args.steps, 3)
    out["fwd_f64_plain_ms"] = _timed(fwd64, args.steps, 3)
    out["speedup_f32_fwd_vs_f64_plain"] = out["fwd_f64_plain_ms"] / out["fwd_f32_ms"]
    out["fwd_f32_gflops"] = 2.0 * total / (out["fwd_f32_ms"] * 1e-3) / 1e9
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="brm", choices=["brm", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--profile", action="store_true", help="two calls only (for ncu captures)")
    ap.add_argument("--profile-n", type=int, default=1 << 20)
    ap.add_argument("--workload", default="er", choices=["er", "rmat", "batched", "diff"],
                    help="er: the headline line; the others print their own JSON line")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale of --workload rmat")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="--profile --workload batched: products of the mix (the first of the 512)")
    ap.add_argument("--long-bucket", action="store_true",
                    help="--profile: long rows' numeric pass by column buckets (option long_bucket)")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.workload == "rmat":
        run_rmat(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "diff":
        run_diff(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
