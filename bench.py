"""Benchmark of the wide-CSC SpMV/SpVTM pair on one GB300 (or N replicas).

A step is one SpMV y = A x followed by one SpVTM u^T = v^T A on the
m=20,000 x n=5,000,000 wide CSC matrix with FP32 values and int32 indices
(about 200M nonzeros, power-law column degrees, 50 dense columns; generated on
the device from seed 1) -- the SpMV-SpVTM "wrap" the paper's drivers repeat
1,000 times (Sec. V).  The default run times 1,000 such steps.

Printed JSON (one line, rank 0):
  value      algorithmic bytes of the pair / device time per step (GB/s), all ranks
  roofline   dominant kernel: algorithmic bytes per launch / its CUDA-event time,
             against the measured HBM copy bandwidth
  e2e        the same metric through the C ABI with host vectors (copies timed): spmv_pair
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample
``--impl reference`` times the FP64 oracle itself (the CPU reference of this
path) on the same workload, one sample per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV/SpVTM GB/s vs 8 TB/s HBM peak; served vectors/s with p50/p99 latency"
WORKLOAD = "wide_csc_m20000_n5000000_fp32_powerlaw2_50dense"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("stream_kernel.cuh", "device_common.cuh", "internal.h"):
        with open(os.path.join(ROOT, "paper_1812_00904_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_name: str, workload: str, order: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(kernel_name)
    if (not e or e.get("source_hash") != kernel_source_hash() or e.get("workload") != workload
            or e.get("nonzero_order", "stored") != order):
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.t = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def rd():
            for line in self.proc.stdout:
                self.samples.append((time.time(), line.strip()))

        self.t = threading.Thread(target=rd, daemon=True)
        self.t.start()

    def stop(self, t0, t1):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        window = [s for s in self.samples if t0 - 0.25 <= s[0] <= t1 + 0.25] or self.samples[-3:]
        for _, line in window:
            parts = [x.strip() for x in line.split(",")]
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                for nm, v in zip(names, parts[3:7]):
                    if v.lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms: float, world: int, device) -> float:
    """The job's time: the longest timed region over the ranks (every rank calls this)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_step: int, steps: int, world: int, ms_max: float) -> float:
    """Aggregate GB/s of all replicas: every rank moves bytes_per_step per step."""
    return bytes_per_step * steps * world / (ms_max / 1e3) / 1e9


def pair_bytes(m, n, nnz, sv=4, sx=4, si=4, sp=4):
    """Algorithmic bytes (wide CSC): SpMV Z(si+sv)+(n+1)sp+n sx+m sx; SpVTM Z(si+sv)+(n+1)sp+m sx+n sx."""
    spmv_b = nnz * (si + sv) + (n + 1) * sp + n * sx + m * sx
    spvtm_b = nnz * (si + sv) + (n + 1) * sp + m * sx + n * sx
    return spmv_b, spvtm_b


def host_cpu():
    """(threads this process may use, CPU model string) of the host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return cores, f"{model or 'unknown'} ({os.uname().machine})"


class OracleSample:
    """A contiguous column block of A on the host, sized so that one FP64 oracle pair on
    `threads` host threads takes about `target_s`."""

    def __init__(self, A, target_s: float, threads: int = 1):
        import numpy as np

        import synth

        self.threads = threads
        ptr = A.ptr.cpu().numpy().astype(np.int64)
        n = A.n
        cols = max(1, n // 64)
        while True:
            z = int(ptr[cols])
            # widened to FP64 once, outside the timed oracle calls
            S = synth.SparseMatrix("csc", A.m, cols, ptr[:cols + 1].astype(np.int32), A.idx[:z].cpu().numpy(),
                                   A.vals[:z].double().cpu().numpy())
            self.S, self.cols, self.z, self.n, self.m = S, cols, z, n, A.m
            self.x = synth.uniform_vector(cols, 5).astype(np.float32).astype(np.float64)
            self.v = synth.uniform_vector(A.m, 6).astype(np.float32).astype(np.float64)
            dt = self.time_pair()
            if dt >= target_s / 2 or cols == n:
                break
            cols = min(n, int(cols * min(8.0, max(1.5, target_s / max(dt, 1e-4)))))
        b1, b2 = pair_bytes(A.m, cols, z)
        self.bytes = b1 + b2

    def time_pair(self, threads: int = None) -> float:
        import oracle

        t = self.threads if threads is None else threads
        t0 = time.perf_counter()
        if t == 1:
            oracle.spmv(self.S, self.x)
            oracle.spvtm(self.S, self.v)
        else:
            oracle.spmv_mt(self.S, self.x, t)
            oracle.spvtm_mt(self.S, self.v, t)
        return time.perf_counter() - t0

    def describe(self, reps: int, threads: int = None) -> str:
        t = self.threads if threads is None else threads
        how = "single thread" if t == 1 else f"{t} threads (each a balanced column range; SpMV into per-thread y, summed)"
        return (f"FP64 oracle SpMV+SpVTM pair on the first {self.cols} of {self.n} columns ({self.z} nonzeros), "
                f"{reps} pair(s), {how}")


def cpu_baseline(A, target_s: float):
    """The FP64 oracle pair on all host cores (the value) and on one core, on the same sample."""
    cores, model = host_cpu()
    smp = OracleSample(A, target_s / 6, threads=1)
    reps1 = 2
    t1 = sum(smp.time_pair(1) for _ in range(reps1)) / reps1
    repsn = 6
    smp.time_pair(cores)
    tn = sum(smp.time_pair(cores) for _ in range(repsn)) / repsn
    return {"value": round(smp.bytes / tn / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": smp.describe(repsn, cores), "cpu_model": model,
            "single_thread": {"value": round(smp.bytes / t1 / 1e9, 3), "cores": 1, "sample": smp.describe(reps1, 1)}}


def run_reference(args):
    """--impl reference: the FP64 oracle (plain CPU loops) on the same workload, all host cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import torch

    import synth

    cores, model = host_cpu()
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A = synth.wide_fp32_large(1, device=dev)
    per_step = min(2.0, 150.0 / (args.steps + args.warmup))
    smp = OracleSample(A, per_step, threads=cores)
    times = []
    for i in range(args.warmup + args.steps):
        t = smp.time_pair()
        if i >= args.warmup:
            times.append(t)
    t = statistics.median(times)
    v = round(smp.bytes / t / 1e9, 3)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * t, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "m": A.m, "n": A.n, "nnz": A.nnz, "step": "one SpMV + one SpVTM",
                      "sample_columns": smp.cols, "sample_nnz": smp.z},
           "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle",
                            "sample": smp.describe(args.steps), "cpu_model": model},
           "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def time_pair_gbs(pkg, plan, m, n, nnz, layout, steps, sv=4, stream=None):
    """GB/s of SpMV + SpVTM pairs on `plan` (one spmv_pair call per pair, device vectors, CUDA events)."""
    import torch

    dev = plan.vals.device
    g = torch.Generator(device=dev)
    g.manual_seed(12)
    x = torch.rand(n, generator=g, device=dev) * 2 - 1
    v = torch.rand(m, generator=g, device=dev) * 2 - 1
    y = torch.empty(m, device=dev)
    u = torch.empty(n, device=dev)
    stream = stream or torch.cuda.current_stream()
    for _ in range(3):
        pkg.spmv_pair(plan.handle, x, y, v, u, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        pkg.spmv_pair(plan.handle, x, y, v, u, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.check()
    ms = e0.elapsed_time(e1) / steps
    long_, short = (n, m) if layout == "csc" else (m, n)
    b = 2 * (nnz * (4 + sv) + (long_ + 1) * 4 + (m + n) * 4)
    return {"gbs": round(b / (ms / 1e3) / 1e9, 1), "ms_per_pair": round(ms, 4), "bytes_per_pair": b,
            "frac_of_hbm_peak": round(b / (ms / 1e3) / 1e9 / load_peaks()[0], 4)}


def small_fp64_flushed(pkg, dev, reps: int = 50):
    """The m=1,000 x n=100,000 FP64 wide matrix (about 0.5M nonzeros, L2-sized): each SpMV and
    SpVTM timed alone with a 256 MB buffer written between repetitions to flush L2."""
    import torch

    import synth

    A = synth.wide_fp64_small(0)
    ptr = torch.from_numpy(A.ptr.astype("int32")).to(dev)
    idx = torch.from_numpy(A.idx.astype("int32")).to(dev)
    vals = torch.from_numpy(A.vals).to(dev)
    plan = pkg.Plan(A.m, A.n, ptr, idx, vals, layout="csc")
    g = torch.Generator(device=dev)
    g.manual_seed(15)
    x = torch.rand(A.n, generator=g, device=dev, dtype=torch.float64) * 2 - 1
    v = torch.rand(A.m, generator=g, device=dev, dtype=torch.float64) * 2 - 1
    y = torch.empty(A.m, device=dev, dtype=torch.float64)
    u = torch.empty(A.n, device=dev, dtype=torch.float64)
    flush = torch.empty(64 << 20, device=dev, dtype=torch.float32)  # 256 MB > L2
    res = {}
    for name, fn in (("spmv", lambda: pkg.spmv(plan.handle, x, y)), ("spvtm", lambda: pkg.spvtm(plan.handle, v, u))):
        fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        b = A.nnz * 12 + (A.n + 1) * 4 + (A.n + A.m) * 8
        res[name] = {"ms_median": round(ms, 4), "ms_min": round(min(ts), 4), "gbs": round(b / (ms / 1e3) / 1e9, 1)}
    plan.check()
    plan.close()
    res.update(workload="wide_csc_m1000_n100000_fp64_zipf2_5dense", nnz=int(A.nnz), l2="flushed between repetitions")
    return res


def ops_alone(pkg, plan, m, n, nnz, reps: int = 15, per: int = 20):
    """Each product timed alone: `reps` batches of `per` back-to-back calls of one op (CUDA events
    per batch on the launching stream); median and min over the batches of the mean call time."""
    import statistics

    import torch

    dev = plan.vals.device
    g = torch.Generator(device=dev)
    g.manual_seed(13)
    x = torch.rand(n, generator=g, device=dev) * 2 - 1
    v = torch.rand(m, generator=g, device=dev) * 2 - 1
    y = torch.empty(m, device=dev)
    u = torch.empty(n, device=dev)
    stream = torch.cuda.current_stream()
    b_spmv, b_spvtm = pair_bytes(m, n, nnz)
    out = {}
    for name, call, b in (("spmv", lambda: pkg.spmv(plan.handle, x, y, stream), b_spmv),
                          ("spvtm", lambda: pkg.spvtm(plan.handle, v, u, stream), b_spvtm)):
        for _ in range(3):
            call()
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(per):
                call()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / per)
        med, mn = statistics.median(times), min(times)
        out[name] = {"ms_median": round(med, 4), "ms_min": round(mn, 4), "gbs_median": round(b / med / 1e6, 1),
                     "gbs_best": round(b / mn / 1e6, 1), "calls": reps * per}
    plan.check()
    return out


def batched_rate(pkg, plan, m, n, nnz, k, steps, ops=("spmv", "spvtm")):
    """Vectors/s and effective GB/s of k-vector SpMV and SpVTM calls (spmv_batch)."""
    import torch

    dev = plan.vals.device
    g = torch.Generator(device=dev)
    g.manual_seed(13)
    X = torch.rand((k, n), generator=g, device=dev) if "spmv" in ops else None
    V = torch.rand((k, m), generator=g, device=dev) if "spvtm" in ops else None
    out = {}
    for op, inp, len_out in ((pkg.SPMV_OP_AX, X, m), (pkg.SPMV_OP_VTA, V, n)):
        if inp is None:
            continue
        Y = torch.empty((k, len_out), device=dev)
        for _ in range(2):
            pkg.spmv_batch(plan.handle, op, k, inp, inp.stride(0), Y, Y.stride(0))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            pkg.spmv_batch(plan.handle, op, k, inp, inp.stride(0), Y, Y.stride(0))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        b = nnz * 8 + (n + 1) * 4 + k * (m + n) * 4
        out["spmv" if op == pkg.SPMV_OP_AX else "spvtm"] = {
            "ms": round(ms, 4), "vectors_per_s": round(k / (ms / 1e3), 1), "gbs": round(b / (ms / 1e3) / 1e9, 1)}
    plan.check()
    return out


def serving_measurement(pkg, dev, seconds: float = 2.0, rates=(0.5, 0.8, 1.0)):
    """Continuous batching over 64 resident matrices with Poisson-arriving requests of 1-32 vectors.

    Capacity is measured first (a burst of requests, vectors completed per second); then requests
    arrive at fractions of it for `seconds` each and every request's submit-to-result latency is
    read back.  Returns vectors/s and p50/p99 latency per arrival rate.
    """
    import numpy as np
    import torch

    import synth

    specs = synth.serving_specs()
    t0 = time.time()
    mats, plans = [], []
    for sp in specs:
        A = synth.serving_matrix(sp, device=dev)
        plan = pkg.Plan(A.m, A.n, A.ptr, A.idx, A.vals, layout=A.layout, flags=pkg.SPMV_PLAN_BANK_ORDER)
        mats.append(A)
        plans.append(plan)
    gen_s = time.time() - t0
    g = torch.Generator(device=dev)
    g.manual_seed(14)
    bufs = []
    for A in mats:
        bufs.append({pkg.SPMV_OP_AX: (torch.rand((32, A.n), generator=g, device=dev), torch.empty((96, A.m), device=dev)),
                     pkg.SPMV_OP_VTA: (torch.rand((32, A.m), generator=g, device=dev), torch.empty((96, A.n), device=dev))})
    torch.cuda.synchronize()
    srv = pkg.serve_create(int(120e9), 32, 4)
    try:
        ids = [pkg.serve_register(srv, p.handle) for p in plans]
        rng = np.random.default_rng(4)
        ring = [0] * len(mats)

        def submit(i, op, k):
            X, Y = bufs[i][op]
            o = ring[i]
            ring[i] = (o + k) % 64
            return pkg.serve_submit(srv, ids[i], op, k, X, Y[o:o + k])

        def draw():
            return int(rng.integers(len(mats))), int(rng.integers(2)), int(rng.integers(1, 33))

        # capacity: a burst of requests, all queued at once
        burst = [draw() for _ in range(600)]
        tb = time.perf_counter()
        rids = [submit(*r) for r in burst]
        for rid in rids:
            pkg.serve_wait(srv, rid, 120_000)
        cap_vps = sum(r[2] for r in burst) / (time.perf_counter() - tb)
        mean_k = 16.5
        res = {"matrices": len(mats), "nonzeros": int(sum(A.nnz for A in mats)), "generate_s": round(gen_s, 1),
               "capacity_vectors_per_s": round(cap_vps, 1), "rates": []}
        for frac in rates:
            lam = frac * cap_vps / mean_k  # requests per second
            st0 = pkg.serve_stats(srv)
            rids, ks = [], []
            t_start = time.perf_counter()
            t_next = t_start
            while True:
                now = time.perf_counter()
                if now - t_start >= seconds:
                    break
                if now < t_next:
                    time.sleep(min(t_next - now, 0.0005))
                    continue
                i, op, k = draw()
                rids.append(submit(i, op, k))
                ks.append(k)
                t_next += rng.exponential(1.0 / lam)
            for rid in rids:
                pkg.serve_wait(srv, rid, 120_000)
            elapsed = time.perf_counter() - t_start
            lat = np.array([pkg.serve_poll(srv, rid)[1] for rid in rids])
            st1 = pkg.serve_stats(srv)
            res["rates"].append({"offered_frac_of_capacity": frac, "requests": len(rids),
                                 "vectors_per_s": round(sum(ks) / elapsed, 1),
                                 "p50_ms": round(float(np.percentile(lat, 50)), 3),
                                 "p99_ms": round(float(np.percentile(lat, 99)), 3),
                                 "launches": st1["launches"] - st0["launches"],
                                 "max_inflight_launches": st1["max_inflight_launches"]})
        res["check"] = serving_check(pkg, srv, ids, mats, bufs, plans)
        res["tracked_requests_after"] = pkg.serve_stats(srv)["tracked_requests"]
        return res
    finally:
        pkg.serve_destroy(srv)
        for p in plans:
            p.close()


def serving_check(pkg, srv, ids, mats, bufs, plans):
    """Served results against the FP64 oracle at the serving workload's scale, outside the timed
    windows: one SpMV request (2 vectors) and one SpVTM request (3 vectors) on every matrix, all
    submitted at once so that they run mixed, each element within 1e-5 of its scale sum_j |a_ij x_j|."""
    import numpy as np
    import torch

    import oracle
    import synth
    from types import SimpleNamespace

    cores, _ = host_cpu()
    checks = []
    for i in range(len(mats)):
        for op, k in ((pkg.SPMV_OP_AX, 2), (pkg.SPMV_OP_VTA, 3)):
            X, Y = bufs[i][op]
            Y[64:64 + k].fill_(float("nan"))
            checks.append((i, op, k, X[:k], Y[64:64 + k]))  # rows 64.. of the outputs are not in the ring
    torch.cuda.synchronize()
    rids = [pkg.serve_submit(srv, ids[i], op, k, X, Y) for i, op, k, X, Y in checks]
    for rid in rids:
        pkg.serve_wait(srv, rid, 600_000)
    worst, bad, vectors = 0.0, 0, 0
    t0 = time.time()
    for i, A in enumerate(mats):
        vals = A.vals.double().cpu().numpy()
        S = synth.SparseMatrix(A.layout, A.m, A.n, A.ptr.cpu().numpy(), A.idx.cpu().numpy(), vals)
        Sabs = SimpleNamespace(layout=A.layout, m=A.m, n=A.n, ptr=S.ptr, idx=S.idx, vals=np.abs(vals))
        for j, op, k, X, Y in checks:
            if j != i:
                continue
            for b in range(k):
                xs = X[b].double().cpu().numpy()
                got = Y[b].double().cpu().numpy()
                if op == pkg.SPMV_OP_AX:
                    ref, scale = oracle.spmv_mt(S, xs, cores), oracle.spmv_mt(Sabs, np.abs(xs), cores)
                else:
                    ref, scale = oracle.spvtm_mt(S, xs, cores), oracle.spvtm_mt(Sabs, np.abs(xs), cores)
                ratio = np.abs(got - ref) / (1e-5 * scale + 1e-300)
                ratio[np.isnan(got)] = np.inf
                worst = max(worst, float(ratio.max()) if ratio.size else 0.0)
                bad += int((ratio > 1.0).sum())
                vectors += 1
        del S, Sabs, vals
    off_chip = sum(1 for p in plans if not p.info()["short_on_chip"])
    return {"checked_requests": len(checks), "checked_vectors": vectors, "matrices": len(mats),
            "short_vector_off_chip": off_chip, "max_err_ratio": worst, "elements_outside": bad,
            "ok": bad == 0, "tolerance": "1e-5 x sum_j |a_ij x_j| per element, FP64 oracle",
            "oracle_s": round(time.time() - t0, 1)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import synth
    import paper_1812_00904_gb300 as pkg
    from paper_1812_00904_gb300 import _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        if args.gpus > 1:
            raise SystemExit(f"--gpus {args.gpus} needs torchrun with {args.gpus} ranks (WORLD_SIZE={world})")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    A = synth.wide_fp32_large(1, device=dev, scale=args.scale)  # every rank holds its own replica
    m, n, nnz = A.m, A.n, A.nnz
    order = 0 if args.stored_order else pkg.SPMV_PLAN_BANK_ORDER
    blocks = pkg.SPMV_PLAN_ROW_BLOCKS if args.row_blocks else 0
    plan = pkg.Plan(m, n, A.ptr, A.idx, A.vals, layout="csc", flags=order | blocks, warps_per_cta=args.warps,
                    tile_items=args.tile_items, stages=args.stages)
    info = plan.info()
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    x = torch.rand(n, generator=g, device=dev) * 2 - 1
    v = torch.rand(m, generator=g, device=dev) * 2 - 1
    y = torch.empty(m, device=dev)
    u = torch.empty(n, device=dev)

    def step():  # the pair call: the SpMV on `stream`, the SpVTM beside it on the plan's second stream
        pkg.spmv_pair(plan.handle, x, y, v, u, stream)

    def step_serial():  # the two products one after the other on `stream` (kernel timings)
        pkg.spmv(plan.handle, x, y, stream)
        pkg.spvtm(plan.handle, v, u, stream)

    for _ in range(args.warmup):
        step()
        step_serial()
    torch.cuda.synchronize()
    plan.check()
    pkg.spmv_profile_reset(plan.handle)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop(t0, t1)
    plan.check()
    # kernel durations: the same K steps again, the two products one after the other on one
    # stream with every launch bracketed by CUDA events (each kernel runs alone: the events make
    # it drain before the next one starts, so the whole-step number above is taken without them)
    pkg.spmv_profile_enable(plan.handle, True)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        step_serial()
    ev3.record(stream)
    torch.cuda.synchronize()
    pkg.spmv_profile_enable(plan.handle, False)
    plan.check()
    ms_profiled = ev2.elapsed_time(ev3)
    kt = {k: pkg.spmv_profile_read(plan.handle, k) for k in range(7)}
    launches = sum(kt[k][1] for k in kt)  # every kernel launch of the K profiled steps (the same as the timed ones)
    ms_max = max_over_ranks(ms, world, dev)
    b_spmv, b_spvtm = pair_bytes(m, n, nnz)
    value = whole_job_gbs(b_spmv + b_spvtm, args.steps, world, ms_max)

    # roofline of the dominant kernel (SpMV local: chunk scatter, or the row-block dot over the
    # row-sorted copy; SpVTM local: chunk dot); algorithmic bytes of the method's data
    peak, peak_src = load_peaks()
    k_scatter = (nnz * 8 + (n + 1) * 4 + n * 4)  # idx + values + pointers + x
    k_segdot = (nnz * 8 + (n + 1) * 4 + m * 4 + n * 4)  # idx + values + pointers + v + u
    cand = {"chunk_scatter": (kt[0], k_scatter), "chunk_segdot": (kt[2], k_segdot),
            "row_block_dot": (kt[5], k_scatter)}
    dom = max(cand, key=lambda k: cand[k][0][0])
    (kms, kl), kbytes = cand[dom]
    avg_s = kms / max(kl, 1) / 1e3
    achieved = kbytes / avg_s / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": ncu_traffic(dom, WORKLOAD, "stored" if args.stored_order else "bank")
            if args.scale == 1.0 else None, "bytes_per_launch": kbytes,
            "avg_launch_us": round(avg_s * 1e6, 2),
            "timing": f"per-kernel CUDA events over a second pass of the {args.steps} steps "
                      f"({ms_profiled / args.steps:.4f} ms per step with the events)"}

    # end to end through the C ABI with host buffers
    e2e = None
    if args.skip_e2e:
        xh = None
    else:
        xh = x.cpu().pin_memory()
        vh = v.cpu().pin_memory()
        yh = torch.empty(m, pin_memory=True)
        uh = torch.empty(n, pin_memory=True)
        e2e_steps = max(5, min(args.steps, 200))

        def e2e_time(step_fn):
            for _ in range(2):
                step_fn()
            torch.cuda.synchronize()
            t0e = time.perf_counter()
            for _ in range(e2e_steps):
                step_fn()  # each call returns after its results have landed in host memory
            torch.cuda.synchronize()
            return (time.perf_counter() - t0e) / e2e_steps

        def separate():
            pkg.spmv(plan.handle, xh, yh, stream)
            pkg.spvtm(plan.handle, vh, uh, stream)

        te_sep = e2e_time(separate)
        te = e2e_time(lambda: pkg.spmv_pair(plan.handle, xh, yh, vh, uh, stream))
        e2e = {"value": round((b_spmv + b_spvtm) / te / 1e9, 1), "unit": "GB/s",
               "h2d_bytes_per_step": 4 * (n + m), "d2h_bytes_per_step": 4 * (m + n), "steps": e2e_steps,
               "ms_per_step": round(te * 1e3, 3),
               "api": "spmv_pair with pinned host vectors (x's copy overlaps the SpVTM, u's the SpMV)",
               "separate_calls": {"value": round((b_spmv + b_spvtm) / te_sep / 1e9, 1),
                                  "ms_per_step": round(te_sep * 1e3, 3), "api": "spmv then spvtm, pinned host vectors"}}

    out = None
    extras = None
    if rank == 0 and world == 1 and not args.skip_extras:
        extras = {}
        extras["ops_alone"] = ops_alone(pkg, plan, m, n, nnz)
        single = {"spmv": 1e3 / extras["ops_alone"]["spmv"]["ms_median"],
                  "spvtm": 1e3 / extras["ops_alone"]["spvtm"]["ms_median"]}
        for kk in (8, 32):
            br = batched_rate(pkg, plan, m, n, nnz, kk, max(10, args.steps // (5 * kk)))
            for op in ("spmv", "spvtm"):
                br[op]["vs_single_vector"] = round(br[op]["vectors_per_s"] / single[op], 2)
            br["path"] = {"spvtm": "one pass per 8 vectors, a vector per lane of a lane group; the 8 short vectors "
                                   f"({m} x 8 x 4 B) do not fit on chip and are read through L2",
                          "spmv": "shared-memory atomic passes, one per vector (the accumulators of 8 vectors do "
                                  "not fit on chip)" if not blocks else
                                  "over the row-sorted copy, one pass per 8 vectors (windows through L2)"}
            extras[f"batched_k{kk}"] = br
        # multi-vector passes where 8 short vectors fit on chip: the same recipe with m = 2,000 rows
        Sm = synth.wide_fp32_short(2000, device=dev)
        ps = pkg.Plan(Sm.m, Sm.n, Sm.ptr, Sm.idx, Sm.vals, layout="csc", flags=order)
        so = ops_alone(pkg, ps, Sm.m, Sm.n, Sm.nnz)
        small_single = {"spmv": 1e3 / so["spmv"]["ms_median"], "spvtm": 1e3 / so["spvtm"]["ms_median"]}
        extras["batched_short_m"] = {"workload": f"wide_csc_m{Sm.m}_n{Sm.n}_fp32_powerlaw2_50dense", "nnz": Sm.nnz,
                                     "single_ms": {"spmv": so["spmv"]["ms_median"], "spvtm": so["spvtm"]["ms_median"]}}
        for kk in (4, 8):
            br = batched_rate(pkg, ps, Sm.m, Sm.n, Sm.nnz, kk, max(10, args.steps // (5 * kk)))
            for op in ("spmv", "spvtm"):
                br[op]["vs_single_vector"] = round(br[op]["vectors_per_s"] / small_single[op], 2)
            extras["batched_short_m"][f"k{kk}"] = br
        ps.close()
        del Sm, ps
        extras["wide_fp64_small"] = small_fp64_flushed(pkg, dev)
        # least squares by CGLS on the same matrix: one SpMV + one SpVTM + vector updates per iteration
        bl = torch.rand(m, generator=g, device=dev) * 2 - 1
        xl = torch.zeros(n, device=dev)
        torch.cuda.synchronize()
        tc0 = time.perf_counter()
        it, rel = pkg.spmv_cgls(plan.handle, bl, xl, 50, 0.0)
        tc = time.perf_counter() - tc0
        extras["cgls"] = {"iterations": it, "ms_per_iteration": round(tc * 1e3 / max(it, 1), 4),
                          "rel_grad": rel, "note": "wall clock of the call, including its setup"}
        # the same matrix multiplied in the caller's stored order (no bank-ordered copy)
        if order:
            ps = pkg.Plan(m, n, A.ptr, A.idx, A.vals, layout="csc", flags=blocks)
            extras["stored_order"] = time_pair_gbs(pkg, ps, m, n, nnz, "csc", max(20, args.steps // 5))
            ps.close()
        # the other SpMV local step: the row-sorted copy, or shared-memory atomic accumulation
        other = order | (0 if blocks else pkg.SPMV_PLAN_ROW_BLOCKS)
        pa = pkg.Plan(m, n, A.ptr, A.idx, A.vals, layout="csc", flags=other)
        pinfo = pa.info()
        extras["atomic_scatter" if blocks else "row_blocks"] = dict(
            time_pair_gbs(pkg, pa, m, n, nnz, "csc", max(20, args.steps // 5)),
            blocks=pinfo["row_blocks"], widest_window=pinfo["row_block_window"])
        if not blocks and pinfo["row_blocks"]:  # 8-vector SpMV passes over the row-sorted copy
            brb = batched_rate(pkg, pa, m, n, nnz, 8, max(10, args.steps // 40), ops=("spmv",))["spmv"]
            brb["vs_single_vector"] = round(brb["vectors_per_s"] / single["spmv"], 2)
            extras["row_blocks"]["batched_k8_spmv"] = brb
        pa.close()
        vb = A.vals.to(torch.bfloat16)
        pb = pkg.Plan(m, n, A.ptr, A.idx, vb, layout="csc", vec_dtype=torch.float32, flags=order | blocks)
        extras["bf16_values"] = dict(time_pair_gbs(pkg, pb, m, n, nnz, "csc", max(20, args.steps // 5), sv=2),
                                     workload=WORKLOAD.replace("fp32", "bf16values"))
        pb.close()
        del vb
    if rank == 0:
        cpu = None
        if not args.skip_cpu_baseline and world == 1:
            cpu = cpu_baseline(A, target_s=args.cpu_seconds)
        spmv_ms = (kt[0][0] + kt[1][0] + kt[5][0] + kt[6][0]) / args.steps
        spvtm_ms = (kt[2][0] + kt[3][0]) / args.steps
        out = {"metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD if args.scale == 1.0 else f"{WORKLOAD}_scale{args.scale}",
                          "m": m, "n": n, "nnz": nnz, "layout": "csc",
                          "step": "one SpMV + one SpVTM (Sec. V wrap): one spmv_pair call, the two products side by side on two streams", "l2": "inputs larger than L2 (no flush)",
                          "parallelism": f"replicas x{world}", "chunks": info["chunks"], "ctas": info["ctas"],
                          "warps_per_cta": info["warps_per_cta"], "tile_items": info["tile_items"],
                          "stages": info["stages"], "zones": info["zones"],
                          "nonzero_order": "stored" if args.stored_order else
                          "bank order (plan-owned copy, permuted within each column)",
                          "plan_setup_ms": round(info["setup_ms"], 3),
                          "spmv_local": (f"row-sorted blocks ({info['row_blocks']} blocks, widest window "
                                         f"{info['row_block_window']} columns)") if info["row_blocks"] else
                          "shared-memory atomic accumulation"},
               "gflops": round(2 * 2 * nnz * args.steps * world / (ms_max / 1e3) / 1e9, 1),
               "frac_of_hbm_peak": round(value / world / peak, 4),
               "ops": {"spmv_gbs": round(b_spmv / (spmv_ms / 1e3) / 1e9, 1),
                       "spvtm_gbs": round(b_spvtm / (spvtm_ms / 1e3) / 1e9, 1),
                       "kernel_ms": {name: round(kt[k][0] / max(kt[k][1], 1), 4) for k, name in
                                     enumerate(["chunk_scatter", "combine", "chunk_segdot", "zone_fixup", "dvalues",
                                                "row_block_dot", "row_block_fixup"])
                                     if kt[k][1]}},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "extras": extras,
               "gpu_launches": launches,
               "clocks": clocks}
    plan.close()
    if extras is not None:
        del A, x, v, y, u
        torch.cuda.empty_cache()
        T = synth.tall_fp32_large(2, device=dev)
        pt = pkg.Plan(T.m, T.n, T.ptr, T.idx, T.vals, layout="csr", flags=order | blocks)
        extras["tall_csr"] = dict(time_pair_gbs(pkg, pt, T.m, T.n, T.nnz, "csr", max(20, args.steps // 5)),
                                  workload=f"tall_csr_m{T.m}_n{T.n}_fp32_powerlaw2.2_20dense", nnz=T.nnz)
        pt.close()
        del T, pt
        torch.cuda.empty_cache()
        if not args.skip_serving:
            extras["serving"] = serving_measurement(pkg, dev)
    if out is not None:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    chk = (extras or {}).get("serving", {}).get("check")
    if chk is not None and not chk["ok"]:
        print(f"served results outside the tolerance: {chk}", file=sys.stderr)
        return 1
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--scale", type=float, default=1.0,
                    help="fraction of the 5M columns (a smaller sample of the same workload, for profiling)")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="skip the tall CSR, BF16-value, batched and serving measurements")
    ap.add_argument("--skip-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--warps", type=int, default=0, help="warps (chunks) per CTA; 0 = library default")
    ap.add_argument("--tile-items", type=int, default=0, help="merge items per staged tile; 0 = library default")
    ap.add_argument("--stages", type=int, default=0, help="staging buffers per warp; 0 = library default")
    ap.add_argument("--stored-order", action="store_true",
                    help="multiply in the stored nonzero order (no bank-ordered plan copy)")
    ap.add_argument("--row-blocks", action="store_true",
                    help="SpMV over the row-sorted plan copy (SPMV_PLAN_ROW_BLOCKS) instead of shared-memory atomics")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
