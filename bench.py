"""Benchmark: factor + solve of one block-tridiagonal SPD system to relative
residual <= 1e-10 on GB300, through the libbtc C ABI.

Workload (default): N = 1024 blocks of n = 64, one right-hand side, seeded
synthetic inputs (B_i ~ N(0, 1/n), D_i = M M^T/n + (||B_{i-1}||+||B_i||+1) I).
A step = btc_factor_solve_refined: the factorization of Alg. 5 with the
forward substitution of Alg. 7 interlaced in the same persistent launch, the
backward substitution, then FP64 residuals and correction solves until
||r|| <= 1e-10 ||A|| ||x||, in the chosen form: FP32 factor and correction
solves, FP64 top-separator (root) Cholesky, FP64 residual and update. The plain
FP64 GPU path (same kernels in FP64, no refinement needed) is timed beside it,
and so is the same step with the double-FP32 root option.

Prints ONE JSON line (rank 0). `--impl reference` times the FP64 CPU oracle
(sequential Alg. 1 factor + block substitution) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
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

import numpy as np  # noqa: E402

METRIC = "factor+solve solves/s at resid<=1e-10 (N=1024, n=64, 1 RHS)"
UNIT = "solves/s"
WORKLOAD = dict(N=1024, n=64, nrhs=1, delta=1.0, seed=0)
TOL = 1e-10
FP32_PEAK_PER_SM_CLK = 128 * 2  # FFMA lanes x 2 flops
FP64_PEAK_PER_SM_CLK = 1.68 * 2  # lane-DFMA per clock per SM on GB300 (measured, four or more warps) x 2 flops
SMS = 152


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


class NvmlClockSampler:
    """SM clock and throttle-reason sampling through NVML (read-only queries, ctypes, no extra package)
    at about 1 ms, so that a timed region of a few tens of milliseconds still gets many samples. Returns
    None from start() when NVML is not available (ClockSampler's nvidia-smi loop is used instead)."""

    # clock-event reason bits (nvml.h): sw power cap, hw slowdown, sw thermal, hw thermal
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, gpu_index, period_s=0.001):
        self.gpu = gpu_index
        self.period = period_s
        self.samples = []
        self.reasons = set()
        self.max_mhz = None
        self.running = False

    def start(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(self.gpu, ctypes.byref(h)) != 0:
                return None
        except (OSError, AttributeError):
            return None
        self.lib, self.h, self.ct = lib, h, ctypes
        mx = ctypes.c_uint(0)
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM = 1
            self.max_mhz = float(mx.value)
        self.running = True
        self.t = threading.Thread(target=self._loop, daemon=True)
        self.t.start()
        while not self.samples and self.t.is_alive():
            time.sleep(0.0005)
        return self

    def _loop(self):
        ct, lib, h = self.ct, self.lib, self.h
        clk, rs = ct.c_uint(0), ct.c_ulonglong(0)
        fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while self.running:
            if lib.nvmlDeviceGetClockInfo(h, 1, ct.byref(clk)) == 0:
                self.samples.append(float(clk.value))
            if fn(h, ct.byref(rs)) == 0:
                for bit, name in self.REASONS.items():
                    if rs.value & bit:
                        self.reasons.add(name)
            time.sleep(self.period)

    def stop(self):
        self.running = False
        self.t.join(timeout=1.0)
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples), "source": "nvml (1 ms)"}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
            return
        # the timed region starts only once the sampler is producing samples
        t0 = time.perf_counter()
        while not self.lines and self.proc.poll() is None and time.perf_counter() - t0 < 5.0:
            time.sleep(0.01)
        self.first = len(self.lines)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # samples taken while the timed region ran (the last pre-region sample when it was shorter than the
        # sampling period)
        for ln in self.lines[max(self.first - 1, 0):]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("btc_factor.cuh", "btc_tile.cuh", "btc_solve.cuh", "btc_fused.cuh"):
        with open(os.path.join(ROOT, "paper_2601_03754_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_from_profile():
    """DRAM bytes per launch of the interlaced factor + forward kernel from the committed ncu summary, if it
    matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "factor_forward_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    if t.get("kernel_sha") != _kernel_hash():
        return None
    return t.get("dram_bytes_per_launch")


def replica_throughput(ms_local, world):
    """Replicas (one independent workload per rank): the job's step time is the slowest rank's mean
    step time (max over ranks), its throughput the units of all ranks over that time (solves/s)."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * 1000.0 / ms


def run_reference(args):
    """The FP64 CPU oracle on the host cores: a bounded sample of the same workload."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import oracle
    from paper_2601_03754_gb300 import gen
    oracle.build()
    W = WORKLOAD
    D, B = gen.bt_random(W["N"], W["n"], delta=W["delta"], seed=W["seed"])
    b = gen.rhs(W["N"], W["n"], W["nrhs"], seed=W["seed"])
    for _ in range(max(args.warmup, 0) and 1):
        oracle.solve(D, B, b)
    times = []
    t_start = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        x = oracle.solve(D, B, b)
        times.append(time.perf_counter() - t0)
    total = time.perf_counter() - t_start
    rel = oracle.relres(D, B, x, b)
    ms = 1000.0 * statistics.mean(times)
    value = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload="bt_random N=1024 n=64 m=1 delta=1, sequential Alg. 1 FP64 factor + solve",
                           **W),
            "relres": rel,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full factor+solve passes of the workload ({total:.1f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(budget_s=12.0, max_reps=200):
    import oracle
    from paper_2601_03754_gb300 import gen
    oracle.build()
    W = WORKLOAD
    D, B = gen.bt_random(W["N"], W["n"], delta=W["delta"], seed=W["seed"])
    b = gen.rhs(W["N"], W["n"], W["nrhs"], seed=W["seed"])
    times = []
    t_start = time.perf_counter()
    while len(times) < max_reps and (time.perf_counter() - t_start) < budget_s:
        t0 = time.perf_counter()
        oracle.solve(D, B, b)
        times.append(time.perf_counter() - t0)
    v = 1.0 / statistics.mean(times)
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} full sequential FP64 factor+solve passes of N=1024, n=64 "
                      f"({time.perf_counter() - t_start:.1f} s, single thread)"}


def run_profile(which):
    """The benchmark workload without timing: warm-up pass + one pass, for ncu launch lists. The
    blocked-256 modes factor N=128, n=256 (TF32 or BF16 tile tasks) twice instead; the small modes run the
    small case N=64, n=16 (mixed path: its solves run as the one-CTA small solve; plain FP64)."""
    import torch
    from paper_2601_03754_gb300 import btc, build, gen
    build.build()
    btc.load()
    if which in ("tiles_tf32", "tiles_bf16"):
        dt = btc.MIXED_TF32 if which == "tiles_tf32" else btc.MIXED_BF16
        D, B = gen.bt_random_torch(128, 256, delta=1.0, seed=7)
        p = btc.btc_plan(128, 256, dt)
        for _ in range(2):
            btc.btc_factor(p, D, B)
        print("profile", which, btc.btc_info(p))
        p.free()
        torch.cuda.synchronize()
        return 0
    W = WORKLOAD
    N, n, m = W["N"], W["n"], W["nrhs"]
    if which == "tf32":  # the tensor-core path on a smaller large-block case (inputs 134 MB > L2)
        N, n = 512, 128
    if which in ("small", "small_f64"):
        N, n, m = 64, 16, 1
    D, B = gen.bt_random(N, n, delta=W["delta"], seed=W["seed"])
    b = gen.rhs(N, n, m, seed=W["seed"])
    Dd, Bd, bd = (torch.from_numpy(a).cuda() for a in (D, B, b))
    xd = torch.zeros_like(bd)
    dts = {"mixed": [btc.MIXED_F32], "f64": [btc.F64], "both": [btc.MIXED_F32, btc.F64],
           "tf32": [btc.MIXED_TF32], "small": [btc.MIXED_F32], "small_f64": [btc.F64]}[which]
    for dt in dts:
        p = btc.btc_plan(N, n, dt)
        btc.btc_plan_set_graphs(p, False)  # ncu does not profile kernels inside graphs with conditional nodes
        btc.btc_plan_set_autotune(p, False)  # the default configuration, without the tuner's timing runs
        for _ in range(2):
            it, rel, rc = btc.btc_factor_solve_refined(p, Dd, Bd, bd, xd, m, tol=TOL, maxit=30)
        print(f"profile dtype={dt} iters={it} relres={rel:.3e}")
        p.free()
    torch.cuda.synchronize()
    return 0


def run_phases():
    """Per-level means of the per-node phase stamps (btc_plan_set_phase_trace) of the interlaced factor +
    forward launch on the benchmark workload (mixed path, default tuned configuration, graphs off); one
    JSON line. The stamps add one CTA barrier per phase, so node times are slightly above the untraced ones."""
    import numpy as np
    import torch
    from paper_2601_03754_gb300 import btc, build, gen
    build.build()
    btc.load()
    W = WORKLOAD
    N, n, m = W["N"], W["n"], W["nrhs"]
    D, B = gen.bt_random(N, n, delta=W["delta"], seed=W["seed"])
    b = gen.rhs(N, n, m, seed=W["seed"])
    Dd, Bd, bd = (torch.from_numpy(a).cuda() for a in (D, B, b))
    p = btc.btc_plan(N, n, btc.MIXED_F32)
    btc.btc_plan_set_graphs(p, False)
    ph = torch.zeros(8 * N, dtype=torch.int64, device="cuda")
    x = bd.clone()
    btc.btc_factor_solve(p, Dd, Bd, x, m)  # tuning pass, unstamped
    btc.btc_plan_set_phase_trace(p, ph)
    for _ in range(3):
        ph.zero_()
        x.copy_(bd)
        btc.btc_factor_solve(p, Dd, Bd, x, m)
        torch.cuda.synchronize()
    P = ph.view(N, 8).cpu().numpy().astype(np.float64)
    ok = P[:, 5] > 0
    t0 = P[ok, 0].min()
    lev = np.array([((i + 1) & -(i + 1)).bit_length() for i in range(N)])
    names = ["operands", "potrf_trsm", "store", "next_diag", "fill"]
    levels = {}
    for lv in sorted(set(lev[ok].tolist())):
        idx = np.where(ok & (lev == lv))[0]
        d = np.diff(P[idx, :6], axis=1) / 1e3
        levels[str(lv)] = {"nodes": int(len(idx)), "start_us": round(float((P[idx, 0].min() - t0) / 1e3), 2),
                           "end_us": round(float((P[idx, 5].max() - t0) / 1e3), 2),
                           "node_us": round(float(d.sum(1).mean()), 2),
                           **{k + "_us": round(float(d[:, j].mean()), 2) for j, k in enumerate(names)}}
    print(json.dumps({"workload": f"bt_random N={N} n={n} mixed, btc_factor_solve (interlaced)",
                      "flow_config": dict(zip(["resident_cap", "ctas_per_sm", "tuned"],
                                              btc.btc_plan_tuning_interlaced(p))),
                      "levels": levels}), flush=True)
    return 0


def _batch_run(btc, torch, specs, dt, chunks, steps, stream, flush, seed0):
    """One batch workload: factor + FP64-refined solve of every instance per step (graph after the first
    two calls); mean ms per batch over `steps` L2-flushed steps, the batch's tuning and its orders."""
    Ds, Bs, bs, xs = [], [], [], []
    for k, (N, n) in enumerate(specs):
        D, B = gen_bt(N, n, seed0 + k)
        Ds.append(D)
        Bs.append(B if B.numel() else torch.zeros((1, n, n), dtype=torch.float64, device="cuda"))
        g = torch.Generator(device="cuda")
        g.manual_seed(4000 + seed0 + k)
        bs.append(torch.randn((N * n, 1), generator=g, device="cuda", dtype=torch.float64))
        xs.append(torch.zeros_like(bs[-1]))
    Ns = [N for N, _ in specs]
    ns = [n for _, n in specs]
    batch = btc.btc_batch_plan(Ns, ns, dt, stream, chunks=chunks)
    q = btc.btc_batch_query(batch)

    def step():
        return btc.btc_batch_factor_solve_refined(batch, Ds, Bs, bs, xs, tol=TOL, maxit=30)

    with torch.cuda.stream(stream):
        step()  # tuning of every group
        step()  # graph capture
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, rel, rc = step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
    ms = statistics.mean(ts)
    tuning = []
    for g in range(q["groups"]):
        np_, cap, ctas, tuned, gms = btc.btc_batch_tuning(batch, g)
        tuning.append({"np": np_, "resident_cap": cap, "ctas_per_sm": ctas, "tuned": tuned,
                       "factor_ms_alone": round(gms, 3)})
    out = {"ms_per_batch": ms, "solves_per_s": len(specs) * 1000.0 / ms, "refine_iters": it, "max_relres": rel,
           "factor_gflop": q["factor_flops"] / 1e9, "factor_tflops": q["factor_flops"] / (ms * 1e-3) / 1e12,
           "groups": q["groups"], "group_tuning": tuning, "device_gb": q["device_bytes"] / 1e9}
    if chunks is not None:
        ch = np.asarray(chunks)
        out["orders"] = {"nested_dissection": int((ch == 0).sum()),
                         "partition_by_chunks": {str(c): int((ch == c).sum()) for c in sorted(set(ch.tolist())) if c}}
    batch.free()
    return out


def gen_bt(N, n, seed):
    from paper_2601_03754_gb300 import gen
    return gen.bt_random_torch(N, n, delta=1e-2, seed=seed)


def batched_measure(btc, gen, torch, steps, stream, flush):
    """Config: 512 instances, n uniform in {8,16,32,64}, N log-uniform in [32, 2048], one RHS each,
    delta = 1e-2; mixed FP32 factor + FP64 refinement to 1e-10, beside the plain FP64 batch. A step is
    btc_batch_factor_solve_refined: after the first (tuning) call, one captured graph with the
    refinement loop on the device. The tuned launch configuration of every block-size group is
    reported. Method dispatch (btc_dispatch_orders) is measured against nested dissection on this mix,
    on a throughput mix of 600 short systems (n in {16, 32}, N log-uniform in [32, 128]) and on a wide
    batch of 2000 systems N=64, n=32; a forced partition order on the benchmark mix's n <= 16 systems
    shows what the model avoids."""
    specs = gen.batch_specs(512, seed=0)
    Ns = [N for N, _ in specs]
    ns = [n for _, n in specs]
    out = {"instances": len(specs), "nodes": int(sum(Ns)), "n_mix": sorted(set(ns))}
    dispatch = btc.btc_dispatch_orders(Ns, ns, btc.MIXED_F32)
    forced = np.asarray([0 if n > 16 or N > 1000 else max(1, min(48, N // 4)) for N, n in specs], dtype=np.int32)
    out["mixed"] = _batch_run(btc, torch, specs, btc.MIXED_F32, None, steps, stream, flush, 1000)
    out["mixed_dispatch"] = _batch_run(btc, torch, specs, btc.MIXED_F32, dispatch, steps, stream, flush, 1000)
    out["mixed_forced_partition_n_le_16"] = _batch_run(btc, torch, specs, btc.MIXED_F32, forced, steps, stream,
                                                       flush, 1000)
    out["plain_f64"] = _batch_run(btc, torch, specs, btc.F64, None, max(2, steps // 4), stream, flush, 1000)
    out["speedup_vs_plain_f64"] = out["plain_f64"]["ms_per_batch"] / out["mixed"]["ms_per_batch"]
    out["dispatch_speedup"] = out["mixed"]["ms_per_batch"] / out["mixed_dispatch"]["ms_per_batch"]
    short = gen.batch_specs(600, seed=4, sizes=(16, 32), nmin=32, nmax=128)
    sd = btc.btc_dispatch_orders([N for N, _ in short], [n for _, n in short], btc.MIXED_F32)
    out["short_systems"] = {"instances": len(short),
                            "nested_dissection": _batch_run(btc, torch, short, btc.MIXED_F32, None, steps, stream,
                                                            flush, 7000),
                            "dispatch": _batch_run(btc, torch, short, btc.MIXED_F32, sd, steps, stream, flush, 7000)}
    out["short_systems"]["dispatch_speedup"] = (out["short_systems"]["nested_dissection"]["ms_per_batch"] /
                                                out["short_systems"]["dispatch"]["ms_per_batch"])
    # a wide batch of identical short systems, where the model takes the partition order
    wide = [(64, 32)] * 2000
    wd = btc.btc_dispatch_orders([N for N, _ in wide], [n for _, n in wide], btc.MIXED_F32)
    out["wide_batch_2000xN64n32"] = {
        "nested_dissection": _batch_run(btc, torch, wide, btc.MIXED_F32, None, steps, stream, flush, 20000),
        "dispatch": _batch_run(btc, torch, wide, btc.MIXED_F32, wd, steps, stream, flush, 20000)}
    w = out["wide_batch_2000xN64n32"]
    w["dispatch_speedup"] = w["nested_dissection"]["ms_per_batch"] / w["dispatch"]["ms_per_batch"]
    return out


def kappa_estimate(btc, torch, D, B, plan, iters=25):
    """2-norm condition number estimate of Psi: lambda_max by power iteration (FP64 block-tridiagonal
    products in torch), lambda_min by inverse iteration with the plan's FP64-refined solve; both as
    Rayleigh quotients. A measurement aid for the report, not part of the timed path."""
    N, n = D.shape[0], D.shape[1]

    def matvec(v):
        V = v.view(N, n, 1)
        y = torch.bmm(D, V)
        if N > 1:
            y[1:] += torch.bmm(B, V[:-1])
            y[:-1] += torch.bmm(B.transpose(1, 2), V[1:])
        return y.view(N * n, 1)

    g = torch.Generator(device="cuda")
    g.manual_seed(1234)
    v = torch.randn((N * n, 1), generator=g, device="cuda", dtype=torch.float64)
    v /= v.norm()
    lmax = 0.0
    for _ in range(iters):
        w = matvec(v)
        lmax = float((v * w).sum())
        v = w / w.norm()
    v = torch.randn((N * n, 1), generator=g, device="cuda", dtype=torch.float64)
    v /= v.norm()
    w = torch.zeros_like(v)
    lmin = 0.0
    for _ in range(iters):
        btc.btc_solve_refined(plan, v, w, 1, tol=1e-12, maxit=60, allow_not_converged=True)
        lmin = float((w * v).sum() / (w * w).sum())
        v = w / w.norm()
    return lmax / lmin if lmin > 0 else float("inf")


def large_block_measure(btc, gen, torch, stream, flush, steps=4):
    """Config: N=4096, n in {128, 256}, delta in {1, 1e-3, 1e-6}: the factor with the four n^3 products
    on tcgen05 tensor cores with TF32 and with BF16 operands (FP32 accumulation), FP64 top-separator
    Cholesky (n = 128; the blocked n = 256 path factors its top separator like every other node),
    FP64 residual and refinement to 1e-10; at n = 128 also the FP32 FMA factor. Per row: factor time
    and TFLOP/s, refined factor + solve time, refinement steps (or "not converged"), the relative
    residual reached (the error against the FP64 bar) and the measured condition number."""
    out = {"N": 4096}
    forms = {128: (("f32_ffma", btc.MIXED_F32), ("tf32", btc.MIXED_TF32), ("bf16", btc.MIXED_BF16)),
             256: (("tf32", btc.MIXED_TF32), ("bf16", btc.MIXED_BF16))}
    for n in (128, 256):
        for delta in (1.0, 1e-3, 1e-6):
            D, B = gen.bt_random_torch(4096, n, delta=delta, seed=7)
            g = torch.Generator(device="cuda")
            g.manual_seed(11)
            b = torch.randn((4096 * n, 1), generator=g, device="cuda", dtype=torch.float64)
            x = torch.zeros_like(b)
            res = {}
            for name, dt in forms[n]:
                p = btc.btc_plan(4096, n, dt, stream)
                info = btc.btc_plan_query(p)
                ts, tf = [], []
                with torch.cuda.stream(stream):
                    for rep in range(steps + 1):
                        flush.fill_(1.0)
                        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                        e0.record(stream)
                        btc.btc_factor(p, D, B)
                        e1.record(stream)
                        e1.synchronize()
                        flush.fill_(1.0)
                        e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                        e2.record(stream)
                        it, rel, rc = btc.btc_factor_solve_refined(p, D, B, b, x, 1, tol=TOL, maxit=60,
                                                                   allow_not_converged=True)
                        e3.record(stream)
                        e3.synchronize()
                        if rep >= 1:
                            tf.append(e0.elapsed_time(e1))
                            ts.append(e2.elapsed_time(e3))
                btc.btc_plan_set_timing(p, True)
                with torch.cuda.stream(stream):
                    btc.btc_factor(p, D, B)
                k_ms, k_n = btc.btc_plan_timing(p)
                btc.btc_plan_set_timing(p, False)
                row = {"ms_factor": statistics.mean(tf), "ms_factor_solve_refined": statistics.mean(ts),
                       "factor_tflops": info["factor_flops"] / (statistics.mean(tf) * 1e-3) / 1e12,
                       "ms_factor_kernel": k_ms[btc.TIME_FACTOR], "ms_root": k_ms[btc.TIME_ROOT] or None,
                       "refine_steps": it if rc == btc.OK else "not converged", "relres": rel}
                if name == "tf32" and "kappa" not in res:
                    row["kappa_estimate"] = kappa_estimate(btc, torch, D, B, p)
                    res["kappa"] = row["kappa_estimate"]
                res[name] = row
                p.free()
            out[f"n{n}_delta{delta:g}"] = res
            del D, B
            torch.cuda.empty_cache()
    return out


def gmres_ir_measure(btc, torch, stream):
    """GMRES-IR against classical refinement on tensor-core factors (n = 128, TF32 and BF16 operands)
    of ill-conditioned block Laplacians (D_i = 2I + small SPD perturbation, B_i = -I,
    kappa ~ 4 (N+1)^2 / pi^2): preconditioned solves (classical: one per step; GMRES-IR: one per outer
    step plus one per Arnoldi step), final relative residual and wall time of each, on the same
    factorization. Where the BF16 factor's error times kappa approaches 1, classical refinement stalls
    and GMRES-IR still reaches the FP64 bar."""
    import numpy as np
    out = {}
    n = 128
    for N in (129, 513, 1025):
        rng = np.random.default_rng(N)
        M = rng.standard_normal((N, n, n)) * 0.05
        D = 2.0 * np.eye(n)[None] + M @ np.swapaxes(M, 1, 2) / n
        B = np.tile(-np.eye(n), (N - 1, 1, 1))
        b = rng.standard_normal((N * n, 1))
        Dd, Bd, bd = (torch.from_numpy(a).cuda() for a in (D, B, b))
        for oname, dt in (("tf32", btc.MIXED_TF32), ("bf16", btc.MIXED_BF16)):
            p = btc.btc_plan(N, n, dt, stream)
            with torch.cuda.stream(stream):
                btc.btc_factor(p, Dd, Bd)
                res = {"kappa_estimate": 4.0 * (N + 1) ** 2 / np.pi ** 2}
                for name in ("classical", "gmres_ir"):
                    x = torch.zeros_like(bd)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    if name == "classical":
                        it, rel, rc = btc.btc_solve_refined(p, bd, x, 1, tol=TOL, maxit=100, allow_not_converged=True)
                        steps = {"steps": it, "preconditioned_solves": it + 1}
                    else:
                        o, i, rel, rc = btc.btc_solve_gmres_ir(p, bd, x, tol=TOL, max_outer=20, restart=60,
                                                               allow_not_converged=True)
                        steps = {"outer_steps": o, "arnoldi_steps": i, "preconditioned_solves": 1 + o + i}
                    torch.cuda.synchronize()
                    res[name] = {**steps, "relres": rel, "converged": rc == btc.OK,
                                 "ms": 1000.0 * (time.perf_counter() - t0)}
            out[f"N{N}_n{n}_{oname}"] = res
            p.free()
    return out


def c2_measure(btc, gen, torch, stream, flush, steps=8):
    """Config C2 beyond the headline row: N=1024, n=64, m in {1, 16}; the bt_random generator at
    delta in {1, 1e-2, 1e-4} and the MPC-like generator. Per input: the measured condition number, then
    per form (mixed FP32 factor + FP64 refinement to 1e-10; plain FP64; plain FP32 factor + one solve,
    no refinement) and m: factor + solve time (L2 flushed), refinement steps and relative residual."""
    N, n = 1024, 64
    out = {}
    inputs = [(f"delta{d:g}", lambda d=d: gen.bt_random(N, n, delta=d, seed=3)) for d in (1.0, 1e-2, 1e-4)]
    inputs.append(("mpc", lambda: gen.mpc(N, n, seed=3)))
    for name, make in inputs:
        D, B = make()
        res = {}
        for dt, form in ((btc.MIXED_F32, "mixed"), (btc.F64, "plain_f64"), (btc.F32, "plain_f32")):
            tdt = torch.float32 if dt == btc.F32 else torch.float64
            Dd, Bd = (torch.from_numpy(a).to("cuda", tdt) for a in (D, B))
            p = btc.btc_plan(N, n, dt, stream)
            if form == "mixed":
                Dk, Bk = (torch.from_numpy(a).cuda() for a in (D, B))
                btc.btc_factor(p, Dk, Bk)
                res["kappa_estimate"] = kappa_estimate(btc, torch, Dk, Bk, p)
            for m in (1, 16):
                b = torch.from_numpy(gen.rhs(N, n, m, seed=4)).to("cuda", tdt)
                x = torch.zeros_like(b)
                ts = []
                with torch.cuda.stream(stream):
                    for rep in range(steps + 2):
                        flush.fill_(1.0)
                        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                        if dt == btc.F32:
                            x.copy_(b)
                            e0.record(stream)
                            btc.btc_factor_solve(p, Dd, Bd, x, m)
                            e1.record(stream)
                            it, rel = 0, None
                        else:
                            e0.record(stream)
                            it, rel, rc = btc.btc_factor_solve_refined(p, Dd, Bd, b, x, m, tol=TOL, maxit=30)
                            e1.record(stream)
                        e1.synchronize()
                        if rep >= 2:
                            ts.append(e0.elapsed_time(e1))
                if dt == btc.F32:
                    r, a, xn = btc.btc_residual(N, n, m, torch.from_numpy(D).cuda(), torch.from_numpy(B).cuda(),
                                                x.double(), b.double())
                    rel = r / (a * xn)
                res[f"{form}_m{m}"] = {"ms": statistics.mean(ts), "solves_per_s": 1000.0 / statistics.mean(ts),
                                      "refine_steps": it, "relres": rel}
            p.free()
        out[name] = res
    return out


def small_case_measure(btc, gen, torch, stream, flush, steps=200):
    """Config C1: N=64, n=16, one RHS: factor + solve latency (p50/p99) of the plain FP64 path and the
    mixed path (both to 1e-10), against a critical-path model: the planner's critical-path flops
    (largest node cost per level, Sec. 4.3 with p = infinity) at one SM's FP64 rate (1.68 DFMA/clock,
    measured with warps on all four sub-partitions)."""
    N, n = 64, 16
    D, B = gen.bt_random(N, n, delta=1.0, seed=0)
    b = gen.rhs(N, n, 1, seed=0)
    Dd, Bd, bd = (torch.from_numpy(a).cuda() for a in (D, B, b))
    out = {"N": N, "n": n}
    for name, dt in (("plain_f64", btc.F64), ("mixed_f32", btc.MIXED_F32)):
        p = btc.btc_plan(N, n, dt, stream)
        info = btc.btc_plan_query(p)
        x = torch.zeros_like(bd)
        ts = []
        with torch.cuda.stream(stream):
            for rep in range(steps + 5):
                e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                e0.record(stream)
                it, rel, _ = btc.btc_factor_solve_refined(p, Dd, Bd, bd, x, 1, tol=TOL, maxit=30)
                e1.record(stream)
                e1.synchronize()
                if rep >= 5:
                    ts.append(1000.0 * e0.elapsed_time(e1))
        model_us = info["critical_path_flops"] / (FP64_PEAK_PER_SM_CLK * 2070e6) * 1e6
        out[name] = {"p50_us": statistics.median(ts), "p99_us": float(np.percentile(np.asarray(ts), 99)),
                     "refine_iters": it, "relres": rel, "levels": info["levels"],
                     "critical_path_model_us": model_us,
                     "critical_path_model": "critical-path flops at one SM's FP64 rate (1.68 DFMA/clock measured, "
                                            "2070 MHz)"}
        p.free()
    return out


def interlace_measure(btc, gen, torch, stream, flush, steps=30):
    """The paper's interlaced factor + forward substitution (Sec. 5, n=64, N=128 in its traces):
    btc_factor_solve against btc_factor followed by btc_solve, one RHS, mixed path, no refinement."""
    out = {}
    for N, n in ((128, 64), (1024, 64)):
        D, B = gen.bt_random(N, n, delta=1.0, seed=0)
        b = gen.rhs(N, n, 1, seed=0)
        Dd, Bd, bd = (torch.from_numpy(a).cuda() for a in (D, B, b))
        p = btc.btc_plan(N, n, btc.MIXED_F32, stream)
        x = bd.clone()
        res = {}
        for name, body in (("sequential", lambda: (btc.btc_factor(p, Dd, Bd), btc.btc_solve(p, x, 1))),
                           ("interlaced", lambda: btc.btc_factor_solve(p, Dd, Bd, x, 1))):
            ts = []
            with torch.cuda.stream(stream):
                for rep in range(steps + 3):
                    flush.fill_(1.0)
                    x.copy_(bd)
                    e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                    e0.record(stream)
                    body()
                    e1.record(stream)
                    e1.synchronize()
                    if rep >= 3:
                        ts.append(1000.0 * e0.elapsed_time(e1))
            res[name + "_us"] = statistics.median(ts)
        res["time_saved"] = 1.0 - res["interlaced_us"] / res["sequential_us"]
        out[f"N{N}_n{n}"] = res
        p.free()
    return out


def _latency_by_n(pool, which, results, ok_status):
    """p50 / p99 latency (us) per block size of the request mix (the service time spans two orders of
    magnitude between the smallest and the largest systems, so the overall p99 is mostly the largest
    ones' service time)."""
    import numpy as np
    by = {}
    for k, r in enumerate(results):
        if r["status"] == ok_status:
            by.setdefault(pool[which[k]]["n"], []).append(r["latency_us"])
    return {str(n): {"p50": round(float(np.percentile(v, 50)), 1), "p99": round(float(np.percentile(v, 99)), 1),
                     "count": len(v)} for n, v in sorted(by.items())}


def serving_measure(btc, torch, rates=(1000.0, 5000.0, 20000.0, 50000.0), count=5000, pool_size=128):
    """Config: Poisson stream of factor+solve requests, n uniform in {12,24,48,96}, N log-uniform
    in [50, 5000], MPC-like generator, 30% re-solves of a cached factor, HBM-footprint admission;
    mixed FP32+FP64-refinement server (FP64 root) vs plain FP64 server; p50/p99 latency and sustained
    solves/s per offered rate, and the knee (the first rate the server does not sustain within 10 %).
    Both servers are prewarmed (plans of every size bucket built, tuned and captured before the
    traffic), so no request pays plan construction. The pool holds `pool_size` distinct systems of
    distinct sizes; every returned x is re-checked by the FP64 residual."""
    from paper_2601_03754_gb300 import serve
    t0 = time.perf_counter()
    pool = serve.make_pool(count=pool_size, seed=0)
    out = {"pool": len(pool), "distinct_shapes": len({(p["N"], p["n"]) for p in pool}), "requests_per_rate": count,
           "slots": 8, "hbm_budget_gb": 64, "prewarm_copies": 2, "pool_build_s": round(time.perf_counter() - t0, 1)}
    for name, dt, rr, cnt in (("mixed", btc.MIXED_F32, rates, count), ("plain_f64", btc.F64, rates[:2], count // 2)):
        srv = btc.btc_server_start(dt, slots=8, hbm_budget_bytes=64 << 30, cache_factors=True)
        t0 = time.perf_counter()
        for n in (12, 24, 48, 96):
            btc.btc_server_prewarm(srv, n, 5000, copies=2)
        res = {"prewarm_s": round(time.perf_counter() - t0, 1)}
        serve.run_stream(srv, pool, 2000.0, 200, seed=1)  # warm-up traffic
        knee = None
        for rate in rr:
            btc.btc_server_reset_stats(srv)
            results, wall, xs, which, rhs, span = serve.run_stream(srv, pool, rate, cnt, seed=2)
            st = btc.btc_server_stats(srv)
            lat = np.asarray([r["latency_us"] for r in results if r["status"] == btc.OK])
            ok = int(lat.size)
            sustained = ok / wall
            statuses = {}
            for r_ in results:
                statuses[str(r_["status"])] = statuses.get(str(r_["status"]), 0) + 1
            row = {"offered_req_per_s": cnt / span if span > 0 else None, "statuses": statuses,
                   "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                   "mean_us": float(lat.mean()), "solves_per_s": sustained, "completed": ok,
                   "cache_hits": st["cache_hits"],
                   "max_relres": max(r["relres"] for r in results if r["status"] == btc.OK),
                   "queue_and_service_us": {k: round(st[k], 1) for k in (
                       "p50_queue_us", "p99_queue_us", "p50_service_us", "p99_service_us")},
                   "latency_by_n_us": _latency_by_n(pool, which, results, btc.OK),
                   **serve.check_results(pool, xs, which, rhs)}
            res[str(int(rate))] = row
            if knee is None and sustained < 0.9 * rate:
                knee = rate
        res["knee_req_per_s"] = knee
        res["device_gb"] = btc.btc_server_stats(srv)["device_bytes"] / 1e9
        srv.stop()
        out[name] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-instance batched measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-server measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the N=4096, n in {128, 256} measurement")
    ap.add_argument("--no-c2", action="store_true", help="skip the N=1024 delta/MPC/16-RHS rows")
    ap.add_argument("--phases", action="store_true", help="per-level node phase times of the factor launch")
    ap.add_argument("--profile", choices=["mixed", "f64", "both", "tf32", "tiles_tf32", "tiles_bf16", "small", "small_f64"],
                    default=None,
                    help="run the workload's factor + refined solve twice (no timing) for an ncu capture")
    args = ap.parse_args()
    if args.profile:
        return run_profile(args.profile)
    if args.phases:
        return run_phases()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_2601_03754_gb300 import btc, build, gen

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    btc.load()
    W = WORKLOAD
    N, n, m = W["N"], W["n"], W["nrhs"]
    D, B = gen.bt_random(N, n, delta=W["delta"], seed=W["seed"] + rank)
    b = gen.rhs(N, n, m, seed=W["seed"] + rank)
    stream = torch.cuda.Stream()
    Dd = torch.from_numpy(D).cuda()
    Bd = torch.from_numpy(B).cuda()
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def timed_steps(plan, steps, body):
        """Per-step CUDA events on the plan's stream, L2 flushed before each step."""
        ts = []
        with torch.cuda.stream(stream):
            for _ in range(steps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out = body()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
        return ts, out

    # ---- chosen form: FP32 factor + FP64 refinement
    pm = btc.btc_plan(N, n, btc.MIXED_F32, stream)
    info = btc.btc_plan_query(pm)

    def mixed_step():
        return btc.btc_factor_solve_refined(pm, Dd, Bd, bd, xd, m, tol=TOL, maxit=30)

    timed_steps(pm, args.warmup, mixed_step)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = NvmlClockSampler(local).start()
    if clocks is None:
        clocks = ClockSampler(local)
        clocks.start()
    t_wall0 = time.perf_counter()
    ts, (iters, rel, rc) = timed_steps(pm, args.steps, mixed_step)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms, value = replica_throughput(statistics.mean(ts), world)
    assert rel <= TOL, rel

    # ---- the same step with the double-FP32 top-separator Cholesky (the option beside the FP64 default)
    pr = btc.btc_plan(N, n, btc.MIXED_F32, stream)
    btc.btc_plan_set_root_precision(pr, btc.ROOT_DOUBLE_FP32)

    def root_df32_step():
        return btc.btc_factor_solve_refined(pr, Dd, Bd, bd, xd, m, tol=TOL, maxit=30)

    timed_steps(pr, 3, root_df32_step)
    tsdr, (itdr, reldr, _) = timed_steps(pr, max(10, min(100, args.steps // 4)), root_df32_step)
    root_double_fp32_option = {"ms_per_step": statistics.mean(tsdr), "refine_iters": itdr, "relres": reldr,
                               "note": "top-separator Cholesky in double-FP32 (pairs of FP32, about 48 bits) "
                                       "instead of FP64"}
    pr.free()

    # ---- per-kernel device times of the same step (library events on the plan's stream, L2 flushed),
    # for the phase split and the roofline of the dominant kernel
    n_phase = max(10, min(200, args.steps // 2))
    btc.btc_plan_set_timing(pm, True)
    timed_steps(pm, n_phase, mixed_step)
    k_ms, k_n = btc.btc_plan_timing(pm)
    btc.btc_plan_set_timing(pm, False)
    phase = {name: (k_ms[c] / k_n[c] if k_n[c] else None) for name, c in
             (("factor_forward_interlaced", btc.TIME_FACTOR_FORWARD), ("root_chol", btc.TIME_ROOT),
              ("solve_tail", btc.TIME_SOLVE_TAIL), ("correction_solve", btc.TIME_SOLVE),
              ("residual", btc.TIME_RESIDUAL))}
    t_fused = phase["factor_forward_interlaced"]

    # ---- the plain FP64 GPU path on the same workload
    p64 = btc.btc_plan(N, n, btc.F64, stream)

    def f64_step():
        return btc.btc_factor_solve_refined(p64, Dd, Bd, bd, xd, m, tol=TOL, maxit=30)

    timed_steps(p64, 3, f64_step)
    ts64, (it64, rel64, _) = timed_steps(p64, max(5, min(50, args.steps // 5)), f64_step)
    ms64 = statistics.mean(ts64)

    # ---- end to end through the host-buffer entry point (pinned host memory)
    Dh = torch.from_numpy(D).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    pe = btc.btc_plan(N, n, btc.MIXED_F32, stream)
    for _ in range(2):
        btc.btc_factor_solve_host(pe, Dh, Bh, bh, xh, m, TOL, 30)
    e2e_ts = []
    for _ in range(max(5, min(100, args.steps // 4))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        btc.btc_factor_solve_host(pe, Dh, Bh, bh, xh, m, TOL, 30)
        e2e_ts.append(time.perf_counter() - t0)
    e2e_v = 1.0 / statistics.mean(e2e_ts)
    # the level-1 loads read D's lower triangles (and, in the diagonal 4x4 tiles of the blocks they read as
    # a tile of D_(e+1), the few entries above the diagonal there) and all of B from the pinned buffers;
    # b is copied
    R = 4
    h2d = (N * n * (n + 1) // 2 + (N // 2) * (n // R) * (R * (R - 1) // 2)) * D.itemsize + B.nbytes + b.nbytes
    d2h = b.nbytes

    batched = (batched_measure(btc, gen, torch, max(3, min(10, args.steps // 5)), stream, flush)
               if not args.no_batch else None)
    serving = serving_measure(btc, torch) if not args.no_serve else None
    large = large_block_measure(btc, gen, torch, stream, flush) if not args.no_large else None
    gmres = gmres_ir_measure(btc, torch, stream) if not args.no_large else None
    small = small_case_measure(btc, gen, torch, stream, flush)
    c2 = c2_measure(btc, gen, torch, stream, flush) if not args.no_c2 else None
    interlace = interlace_measure(btc, gen, torch, stream, flush)
    # solve roofline: each factor block read once per direction (the compulsory bytes of Alg. 7, m = 1)
    solve_bytes = 2.0 * (N + info["offdiag_blocks"]) * n * n * 4
    t_solve = phase["correction_solve"]
    solve_roof = {"kernel": "k_solve_flow (one correction solve, forward + backward)", "bound": "hbm",
                  "achieved": solve_bytes / (t_solve * 1e-3) / 1e9, "peak": None, "unit": "GB/s",
                  "algorithmic_bytes": solve_bytes,
                  "note": "bound by 22 dependent levels; part of the factor is still in L2 from the factorization"}

    peaks, pk_kind = _peaks()
    solve_roof["peak"] = peaks.get("hbm_gbs")
    solve_roof["frac"] = solve_roof["achieved"] / solve_roof["peak"] if solve_roof["peak"] else None
    sm_max = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SMS * FP32_PEAK_PER_SM_CLK * sm_max * 1e6 / 1e12
    # algorithmic work of the interlaced launch: Table 1 factor costs without the top separator's
    # potrf (its own FP64 kernel), plus the forward sweep (Alg. 7: n^2 m per eliminated node, 2 n^2 m
    # per off-diagonal block)
    root_flops = n ** 3 / 3.0
    fwd_flops = m * (N * n * n + 2.0 * info["offdiag_blocks"] * n * n)
    fused_flops = info["factor_flops"] - root_flops + fwd_flops
    achieved = fused_flops / (t_fused * 1e-3) / 1e12
    traffic = _traffic_from_profile()
    # graph of one step: pack, interlaced factor + forward, FP64 root, solve tail, unpack, residual,
    # stopping test; per refinement step: solve, update, residual, stopping test
    launches = 7 + 4 * iters

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (factor, solves) + f64 (root chol) + f64 (residual, update)",
        "data": "synthetic",
        "config": {"workload": "bt_random N=1024 n=64 nrhs=1 delta=1 seed=0; mixed FP32 factor + FP64 refinement "
                               "to relres<=1e-10", "N": N, "n": n, "nrhs": m, "delta": W["delta"],
                   "l2": "flushed before every step (256 MB write, outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "latency_us": {"p50": 1000 * statistics.median(ts),
                       "p99": 1000 * float(np.percentile(np.asarray(ts), 99)), "mean": 1000 * ms},
        "refine_iters": iters, "relres": rel,
        "plain_f64": {"ms_per_step": ms64, "solves_per_s": 1000.0 / ms64, "refine_iters": it64, "relres": rel64,
                      "p99_us": 1000 * float(np.percentile(np.asarray(ts64), 99))},
        "speedup_vs_plain_f64": ms64 / ms,
        "phases_ms": phase,
        "flow_config": dict(zip(("resident_cap", "ctas_per_sm", "tuned"), btc.btc_plan_tuning_interlaced(pm))),
        "root_double_fp32_option": root_double_fp32_option,
        "gmres_ir_vs_classical": gmres,
        "roofline": {"kernel": "k_factor_fwd_flow (interlaced factor + forward sweep, one launch per step)",
                     "bound": "alu",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": traffic,
                     "peak_kind": f"FP32 FFMA: {SMS} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz (derived)",
                     "algorithmic": f"{fused_flops:.4g} flop per launch (Alg. 5 Table 1 costs without the top "
                                    f"separator + Alg. 7 forward sweep)"},
        "e2e": {"value": e2e_v * world, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "entry_point": "btc_factor_solve_host (pinned host buffers; the level-1 eliminations read D, B "
                               "over the CPU-GPU link while level 1 runs)"},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "peaks_source": pk_kind,
        "batched": batched,
        "serving": serving,
        "large_blocks": large,
        "small_case": small,
        "c2_delta_mpc_m16": c2,
        "interlaced_vs_sequential": interlace,
        "solve_roofline": solve_roof,
        "wall_s_timed": t_wall,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
