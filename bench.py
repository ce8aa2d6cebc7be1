#!/usr/bin/env python3
"""Benchmark of the Discrete Projection Moment hot path on GB300.

One step = one call of the whole pipeline (clear images, fused projection,
image moments, combine) for the 512^3 float32 MRI-like volume at K = 6
(84 moments), the configuration the headline metric is quoted on.  The
volume (537 MB) is larger than the 129 MB L2, so successive steps cannot
hit in L2 and no flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own replica on its own GPU
(weak scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
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

METRIC = "voxels/s and % HBM peak for M_pqr (K=6) at 512^3; batched vol/s, p50/p99 latency"
UNIT = "voxel/s"
L = M = N = 512
K = 6
SEED = 3
WORKLOAD = "mri_like_f32_512x512x512_K6"
CASE = "f32"  # volume recipe: f32 MRI-like, u16 CT-like phantom, u8 uniform
KERNEL_SRC = os.path.join(ROOT, "paper_2012_08099_gb300", "csrc", "k1_int.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k1_int_mri512_f32_k6_traffic.json")
K1_NAME = "k1_int_kernel (fused projection; float32 as two quantised int32 limbs)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-single-rows", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=400)
    ap.add_argument("--shape", default=None,
                    help="L,M,N of a smaller volume of the same recipe (profiling runs)")
    ap.add_argument("--case", default=None,
                    help="dtype:K of a profiling run (u16 = CT-like phantom, u8 = uniform "
                         "0-255, f32 = MRI-like); the headline line is f32:6")
    args = ap.parse_args()
    global L, M, N, WORKLOAD, CASE, K
    if args.shape:
        L, M, N = (int(v) for v in args.shape.split(","))
    if args.case:
        CASE, k = args.case.split(":")
        K = int(k)
    if args.shape or args.case:
        recipe = {"f32": "mri_like_f32", "u16": "ct_phantom_u16", "u8": "uniform_u8"}[CASE]
        WORKLOAD = f"{recipe}_{L}x{M}x{N}_K{K}"
    return args


def make_volume(seed):
    from paper_2012_08099_gb300 import synth
    if CASE == "u16":
        return synth.ct_phantom_u16(L, M, N, seed=seed)
    if CASE == "u8":
        return synth.uniform_volume((N, M, L), np.uint8, seed=seed)
    return synth.mri_like_f32(L, M, N, seed=seed)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the slowest replica's time); x itself
    without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all replicas processed per second of the slowest one."""
    return world * units_per_rank / seconds


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        with open(self.tmp.name) as f:
            rows = [r.strip() for r in f if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU baseline


def oracle_rate(vol_slab: np.ndarray, threads: int):
    import oracle
    t0 = time.perf_counter()
    oracle.moments(vol_slab, K, nthreads=threads)
    return time.perf_counter() - t0


def cpu_baseline(vol: np.ndarray, budget_s: float):
    """The oracle (Eq. 2, FP64) on a z-slab of the same volume, all host cores."""
    threads = os.cpu_count() or 1
    t1 = oracle_rate(np.ascontiguousarray(vol[:2]), threads) / 2.0
    nz = int(max(2, min(vol.shape[0], budget_s / max(t1, 1e-6))))
    nz = max(threads, nz - nz % threads) if nz >= threads else nz
    nz = min(nz, vol.shape[0])
    slab = np.ascontiguousarray(vol[:nz])
    dt = oracle_rate(slab, threads)
    vox = slab.size
    return {"value": vox / dt, "unit": UNIT, "cores": min(threads, nz), "kind": "oracle",
            "sample": f"z-slab {L}x{M}x{nz} of the {WORKLOAD} volume, K={K}, "
                      f"{vox} voxels in {dt:.2f} s"}


def cpu_dpma_baseline(vol: np.ndarray, reps: int = 5):
    """The multithreaded CPU DPMA (projections, 1-D integrals, exact
    combine) on the whole volume, all host cores; median of `reps` runs."""
    import cpu_dpma
    cpu_dpma.moments(vol, K)  # plan and page-in
    ts = []
    used = 0
    for _ in range(reps):
        t0 = time.perf_counter()
        _, used = cpu_dpma.moments(vol, K, return_threads=True)
        ts.append(time.perf_counter() - t0)
    dt = statistics.median(ts)
    return {"value": vol.size / dt, "unit": UNIT, "cores": used, "kind": "cpu_dpma",
            "sample": f"the whole {WORKLOAD} volume ({vol.size} voxels), median of {reps} runs "
                      f"of {dt:.3f} s"}


# ------------------------------------------------------------------- ours


def counters_if_current():
    """ncu counters of the projection kernel for this workload, per launch
    (dram bytes, warp instructions), if they were taken on the kernel source
    as it stands; else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
        with open(KERNEL_SRC, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
        if rec.get("k1_int_sha256") == h:
            return rec
    except Exception:
        pass
    return None


def run_ours(args):
    import torch

    import paper_2012_08099_gb300 as dpma
    from paper_2012_08099_gb300 import synth

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    lib = dpma.lib()
    vol = make_volume(SEED + rank)
    DT = {"f32": dpma.F32, "u16": dpma.U16, "u8": dpma.U8}[CASE]
    t = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda()
    nm = dpma.num_moments(K)
    ws = torch.empty(dpma.workspace_size(L, M, N, DT, K), dtype=torch.uint8, device="cuda")
    out = torch.empty(nm * 2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    vp, op, wp = (ctypes.c_void_p(x.data_ptr()) for x in (t, out, ws))
    wbytes = ws.numel()

    def step():
        rc = lib.dpma_moments_async(vp, L, M, N, DT, K, op, sp, wp, wbytes)
        if rc:
            raise dpma.DpmaError(rc, lib.dpma_last_error().decode())

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            step()
    stream.synchronize()
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    dpma.stage_timing(True)
    dpma.stage_times(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    e1.synchronize()
    barrier()
    stage_ms, stage_launches = dpma.stage_times(reset=True)
    dpma.stage_timing(False)
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    ms_step = max_over_ranks(ms_total / args.steps, dist, "cuda")
    voxels = float(L * M * N)
    value = whole_job_rate(voxels, world, ms_step * 1e-3)

    # roofline of the dominant kernel (fused projection): algorithmic bytes =
    # every voxel read once
    k1_ms = stage_ms[1] / args.steps
    algo_bytes = float(vol.nbytes)
    peak, peak_kind = measured_hbm_peak()
    achieved = algo_bytes / (k1_ms * 1e-3) / 1e9
    ctr = counters_if_current() if (L, M, N) == (512, 512, 512) else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": float(ctr["dram_bytes_per_launch"]) if ctr else None,
                "peak_source": f"{peak_kind} hbm_gbs",
                "kernel": K1_NAME, "kernel_ms": round(k1_ms, 5),
                "pipeline_frac": round(algo_bytes / (ms_step * 1e-3) / 1e9 / peak, 4),
                "stage_ms_per_step": [round(s / args.steps, 5) for s in stage_ms],
                "stage_launches_per_step": [round(n / args.steps, 3) for n in stage_launches]}
    gpu_launches = int(sum(stage_launches))
    # The integer-lane projection does its exact sums on the integer/ALU
    # pipes; what bounds it is instruction issue: 4 schedulers per SM, one
    # warp instruction each per clock.  Instructions per launch come from the
    # ncu capture of the same kernel source (scaled to 512 slices).
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    issue_roofline = None
    if clk and clk.get("sm_mhz") and ctr and ctr.get("warp_inst_per_launch"):
        inst = float(ctr["warp_inst_per_launch"])
        ipk = sms * 4 * clk["sm_mhz"] * 1e6 / 1e12
        ach = inst / (k1_ms * 1e-3) / 1e12
        issue_roofline = {"bound": "issue", "achieved": round(ach, 4), "peak": round(ipk, 4),
                          "unit": "Twarp-inst/s", "frac": round(ach / ipk, 4), "kernel": K1_NAME,
                          "thread_inst_per_voxel": round(inst * 32 / voxels, 2),
                          "peak_source": f"{sms} SMs x 4 schedulers x median SM clock"}

    # end to end through the C ABI from pinned host memory
    hv = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).pin_memory()
    out_bytes = nm * (8 if CASE == "f32" else 16)
    ho = torch.empty(nm * 2, dtype=torch.float64).pin_memory()
    hvp, hop = ctypes.c_void_p(hv.data_ptr()), ctypes.c_void_p(ho.data_ptr())
    for _ in range(3):
        lib.dpma_moments_host(hvp, L, M, N, DT, K, hop)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        rc = lib.dpma_moments_host(hvp, L, M, N, DT, K, hop)
        if rc:
            raise dpma.DpmaError(rc, lib.dpma_last_error().decode())
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist, "cuda")
    e2e = {"value": whole_job_rate(voxels, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(vol.nbytes), "d2h_bytes_per_step": int(out_bytes + 8),
           "ms_per_step": round(e2e_s * 1e3, 4)}

    batched = serving = singles = None
    if rank == 0 and not args.no_single_rows:
        singles = run_single_rows(dpma, torch, peak)
    if rank == 0 and not args.no_batched:
        batched = run_batched(dpma, torch)
    if rank == 0 and not args.no_serving:
        serving = run_serving(dpma, args.serving_requests)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(vol, args.cpu_budget_s)
        cpu["cpu_dpma"] = cpu_dpma_baseline(vol)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "u16": "u16", "u8": "u8"}[CASE], "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": L, "M": M, "N": N, "K": K,
                       "moments": nm, "images": dpma.num_images(K),
                       "volume_bytes": int(vol.nbytes), "parallelism": f"replicas{world}",
                       "l2": f"input {vol.nbytes / 1e6:.0f} MB vs 129 MB L2"
                             + (" (larger: no flush needed)" if vol.nbytes > 129e6 else "")},
            "roofline": roofline, "issue_roofline": issue_roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": gpu_launches, "clocks": clk,
            "single_volume_rows": singles, "batched": batched, "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------ single-volume rows


def run_single_rows(dpma, torch, peak):
    """The two smaller single-volume workloads: 64^3 u8 (uniform 0-255) at
    K = 3, and the 256^3 u16 CT-like phantom at K = 6.  Both fit in the
    129 MB L2, so every timed call of the phantom follows a 256 MB write
    that flushes it; the 64^3 volume (256 KB) is timed as a call rate
    (back-to-back asynchronous calls) and as the latency of the synchronous
    call, each with the projection kernel's own event time."""
    from paper_2012_08099_gb300 import synth
    lib = dpma.lib()
    rows = []
    s = torch.cuda.Stream()
    sp = ctypes.c_void_p(s.cuda_stream)

    def setup(vol, dt, K):
        t = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda()
        L_, M_, N_ = vol.shape[2], vol.shape[1], vol.shape[0]
        ws = torch.empty(dpma.workspace_size(L_, M_, N_, dt, K), dtype=torch.uint8, device="cuda")
        out = torch.empty(dpma.num_moments(K) * 2, dtype=torch.int64, device="cuda")
        args = (ctypes.c_void_p(t.data_ptr()), L_, M_, N_, dt, K, ctypes.c_void_p(out.data_ptr()),
                sp, ctypes.c_void_p(ws.data_ptr()), ws.numel())

        def call():
            rc = lib.dpma_moments_async(*args)
            if rc:
                raise dpma.DpmaError(rc, lib.dpma_last_error().decode())
        return t, out, call

    def k1_stage(call, reps, between=None):
        dpma.stage_timing(True)
        dpma.stage_times(reset=True)
        with torch.cuda.stream(s):
            for _ in range(reps):
                if between:
                    between()
                call()
        s.synchronize()
        ms, n = dpma.stage_times(reset=True)
        dpma.stage_timing(False)
        return [m / reps for m in ms], [x / reps for x in n]

    # 64^3 u8, K = 3
    vol = synth.uniform_volume((64, 64, 64), np.uint8, seed=1)
    t, out, call = setup(vol, dpma.U8, 3)
    with torch.cuda.stream(s):
        for _ in range(20):
            call()
    s.synchronize()
    reps = 2000
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        e0.record(s)
        for _ in range(reps):
            call()
        e1.record(s)
    e1.synchronize()
    us_async = e0.elapsed_time(e1) * 1e3 / reps
    lat = []
    for _ in range(300):
        t0 = time.perf_counter()
        dpma.moments(t, 3, dpma.U8, out=out.view(-1, 2))
        lat.append((time.perf_counter() - t0) * 1e6)
    st_ms, st_n = k1_stage(call, 500)
    k1_us = st_ms[1] * 1e3
    rows.append({"workload": "uniform_u8_64x64x64_K3", "metric": "us per call",
                 "us_per_call_async": round(us_async, 3),
                 "us_per_call_sync_p50": round(statistics.median(lat), 2),
                 "k1_us": round(k1_us, 3),
                 "stage_us": [round(m * 1e3, 3) for m in st_ms],
                 "roofline": {"bound": "hbm", "achieved": round(vol.nbytes / (k1_us * 1e-6) / 1e9, 1),
                              "peak": peak, "unit": "GB/s",
                              "frac": round(vol.nbytes / (k1_us * 1e-6) / 1e9 / peak, 4),
                              "note": "256 KB volume, L2-resident between calls"},
                 "gpu_launches_per_call": sum(st_n)})

    # 256^3 u16 CT-like phantom, K = 6, L2 flushed before every call
    vol = synth.ct_phantom_u16(256, 256, 256, seed=2)
    t, out, call = setup(vol, dpma.U16, 6)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def do_flush():
        flush.fill_(1)
    with torch.cuda.stream(s):
        for _ in range(5):
            call()
    s.synchronize()
    reps = 200
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    with torch.cuda.stream(s):
        for a, b in evs:
            do_flush()
            a.record(s)
            call()
            b.record(s)
    s.synchronize()
    us_call = statistics.median(a.elapsed_time(b) for a, b in evs) * 1e3
    st_ms, st_n = k1_stage(call, 100, do_flush)
    k1_us = st_ms[1] * 1e3
    ach = vol.nbytes / (k1_us * 1e-6) / 1e9
    rows.append({"workload": "ct_phantom_u16_256x256x256_K6", "metric": "voxel/s",
                 "value": vol.size / (us_call * 1e-6), "us_per_call_p50": round(us_call, 2),
                 "k1_us": round(k1_us, 3), "stage_us": [round(m * 1e3, 3) for m in st_ms],
                 "l2": "256 MB buffer written before every timed call (L2 flush)",
                 "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak,
                              "unit": "GB/s", "frac": round(ach / peak, 4)},
                 "gpu_launches_per_call": sum(st_n),
                 "step2_us": step2_routes(dpma, torch, t, 256, 256, 256, dpma.U16, 6, s)})
    return rows


def step2_routes(dpma, torch, t, L_, M_, N_, dt, K, s, reps=50):
    """Device time of step 2 alone on the same projection images (already
    in L2), by the separable power sums (the pipeline's default) and by the
    discrete Radon route of Sec. 3.2; both give the same int128 moments."""
    lib = dpma.lib()
    P = dpma.num_images(K)
    npairs = (K + 1) * (K + 2) // 2
    imgs = torch.empty(dpma.images_size(L_, M_, N_, dt, K) // 4, dtype=torch.int32, device="cuda")
    m_pow = torch.empty(P * npairs * 4, dtype=torch.int32, device="cuda")
    m_drt = torch.empty_like(m_pow)
    ws = torch.empty(dpma.workspace_size(L_, M_, N_, dt, K), dtype=torch.uint8, device="cuda")
    nd = lib.dpma_drt_workspace_size(L_, M_, N_, dt, K)
    wd = torch.empty(nd, dtype=torch.uint8, device="cuda")
    sp = ctypes.c_void_p(s.cuda_stream)
    ip = ctypes.c_void_p(imgs.data_ptr())
    lib.dpma_project(ctypes.c_void_p(t.data_ptr()), L_, M_, N_, dt, K, ip, sp)

    def power():
        lib.dpma_image_moments(ip, L_, M_, N_, dt, K, ctypes.c_void_p(m_pow.data_ptr()), sp,
                               ctypes.c_void_p(ws.data_ptr()), ws.numel())

    def drt():
        lib.dpma_image_moments_drt(ip, L_, M_, N_, dt, K, ctypes.c_void_p(m_drt.data_ptr()), sp,
                                   ctypes.c_void_p(wd.data_ptr()), nd, None)
    res = {}
    for name, fn in (("power_sums", power), ("drt", drt)):
        with torch.cuda.stream(s):
            for _ in range(5):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
        e1.synchronize()
        res[name] = round(e0.elapsed_time(e1) * 1e3 / reps, 2)
    res["identical"] = bool(torch.equal(m_pow, m_drt))
    return res


# ------------------------------------------------ batched and serving rows


def run_batched(dpma, torch, reps=20):
    """4096 binary ROI masks (u8, sizes log-uniform 8..96, fill 20-80%), K = 4:
    one graph-captured batched run vs. the same ROIs launched one by one."""
    from paper_2012_08099_gb300 import synth
    rb = synth.roi_batch(4096, seed=4)
    tv = [torch.from_numpy(v).cuda() for v in rb.volumes]
    n = len(tv)
    voxels = float(sum(v.size for v in rb.volumes))
    b = dpma.Batch(tv, [4] * n, [dpma.U8] * n, autotune=True)
    out = b.out_buffer()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(out)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(out)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    e1.synchronize()
    ms_batch = e0.elapsed_time(e1) / reps
    b.status()
    # per-volume launches of the single-volume pipeline on one stream
    lib = dpma.lib()
    wsb = max(dpma.workspace_size(v.shape[2], v.shape[1], v.shape[0], dpma.U8, 4) for v in rb.volumes)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    out1 = torch.zeros_like(out)
    sp = ctypes.c_void_p(s.cuda_stream)
    args = [(ctypes.c_void_p(t.data_ptr()), t.shape[2], t.shape[1], t.shape[0],
             ctypes.c_void_p(out1.data_ptr() + off)) for t, off in zip(tv, b.offsets)]

    def per_volume():
        for vp, L_, M_, N_, op in args:
            rc = lib.dpma_moments_async(vp, L_, M_, N_, dpma.U8, 4, op, sp,
                                        ctypes.c_void_p(ws.data_ptr()), wsb)
            if rc:
                raise dpma.DpmaError(rc, lib.dpma_last_error().decode())

    with torch.cuda.stream(s):
        per_volume()
        s.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(s)
        for _ in range(2):
            per_volume()
        f1.record(s)
    f1.synchronize()
    ms_single = f0.elapsed_time(f1) / 2
    return {"workload": "roi_masks_u8_4096_K4", "value": n / (ms_batch * 1e-3),
            "unit": "volume/s", "voxels_per_s": voxels / (ms_batch * 1e-3),
            "ms_per_batch": round(ms_batch, 4), "volumes": n, "voxels": int(voxels),
            "graph_captured": True, "fused_launches": b.info(5),
            "fused_threads": b.info(2), "fused_ctas": b.info(3),
            "second_launch": {"volumes": b.info(6), "threads": b.info(7), "ctas": b.info(8)},
            "per_volume_launches": {"value": n / (ms_single * 1e-3), "unit": "volume/s",
                                    "ms_per_batch": round(ms_single, 3)},
            "speedup_vs_per_volume": round(ms_single / ms_batch, 2),
            "identical": bool(torch.equal(out, out1))}


def run_serving(dpma, n_requests, distinct=48, rate_hz=200.0):
    """Poisson request stream (mean 200 req/s) of u16 CT-like phantoms, x, y
    log-uniform 32..512, z 32..300, K uniform in {3,4,6,8}; then the same
    requests submitted at once (saturation)."""
    import threading
    from paper_2012_08099_gb300 import synth
    reqs = synth.serving_stream(distinct, seed=5, rate_hz=rate_hz)
    g = np.random.Generator(np.random.PCG64(55))
    arrivals = np.cumsum(g.exponential(1.0 / rate_hz, size=n_requests))
    pick = g.integers(0, distinct, size=n_requests)
    res = {}
    with dpma.Server(max_inflight=64, streams=4) as srv:
        for r in reqs[:4]:                       # warm the pinned pools
            srv.wait(srv.submit(r.volume, r.K))
        srv.stats(reset=True)
        tickets = []

        def waiter():
            for t in iter_tickets():
                srv.wait(t)

        def iter_tickets():
            i = 0
            while i < n_requests:
                while len(tickets) <= i:
                    time.sleep(0.0002)
                yield tickets[i]
                i += 1

        w = threading.Thread(target=waiter)
        w.start()
        t0 = time.perf_counter()
        for a, j in zip(arrivals, pick):
            dt = a - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(reqs[j].volume, reqs[j].K))
        w.join()
        st = srv.stats(reset=True)
        vox = float(sum(reqs[j].volume.size for j in pick))
        res["poisson"] = {"offered_req_per_s": rate_hz, "requests": n_requests,
                          "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                          "mean_ms": round(st["mean_ms"], 3), "max_ms": round(st["max_ms"], 3),
                          "volumes_per_s": round(st["volumes_per_s"], 1),
                          "voxels_per_s": st["voxels_per_s"], "failed": st["failed"],
                          "launches": st["launches"]}
        # saturation: every request at once
        t0 = time.perf_counter()
        ts = [srv.submit(reqs[j].volume, reqs[j].K) for j in pick]
        for t in ts:
            srv.wait(t)
        wall = time.perf_counter() - t0
        st = srv.stats(reset=True)
        res["saturation"] = {"requests": n_requests, "volumes_per_s": round(n_requests / wall, 1),
                             "voxels_per_s": vox / wall, "p50_ms": round(st["p50_ms"], 3),
                             "p99_ms": round(st["p99_ms"], 3), "failed": st["failed"]}
    res["workload"] = "ct_phantom_u16_poisson_200hz_mixedK"
    res["distinct_volumes"] = distinct
    return res


# -------------------------------------------------------------- reference


def run_reference(args):
    """The oracle (plain Eq. 2 in FP64) on the host cores, bounded samples."""
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from paper_2012_08099_gb300 import synth
    import oracle

    oracle.build()
    vol = make_volume(SEED)
    threads = os.cpu_count() or 1
    per_slice = oracle_rate(np.ascontiguousarray(vol[:2]), threads) / 2.0
    budget = 150.0 / max(1, args.steps + args.warmup)
    nz = int(max(1, min(N, budget / max(per_slice, 1e-6))))
    slab = np.ascontiguousarray(vol[:nz])
    for _ in range(args.warmup):
        oracle.moments(slab, K, nthreads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.moments(slab, K, nthreads=threads)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = slab.size / dt
    sample = f"z-slab {L}x{M}x{nz} of the {WORKLOAD} volume per step, K={K}"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "L": L, "M": M, "N": N, "K": K,
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(threads, nz),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
