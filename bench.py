#!/usr/bin/env python
"""Benchmark: LM iterations per second of exact LM bundle adjustment on GB300.

Workload (default ``aerial5k``): 5,000 nadir cameras on a 50 x 100 flight grid
(60% forward / 30% side overlap), 1M points on sinusoidal terrain, tracks of
2 + Geometric (mean 5, max 20) cameras, N(0, 1 px) noise; FP32 Jacobians,
RCS assembly, SpMV and PCG with FP64 cost / gain-ratio sums and FP64
refinement residual; PCG stop at the paper's inexact-Newton T = 0.1.

A step is one LM iteration (linearize, RCS formation, PCG solve,
back-substitution, trial evaluation, accept/reject) through the C ABI.  The
timed steps are LM iterations 1..K from the initial state (the state is reset
after the warm-up).  ``value`` is K / device time with all inputs resident in
HBM; ``e2e`` is the same metric with each step's state copied in from host
memory and the result copied back.  ``roofline`` is for the dominant kernel
(the PCG), ``rcs_assembly`` for the RCS formation, both from CUDA events the
library records around each launch.  After the timed steps, untimed: the
storage formats' products (``spmv_formats``), the variable-size BSMC at
c = 11 (``vbsmc``), triangulation, the solver comparison (``solver``) and the
oracle's rate and phase times on the host (``cpu_baseline``).

``cpu_baseline`` is the FP64 CPU oracle timed on the host in a spawned process
(one LM iteration on the full workload; a scaled 200-camera sample beside it).
``--impl reference`` times the oracle on bounded samples of the same workload
(a 100-camera sample per step), scaled to the full observation count.
Multi-GPU: independent replicas (one problem per rank), max time over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
METRIC = "LM iters/s"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return d, "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of a per-rank float over all ranks (a job takes as long as
    its slowest rank); the value itself without a process group."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_scene(workload: str, rank: int = 0):
    import scenes
    if workload == "aerial5k":
        return scenes.aerial_scene(seed=2001 + rank)
    if workload == "ring50":
        return scenes.ring_scene(seed=1001 + rank)
    if workload == "aerial_small":
        return scenes.aerial_small(seed=2101 + rank)
    if workload == "aerial2400":
        return scenes.aerial_small(n_along=60, n_across=40, pts_per_cam=200, seed=2201 + rank)
    if workload == "blocks50k":
        # 20 overlapping 50 x 50 aerial blocks, 10M points, tracks 2 + Geom (mean 6, max 40),
        # 1% outlier observations
        return scenes.blocks_scene(seed=3001 + rank)
    if workload == "capacity":
        # 200,000 cameras (400 x 500 grid), 40M points, ~243M observations, ~33 co-visible
        return scenes.capacity_scene(seed=5001 + rank)
    raise ValueError(workload)


def workload_opts(workload: str, B):
    if workload == "ring50":
        return dict(precision=B.BA_FP64, pcg_rel_tol=1e-10)
    if workload == "blocks50k":
        return dict(precision=B.BA_FP32, pcg_rel_tol=0.1, inner_rel_tol=1e-4, robust=B.BA_LOSS_HUBER,
                    huber_delta=2.0)
    return dict(precision=B.BA_FP32, pcg_rel_tol=0.1, inner_rel_tol=1e-4)


def workload_config(workload: str, s, opts):
    return {"workload": workload, "n_cams": s.n_cams, "n_pts": s.n_pts, "n_obs": s.n_obs,
            "mean_track": round(s.n_obs / s.n_pts, 3), "precision": "fp32+fp64-refine"
            if opts.get("precision") == 1 else "fp64", "pcg_rel_tol": opts["pcg_rel_tol"],
            "lm_iterations_timed": "1..K from the initial state",
            "robust": "huber 2 px" if opts.get("robust") else "none",
            "l2": "inputs larger than L2 (stored Jacobians %.0f MB > 129 MB)" % (s.n_obs * 80 / 1e6)}


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
            os.unlink(self.path)
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except Exception:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


def rcs_bytes_and_flops(st, esz=4):
    """Algorithmic traffic and flops of one RCS-formation launch (K2).

    reads: stored Jacobian rows (20 values / observation), the (a, b) product
    list (4 B / product), local-block descriptors (4 B), track starts (4 B /
    point), group descriptors (40 B); writes: sub-RCS partials (36 values)
    and per-point L^-1, l_p (9 values)."""
    m, P, pairs, npart, ng = st["n_obs"], st["n_pts"], st["n_pairs"], st["n_partials"], st["n_groups"]
    byts = m * 20 * esz + pairs * 4 + npart * 4 + (P + 1) * 4 + ng * 40 + npart * 36 * esz + P * 9 * esz
    offd = pairs - m
    # per obs: V 9x2, l_p 6, P 2x6x... (30), e^ 12; per point: Cholesky ~40; per diag product 75 FMA,
    # per off-diagonal product 108 FMA
    flops = m * 2 * (9 + 6 + 15 + 6) + P * 60 + m * 2 * 75 + offd * 2 * 108
    return byts, flops


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2307_08383_gb300 as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    s = make_scene(args.workload, rank)
    opts = workload_opts(args.workload, B)
    stream = torch.cuda.current_stream()
    t_create = time.perf_counter()
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, stream=stream.cuda_stream, profile=1, **opts)
    t_create = time.perf_counter() - t_create
    lam0 = g.opts.lambda0
    net = None
    if args.workload == "capacity":
        # the learned correction (packaged weights), block-Jacobi as its fallback
        net = B.PrecondNet.load()
        B.ba_set_precond_net(g, net)

    for _ in range(args.warmup):
        g.lm_step()
    g.set_state(s.cams0, s.pts0, lam0, 2.0)
    torch.cuda.synchronize()
    g.reset_kernel_times()
    st0 = g.stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    infos = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(g.lm_step())
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st1 = g.stats()
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    ktimes = g.kernel_times()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = world * args.steps / (ms_max / 1e3)

    # ---- end-to-end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        g.set_state(s.cams0, s.pts0, lam0, 2.0)
        hc = torch.empty((s.n_cams, 6), dtype=torch.float64, pin_memory=True).numpy()
        hp = torch.empty((s.n_pts, 3), dtype=torch.float64, pin_memory=True).numpy()
        hc[:] = s.cams0
        hp[:] = s.pts0
        lam, nu = lam0, 2.0
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g.set_state(hc, hp, lam, nu)
            g.lm_step()
            B.ba_get_cameras(g.h, s.n_cams, hc)
            B.ba_get_points(g.h, s.n_pts, hp)
            lam, nu, _ = g.lm_state()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": world * args.steps / max_over_ranks(dt, dist, "cuda"), "unit": "LM iters/s",
               "h2d_bytes_per_step": int(hc.nbytes + hp.nbytes),
               "d2h_bytes_per_step": int(hc.nbytes + hp.nbytes + 8)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks, peak_kind = load_peaks()
    total_timed = sum(v[1] for v in ktimes.values())
    esz = 4 if opts["precision"] == B.BA_FP32 else 8
    # the dominant kernel: the PCG loop (one launch per refinement sweep)
    n_pcg, t_pcg = ktimes["pcg_loop"]
    iters = sum(i["pcg_iters"] for i in infos)
    per_iter = pcg_bytes_per_iteration(st1, esz)
    us_iter = 1e3 * t_pcg / max(iters, 1)
    achieved = per_iter / (us_iter / 1e6) / 1e9
    traffic = captured_traffic("pcg_split", args.workload) if opts["precision"] == B.BA_FP32 and \
        ktimes.get("split_prepare", (0, 0.0))[0] > 0 else None
    split_ran = ktimes.get("split_prepare", (0, 0.0))[0] > 0
    roof = {"kernel": "pcg_loop (k_pcg_split)" if split_ran else "pcg_loop (k_pcg_persist)", "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
            "peak_kind": peak_kind, "traffic": traffic, "per": "PCG iteration",
            "algorithmic_bytes": int(per_iter), "iterations": iters, "launches": n_pcg,
            "us_per_iteration": round(us_iter, 2),
            "note": ("S (%.0f MB) fits in L2: its DRAM traffic is the vectors" % (st1["nnzb"] * 36 * esz / 1e6))
            if st1["nnzb"] * 36 * esz < 100e6 else "S (%.0f MB) streams from HBM" % (st1["nnzb"] * 36 * esz / 1e6),
            "share_of_timed_kernels": round(t_pcg / total_timed, 3) if total_timed else None}
    # RCS assembly (K2), the metric's second figure
    n_l, tot = ktimes["form_rcs"]
    byts, flops = rcs_bytes_and_flops(st1, esz)
    avg_ms = tot / max(n_l, 1)
    ach_rcs = byts / (avg_ms / 1e3) / 1e9
    rcs = {"kernel": "form_rcs", "bound": "hbm", "achieved": round(ach_rcs, 1), "peak": peaks["hbm_gbs"],
           "unit": "GB/s", "frac": round(ach_rcs / peaks["hbm_gbs"], 4), "peak_kind": peak_kind,
           "traffic": captured_traffic("form_rcs", args.workload) if opts["precision"] == B.BA_FP32 else None,
           "algorithmic_bytes": int(byts), "launches": n_l, "avg_ms": round(avg_ms, 4),
           "fp32_tflops": round(flops / (avg_ms / 1e3) / 1e12, 2),
           "share_of_timed_kernels": round(tot / total_timed, 3) if total_timed else None}
    kernels = {nm: {"launches": v[0], "ms": round(v[1], 3)} for nm, v in ktimes.items() if v[0]}
    # the oracle's host timing runs in a spawned process beside the untimed
    # measurements below (it starts after the timed regions)
    cpu_handle = None if args.no_cpu_baseline else start_cpu_baseline(args.workload)
    formats = None if args.no_formats else formats_bench(B, torch, g, st1, esz, peaks, peak_kind, stream)
    tri = triangulation_bench(g, st1, ktimes)
    vbs = None if args.no_vbsmc else vbsmc_bench(B, torch, g, peaks, peak_kind, esz)
    g.close()
    vbi = None if args.no_vbsmc or args.workload != "aerial5k" else interiors_lm_bench(B, torch, s, stream)
    solver = None if args.no_solver else solver_bench(B, torch)
    cpu = None if cpu_handle is None else finish_cpu_baseline(cpu_handle, s.n_obs)
    acc = sum(i["accepted"] for i in infos)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "LM iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if opts["precision"] == B.BA_FP32 else "f64", "data": "synthetic",
        "config": workload_config(args.workload, s, opts),
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roof, "rcs_assembly": rcs, "cpu_baseline": cpu,
        "clocks": clk.summary(),
        "lm": {"accepted": acc, "pcg_iters": [i["pcg_iters"] for i in infos],
               "cost": [infos[0]["cost_before"], infos[-1]["cost_after"]],
               "rcs_rel_resid_max": max(i["rcs_rel_resid"] for i in infos)},
        "kernels_ms": kernels, "solver": solver, "spmv_formats": formats, "triangulation": tri, "vbsmc": vbs,
        "interiors_lm": vbi,
        "impl": "ours",
        "setup": {"problem_create_s": round(t_create, 2), "device_bytes": int(st1["device_bytes"]),
                  "preconditioner": "learned (packaged weights), block-Jacobi fallback" if net else "block-Jacobi",
                  "used_fallback": [i["used_fallback"] for i in infos]},
    }
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


# DRAM traffic per unit (dram__bytes_read.sum + dram__bytes_write.sum from one
# ncu capture of the kernel on the workload), keyed by the digest of the
# kernel's source file at the time of the capture: once the source changes
# the stored figure no longer describes the kernel that runs, and the bench
# line reports null instead.
NCU_TRAFFIC = {
    "pcg_split": {"source": "k_pcg.cu", "digest": "a79cea617bb62c35", "workload": "aerial5k",
                  "bytes_per_unit": (47_371_776 + 44_544) // 41},
    "form_rcs": {"source": "k_rcs.cu", "digest": None, "workload": "aerial5k", "bytes_per_unit": None},
}


def source_digest(name):
    """First 16 hex digits of the SHA-256 of a CUDA source file of the library."""
    import hashlib
    path = os.path.join(ROOT, "paper_2307_08383_gb300", "csrc", name)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def captured_traffic(kernel, workload):
    """The stored ncu DRAM bytes per unit of a kernel, if they were captured
    on this workload from the source that is built now; else None."""
    t = NCU_TRAFFIC[kernel]
    if t["digest"] is None or t["workload"] != workload or t["digest"] != source_digest(t["source"]):
        return None
    return t["bytes_per_unit"]


def formats_bench(B, torch, g, st, esz, peaks, peak_kind, stream, repeats=7):
    """y = S x with the current RCS in each storage format of Sec. 4 (the
    library's BSMC, block CSR of the full symmetric matrix, scalar CSR), one
    launch per format through ba_rcs_spmv, L2 flushed before each launch (a
    256 MB write), CUDA events on the problem's stream, median of repeats.
    Bytes: the format's arrays read once plus x and y (6n values each)."""
    import statistics
    n = st["n_cams"]
    # an accepted LM step drops the RCS: form the one of the final state
    g.linearize()
    g.form_rcs(g.lm_state()[0])
    dt = torch.float32 if esz == 4 else torch.float64
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(6 * n, dtype=dt, device="cuda", generator=gen)
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    res = {}
    for name, fmt in (("bsmc", B.BA_FMT_BSMC), ("bsmc_once", B.BA_FMT_BSMC_ONCE), ("bsr_full", B.BA_FMT_BSR_FULL),
                      ("csr", B.BA_FMT_CSR), ("implicit", B.BA_FMT_IMPLICIT)):
        nbytes = g.rcs_spmv(fmt, x, y)  # builds the format's arrays (untimed)
        torch.cuda.synchronize()
        ts = []
        for _ in range(repeats):
            flush.zero_()
            e0.record(stream)
            g.rcs_spmv(fmt, x, y)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        us = 1e3 * statistics.median(ts)
        moved = nbytes + 2 * 6 * n * esz
        res[name] = {"us": round(us, 2), "format_bytes": int(nbytes), "bytes_per_spmv": int(moved),
                     "achieved_gbs": round(moved / us / 1e3, 1),
                     "frac_hbm": round(moved / us / 1e3 / peaks["hbm_gbs"], 4)}
    return {"what": "y = S x per RCS storage format (Sec. 4, Table 1, Eqs. 8-10)", "l2": "flushed before each launch",
            "peak_gbs": peaks["hbm_gbs"], "peak_kind": peak_kind, "formats": res,
            "bytes_csr_over_bsmc": round(res["csr"]["format_bytes"] / res["bsmc"]["format_bytes"], 3),
            "time_csr_over_bsmc": round(res["csr"]["us"] / res["bsmc"]["us"], 3),
            "time_bsr_full_over_bsmc": round(res["bsr_full"]["us"] / res["bsmc"]["us"], 3),
            "time_implicit_over_bsmc": round(res["implicit"]["us"] / res["bsmc"]["us"], 3),
            "note": "implicit: no stored S; its bytes are what one product reads instead (stored J rows, "
                    "per-point factors, a work vector, a camera-major index)"}


def vbsmc_bench(B, torch, g, peaks, peak_kind, esz, c=11, tol=1e-10, repeats=7):
    """The RCS pattern of the workload with c unknowns per camera (c = 11:
    six exterior and five interior, Sec. 4.1) in variable-size BSMC
    (ba_vbsmc_*): y = S x with L2 flushed before each launch (CUDA events on
    the current stream, median of repeats), and a block-Jacobi PCG solve
    timed by the library's CUDA events.  Values from a seeded SPD generator
    (off-diagonal blocks N(0, 1), diagonal blocks dominant), so the iteration
    count says nothing about BA conditioning; the times per product and per
    iteration are what this measures.  Bytes: the stored format read once plus
    x and y."""
    import numpy as np

    import scenes
    g.linearize()
    g.form_rcs(g.lm_state()[0])
    row_ptr, col, _, _ = g.rcs()
    n = len(row_ptr) - 1
    cdim = np.full(n, c, dtype=np.int32)
    val, _ = scenes.random_block_spd(row_ptr, col, cdim, seed=7)
    b = np.random.default_rng(8).standard_normal(c * n)
    prec = B.BA_FP32 if esz == 4 else B.BA_FP64
    vb = B.VBSMC(cdim, row_ptr, col, val, b, precision=prec)
    N, nbytes = vb.info()
    dt = torch.float32 if esz == 4 else torch.float64
    x = torch.randn(N, dtype=dt, device="cuda", generator=torch.Generator(device="cuda").manual_seed(9))
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    vb.spmv(x, y)
    torch.cuda.synchronize()
    ts = []
    for _ in range(repeats):
        flush.zero_()
        e0.record(stream)
        vb.spmv(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    us = 1e3 * statistics.median(ts)
    moved = nbytes + 2 * N * esz
    # per iteration: the difference of a loose and a tight solve (the start
    # phase and the launch cancel), medians of three
    vb.solve(tol)  # warm-up
    lo = [vb.solve(1e-1) for _ in range(3)]
    hi = [vb.solve(tol) for _ in range(3)]
    its = hi[-1][1]
    d_it = max(its - lo[-1][1], 1)
    us_it = 1e3 * (statistics.median([r[3] for r in hi]) - statistics.median([r[3] for r in lo])) / d_it
    vb.close()
    return {"what": "variable-size BSMC (Sec. 4: c_i x c_j blocks), c = %d on every camera" % c,
            "cameras": n, "blocks": len(col), "unknowns": N, "storage_bytes": int(nbytes),
            "spmv_us": round(us, 2), "bytes_per_spmv": int(moved), "achieved_gbs": round(moved / us / 1e3, 1),
            "frac_hbm": round(moved / us / 1e3 / peaks["hbm_gbs"], 4), "peak_kind": peak_kind,
            "l2": "flushed before each product",
            "pcg": {"tol": tol, "iterations": its, "us_per_iteration": round(us_it, 2),
                    "per_iteration": "(t(tol) - t(1e-1)) / (iterations(tol) - iterations(1e-1))",
                    "values": "seeded SPD generator, diagonally dominant blocks"}}


def interiors_lm_bench(B, torch, s, stream, steps=5, warmup=2):
    """LM iterations with five interiors per camera (c = 11 on every camera:
    self-calibration, Sec. 4.1) on the workload's scene, through ba_vbi_*:
    linearize with 11 camera columns, the variable-size RCS, block-Jacobi PCG
    to the paper's T = 0.1, Eq. 5, trial evaluation, gain ratio.  FP32 RCS
    and PCG (FP64 V_k factors, sums and state).  The initial interiors are
    the observing pinhole perturbed (1% on f, 2 px on the principal point,
    0.01 on k1, k2).  Timed with CUDA events on the current stream after
    warm-up steps from the initial state, the state reset before the timed
    steps."""
    import numpy as np

    import scenes
    intr = scenes.interiors0(s.n_cams, seed=11)
    cdim = np.full(s.n_cams, 11, dtype=np.int32)
    t0 = time.perf_counter()
    g = B.VBIProblem(s.cams0, intr, cdim, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, precision=B.BA_FP32,
                     pcg_rel_tol=0.1)
    t_create = time.perf_counter() - t0
    lam0 = g.lm_state()[0]
    for _ in range(warmup):
        g.lm_step()
    g.set_state(s.cams0, intr, s.pts0, lam0, 2.0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [g.lm_step() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    info = g.info()
    g.close()
    names = ("linearize", "form_rcs", "pcg", "backsub_trial_cameras", "trial_cost")
    return {"what": "LM with c = 11 (6 exterior + 5 interior unknowns) on every camera, FP32 RCS and PCG, "
                    "T = 0.1", "lm_iters_per_s": round(steps / (ms / 1e3), 3), "ms_per_step": round(ms / steps, 3),
            "steps": steps, "unknowns": info["unknowns"], "blocks": info["blocks"],
            "device_bytes": info["device_bytes"], "problem_create_s": round(t_create, 2),
            "accepted": sum(i["accepted"] for i in infos), "pcg_iters": [i["pcg_iters"] for i in infos],
            "cost": [infos[0]["cost_before"], infos[-1]["cost_after"]],
            "phase_ms_mean": {k: round(sum(i["ms"][q] for i in infos) / steps, 3) for q, k in enumerate(names)}}


def triangulation_bench(g, st, ktimes, gn_iters=3, repeats=3):
    """Every point re-triangulated from the final cameras (ba_triangulate:
    linear solve + Gauss-Newton, FP64), after the timed LM steps, timed by the
    library's CUDA events; beside it the point pass of the LM step (Eq. 5
    back-substitution with the trial evaluation) from the timed steps."""
    g.reset_kernel_times()
    fails = []
    for _ in range(repeats):
        fails.append(g.triangulate(gn_iters)[0])
    n, ms = g.kernel_times()["triangulate"]
    avg = ms / max(n, 1)
    sp = ktimes.get("step_points", (0, 0.0))
    return {"gn_iters": gn_iters, "ms": round(avg, 4), "points_per_s": round(st["n_pts"] / (avg / 1e3)),
            "points_unchanged": fails[-1],
            "lm_point_pass_ms": round(sp[1] / sp[0], 4) if sp[0] else None}


def pcg_bytes_per_iteration(st, esz=4):
    """Algorithmic DRAM bytes of one block-Jacobi PCG iteration if nothing
    stayed on chip: every stored block of S once (36 values) and ten camera
    vectors (6 values each) read or written."""
    return st["nnzb"] * 36 * esz + st["n_cams"] * 6 * esz * 10


def solver_bench(B, torch, seeds=tuple(range(200, 220)), repeats=3):
    """PCG time to a true relative residual of 1e-8 on the RCS of the 20
    held-out aerial-shaped scenes (2,000-8,000 cameras; LM iterations 0 and 1
    of each, 40 systems): FP64 block-Jacobi PCG against FP32 PCG inside FP64
    refinement, with block-Jacobi and with the packaged learned correction.
    Times are host wall-clock around synchronised calls (the solve
    synchronises internally), median over repeats per system; the summary
    gives, per arm, the median over the systems and, per FP32 arm, the median
    of its per-system speedup over FP64."""
    from paper_2307_08383_gb300.precond_training import _instances_of_scene
    net = B.PrecondNet.load()
    arms = {"fp64_block_jacobi": (dict(precision=B.BA_FP64), False),
            "fp32_block_jacobi": (dict(precision=B.BA_FP64, solve_precision=B.BA_FP32, inner_rel_tol=1e-4), False),
            "fp32_learned": (dict(precision=B.BA_FP64, solve_precision=B.BA_FP32, inner_rel_tol=1e-4), True)}
    res = {k: {"ms": [], "pcg_iters": [], "true_rel_resid": [], "used_fallback": []} for k in arms}
    sizes = []
    for seed in seeds:
        _, insts = _instances_of_scene(seed)
        for row_ptr, col, val, b, lam in insts:
            sizes.append((len(row_ptr) - 1, len(col)))
            for name, (kw, use_net) in arms.items():
                g = B.Problem.from_rcs(row_ptr, col, val, b, pcg_rel_tol=1e-8, pcg_max_iters=50000, **kw)
                if use_net:
                    B.ba_set_precond_net(g, net)
                g.solve_rcs()
                ts = []
                for _ in range(repeats):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    info, conv = g.solve_rcs()
                    torch.cuda.synchronize()
                    ts.append((time.perf_counter() - t0) * 1e3)
                    if not conv:
                        raise RuntimeError(f"{name} did not reach 1e-8 (seed {seed})")
                ts.sort()
                r = res[name]
                r["ms"].append(round(ts[len(ts) // 2], 3))
                r["pcg_iters"].append(info["pcg_iters"])
                r["true_rel_resid"].append(info["rcs_rel_resid"])
                r["used_fallback"].append(info["used_fallback"])
                B.ba_set_precond_net(g, None)
                g.close()
    net.close()
    med = statistics.median
    t64 = res["fp64_block_jacobi"]["ms"]
    summary = {k: {"median_ms": round(med(v["ms"]), 3), "median_pcg_iters": med(v["pcg_iters"]),
                   "max_true_rel_resid": max(v["true_rel_resid"]), "fallbacks": int(sum(v["used_fallback"]))}
               for k, v in res.items()}
    for k in ("fp32_block_jacobi", "fp32_learned"):
        summary[k]["median_speedup_vs_fp64"] = round(med([a / b for a, b in zip(t64, res[k]["ms"])]), 3)
    return {"metric": "PCG time to true rel. residual 1e-8", "unit": "ms", "scene_seeds": [seeds[0], seeds[-1]],
            "systems": len(sizes), "n_cams_range": [min(x[0] for x in sizes), max(x[0] for x in sizes)],
            "nnzb_range": [min(x[1] for x in sizes), max(x[1] for x in sizes)], "summary": summary,
            "learned_weights": _weights_note(),
            "arms": res}


def _weights_note():
    """What the packaged learned correction is: its training record's kept
    epoch and learning rate (epoch -1: the zero-output start, i.e. plain
    block-Jacobi, kept because no trained epoch beat it on validation)."""
    import numpy as np
    path = os.path.join(ROOT, "paper_2307_08383_gb300", "weights", "precond_net_aerial.npz")
    with np.load(path, allow_pickle=False) as d:
        meta = json.loads(str(d["meta"]))
    ep, lr = meta.get("kept_epoch"), meta.get("kept_lr")
    if ep is None or ep < 0:
        return "packaged weights are the zero-output start (plain block-Jacobi): no trained epoch beat it on " \
               "the validation systems"
    return f"packaged weights: epoch {ep} at learning rate {lr} ({meta.get('loss', 'see training record')})"


def _oracle_steps(workload, n_steps, sample_cams, phases=False):
    """Times n_steps oracle LM iterations on a sample of the workload (and,
    with phases, the phases of one more)."""
    import oracle as O
    import scenes
    if workload == "ring50":
        s = scenes.ring_scene(seed=1001)
        tol = 1e-10
    else:
        na, nc = sample_cams
        s = scenes.aerial_small(n_along=na, n_across=nc, pts_per_cam=200, seed=2101)
        tol = 0.1
    pb = O.Problem(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt, s.obs_uv, pcg_tol=tol)
    st = O.LMState(s.cams0.copy(), s.pts0.copy())
    times = []
    c0 = time.process_time()
    for _ in range(n_steps):
        t0 = time.perf_counter()
        st, _, _ = pb.step(st)
        times.append(time.perf_counter() - t0)
    # threads the oracle kept busy: process CPU time over wall time
    _oracle_steps.cores = round(max(1.0, (time.process_time() - c0) / max(sum(times), 1e-9)), 2)
    if not phases:
        return s, times
    # one more iteration's phases, each timed alone: linearize, RCS (Eq. 3-4),
    # PCG, back-substitution (Eq. 5)
    t = [time.perf_counter()]
    e, Jc, Jp = pb.linearize(st.cams, st.pts)
    t.append(time.perf_counter())
    blk, A, b = pb.rcs(e, Jc, Jp, st.lam)
    t.append(time.perf_counter())
    res = pb.solve(A, b)
    t.append(time.perf_counter())
    O.back_substitute(blk, pb.obs_cam, pb.obs_pt, pb.P, res.y.reshape(-1, 6))
    t.append(time.perf_counter())
    names = ("linearize", "form_rcs", "pcg", "back_substitute")
    return s, times, {k: t[q + 1] - t[q] for q, k in enumerate(names)}


def _cpu_worker(workload, q):
    """The FP64 oracle on the host, in a process of its own (spawned; it
    imports nothing of the GPU path): one LM iteration on the full workload
    (the first, from the initial state), then three on a 200-camera sample of
    the same layout with one further iteration's phases timed alone.  Puts a
    dict of timings on q."""
    try:
        import oracle as O
        out = {}
        full = make_scene(workload)
        tol = 1e-10 if workload == "ring50" else 0.1
        pb = O.Problem(full.n_cams, full.n_pts, full.obs_cam, full.obs_pt, full.obs_uv, pcg_tol=tol)
        st = O.LMState(full.cams0.copy(), full.pts0.copy())
        c0, t0 = time.process_time(), time.perf_counter()
        _, info, _ = pb.step(st)
        wall = time.perf_counter() - t0
        out["full"] = {"seconds": wall, "cores": round(max(1.0, (time.process_time() - c0) / wall), 2),
                       "pcg_iters": int(info.pcg_iters), "n_cams": full.n_cams, "n_pts": full.n_pts,
                       "n_obs": full.n_obs}
        del pb, st, full
        s, times, ph = _oracle_steps(workload, 3, (20, 10), phases=True)
        out["sample"] = {"seconds": times, "n_cams": s.n_cams, "n_pts": s.n_pts, "n_obs": s.n_obs,
                         "cores": _oracle_steps.cores, "phases": ph}
        q.put(out)
    except Exception as e:  # reported in the bench line, never raised into the GPU process
        q.put({"error": repr(e)})


def start_cpu_baseline(workload):
    """Starts the oracle's host timing in a spawned process; returns a handle
    for finish_cpu_baseline."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    proc = ctx.Process(target=_cpu_worker, args=(workload, q), daemon=True)
    proc.start()
    return proc, q


def finish_cpu_baseline(handle, m_full, timeout_s=1800):
    """cpu_baseline from the spawned oracle run: value = one LM iteration on
    the full workload; the 200-camera sample, scaled to the full observation
    count by time per observation, beside it."""
    import queue
    proc, q = handle
    try:
        r = q.get(timeout=timeout_s)
    except queue.Empty:
        r = {"error": f"the oracle did not finish within {timeout_s} s"}
    proc.join(timeout=10)
    if proc.is_alive():
        proc.terminate()
    if "error" in r:
        return {"value": None, "unit": "LM iters/s", "kind": "oracle", "error": r["error"]}
    f, sm = r["full"], r["sample"]
    per_obs = sum(sm["seconds"]) / len(sm["seconds"]) / sm["n_obs"]
    return {"value": round(1.0 / f["seconds"], 6), "unit": "LM iters/s", "cores": f["cores"], "kind": "oracle",
            "sample": f"one FP64 oracle LM iteration (the first, from the initial state: {f['pcg_iters']} PCG "
                      f"iterations) on the full workload, {f['n_cams']} cameras, {f['n_pts']} points, "
                      f"{f['n_obs']} observations: {f['seconds']:.1f} s",
            "seconds_full_iteration": round(f["seconds"], 2),
            "sample_scaled": {
                "value": round(1.0 / (per_obs * m_full), 6),
                "what": f"3 oracle LM iterations on a {sm['n_cams']}-camera, {sm['n_obs']}-observation sample of "
                        f"the same layout ({sum(sm['seconds']):.1f} s), scaled to {m_full} observations by time "
                        f"per observation (an estimate, not a measurement)",
                "phases_s_scaled": {k: round(v / sm["n_obs"] * m_full, 3) for k, v in sm["phases"].items()}},
            "cores_note": "process CPU time over wall time of the oracle process"}


def run_reference(args):
    """The oracle arm: each step is one FP64 oracle LM iteration on a
    100-camera sample of the workload's layout (seconds each, so that the
    whole --steps K --warmup W run ends within minutes); the reported rate is
    scaled to the full workload by time per observation, which the config
    states.  The full-size measurement is the cpu_baseline of the GPU arm."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    full = make_scene(args.workload) if args.workload == "ring50" else None
    m_full = full.n_obs if full is not None else _aerial5k_obs()
    sample = (10, 10)
    if args.warmup:
        _oracle_steps(args.workload, args.warmup, sample)
    s, times = _oracle_steps(args.workload, args.steps, sample)
    per_obs = sum(times) / len(times) / s.n_obs
    est = per_obs * m_full
    value = 1.0 / est
    scaled = s.n_obs != m_full
    desc = (f"each step one FP64 oracle LM iteration on a {s.n_cams}-camera, {s.n_pts}-point, {s.n_obs}-observation "
            f"sample of the workload's layout" + (f", the rate scaled to {m_full} observations by time per "
                                                   f"observation" if scaled else ""))
    out = {"metric": METRIC, "value": round(value, 6), "unit": "LM iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "n_obs": m_full,
                      "sample": {"n_cams": s.n_cams, "n_pts": s.n_pts, "n_obs": s.n_obs},
                      "scaling": "value = sample observations per second / workload observations" if scaled
                      else "none: the whole workload", "ms_per_step": "measured, per sample step",
                      "ms_per_step_scaled": round(est * 1e3, 1)},
           "impl": "reference",
           "cpu_baseline": {"value": round(value, 6), "unit": "LM iters/s", "cores": _oracle_steps.cores,
                            "kind": "oracle", "sample": desc},
           "e2e": {"value": round(value, 6), "unit": "LM iters/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_kernel_case(args):
    """A short driver for ncu captures: builds the problem for the workload,
    linearizes once and runs the chosen kernel family three times."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2307_08383_gb300 as B
    s = make_scene(args.workload)
    opts = workload_opts(args.workload, B)
    if args.pcg_tol:
        opts.update(pcg_rel_tol=args.pcg_tol, inner_rel_tol=args.pcg_tol, refine_max=1)
    if args.pcg_variant:
        opts["pcg_variant"] = {"standard": B.BA_PCG_STANDARD, "split": B.BA_PCG_SPLIT,
                               "implicit": B.BA_PCG_IMPLICIT}[args.pcg_variant]
    if args.group_obs:
        opts["group_max_obs"] = args.group_obs
    g = B.Problem(s.cams0, s.pts0, s.obs_cam, s.obs_pt, s.obs_uv, profile=2, **opts)
    g.linearize()
    iters = []
    for _ in range(3):
        g.form_rcs(1e-6 if args.pcg_tol else 1e-4)
        if args.kernel_case == "pcg":
            info, _ = g.solve_rcs()
            iters.append(info["pcg_iters"])
    torch.cuda.synchronize()
    kt = {k: v for k, v in g.kernel_times().items() if v[0]}
    out = {"kernel_case": args.kernel_case, "workload": args.workload, "stats": g.stats(), "kernel_ms": kt}
    if args.kernel_case == "form_rcs":
        st = g.stats()
        out["rcs_phase_us_per_group"] = [round(x, 2) for x in st["rcs_phase_us"]]
        out["form_rcs_us"] = round(1e3 * kt["form_rcs"][1] / kt["form_rcs"][0], 1)
        out["rcs_reduce_us"] = round(1e3 * kt["rcs_reduce"][1] / kt["rcs_reduce"][0], 1)
    if iters:
        n_l, ms = kt["pcg_loop"]
        out.update(pcg_iters=iters, pcg_variant=args.pcg_variant or "auto",
                   us_per_iteration=round(1e3 * ms / max(sum(iters), 1), 2),
                   split_phase_us=[round(x, 2) for x in g.stats()["pcg_phase_us"]],
                   split_work_imbalance=round(g.stats()["pcg_work_imbalance"], 3))
    print(json.dumps(out))
    g.close()


def run_spmv_case(args, repeats=5):
    """A short driver for the storage-format products at a workload's RCS
    pattern without the rest of its problem: the pattern of the workload's
    observations (ba_symbolic_pattern, on the host), seeded SPD values
    (off-diagonal blocks N(0, 1), dominant diagonal blocks), an RCS-only FP32
    problem (ba_problem_create_rcs), then y = S x in BSMC, full block CSR and
    scalar CSR, each after an L2 flush, timed with CUDA events (median of
    repeats).  The device holds the system and the formats only (about 1.1 GB
    at 50,000 cameras with BSMC alone, 3.5 GB with all three)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2307_08383_gb300 as B
    import scenes
    s = make_scene(args.workload)
    row_ptr, col = B.ba_symbolic_pattern(s.n_cams, s.n_pts, s.obs_cam, s.obs_pt)
    del s
    n = len(row_ptr) - 1
    val, _ = scenes.random_block_spd(row_ptr, col, np.full(n, 6, dtype=np.int32), seed=7)
    b = np.random.default_rng(8).standard_normal(6 * n)
    g = B.Problem.from_rcs(row_ptr, col, val.reshape(-1, 36), b, precision=B.BA_FP32)
    del val
    stream = torch.cuda.current_stream()
    x = torch.randn(6 * n, dtype=torch.float32, device="cuda", generator=torch.Generator(device="cuda").manual_seed(9))
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    peaks, peak_kind = load_peaks()
    fmts = [("bsmc", B.BA_FMT_BSMC), ("bsmc_once", B.BA_FMT_BSMC_ONCE)] + \
        ([] if args.spmv_bsmc_only else [("bsr_full", B.BA_FMT_BSR_FULL), ("csr", B.BA_FMT_CSR)])
    res = {}
    for name, fmt in fmts:
        nbytes = g.rcs_spmv(fmt, x, y)
        torch.cuda.synchronize()
        ts = []
        for _ in range(repeats):
            flush.zero_()
            e0.record(stream)
            g.rcs_spmv(fmt, x, y)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        us = 1e3 * statistics.median(ts)
        moved = nbytes + 2 * 6 * n * 4
        res[name] = {"us": round(us, 2), "format_bytes": int(nbytes), "achieved_gbs": round(moved / us / 1e3, 1),
                     "frac_hbm": round(moved / us / 1e3 / peaks["hbm_gbs"], 4)}
    print(json.dumps({"kernel_case": "spmv", "workload": args.workload, "n_cams": n, "nnzb": len(col),
                      "peak_kind": peak_kind, "formats": res}))
    g.close()


def _aerial5k_obs():
    # observation count of the full aerial workload (seeded, deterministic)
    return make_scene("aerial5k").n_obs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="aerial5k",
                    choices=["aerial5k", "ring50", "aerial_small", "aerial2400", "blocks50k", "capacity"])
    ap.add_argument("--kernel-case", default=None, choices=["form_rcs", "pcg", "spmv"],
                    help="profiling driver: run one kernel family a few times on the workload and exit")
    ap.add_argument("--pcg-tol", type=float, default=None, help="kernel case: PCG relative tolerance")
    ap.add_argument("--spmv-bsmc-only", action="store_true", help="spmv kernel case: the BSMC product only")
    ap.add_argument("--pcg-variant", default=None, choices=["standard", "split", "implicit"], help="kernel case: PCG variant")
    ap.add_argument("--group-obs", type=int, default=0, help="kernel case: observations per point group")
    ap.add_argument("--no-formats", action="store_true", help="skip the RCS storage-format SpMV comparison")
    ap.add_argument("--no-vbsmc", action="store_true",
                    help="skip the variable-size BSMC (c = 11) measurements: product, PCG and the LM with interiors")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solver", action="store_true", help="skip the PCG time-to-1e-8 comparison")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.kernel_case == "spmv":
        run_spmv_case(args)
    elif args.kernel_case:
        run_kernel_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
