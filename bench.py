"""Benchmark of the SegSALSA-STR SALSA sweep on GB300 (one JSON line on stdout).

Workload (default): the 2048x2048, K=16 synthetic scene (64 Voronoi seeds, logits
3*onehot + N(0,1), softmax probabilities), 3x3 patch with Gaussian weights sigma=0.5,
lambda=2, mu=1, Schatten p=1, 200 SALSA iterations. Its working set (about 6.5 GB) is far
larger than L2, so the sweep's fraction of the HBM roofline means what it says. One step =
set_probs (device-resident p), 200 iterations with the residual/objective trace every 10
iterations, label readout. value = ADMM iterations per second (all ranks). `--workload 145x145`
runs the 145x145, K=16 scene (the shape of the paper's Indian Pines subscene) for each
Schatten p in {1, 2, inf}; other workloads are listed under --help.

`--impl reference` times the FP64 CPU oracle (the only reference there is: the paper has no
code) on the host cores, on a bounded sample of the same workload (a 256x256 crop for images
above 512x512, scaled to the full image by pixel count).
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
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("ADMM iters/s and Mpixel·class·iter/s at 1e-4 vs FP64; % HBM roofline")
SP_LIST = (1, 2, np.inf)


def _sweep_traffic(workload):
    """DRAM bytes per sweep launch from the committed ncu summary, or None when the summary is
    for another workload or the kernel sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"sweep_traffic_{workload}_k16.json")
    try:
        with open(path) as f:
            d = json.load(f)
        src = "".join(open(os.path.join(ROOT, p)).read() for p in d["source_files"])
        if hashlib.sha256(src.encode()).hexdigest() != d["source_sha256"]:
            return None
        return float(d["dram_bytes_read_per_launch"] + d["dram_bytes_write_per_launch"])
    except Exception:
        return None


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (the slowest replica defines the step time); the
    identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of `world` replicas that each processed `units_per_rank` units,
    timed by the slowest rank."""
    return units_per_rank * world / seconds_max


def cpu_info():
    """Host cores this process may run on and the BLAS thread setting the oracle runs under."""
    try:
        host = len(os.sched_getaffinity(0))
    except Exception:
        host = os.cpu_count() or 1
    blas = None
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            blas = f"{var}={os.environ[var]}"
            break
    if blas is None:
        try:
            from threadpoolctl import threadpool_info
            n = [d.get("num_threads") for d in threadpool_info() if d.get("user_api") == "blas"]
            blas = f"threadpoolctl: {n[0]}" if n else "unset (numpy default)"
        except Exception:
            blas = "unset (numpy default)"
    return {"host_cores": host, "blas_threads": blas}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(name, patch=None):
    """Scene, solver settings and description of a workload; `patch` (M) replaces the 3x3
    patch of the HxW workloads by a (2M+1)x(2M+1) one (Gaussian sigma = max(0.5, M/2))."""
    import dataclasses
    from paper_1504_07028_gb300 import synth
    if name == "145x145":
        sc = synth.scene_145x145_k16()
        cfgs = [synth.CFG_145[sp] for sp in SP_LIST]
        desc = ("145x145 K=16, 3x3 Gaussian patch sigma=0.5, lambda=1.5, mu=1, 300 iterations "
                "for each Schatten p in {1,2,inf}")
    elif name == "patchsweep":
        sc = synth.scene_145x145_k16()
        cfgs = [synth.SolverConfig(M=m, sigma=max(0.5, 0.5 * m), lam=1.5, mu=1.0,
                                   schatten_p=1, iters=300) for m in (0, 1, 2, 3, 4, 5)]
        desc = ("145x145 K=16, Schatten p=1, lambda=1.5, mu=1, 300 iterations for each patch "
                "1x1, 3x3, 5x5, 7x7, 9x9 and 11x11 (Gaussian sigma = M/2, 0.5 for 1x1): time "
                "against L (Fig. 1's patch sweep without the dataset)")
    elif name == "64x64":
        sc = synth.scene_64x64_k4()
        cfgs = [synth.CFG_64]
        desc = "64x64 K=4, 3x3 Gaussian patch sigma=0.5, lambda=2, mu=1, 200 iterations, p=1"
    elif name == "2048x2048":
        sc = synth.scene_2048x2048_k16()
        cfgs = [synth.CFG_BATCH]
        desc = "2048x2048 K=16, 3x3 Gaussian patch sigma=0.5, lambda=2, mu=1, 200 iterations, p=1"
    elif "x" in name:
        H, W = (int(v) for v in name.split("x"))
        sc = synth.scene(H, W, 16, S=64, gap=3.0, noise_std=1.0, wrong_frac=0.0, seed=56)
        cfgs = [synth.CFG_BATCH]
        desc = f"{H}x{W} K=16, 3x3 Gaussian patch sigma=0.5, lambda=2, mu=1, 200 iterations, p=1"
    else:
        raise SystemExit(f"unknown workload {name}")
    if patch is not None:
        if "x" not in name or name in ("145x145", "64x64"):
            raise SystemExit("--patch applies to the HxW workloads only")
        cfgs = [dataclasses.replace(c, M=patch, sigma=max(0.5, 0.5 * patch)) for c in cfgs]
        desc = desc.replace("3x3 Gaussian patch sigma=0.5",
                            f"{2 * patch + 1}x{2 * patch + 1} Gaussian patch sigma={max(0.5, 0.5 * patch)}")
    return sc, cfgs, desc


# -------------------------------------------------------------------- reference arm (oracle)

def oracle_sample(sc, cfgs, iters_per_p):
    """Time the FP64 oracle for `iters_per_p` iterations of each solve of the workload (on the
    crop of `oracle_crop` for large images). Returns (full-image iterations, wall s, threads
    used, crop scale)."""
    from oracle import segsalsa_str_oracle as O
    pc, scale = oracle_crop(sc)
    p = pc.astype(np.float32).astype(np.float64)
    t0, c0 = time.perf_counter(), time.process_time()
    n = 0
    for cfg in cfgs:
        O.solve(p, cfg.M, cfg.sigma, cfg.lam, cfg.mu, cfg.schatten_p, iters_per_p,
                trace_every=10)
        n += iters_per_p
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    return n * scale, wall, (max(1, round(cpu / wall)) if wall > 0 else 1), scale


def sample_note(sc, iters, nsolves, wall):
    """What the oracle sample was, in words."""
    pc, scale = oracle_crop(sc)
    what = (f"{iters} iterations of each of the {nsolves} solves" if nsolves > 1
            else f"{iters} iterations")
    if scale < 1.0:
        return (f"{what} on the top-left {pc.shape[1]}x{pc.shape[2]} crop of the {sc.H}x{sc.W} "
                f"scene ({wall:.1f} s), scaled to the full image by pixel count (x{scale:.5f})")
    return f"{what} of the full workload ({wall:.1f} s)"


CROP = 256          # oracle sample side for images above 512x512


def oracle_crop(sc):
    """The oracle's sample of a large scene: its top-left CROP x CROP probabilities, or the
    whole scene when it is at most 512x512. Returns (p, pixel-count scale to the full image)."""
    if sc.H * sc.W <= 512 * 512:
        return sc.p, 1.0
    p = np.ascontiguousarray(sc.p[:, :CROP, :CROP])
    return p, (CROP * CROP) / (sc.H * sc.W)


BATCH_DESC = ("64 images, H and W uniform in [96, 512], K uniform in {4, 8, 16}, 3x3 Gaussian "
              "patch sigma=0.5, lambda=2, mu=1, 200 iterations each, p=1, autotuned tiling")


def oracle_batch_sample(scenes, cfg, images, iters):
    """Time the FP64 oracle for `iters` iterations of each image index in `images`; returns
    (pixel-class-iterations, wall seconds, cores)."""
    from oracle import segsalsa_str_oracle as O
    t0, c0 = time.perf_counter(), time.process_time()
    units = 0
    for j in images:
        sc = scenes[j]
        O.solve(sc.p.astype(np.float32).astype(np.float64), cfg.M, cfg.sigma, cfg.lam, cfg.mu,
                cfg.schatten_p, iters)
        units += sc.H * sc.W * sc.K * iters
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    return units, wall, max(1, round(cpu / wall)) if wall > 0 else 1


def run_reference_batch(args):
    from paper_1504_07028_gb300 import synth
    scenes = synth.batch_scenes()
    cfg = synth.CFG_BATCH
    mean_units = np.mean([s.H * s.W * s.K for s in scenes])
    for _ in range(args.warmup):
        oracle_batch_sample(scenes, cfg, [0], 1)
    tot_u, tot_t, cores = 0, 0.0, 1
    for k in range(args.steps):
        imgs = [(8 * k + j) % len(scenes) for j in range(8)]
        u, t, cores = oracle_batch_sample(scenes, cfg, imgs, 1)
        tot_u += u
        tot_t += t
    v = tot_u / tot_t / mean_units     # image-iterations per second of the batch's mean image
    sample = (f"1 iteration of 8 batch images per step ({args.steps} steps), converted to "
              f"iterations of the batch's mean image (pixel-class rate / mean H*W*K)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ADMM iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": BATCH_DESC, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "ADMM iter/s", "cores": cores, "kind": "oracle",
                         "sample": sample, **cpu_info()},
        "e2e": {"value": v, "unit": "ADMM iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


MLR_CROP = (122, 68)   # 1/25 of the 610x340 pixels


def oracle_mlr_sample(iters):
    """FP64 oracle on a 122x68 crop of the MLR workload (same K, d, patch): MLR probabilities
    plus `iters` iterations. Returns (full-image iterations per second, wall s, cores)."""
    import torch
    from oracle import segsalsa_str_oracle as O
    from paper_1504_07028_gb300 import synth
    sc = synth.scene_610x340_mlr()
    cfg = synth.CFG_MLR
    ch, cw = MLR_CROP
    xc = np.ascontiguousarray(sc.x[:ch, :cw])
    x = torch.from_numpy(xc.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    w = torch.from_numpy(sc.Wc.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    t0, c0 = time.perf_counter(), time.process_time()
    O.solve(O.mlr_probs(x, w), cfg.M, cfg.sigma, cfg.lam, cfg.mu, cfg.schatten_p, iters)
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    scale = (ch * cw) / (sc.H * sc.W)
    return iters * scale / wall, wall, max(1, round(cpu / wall))


def run_reference_mlr(args):
    per = max(1, args.ref_iters)
    for _ in range(args.warmup):
        oracle_mlr_sample(1)
    rates, walls, cores = [], 0.0, 1
    for _ in range(args.steps):
        r, wall, cores = oracle_mlr_sample(per)
        rates.append(r)
        walls += wall
    v = float(np.mean(rates))
    tot_t = walls
    sample = (f"MLR probabilities + {per} iterations of a {MLR_CROP[0]}x{MLR_CROP[1]} crop per "
              f"step ({args.steps} steps), scaled to the 610x340 image by pixel count")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ADMM iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": MLR_DESC, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "ADMM iter/s", "cores": cores, "kind": "oracle",
                         "sample": sample, **cpu_info()},
        "e2e": {"value": v, "unit": "ADMM iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload == "batch64":
        run_reference_batch(args)
        return
    if args.workload == "mlr610x340":
        run_reference_mlr(args)
        return
    if args.workload == "diff256":
        run_reference_diff(args)
        return
    sc, cfgs, desc = make_workload(args.workload, args.patch)
    per_p = max(1, args.ref_iters)
    for _ in range(min(args.warmup, 1)):
        oracle_sample(sc, cfgs, 1)
    tot_n, tot_t, cores = 0.0, 0.0, 1
    for _ in range(args.steps):
        n, t, cores, _ = oracle_sample(sc, cfgs, per_p)
        tot_n += n
        tot_t += t
    v = tot_n / tot_t
    sample = (sample_note(sc, per_p, len(cfgs), tot_t / max(1, args.steps)) +
              f"; per step, {args.steps} steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ADMM iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "ADMM iter/s", "cores": cores, "kind": "oracle",
                         "sample": sample, **cpu_info()},
        "e2e": {"value": v, "unit": "ADMM iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1504_07028_gb300 import binding as B
    from paper_1504_07028_gb300 import build as Bu

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    Bu.build()
    sc, cfgs, desc = make_workload(args.workload, args.patch)
    K, H, W = sc.K, sc.H, sc.W
    n = H * W
    # the solves of a step are independent: each gets its own handle, stream and host thread,
    # so their kernels overlap on the GPU (ctypes releases the GIL during the C calls)
    stream = torch.cuda.current_stream(dev)
    streams = [torch.cuda.Stream(dev) for _ in cfgs]
    solvers = []
    for cfg, sx in zip(cfgs, streams):
        solvers.append((cfg, B.Solver(B.make_params(
            H, W, K, M=cfg.M, sigma=cfg.sigma, lam=cfg.lam, mu=cfg.mu,
            schatten_p=cfg.schatten_p, precision="fp32", stream=sx.cuda_stream))))
    p_dev = torch.from_numpy(sc.p.astype(np.float32)).to(dev)          # (K, H, W)
    labs_dev = [torch.empty((H, W), dtype=torch.int32, device=dev) for _ in cfgs]
    iters_per_step = sum(cfg.iters for cfg in cfgs)
    ws_bytes = B.segsalsa_str_workspace_bytes(B.make_params(
        H, W, K, M=cfgs[0].M, sigma=cfgs[0].sigma, lam=cfgs[0].lam, mu=cfgs[0].mu,
        schatten_p=cfgs[0].schatten_p, precision="fp32"))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    pool = ThreadPoolExecutor(max_workers=len(cfgs))

    if args.profile_run:                     # eager launches (profiling mode), one thread
        for _, s in solvers:
            s.set_profiling(True)

    def run_all(p_src, labs):
        def one(i):
            cfg, s = solvers[i]
            s.set_probs(p_src)
            s.solve(cfg.iters, trace_every=10)
            s.get_labels(labs[i])
        if args.profile_run:
            for i in range(len(solvers)):
                one(i)
        else:
            list(pool.map(one, range(len(solvers))))

    def step():
        stream.synchronize()                 # p and the L2 flush are ready
        run_all(p_dev, labs_dev)             # each call returns after its stream finished

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(nsteps):
        out = []
        for _ in range(nsteps):
            flush.zero_()                       # L2 flushed between timed steps (untimed)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return out

    for _, s in solvers:
        s.reset_stats()
    clocks = Clocks(local_rank)
    barrier()
    clocks.start()
    times = timed(args.steps)
    barrier()
    ck = clocks.stop()
    total_ms = max_over_ranks(float(sum(times)), dev)
    launches = 0
    for _, s in solvers:
        launches += sum(c for c, _ in s.kernel_stats().values())
    # each solve alone, CUDA-graph replay as in the timed steps (events on its own stream): the
    # time per iteration of one image without the overlap of the concurrent solves
    single_us = []
    if not args.profile_run:
        for (cfg, s), sx in zip(solvers, streams):
            s.set_probs(p_dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(sx)
            s.solve(cfg.iters, trace_every=10)
            b.record(sx)
            b.synchronize()
            single_us.append(1e3 * a.elapsed_time(b) / cfg.iters)
    # per-kernel device times: CUDA events around every launch, recorded on the launch stream
    # during a replay of the same steps (the events add ~1 us gaps, so they stay out of `value`)
    for _, s in solvers:
        s.reset_stats()
        s.set_profiling(True)
    prof_ms = 0.0
    for _ in range(args.steps):          # one solve at a time: durations without overlap
        for i, (cfg, s) in enumerate(solvers):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.set_probs(p_dev)
            s.solve(cfg.iters, trace_every=10)
            s.get_labels(labs_dev[i])
            b.record(stream)
            b.synchronize()
            prof_ms += a.elapsed_time(b)
    stats = {}
    hbm_peak, peak_kind = _peaks()
    per_solve = []
    sw_bytes_tot = 0.0
    for cfg, s in solvers:
        st = s.kernel_stats()
        for kname, (cnt, ms) in st.items():
            c0, m0 = stats.get(kname, (0, 0.0))
            stats[kname] = (c0 + cnt, m0 + ms)
        sb, ib = s.traffic_model()
        c_sw, m_sw = st["sweep"]
        n_sw = args.steps * cfg.iters          # sweeps (a wide-patch sweep is three launches)
        sw_bytes_tot += sb * n_sw
        per_solve.append({
            "M": cfg.M, "L": (2 * cfg.M + 1) ** 2, "schatten_p": str(cfg.schatten_p),
            "sweep_us": m_sw / n_sw * 1e3, "sweep_gbs": sb / (m_sw / n_sw * 1e-3) / 1e9,
            "sweep_frac_of_hbm": sb / (m_sw / n_sw * 1e-3) / 1e9 / hbm_peak,
            "kernel_ms_per_iteration": sum(m for _, m in st.values()) / (args.steps * cfg.iters)})
        if single_us:
            per_solve[-1]["graph_us_per_iteration_alone"] = single_us[len(per_solve) - 1]
        s.set_profiling(args.profile_run)
    dom = max(stats.items(), key=lambda kv: kv[1][1])
    sweep_bytes, iter_bytes = solvers[0][1].traffic_model()
    sw_cnt, sw_ms = stats["sweep"]
    sw_cnt = args.steps * iters_per_step     # sweeps, as above
    achieved = sw_bytes_tot / (sw_ms * 1e-3) / 1e9
    # the z-update (12) as a second roofline: the three passes of one z-update against its
    # algorithmic bytes (rhs read and z written once, 8 B per pixel and class in FP32)
    z_cnt = stats["column_solve"][0]
    z_ms = sum(stats[k][1] for k in ("row_fft_forward", "column_solve", "row_fft_inverse"))
    z_roof = None
    if z_cnt:
        z_us = z_ms / z_cnt * 1e3
        z_gbs = 8.0 * n * K / (z_us * 1e-6) / 1e9
        z_roof = {"bound": "hbm", "kernels": "row DFT forward + column solve + row DFT inverse",
                  "achieved": z_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": z_gbs / hbm_peak,
                  "peak_source": peak_kind, "algorithmic_bytes_per_zupdate": 8.0 * n * K,
                  "avg_zupdate_us": z_us}
    value = whole_job_rate(iters_per_step * args.steps, world, total_ms * 1e-3)
    mpix = value * n * K / 1e6

    # ---- end to end through the public API with host buffers (pinned p in, labels out)
    p_host = torch.from_numpy(sc.p.astype(np.float32)).pin_memory()
    labs_host = [torch.empty((H, W), dtype=torch.int32).pin_memory() for _ in cfgs]
    e2e_times = []
    for i in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_all(p_host, labs_host)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_times), dev)
    e2e_value = whole_job_rate(iters_per_step * len(e2e_times), world, e2e_s)
    h2d = 4 * n * K * len(solvers)
    d2h = 4 * n * len(solvers) + sum(48 * (cfg.iters // 10 + 1) for cfg, _ in solvers)

    # ---- accuracy of the timed FP32 path against FP64 (GPU FP64 path, validated against the
    #      FP64 oracle in the GPU tests): max |z32 - z64| and label agreement off the margin band
    err, lab_ok = 0.0, True
    fp64_form = None
    if rank == 0 and not args.skip_fp64_check:
        streams64 = [torch.cuda.Stream(dev) for _ in cfgs]
        solvers64 = [(cfg, B.Solver(B.make_params(H, W, K, M=cfg.M, sigma=cfg.sigma, lam=cfg.lam,
                                                  mu=cfg.mu, schatten_p=cfg.schatten_p,
                                                  precision="fp64", stream=sx.cuda_stream)))
                     for cfg, sx in zip(cfgs, streams64)]
        p64 = p_dev.to(torch.float64)
        labs64 = [torch.empty((H, W), dtype=torch.int32, device=dev) for _ in cfgs]

        def step64():
            def one(i):
                cfg, s64 = solvers64[i]
                s64.set_probs(p64)
                s64.solve(cfg.iters, trace_every=10)
                s64.get_labels(labs64[i])
            stream.synchronize()
            list(pool.map(one, range(len(solvers64))))

        step64()                                  # warm-up (graphs built)
        flush.zero_()
        a64 = torch.cuda.Event(enable_timing=True)
        b64 = torch.cuda.Event(enable_timing=True)
        a64.record(stream)
        step64()
        b64.record(stream)
        b64.synchronize()
        v64 = iters_per_step / (a64.elapsed_time(b64) * 1e-3)
        fp64_form = {"value": v64, "unit": "ADMM iter/s",
                     "note": "the same step (solves, streams, trace) with the FP64 handles",
                     "fp32_speedup": value / v64}
        for (cfg, s), (_, s64) in zip(solvers, solvers64):
            s.set_probs(p_dev)
            s.solve(cfg.iters)
            z32 = s.get_z()
            z64 = s64.get_z()
            err = max(err, float(np.abs(z32 - z64).max()))
            srt = np.sort(z64, axis=0)
            clear = srt[-1] - srt[-2] >= 1e-3
            lab_ok &= bool(np.array_equal(np.argmax(z32, 0)[clear], np.argmax(z64, 0)[clear]))
        for _, s64 in solvers64:
            s64.close()

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        it = max(1, args.cpu_iters)
        nn, wall, cores, _ = oracle_sample(sc, cfgs[:1], it)
        cpu = {"value": nn / wall, "unit": "ADMM iter/s", "cores": cores, "kind": "oracle",
               "sample": sample_note(sc, it, 1, wall) +
                         (" (the p=1 solve)" if len(cfgs) > 1 else ""),
               **cpu_info()}

    line = {
        "metric": METRIC, "value": value, "unit": "ADMM iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": desc, "H": H, "W": W, "K": K, "iters_per_step": iters_per_step,
                   "concurrency": f"{len(cfgs)} independent solves per step, one stream and host "
                                  "thread each",
                   "l2": ("flushed between timed steps (256 MB write); the "
                          f"{ws_bytes / 1e6:.0f} MB working set per solve "
                          + ("exceeds L2" if ws_bytes > 129e6 else "is L2-resident within a step")),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "mpixel_class_iter_per_s": mpix,
        "accuracy": {"max_abs_z_vs_fp64": err, "labels_match_off_1e-3_margin": lab_ok},
        "fp64_form": fp64_form,
        "roofline": {"bound": "hbm", "kernel": "sweep (fused prox + dual + rhs partials)",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_source": peak_kind,
                     "traffic": _sweep_traffic(args.workload),
                     "algorithmic_bytes_per_launch": sw_bytes_tot / sw_cnt,
                     "avg_launch_us": sw_ms / sw_cnt * 1e3},
        "zupdate_roofline": z_roof,
        "kernel_ms": {k: {"launches": c, "ms": round(m, 4)} for k, (c, m) in stats.items()},
        "us_per_iteration_one_solve_alone": (sum(single_us) / len(single_us)) if single_us else None,
        "per_solve": per_solve,
        "kernel_timing": ("CUDA events around every launch on the launch stream, in a replay "
                          f"of the {args.steps} timed steps with the solves run one at a time "
                          f"({prof_ms:.1f} ms with the events; the events break the programmatic "
                          "dependent launches and add gaps, so kernel_ms overstates the "
                          "iteration: us_per_iteration_one_solve_alone is the graph-replay time "
                          "of one solve)"),
        "dominant_kernel": dom[0],
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "ADMM iter/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    for _, s in solvers:
        s.close()
    pool.shutdown()
    return line if rank == 0 else None


def run_batch(args, rank, world, local_rank):
    """The serving-style batch: 64 uneven images in one batch handle (CUDA-graph chunks over
    concurrent lanes). One step = set_probs of every image (device-resident p), 200 iterations
    of the whole batch, label readout of every image. value = image-iterations per second."""
    import torch
    from paper_1504_07028_gb300 import binding as B
    from paper_1504_07028_gb300 import build as Bu
    from paper_1504_07028_gb300 import synth

    from paper_1504_07028_gb300 import shard

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    Bu.build()
    all_scenes = synth.batch_scenes()
    cfg = synth.CFG_BATCH
    # the images are independent problems: each rank takes its share (longest processing time
    # first on the per-iteration bytes), no collective on the data path
    costs = [shard.iteration_bytes(s.H, s.W, s.K, cfg.M) for s in all_scenes]
    mine = shard.partition(costs, world)[rank]
    scenes = [all_scenes[j] for j in mine]
    nimg = len(scenes)
    params = [B.make_params(s.H, s.W, s.K, M=cfg.M, sigma=cfg.sigma, lam=cfg.lam, mu=cfg.mu,
                            schatten_p=cfg.schatten_p) for s in scenes]
    bt = B.Batch(params)
    tune_s, chosen = 0.0, None
    if not args.no_autotune:
        t0 = time.perf_counter()
        chosen = bt.autotune(args.tune_iters)
        tune_s = time.perf_counter() - t0
    p_dev = [torch.from_numpy(s.p.astype(np.float32)).to(dev) for s in scenes]
    labs_dev = [torch.empty((s.H, s.W), dtype=torch.int32, device=dev) for s in scenes]
    torch.cuda.synchronize()            # the batch's streams do not wait for torch's stream
    units = [s.H * s.W * s.K for s in scenes]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_all(p_src, labs):
        for j in range(nimg):
            bt.image(j).set_probs(p_src[j])
        bt.solve(cfg.iters)
        for j in range(nimg):
            bt.image(j).get_labels(labs[j])

    for _ in range(args.warmup):
        run_all(p_dev, labs_dev)
    torch.cuda.synchronize()
    for j in range(nimg):
        bt.image(j).reset_stats()
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_all(p_dev, labs_dev)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_ms = max_over_ranks(float(sum(times)), dev)
    launches = sum(sum(c for c, _ in bt.image(j).kernel_stats().values()) for j in range(nimg))
    iters_per_step = len(all_scenes) * cfg.iters          # the whole batch, all ranks
    value = iters_per_step * args.steps / (total_ms * 1e-3)
    all_units = sum(s.H * s.W * s.K for s in all_scenes)
    mpix = all_units * cfg.iters * args.steps / (total_ms * 1e-3) / 1e6
    iter_bytes = sum(bt.image(j).traffic_model()[1] for j in range(nimg))
    ws_total = sum(B.segsalsa_str_workspace_bytes(p) for p in params)
    path_gbs = iter_bytes * cfg.iters * args.steps / (total_ms * 1e-3) / 1e9

    # per-kernel device times: each image alone, eager launches with CUDA events around each
    # (a serial replay; the batch itself overlaps the images)
    prof_iters = 20
    stats = {}
    sweep_bytes_total = 0.0
    for j in range(nimg):
        im = bt.image(j)
        im.reset_stats()
        im.set_profiling(True)
        im.set_probs(p_dev[j])
        im.solve(prof_iters)
        for kname, (cnt, ms) in im.kernel_stats().items():
            c0, m0 = stats.get(kname, (0, 0.0))
            stats[kname] = (c0 + cnt, m0 + ms)
        sweep_bytes_total += im.traffic_model()[0] * prof_iters
        im.set_profiling(False)
    sw_cnt, sw_ms = stats["sweep"]
    hbm_peak, peak_kind = _peaks()
    achieved = sweep_bytes_total / (sw_ms * 1e-3) / 1e9
    dom = max(stats.items(), key=lambda kv: kv[1][1])

    # end to end with host buffers: pinned p in, labels out
    p_host = [torch.from_numpy(s.p.astype(np.float32)).pin_memory() for s in scenes]
    labs_host = [torch.empty((s.H, s.W), dtype=torch.int32).pin_memory() for s in scenes]
    e2e_times = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_all(p_host, labs_host)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_times), dev)
    e2e_value = iters_per_step * len(e2e_times) / e2e_s

    # accuracy against the FP64 GPU path on sampled images (smallest, largest, first)
    err, lab_ok = 0.0, True
    sample = sorted({int(np.argmin(units)), int(np.argmax(units)), 0})
    if rank == 0 and not args.skip_fp64_check:
        for j in range(nimg):
            bt.image(j).set_probs(p_dev[j])
        bt.solve(cfg.iters)
        for j in sample:
            s = scenes[j]
            z32 = bt.image(j).get_z()
            s64 = B.Solver(B.make_params(s.H, s.W, s.K, M=cfg.M, sigma=cfg.sigma, lam=cfg.lam,
                                         mu=cfg.mu, schatten_p=cfg.schatten_p, precision="fp64"))
            s64.set_probs(s.p.astype(np.float32).astype(np.float64))
            s64.solve(cfg.iters)
            z64 = s64.get_z()
            s64.close()
            err = max(err, float(np.abs(z32 - z64).max()))
            srt = np.sort(z64, axis=0)
            clear = srt[-1] - srt[-2] >= 1e-3
            lab_ok &= bool(np.array_equal(np.argmax(z32, 0)[clear], np.argmax(z64, 0)[clear]))

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        u, wall, cores = oracle_batch_sample(scenes, cfg, [int(np.argmin(units)), 0],
                                             max(1, args.cpu_iters // 2))
        v = u / wall / np.mean(units)
        cpu = {"value": v, "unit": "ADMM iter/s", "cores": cores, "kind": "oracle",
               "sample": f"{max(1, args.cpu_iters // 2)} iterations of two batch images "
                         f"({wall:.1f} s), converted to iterations of the batch's mean image",
               **cpu_info()}

    line = {
        "metric": METRIC, "value": value, "unit": "ADMM iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "scaling": "strong",               # the batch's total work is fixed, whatever N
        "config": {"workload": BATCH_DESC, "images": len(all_scenes), "images_this_rank": nimg,
                   "iters_per_image": cfg.iters,
                   "pixel_class_total": int(all_units), "lanes": bt.lanes(),
                   "autotune_s": round(tune_s, 2), "tilings": chosen,
                   "l2": "flushed between timed steps (256 MB write); the batch's working set "
                         f"({ws_total / 1e9:.1f} GB of workspaces) exceeds L2",
                   "parallelism": (f"images sharded over {world} ranks by per-iteration "
                                   "bytes, no collective" if world > 1 else "single GPU")},
        "mpixel_class_iter_per_s": mpix,
        "path_effective_gbs": path_gbs,
        "path_frac_of_hbm": path_gbs / hbm_peak,
        "accuracy": {"max_abs_z_vs_fp64": err, "labels_match_off_1e-3_margin": lab_ok,
                     "sampled_images": sample},
        "roofline": {"bound": "hbm", "kernel": "sweep (fused prox + dual + rhs partials)",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_source": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": sweep_bytes_total / sw_cnt,
                     "avg_launch_us": sw_ms / sw_cnt * 1e3},
        "kernel_ms": {k: {"launches": c, "ms": round(m, 4)} for k, (c, m) in stats.items()},
        "kernel_timing": (f"CUDA events around every launch, each image alone for {prof_iters} "
                          "eager iterations (the batch overlaps images; this replay does not)"),
        "dominant_kernel": dom[0],
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "ADMM iter/s",
                "h2d_bytes_per_step": 4 * int(all_units),
                "d2h_bytes_per_step": 4 * int(sum(s.H * s.W for s in all_scenes))},
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    bt.close()


MLR_DESC = ("610x340 K=9, d=103 bands, MLR class model p = softmax(W x) as BF16 tensor-core GEMM "
            "(FP32 accumulation) + softmax, 5x5 Gaussian patch sigma=1, lambda=1.5, mu=1, Schatten "
            "p=1, 400 iterations")


def run_mlr(args, rank, world, local_rank):
    """Mixed-precision workload with the MLR front end. One step = set_spectra (BF16 spectra and
    weights resident on the device: tensor-core GEMM + softmax + validation + init), 400 FP32
    SALSA iterations with the trace every 10, label readout. value = ADMM iterations/s."""
    import torch
    from paper_1504_07028_gb300 import binding as B
    from paper_1504_07028_gb300 import build as Bu
    from paper_1504_07028_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    Bu.build()
    sc = synth.scene_610x340_mlr()
    cfg = synth.CFG_MLR
    H, W, K, d = sc.H, sc.W, sc.K, sc.d
    n = H * W
    mk = lambda prec: B.make_params(H, W, K, M=cfg.M, sigma=cfg.sigma, lam=cfg.lam, mu=cfg.mu,
                                    schatten_p=cfg.schatten_p, precision=prec)
    s = B.Solver(mk("fp32"))
    xh = torch.from_numpy(sc.x.astype(np.float32)).to(torch.bfloat16)
    wh = torch.from_numpy(sc.Wc.astype(np.float32)).to(torch.bfloat16)
    xd, wd = xh.to(dev), wh.to(dev)
    lab = torch.empty((H, W), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()

    def step(x, w, out):
        s.set_spectra(x, w)
        s.solve(cfg.iters, trace_every=10)
        s.get_labels(out)

    if args.profile_run:                     # eager launches for runs under a profiler
        s.set_profiling(True)
    for _ in range(args.warmup):
        step(xd, wd, lab)
    torch.cuda.synchronize()
    s.reset_stats()
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(xd, wd, lab)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_ms = max_over_ranks(float(sum(times)), dev)
    launches = sum(c for c, _ in s.kernel_stats().values())
    value = whole_job_rate(cfg.iters * args.steps, world, total_ms * 1e-3)
    # per-kernel device times: a profiled (eager) replay of the timed steps
    s.reset_stats()
    s.set_profiling(True)
    for _ in range(args.steps):
        flush.zero_()
        step(xd, wd, lab)
    stats = s.kernel_stats()
    s.set_profiling(args.profile_run)
    hbm_peak, peak_kind = _peaks()
    sweep_bytes, _ = s.traffic_model()
    sw_cnt, sw_ms = stats["sweep"]
    achieved = sweep_bytes / (sw_ms / sw_cnt * 1e-3) / 1e9
    ml_cnt, ml_ms = stats["mlr"]
    dpad, npad = (d + 15) // 16 * 16, (16 if K <= 16 else 32)
    mlr_bytes = n * d * 2 + K * d * 2 + n * K * 4
    mlr_s = ml_ms / ml_cnt * 1e-3
    dom = max(stats.items(), key=lambda kv: kv[1][1])
    # end to end with host buffers (pinned BF16 spectra and weights in, labels out)
    xp = xh.view(torch.int16).pin_memory()
    wp = wh.view(torch.int16).pin_memory()
    xp_np, wp_np = xp.numpy().view(np.uint16), wp.numpy().view(np.uint16)
    labh = torch.empty((H, W), dtype=torch.int32).pin_memory()
    e2e = []
    for _ in range(max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(xp_np, wp_np, labh)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e), dev)
    e2e_value = whole_job_rate(cfg.iters * len(e2e), world, e2e_s)
    # accuracy against the FP64 GPU path from the same BF16 inputs
    err, lab_ok = 0.0, True
    if rank == 0 and not args.skip_fp64_check:
        s.set_spectra(xd, wd)
        s.solve(cfg.iters)
        z32 = s.get_z()
        s64 = B.Solver(mk("fp64"))
        s64.set_spectra(xd, wd)
        s64.solve(cfg.iters)
        z64 = s64.get_z()
        s64.close()
        err = float(np.abs(z32 - z64).max())
        srt = np.sort(z64, axis=0)
        clear = srt[-1] - srt[-2] >= 1e-3
        lab_ok = bool(np.array_equal(np.argmax(z32, 0)[clear], np.argmax(z64, 0)[clear]))
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        it = max(1, args.cpu_iters)
        v_cpu, wall, cores = oracle_mlr_sample(it)
        cpu = {"value": v_cpu, "unit": "ADMM iter/s", "cores": cores, "kind": "oracle",
               "sample": f"MLR probabilities + {it} iterations of a {MLR_CROP[0]}x{MLR_CROP[1]} "
                         f"crop ({wall:.1f} s), scaled to the full image by pixel count",
               **cpu_info()}
    line = {
        "metric": METRIC, "value": value, "unit": "ADMM iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
        "data": "synthetic",
        "config": {"workload": MLR_DESC, "H": H, "W": W, "K": K, "d": d, "iters_per_step": cfg.iters,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "mpixel_class_iter_per_s": value * n * K / 1e6,
        "accuracy": {"max_abs_z_vs_fp64": err, "labels_match_off_1e-3_margin": lab_ok},
        "roofline": {"bound": "hbm", "kernel": "sweep (fused prox + dual + rhs partials)",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_source": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": sweep_bytes,
                     "avg_launch_us": sw_ms / sw_cnt * 1e3},
        "mlr_kernel": {"bound": "hbm", "avg_launch_us": mlr_s * 1e6,
                       "algorithmic_bytes": mlr_bytes, "achieved_gbs": mlr_bytes / mlr_s / 1e9,
                       "frac_of_hbm": mlr_bytes / mlr_s / 1e9 / hbm_peak,
                       "tensor_flops": 2 * n * dpad * npad,
                       "achieved_tflops": 2 * n * dpad * npad / mlr_s / 1e12},
        "kernel_ms": {k: {"launches": c, "ms": round(m, 4)} for k, (c, m) in stats.items()},
        "kernel_timing": "CUDA events around every launch on the launch stream, in an eager "
                         "replay of the timed steps",
        "dominant_kernel": dom[0],
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "ADMM iter/s", "h2d_bytes_per_step": n * d * 2 + K * d * 2,
                "d2h_bytes_per_step": 4 * n + 48 * (cfg.iters // 10 + 1)},
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()


DIFF_DESC = ("256x256 K=8, 3x3 Gaussian patch sigma=0.5, lambda=2, mu=1, Schatten p=1: gradient of "
             "<zbar, z^50> with respect to log p, lambda and the 9 shift weights (forward pass, "
             "checkpoints every 10 iterations, reverse pass)")


def oracle_grad_sample():
    """FP64 reference gradient (oracle autograd) on a 64x64 crop of the differentiable
    workload; returns (full-image differentiated iterations per second, wall s, cores)."""
    from oracle import segsalsa_str_oracle as O
    from oracle import unrolled_grad as U
    from paper_1504_07028_gb300 import synth
    sc = synth.scene_256x256_k8()
    cfg = synth.CFG_256
    lp = np.log(sc.p[:, :64, :64])
    zb = np.random.default_rng(7).normal(size=lp.shape)
    t0, c0 = time.perf_counter(), time.process_time()
    U.reference_gradient(lp, cfg.lam, O.gaussian_weights(cfg.M, cfg.sigma), cfg.M, cfg.mu,
                         cfg.schatten_p, cfg.iters, zb)
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    return cfg.iters * (64 * 64) / (256 * 256) / wall, wall, max(1, round(cpu / wall))


def run_diff(args, rank, world, local_rank):
    """Differentiable solver. One step = set_log_probs (device log p) + segsalsa_str_backward
    (forward pass with checkpoints, reverse pass) giving d/dlog p on the device and d/dlambda,
    d/domega on the host. value = differentiated ADMM iterations per second."""
    import torch
    from paper_1504_07028_gb300 import binding as B
    from paper_1504_07028_gb300 import build as Bu
    from paper_1504_07028_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    Bu.build()
    sc = synth.scene_256x256_k8()
    cfg = synth.CFG_256
    H, W, K = sc.H, sc.W, sc.K
    mk = lambda prec: B.Solver(B.make_params(H, W, K, M=cfg.M, sigma=cfg.sigma, lam=cfg.lam,
                                             mu=cfg.mu, schatten_p=cfg.schatten_p, precision=prec))
    s = mk("fp32")
    lp = torch.tensor(np.log(sc.p), dtype=torch.float32, device=dev)
    zb = torch.tensor(np.random.default_rng(7).normal(size=(K, H, W)), dtype=torch.float32,
                      device=dev)
    g = torch.empty_like(lp)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    every = 10

    def step(lp_in, zb_in, out):
        s.set_log_probs(lp_in)
        return s.backward(cfg.iters, zb_in, every, out=out)

    for _ in range(args.warmup):
        step(lp, zb, g)
    torch.cuda.synchronize()
    s.reset_stats()
    clocks = Clocks(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = step(lp, zb, g)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    total_ms = max_over_ranks(float(sum(times)), dev)
    launches = sum(c for c, _ in s.kernel_stats().values())
    value = whole_job_rate(cfg.iters * args.steps, world, total_ms * 1e-3)
    # forward alone, for the cost of differentiation
    t_fwd = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.set_log_probs(lp)
        s.solve(cfg.iters)
        b.record(stream)
        b.synchronize()
        t_fwd.append(a.elapsed_time(b))
    # per-kernel device times (profiled eager replay of one step)
    s.reset_stats()
    s.set_profiling(True)
    step(lp, zb, g)
    stats = s.kernel_stats()
    s.set_profiling(False)
    hbm_peak, peak_kind = _peaks()
    sweep_bytes, _ = s.traffic_model()
    sw_cnt, sw_ms = stats["sweep"]
    achieved = sweep_bytes / (sw_ms / sw_cnt * 1e-3) / 1e9
    dom = max(stats.items(), key=lambda kv: kv[1][1])
    # FP64 form: time and agreement of the gradients and of z
    g32 = g.double().cpu().numpy()
    glam32, gom32 = res[1], res[2]
    s64 = mk("fp64")
    lp64 = lp.double()
    zb64 = zb.double()
    g64t = torch.empty_like(lp64)
    s64.set_log_probs(lp64)
    s64.backward(cfg.iters, zb64, every, out=g64t)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s64.set_log_probs(lp64)
    _, glam64, gom64 = s64.backward(cfg.iters, zb64, every, out=g64t)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    g64 = g64t.cpu().numpy()
    scale = max(np.abs(g64).max(), abs(glam64), np.abs(gom64).max())
    grad_err = max(np.abs(g32 - g64).max(), abs(glam32 - glam64), np.abs(gom32 - gom64).max()) / scale
    z32 = s.get_z()
    z64 = s64.get_z()
    s64.close()
    # end to end with host buffers
    lph = torch.tensor(np.log(sc.p), dtype=torch.float32).pin_memory()
    zbh = zb.cpu().pin_memory()
    gh = torch.empty_like(lph).pin_memory()
    e2e = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(lph, zbh, gh)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    e2e_value = whole_job_rate(cfg.iters * len(e2e), world, max_over_ranks(sum(e2e), dev))
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        v, wall, cores = oracle_grad_sample()
        cpu = {"value": v, "unit": "ADMM iter/s", "cores": cores, "kind": "oracle",
               "sample": f"reference gradient (FP64 autograd through the oracle iteration) of a "
                         f"64x64 crop, 50 iterations ({wall:.1f} s), scaled by pixel count",
               **cpu_info()}
    line = {
        "metric": METRIC, "value": value, "unit": "ADMM iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": DIFF_DESC, "H": H, "W": W, "K": K, "iters": cfg.iters,
                   "checkpoint_every": every, "unit_note": "differentiated iterations "
                   "(forward + reverse pass) per second",
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "forward_only_ms": float(np.mean(t_fwd)),
        "gradient_vs_fp64": {"max_abs_error_over_max_entry": grad_err,
                             "max_abs_z_vs_fp64": float(np.abs(z32 - z64).max())},
        "fp64_form_ms_per_step": t64 * 1e3,
        "roofline": {"bound": "hbm", "kernel": "sweep (fused prox + dual + rhs partials)",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_source": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": sweep_bytes,
                     "avg_launch_us": sw_ms / sw_cnt * 1e3},
        "kernel_ms": {k: {"launches": c, "ms": round(m, 4)} for k, (c, m) in stats.items()},
        "kernel_timing": "CUDA events around every launch, eager replay of one step",
        "dominant_kernel": dom[0],
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": "ADMM iter/s", "h2d_bytes_per_step": 2 * 4 * H * W * K,
                "d2h_bytes_per_step": 4 * H * W * K + 8 * 10},
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()


def run_reference_diff(args):
    rates, cores, walls = [], 1, 0.0
    for _ in range(args.warmup):
        oracle_grad_sample()
    for _ in range(args.steps):
        r, wall, cores = oracle_grad_sample()
        rates.append(r)
        walls += wall
    v = float(np.mean(rates))
    sample = ("reference gradient of a 64x64 crop, 50 iterations, per step, scaled to 256x256 "
              "by pixel count")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ADMM iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * walls / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": DIFF_DESC, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "ADMM iter/s", "cores": cores, "kind": "oracle",
                         "sample": sample, **cpu_info()},
        "e2e": {"value": v, "unit": "ADMM iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


DEFAULT_WORKLOAD = "2048x2048"
# short runs of the other workloads appended to the default line (keys kept per workload)
EXTRAS = [("145x145", ["--steps", "5", "--warmup", "3"]),
          ("batch64", ["--steps", "3", "--warmup", "3"]),
          ("mlr610x340", ["--steps", "3", "--warmup", "3"]),
          ("patchsweep", ["--steps", "2", "--warmup", "3"])]
EXTRA_KEYS = ("value", "unit", "ms_per_step", "steps", "warmup", "us_per_iteration_one_solve_alone",
              "gpu_launches", "clocks")


def run_extras():
    """Each other workload in a child process of this script (fresh handles and memory, the
    same GPU), without the CPU baseline and the FP64 check; a compact summary of its line."""
    out = {}
    for name, extra in EXTRAS:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", name, "--skip-cpu",
               "--skip-fp64-check", *extra]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
            ln = [x for x in r.stdout.splitlines() if x.startswith("{")]
            if r.returncode != 0 or not ln:
                out[name] = {"error": (r.stderr.strip().splitlines() or ["no output"])[-1][:200]}
                continue
            d = json.loads(ln[-1])
            rec = {k: d[k] for k in EXTRA_KEYS if k in d}
            rec["workload"] = d.get("config", {}).get("workload")
            if "roofline" in d:
                rec["roofline"] = {k: d["roofline"].get(k) for k in
                                   ("kernel", "achieved", "peak", "unit", "frac")}
            if "e2e" in d:
                rec["e2e"] = d["e2e"]
            if "per_solve" in d:
                rec["per_solve"] = d["per_solve"]
            out[name] = rec
        except Exception as e:  # a failed extra never costs the headline line
            out[name] = {"error": str(e)[:200]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the short runs of the other workloads")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    help="2048x2048 (default), 145x145, 64x64, HxW (K=16 synthetic scene), patchsweep, or "
                         "batch64 (64 uneven images in one batch), mlr610x340 (MLR front end), or diff256 "
                         "(differentiable solver)")
    ap.add_argument("--patch", type=int, default=None,
                    help="HxW workloads: patch radius M (default 1, the 3x3 patch)")
    ap.add_argument("--no-autotune", action="store_true", help="batch64: default tilings")
    ap.add_argument("--tune-iters", type=int, default=4, help="batch64: iterations per trial")
    ap.add_argument("--cpu-iters", type=int, default=4)
    ap.add_argument("--ref-iters", type=int, default=2)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64-check", action="store_true")
    ap.add_argument("--profile-run", action="store_true",
                    help="for runs under a profiler: eager kernel launches (no CUDA-graph "
                         "replay) and the solves of a step one after another")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        if args.workload == "batch64":
            run_batch(args, rank, world, local_rank)
        elif args.workload == "mlr610x340":
            run_mlr(args, rank, world, local_rank)
        elif args.workload == "diff256":
            run_diff(args, rank, world, local_rank)
        else:
            line = run_ours(args, rank, world, local_rank)
            if line is not None:
                if world == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_extras \
                        and not args.profile_run:
                    line["other_workloads"] = run_extras()
                print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
