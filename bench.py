"""Benchmark: light paths per second of the learned sphere tracer (CVAE decoders + NEE) on one B300.

Workload (one step): the displaced-sphere object 0.1 sin(6x) sin(6y) sin(6z) lit by a point light, rendered at
512 x 512 pixels with 256 samples per pixel at the four densities sigma_t in {16, 32, 64, 128} (density
doubling, g = 0.8, albedo 0.999), with the three decoders trained by ``paper_2011_03082_b300.pipeline`` —
the four images in one persistent ``ms_render_batch`` launch.  The decoders are the model set
``pipeline.RENDER_SET`` (trained for the exact N = 1 step and centre event; ``--models paper`` for the set in the
paper's form).  ``value`` counts camera paths (light paths)
per second over all ranks.  The brute-force tracer is timed on the same workload for context, with its own
autotuned kernel variant.

``python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]``; under torchrun every rank renders
its own samples (sample offset = rank * spp): weak scaling, no collective on the data path.
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
METRIC = "light paths/s: CVAE sphere-trace vs brute-force GPU walk at equal RMSE; % roofline"
UNIT = "light paths/s"
SIGMAS = (16.0, 32.0, 64.0, 128.0)
WORKLOAD = ("render of the displaced sphere 0.1 sin(6x)sin(6y)sin(6z), point light, 512x512 px, 256 spp, "
            "sigma_t {16,32,64,128}, g 0.8, albedo 0.999, CVAE sphere tracing + NEE (trained decoders)")

# Algorithmic work per counted unit of the renderer's roofline: special-function (MUFU) operations, split into
# 2^x (which issues at twice the rate of the unit's other functions on this GPU) and the others (log2, sin, cos,
# reciprocal square root, reciprocal), as (ex2, other):
#   march step: f and its derivative along the ray, sqrt + 3 sin/cos pairs               (0, 7)
#   sphere radius at a collision: f alone, sqrt + 3 sin                                   (0, 4)
#   sphere step: the Table 1 decoders' Softplus (2 x width per decoder: 80 units, exp + log each), the 10
#     posterior standard deviations exp(log Sigma / 2), N = exp(y), phi^N; 11 Box-Muller pairs (log, sqrt,
#     sin, cos), log tau and log N, the rotation angle's sin/cos                          (92, 128)
#   brute-force event: HG cosine (reciprocal), the scattering rotation (sin, cos, sqrt, rsqrt)  (0, 5)
#   next-event estimate: the segment's length and direction (sqrt, reciprocal), rho_g (rsqrt, reciprocal),
#     transmittance exp(-sigma_t d), 1 / d^2                                              (1, 5)
#   flight: -log(1 - u) / sigma_t                                                         (0, 2)
MUFU_MARCH = (0, 7)
MUFU_RADIUS = (0, 4)
MUFU_SPHERE = (2 * (8 + 16 + 16) + 10 + 1 + 1, 2 * (8 + 16 + 16) + 11 * 4 + 2 + 2)
MUFU_EVENT = (0, 5)
MUFU_NEE = (1, 5)
MUFU_FLIGHT = (0, 2)


def nproc():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: Path):
        self.path = path
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path.exists():
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.path.read_text().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {}


def recorded_traffic(pixels: int):
    """DRAM bytes of one render launch of ``pixels`` image pixels, from the committed ncu capture of a smaller
    launch of the same four-density batch (one launch, 16 spp, ``profiles/``): the traffic is the images' reads
    and write-backs plus a few register spills, so it follows the pixels, not the paths.  Captured with the
    default kernel variant; the variants differ only in scheduling constants.  None when the kernel's sources
    changed since the capture."""
    import hashlib
    rec = json.loads((ROOT / "paper_2011_03082_b300" / "measured_traffic.json").read_text())["render_kernel"]
    h = hashlib.sha256()
    for f in rec["sources"]:
        h.update((ROOT / f).read_bytes())
    if h.hexdigest() != rec["sha256"]:
        return None
    return float(rec["bytes_per_pixel"]) * pixels


# --------------------------------------------------------------------------------------------- CPU oracle

def oracle_paths_per_second(models_np, budget_s: float, sigmas=SIGMAS, mode=1, opts=None):
    """Time the oracle renderer (as it stands) on a bounded sample of the workload: every density, a square
    image and spp sized so that the whole sample takes about ``budget_s`` seconds on all host cores."""
    import oracle
    from paper_2011_03082_b300 import synth
    decs = [(models_np[k].astype(np.float64), *synth.MODEL_SHAPES[k]) for k in ("length", "path", "event")]
    side = 64

    def sample(spp):
        paths, threads = 0, 0
        t0 = time.perf_counter()
        for s in sigmas:
            _, st, threads = oracle.render(dict(synth.render_scene(s, width=side, height=side, spp=spp, mode=mode),
                                                **(opts or {})), decs)
            paths += int(st[0])
        return paths, time.perf_counter() - t0, threads

    # grow the sample (same image, more samples per pixel) until one run fills at least half the budget;
    # the last run is the one reported
    spp = 1
    while True:
        paths, dt, threads = sample(spp)
        if dt >= 0.5 * budget_s or spp >= 1 << 16:
            break
        spp = int(min(max(2 * spp, spp * 0.9 * budget_s / max(dt, 1e-3)), 1 << 16))
    return dict(value=paths / dt, unit=UNIT, cores=int(threads), kind="oracle",
                sample=f"{side}x{side} px x {spp} spp at each sigma_t in {list(sigmas)} "
                       f"({'sphere tracing' if mode else 'brute force'} + NEE, same scene and decoders), "
                       f"{paths} paths in {dt:.1f} s")


def run_reference(args):
    """--impl reference: the CPU oracle timed as the reference arm, on the same config and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2011_03082_b300 import pipeline
    models = pipeline.load_set(args.models or pipeline.RENDER_SET)
    opts = pipeline.render_options(models)
    dec = {k: pipeline.decoder_part(k, models[k]["params"]) for k in pipeline.MODELS}
    # each step is a bounded sample; the budget keeps the whole run within a few minutes
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_paths_per_second(dec, budget * 0.25, opts=opts)
    vals, samples, cores = [], [], 0
    for _ in range(args.steps):
        r = oracle_paths_per_second(dec, budget, opts=opts)
        vals.append(r["value"])
        samples.append(r["sample"])
        cores = r["cores"]
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "note": "CPU oracle (FP64, all host cores) on a bounded sample"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": samples[-1]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------------------- GPU arm

def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--width", type=int, default=512)
    ap.add_argument("--spp", type=int, default=256)
    ap.add_argument("--no-brute", action="store_true", help="skip the brute-force context measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-equal-rmse", action="store_true", help="skip the equal-RMSE comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-request batch")
    ap.add_argument("--eq-res", type=int, default=512, help="image side of the equal-RMSE comparison")
    ap.add_argument("--eq-ref-spp", type=int, default=16384, help="spp of its brute-force reference")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="resolution and spp scale of the 64 requests")
    ap.add_argument("--variant", type=int, default=None, help="renderer variant to use instead of autotuning")
    ap.add_argument("--models", default=None, help="model set (paper_2011_03082_b300.pipeline.MODEL_SETS); "
                                                   "pipeline.RENDER_SET when not given")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2011_03082_b300 import build, ms, pipeline, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    set_name = args.models or pipeline.RENDER_SET
    models = pipeline.load_set(set_name)
    opts = pipeline.render_options(models)
    dm = pipeline.device_decoders(models, dev)
    cset = ms.cvae_set(dm)

    W = H = args.width
    spp = args.spp
    reqs = [dict(synth.render_scene(s, width=W, height=H, spp=spp, mode=ms.MS_SPHERE, seed=1,
                                    sample_offset=rank * spp), **opts) for s in SIGMAS]
    preqs = [ms.render_params(r) for r in reqs]
    npx = W * H * len(reqs)
    images = torch.zeros(npx, dtype=torch.float64, device=dev)
    stats = torch.zeros(len(reqs), ms.MS_RENDER_STATS if hasattr(ms, "MS_RENDER_STATS") else 16, dtype=torch.int64,
                        device=dev)
    ws = ms.workspace(ms.ms_render_workspace_size(preqs), dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2
    stream = torch.cuda.current_stream(dev)

    def one_step(p, images, stats):
        ms.ms_render_batch(p, cset, images, stats, ws=ws)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # measured issue rates of the ALU units (the roofline's denominators), with the SM clock while they ran
    clock_dir = tempfile.mkdtemp(prefix="ms_bench_clocks_")
    with ClockSampler(local, Path(clock_dir) / f"peaks_rank{rank}.csv") as pclk:
        time.sleep(1.5)             # let the sampler start
        alu = ms.ms_alu_peaks(dev)
        alu = ms.ms_alu_peaks(dev)  # the second pass, with the clocks settled, is the one kept
    alu_clocks = pclk.summary()

    # autotune the renderer's scheduling variant on a reduced sample of the same requests (untimed), unless a
    # variant is given
    # (brute force, the comparison method, gets its own pick on the same sample)
    if args.variant is None:
        tune_reqs = [ms.render_params(dict(r, spp=max(1, spp // 16))) for r in reqs]
        variant, variant_ms = ms.ms_render_autotune(tune_reqs, cset, images, stats, repeats=1, ws=ws)
        tune_bf = [ms.render_params(dict(r, spp=max(1, spp // 16), mode=ms.MS_BRUTE)) for r in reqs]
        bf_variant, bf_variant_ms = ms.ms_render_autotune(tune_bf, None, images, stats, repeats=1, ws=ws)
    else:
        variant, variant_ms = args.variant, []
        bf_variant, bf_variant_ms = args.variant, []
    for r in preqs:
        r.variant = variant
    for _ in range(args.warmup):
        images.zero_()
        stats.zero_()
        one_step(preqs, images, stats)
    barrier()

    # ---------------- timed region: K steps, L2 flushed between steps ----------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats_acc = torch.zeros_like(stats)
    with ClockSampler(local, Path(clock_dir) / f"clocks_rank{rank}.csv") as clk:
        barrier()
        for k in range(args.steps):
            images.zero_()
            stats.zero_()
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            one_step(preqs, images, stats)
            ev[k][1].record(stream)
            stats_acc += stats
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    img_fp32 = images.clone()        # the last timed step's images (FP32 decoders), for the precision form below
    t_ms = float(np.sum(step_ms))
    paths_rank = float(stats_acc[:, 0].sum().item())
    t_max = t_ms
    paths_all = paths_rank
    if world > 1:
        tt = torch.tensor([t_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
        pp = torch.tensor([paths_rank], device=dev, dtype=torch.float64)
        dist.all_reduce(pp)
        paths_all = float(pp.item())
    value = paths_all / (t_max / 1e3)
    # light paths that enter the medium (the rest miss the object and cost one march)
    entering = float(stats_acc[:, 1].sum().item()) * world / (t_max / 1e3)
    st = stats_acc.sum(dim=0).cpu().numpy().astype(np.float64)
    per_req = (stats_acc.cpu().numpy() / args.steps).astype(np.int64).tolist()

    # ---------------- roofline of the render kernel (special-function pipe) ----------------
    peaks = measured_peaks()
    clocks = clk.summary()
    sm_mhz_max = float(peaks.get("sm_max_mhz", 2032.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # every collision of a sphere-tracing request evaluates f once for the sphere's radius (counted in st[8])
    radius_evals = st[3] + st[4]
    units = ((st[8] - radius_evals, MUFU_MARCH), (radius_evals, MUFU_RADIUS), (st[3], MUFU_SPHERE),
             (st[4], MUFU_EVENT), (st[7], MUFU_NEE), (st[2], MUFU_FLIGHT))
    ex2_ops = sum(n * c[0] for n, c in units)
    other_ops = sum(n * c[1] for n, c in units)
    # the special-function unit's shortest time for this mix at the measured rates, hence its effective peak
    t_min = ex2_ops / alu["ex2"] + other_ops / min(alu["lg2"], alu["sin"], alu["rsqrt"])
    mufu_ops = ex2_ops + other_ops
    mufu_peak = mufu_ops / t_min / 1e12
    achieved = mufu_ops / (t_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": mufu_peak, "unit": "Tops/s (MUFU)",
                "frac": achieved / mufu_peak, "traffic": recorded_traffic(W * H * len(reqs)),
                "traffic_unit": "DRAM bytes per launch (ncu capture of a smaller launch scaled by pixels; null if the "
                                "kernel changed)",
                "kernel": "render_kernel",
                "peak_source": "measured (ms_alu_peaks, of measured): the special-function unit's rate for this "
                               f"kernel's mix of {ex2_ops:.3e} 2^x and {other_ops:.3e} other operations per step "
                               "(2^x at its own measured rate, the rest at that of log2 / sin / rsqrt); SM clock "
                               f"{alu_clocks.get('sm_mhz')} MHz while measured",
                "mufu_ops_per_step": {"ex2": ex2_ops / args.steps, "other": other_ops / args.steps},
                "alu_peaks_tops": {k: v / 1e12 for k, v in alu.items()}}

    # ---------------- end to end through the C ABI with host buffers ----------------
    host_w = {k: (torch.from_numpy(pipeline.decoder_part(k, models[k]["params"])).pin_memory(), *synth.MODEL_SHAPES[k])
              for k in pipeline.MODELS}
    dev_w = {k: (torch.empty_like(v[0], device=dev), *v[1:]) for k, v in host_w.items()}
    cset_e2e = ms.cvae_set(dev_w)
    host_img = torch.empty(npx, dtype=torch.float64).pin_memory()
    host_stats = torch.empty_like(stats, device="cpu").pin_memory()
    h2d = sum(v[0].numel() * 4 for v in host_w.values())
    d2h = host_img.numel() * 8 + host_stats.numel() * 8
    e2e_ms = []
    for k in range(max(1, args.steps // 2)):
        images.zero_()
        stats.zero_()
        flush.fill_(k & 0xFF)
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for name in pipeline.MODELS:
            dev_w[name][0].copy_(host_w[name][0], non_blocking=True)
        ms.ms_render_batch(preqs, cset_e2e, images, stats, ws=ws)
        host_img.copy_(images, non_blocking=True)
        host_stats.copy_(stats, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_paths = float(host_stats[:, 0].sum().item()) * world
    e2e_t = float(np.mean(e2e_ms))
    if world > 1:
        tt = torch.tensor([e2e_t], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = float(tt.item())
    e2e = {"value": e2e_paths / (e2e_t / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    # ---------------- brute force on the same workload (context: paths/s at equal spp) ----------------
    brute = None
    if not args.no_brute:
        breqs = [ms.render_params(dict(r, mode=ms.MS_BRUTE, variant=bf_variant)) for r in reqs]
        images.zero_()
        stats.zero_()
        ms.ms_render_batch(breqs, None, images, stats, ws=ws)   # warm-up
        barrier()
        images.zero_()
        stats.zero_()
        flush.fill_(7)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ms.ms_render_batch(breqs, None, images, stats, ws=ws)
        b.record(stream)
        b.synchronize()
        bt = a.elapsed_time(b)
        bpaths = float(stats[:, 0].sum().item())
        brute = {"paths_per_s": bpaths / (bt / 1e3), "ms_per_step": bt,
                 "speedup_equal_spp": (bpaths / (bt / 1e3)) and value / world / (bpaths / (bt / 1e3)),
                 "events_per_path": float(stats[:, 4].sum().item()) / max(1.0, float(stats[:, 1].sum().item()))}

    # ---------------- the precision form: the same step with FP16 and BF16 decoders (context) ----------------
    precision = {}
    for name, code in (("fp16", ms.MS_FP16), ("bf16", ms.MS_BF16)):
        cs_h = ms.cvae_set(dm, precision=code)
        images.zero_()
        stats.zero_()
        ms.ms_render_batch(preqs, cs_h, images, stats, ws=ws)      # warm-up
        images.zero_()
        stats.zero_()
        flush.fill_(9)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ms.ms_render_batch(preqs, cs_h, images, stats, ws=ws)
        b.record(stream)
        b.synchronize()
        th = a.elapsed_time(b)
        d = (images - img_fp32).double()
        precision[name] = {"paths_per_s": float(stats[:, 0].sum().item()) / (th / 1e3), "ms_per_step": th,
                           "image_rmse_vs_fp32_decoders": float(torch.sqrt(torch.mean(d * d)).item()) / spp,
                           "image_rms": float(torch.sqrt(torch.mean(img_fp32.double() ** 2)).item()) / spp}

    # ---------------- equal-RMSE comparison with brute force and the fallback policy (after the timed region) --
    equal = policy = batch = breakdown = None
    if rank == 0 and world == 1 and not args.no_equal_rmse:
        from paper_2011_03082_b300 import experiments
        refs = experiments.reference_images(SIGMAS, args.eq_res, args.eq_ref_spp, bf_variant, cset)
        rows = experiments.equal_rmse(SIGMAS, res=args.eq_res, ref_spp=args.eq_ref_spp, st_spp=spp, cset=cset,
                                      variant=variant, refs=refs, tau_min=1.0, opts=opts, bf_variant=bf_variant)
        # the library's per-density threshold (min_optical_radius 0); when it is 1 at every density the rows
        # above are already its rows
        policy_tau = [float(ms.lib().ms_render_default_min_optical_radius(s)) for s in SIGMAS]
        rows_auto = rows if all(t == 1.0 for t in policy_tau) else experiments.equal_rmse(
            SIGMAS, res=args.eq_res, ref_spp=args.eq_ref_spp, st_spp=spp, cset=cset, variant=variant, refs=refs,
            tau_min=0.0, opts=opts, bf_variant=bf_variant)
        keys = ("sigma_t", "tau_min", "rmse_st", "spp_bf_equal", "t_st_s", "t_bf_equal_s", "speedup", "note")
        equal = {"res": args.eq_res, "ref_spp": args.eq_ref_spp, "st_spp": spp,
                 "per_sigma": [{k: r[k] for k in keys} for r in rows],
                 "per_sigma_default_policy": [dict({k: r[k] for k in keys},
                                                   tau_min_used=float(
                                                       ms.lib().ms_render_default_min_optical_radius(r["sigma_t"])))
                                              for r in rows_auto]}
        pol = experiments.fallback_policy(SIGMAS, res=args.eq_res, spp=spp, ref_spp=args.eq_ref_spp, cset=cset,
                                          variant=variant, refs=refs, opts=opts, bf_variant=bf_variant)
        policy = [{"sigma_t": r["sigma_t"], "best_tau_min": r["best_tau_min"],
                   "library_default": r["library_default"],
                   "sweep": [{k: v for k, v in x.items() if k != "mode"} for x in r["sweep"]]} for r in pol]
        del refs
        breakdown = experiments.time_breakdown((64.0, 128.0), res=W, spp=64, cset=cset, opts=opts)
    if rank == 0 and world == 1 and not args.no_batched:
        from paper_2011_03082_b300 import experiments
        b = experiments.batched(seed=5, n=64, scale=args.batch_scale, repeats=1, cset=cset, sequential=False,
                                opts=opts)
        batch = {k: b[k] for k in ("requests", "scale", "paths", "seconds", "paths_per_s", "variant", "p50_ms",
                                   "p99_ms", "launch")}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        dec_np = {k: pipeline.decoder_part(k, models[k]["params"]) for k in pipeline.MODELS}
        cpu = oracle_paths_per_second(dec_np, args.cpu_budget, opts=opts)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "width": W, "height": H, "spp": spp, "sigma_t": list(SIGMAS),
                           "g": 0.8, "albedo": 0.999, "mode": "sphere", "launch": "one ms_render_batch per step",
                           "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if world > 1
                           else "single GPU", "stats_per_request": per_req,
                           "kernel_variant": dict(index=variant, **ms.ms_render_variant_info(variant)),
                           "autotune_ms": [round(t, 2) for t in variant_ms],
                           "brute_force_variant": dict(index=bf_variant, **ms.ms_render_variant_info(bf_variant)),
                           "brute_force_autotune_ms": [round(t, 2) for t in bf_variant_ms]},
                "model_set": {"name": set_name, "file": "paper_2011_03082_b300/weights/" + pipeline.MODEL_SETS[set_name],
                              "render_options": opts},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
                "clocks": clocks, "entering_paths_per_s": entering, "brute_force": brute,
                "decoder_precision": precision, "equal_rmse": equal, "time_breakdown": breakdown,
                "fallback_policy": policy, "batched_64": batch, "step_ms": step_ms}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
