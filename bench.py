"""Benchmark: light paths per second of the learned sphere tracer (CVAE decoders + NEE) on one B300.

Workload (one step): the displaced-sphere object 0.1 sin(6x) sin(6y) sin(6z) lit by a point light, rendered at
512 x 512 pixels with 256 samples per pixel at the four densities sigma_t in {16, 32, 64, 128} (density
doubling, g = 0.8, albedo 0.999), with the three decoders trained by ``paper_2011_03082_b300.pipeline`` —
the four images in one persistent ``ms_render_batch`` launch.  ``value`` counts camera paths (light paths)
per second over all ranks.  The brute-force tracer is timed on the same workload for context.

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
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
METRIC = "light paths/s: CVAE sphere-trace vs brute-force GPU walk at equal RMSE; % roofline"
UNIT = "light paths/s"
SIGMAS = (16.0, 32.0, 64.0, 128.0)
WORKLOAD = ("render of the displaced sphere 0.1 sin(6x)sin(6y)sin(6z), point light, 512x512 px, 256 spp, "
            "sigma_t {16,32,64,128}, g 0.8, albedo 0.999, CVAE sphere tracing + NEE (trained decoders)")

# Algorithmic work per counted unit of the renderer's roofline: special-function (MUFU) operations per march
# step (f and its derivative along the ray: sqrt + 3 sin/cos pairs), per sphere-radius evaluation at a
# collision (f alone: sqrt + 3 sin), per sphere step (the three decoders' 2 x width Softplus each, as exp +
# log; 10 posterior exps; 11 Box-Muller pairs x 4; 3 logs) and per brute-force event (log, sin/cos, rsqrt,
# divide).
MUFU_PER_MARCH = 7
MUFU_PER_RADIUS = 4
MUFU_PER_SPHERE = sum(2 * shape[3] * 2 for shape in (
    (2, 1, 2, 8), (3, 3, 5, 16), (7, 6, 5, 16))) + 10 + 11 * 4 + 3      # Table 1 decoder shapes: 217
MUFU_PER_EVENT = 5
MUFU_PER_NEE = 4


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


def recorded_traffic(variant: dict):
    """DRAM bytes per launch of the render kernel from the committed one-pass ncu captures of the benchmark
    launch (one per kernel variant), or None when the kernel sources changed since or the selected variant was
    not captured."""
    import hashlib
    rec = json.loads((ROOT / "paper_2011_03082_b300" / "measured_traffic.json").read_text())["render_kernel"]
    h = hashlib.sha256()
    for f in rec["sources"]:
        h.update((ROOT / f).read_bytes())
    if h.hexdigest() != rec["sha256"]:
        return None
    key = "{decode_batch},{trans_batch},{steps},{min_blocks}".format(**variant)
    v = rec["dram_bytes_per_launch"].get(key)
    return None if v is None else float(v)


# --------------------------------------------------------------------------------------------- CPU oracle

def oracle_paths_per_second(models_np, budget_s: float, sigmas=SIGMAS, mode=1):
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
            _, st, threads = oracle.render(synth.render_scene(s, width=side, height=side, spp=spp, mode=mode), decs)
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
    models = pipeline.load()
    dec = {k: pipeline.decoder_part(k, models[k]["params"]) for k in pipeline.MODELS}
    # each step is a bounded sample; the budget keeps the whole run within a few minutes
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_paths_per_second(dec, budget * 0.25)
    vals, samples, cores = [], [], 0
    for _ in range(args.steps):
        r = oracle_paths_per_second(dec, budget)
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
    ap.add_argument("--variant", type=int, default=None, help="renderer variant to use instead of autotuning")
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
    models = pipeline.load()
    dm = pipeline.device_decoders(models, dev)
    cset = ms.cvae_set(dm)

    W = H = args.width
    spp = args.spp
    reqs = [synth.render_scene(s, width=W, height=H, spp=spp, mode=ms.MS_SPHERE, seed=1,
                               sample_offset=rank * spp) for s in SIGMAS]
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

    # autotune the renderer's scheduling variant on a reduced sample of the same requests (untimed), unless a
    # variant is given
    if args.variant is None:
        tune_reqs = [ms.render_params(dict(r, spp=max(1, spp // 16))) for r in reqs]
        variant, variant_ms = ms.ms_render_autotune(tune_reqs, cset, images, stats, repeats=1, ws=ws)
    else:
        variant, variant_ms = args.variant, []
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
    out_dir = ROOT / "gpurun_out"
    out_dir.mkdir(exist_ok=True)
    with ClockSampler(local, out_dir / f"bench_clocks_rank{rank}.csv") as clk:
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
    st = stats_acc.sum(dim=0).cpu().numpy().astype(np.float64)
    per_req = (stats_acc.cpu().numpy() / args.steps).astype(np.int64).tolist()

    # ---------------- roofline of the render kernel (special-function pipe) ----------------
    peaks = measured_peaks()
    clocks = clk.summary()
    sm_mhz_max = float(peaks.get("sm_max_mhz", 2032.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mufu_peak = n_sm * 16 * sm_mhz_max * 1e6 / 1e12              # Tops/s at the maximum SM clock
    # every collision of a sphere-tracing request evaluates f once for the sphere's radius (counted in st[8])
    radius_evals = st[3] + st[4]
    mufu_ops = ((st[8] - radius_evals) * MUFU_PER_MARCH + radius_evals * MUFU_PER_RADIUS + st[3] * MUFU_PER_SPHERE
                + st[4] * MUFU_PER_EVENT + st[7] * MUFU_PER_NEE + st[2] * 2)
    achieved = mufu_ops / (t_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": mufu_peak, "unit": "Tops/s (MUFU)",
                "frac": achieved / mufu_peak, "traffic": recorded_traffic(ms.ms_render_variant_info(variant)),
                "traffic_unit": "DRAM bytes per launch (committed ncu capture; null if the kernel changed)",
                "kernel": "render_kernel",
                "peak_source": f"{n_sm} SMs x 16 MUFU ops/clk x {sm_mhz_max:.0f} MHz (recipe unit counts, max clock)"}

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
        breqs = [ms.render_params(dict(r, mode=ms.MS_BRUTE, variant=variant)) for r in reqs]
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

    # ---------------- equal-RMSE comparison with brute force (context; after the timed region) ----------------
    equal = None
    if rank == 0 and not args.no_equal_rmse:
        from paper_2011_03082_b300 import experiments
        rows = experiments.equal_rmse(res=128, ref_spp=8192, st_spp=256, cset=cset, variant=variant)
        equal = {"res": 128, "ref_spp": 8192, "st_spp": 256,
                 "per_sigma": [{k: r[k] for k in ("sigma_t", "rmse_st", "spp_bf_equal", "t_st_s", "t_bf_equal_s",
                                                  "speedup", "note")} for r in rows]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        dec_np = {k: pipeline.decoder_part(k, models[k]["params"]) for k in pipeline.MODELS}
        cpu = oracle_paths_per_second(dec_np, args.cpu_budget)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "width": W, "height": H, "spp": spp, "sigma_t": list(SIGMAS),
                           "g": 0.8, "albedo": 0.999, "mode": "sphere", "launch": "one ms_render_batch per step",
                           "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if world > 1
                           else "single GPU", "stats_per_request": per_req,
                           "kernel_variant": dict(index=variant, **ms.ms_render_variant_info(variant)),
                           "autotune_ms": [round(t, 2) for t in variant_ms]},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
                "clocks": clocks, "brute_force": brute, "equal_rmse": equal, "step_ms": step_ms}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
