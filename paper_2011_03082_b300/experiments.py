"""Equal-error comparison of sphere tracing (learned decoders) against brute-force path tracing on the GPU.

For each density (the density-doubling protocol of Fig. 1 and Sec. 5.2, synthetic displaced-sphere scene):

1. a brute-force reference image at ``ref_spp`` samples per pixel;
2. the sphere-traced image at ``st_spp`` and its RMSE against the reference;
3. brute-force images at doubling spp until their RMSE drops below the sphere tracer's; the spp at equal RMSE
   is interpolated with RMSE ~ spp^(-1/2) between the two bracketing runs;
4. time per path of both methods (CUDA events), hence the time each needs for that RMSE and the speed-up.

The sphere tracer is biased (its samplers are learned approximations): when its error is above the brute-force
error of the smallest ladder run, the speed-up is bounded above by that run, and the result says so.

Every study renders with a model set and the request fields it needs (``pipeline.render_set``): by default
``pipeline.RENDER_SET``; pass ``cset`` and ``opts`` to use another.

``python -m paper_2011_03082_b300.experiments [--res 128] [--ref-spp 8192] [--st-spp 256]``, and
``python -m paper_2011_03082_b300.experiments --batched [--scale 0.25]`` for the 64-request batch.

Two further studies:

* ``--absorption``: the absorption experiment of Sec. 5 (Fig. 8).  RGB media with absorption 1 - phi of
  (2e-3, 2e-4, 2e-3), doubled between settings; each colour channel is one request of a three-request batch with
  a shared seed, rendered by sphere tracing and by brute force, timed with CUDA events.
* ``--fallback``: the sphere / brute-force threshold (the minimum optical radius sigma_t r of a sphere step, the
  thin-region fallback of Sec. 6): render time and RMSE against a brute-force reference for several thresholds.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import ms, pipeline, synth


def _model_set(cset, opts):
    """The (cvae_set, request fields) to render with: the default set when ``cset`` is None."""
    if cset is None:
        return pipeline.render_set()
    return cset, dict(opts or {})


def _render(p: dict, cset, variant=0):
    img = torch.zeros(p["width"] * p["height"], dtype=torch.float64, device="cuda")
    st = torch.zeros(ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
    rp = ms.render_params(dict(p, variant=variant))
    ws = ms.workspace(ms.ms_render_workspace_size([rp]))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    ms.ms_render(rp, cset if p["mode"] == ms.MS_SPHERE else None, img, st, ws=ws)
    b.record()
    b.synchronize()
    return img.cpu().numpy() / p["spp"], a.elapsed_time(b) / 1e3


def reference_images(sigmas=(16.0, 32.0, 64.0, 128.0), res=128, ref_spp=8192, variant=0, cset=None) -> dict:
    """Brute-force reference images (seed 101) per density: {sigma_t: per-pixel mean image}."""
    return {s: _render(synth.render_scene(s, width=res, height=res, spp=ref_spp, mode=ms.MS_BRUTE, seed=101), cset,
                       variant)[0] for s in sigmas}


def equal_rmse(sigmas=(16.0, 32.0, 64.0, 128.0), res=128, ref_spp=8192, st_spp=256, cset=None, variant=0, refs=None,
               tau_min=1.0, opts=None, bf_variant=None):
    """``refs``: reference images from ``reference_images`` at the same res and ref_spp (rendered here when None).
    ``tau_min``: the sphere tracer's minimum optical radius (0: the library's per-density default).
    ``variant`` / ``bf_variant``: the renderer variants of the sphere tracer and of brute force (each method's
    own autotuned pick; ``bf_variant`` None: the same as ``variant``)."""
    cset, opts = _model_set(cset, opts)
    bfv = variant if bf_variant is None else bf_variant
    out = []
    for s in sigmas:
        base = dict(synth.render_scene(s, width=res, height=res, spp=ref_spp, mode=ms.MS_BRUTE, seed=101), **opts)
        ref = refs[s] if refs is not None else _render(base, cset, bfv)[0]
        st_img, t_st = _render(dict(base, mode=ms.MS_SPHERE, spp=st_spp, seed=202, min_optical_radius=tau_min),
                               cset, variant)
        rmse_st = float(np.sqrt(np.mean((st_img - ref) ** 2)))
        ladder = []
        spp = 16
        while spp <= ref_spp // 2:
            img, t = _render(dict(base, spp=spp, seed=303 + spp), cset, bfv)
            ladder.append((spp, float(np.sqrt(np.mean((img - ref) ** 2))), t))
            if ladder[-1][1] <= rmse_st:
                break
            spp *= 2
        per_spp_bf = ladder[-1][2] / ladder[-1][0]
        if ladder[0][1] <= rmse_st:
            spp_eq, note = float(ladder[0][0]), "sphere-tracing error above the smallest brute-force run (upper bound)"
        elif ladder[-1][1] > rmse_st:
            spp_eq, note = float(ladder[-1][0]), "brute force did not reach the sphere-tracing error (lower bound)"
        else:
            (s0, e0, _), (s1, e1, _) = ladder[-2], ladder[-1]
            # RMSE = c / sqrt(spp): fit through the bracketing pair (geometric mean of the two estimates)
            spp_eq = float(np.sqrt(s0 * (e0 / rmse_st) ** 2 * s1 * (e1 / rmse_st) ** 2))
            note = "interpolated"
        t_bf = per_spp_bf * spp_eq
        out.append(dict(sigma_t=s, res=res, ref_spp=ref_spp, st_spp=st_spp, tau_min=tau_min, rmse_st=rmse_st,
                        spp_bf_equal=spp_eq, t_st_s=t_st, t_bf_equal_s=t_bf, speedup=t_bf / t_st, note=note,
                        ladder=[dict(spp=a, rmse=b, t_s=c) for a, b, c in ladder]))
    return out


def batched(seed=5, n=64, scale=0.25, repeats=3, cset=None, sequential=True, tune_div=64, opts=None):
    """The heterogeneous batch: ``n`` requests (resolution, spp, density, g, albedo, displacement frequency
    drawn with ``seed``; ``scale`` shrinks resolution and spp) in one persistent launch, the renderer variant
    autotuned on the same requests at 1/``tune_div`` of their spp, captured in a CUDA graph and replayed; reports
    light paths per second, per-request completion p50 / p99 (ns counters written by the kernel when each
    request's last path ends) and, with ``sequential``, the time of the same requests rendered one launch at a
    time."""
    cset, opts = _model_set(cset, opts)
    raw = [dict(r, **opts) for r in synth.batch_requests(seed, n, scale=scale)]
    reqs = [ms.render_params(r) for r in raw]
    npx = sum(r.width * r.height for r in reqs)
    paths = sum(r.width * r.height * r.spp for r in reqs)
    imgs = torch.zeros(npx, dtype=torch.float64, device="cuda")
    st = torch.zeros(n, ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
    ws = ms.workspace(ms.ms_render_workspace_size(reqs))
    tune = [ms.render_params(dict(raw[i], spp=max(1, reqs[i].spp // tune_div))) for i in range(n)]
    variant, _ = ms.ms_render_autotune(tune, cset, imgs, st, ws=ws)
    for r in reqs:
        r.variant = variant
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            imgs.zero_()
            st.zero_()
            ms.ms_render_batch(reqs, cset, imgs, st, ws=ws)
    g.replay()
    torch.cuda.synchronize()
    times = []
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
    done_ms = st[:, 10].double().cpu().numpy() / 1e6
    t = float(np.median(times))
    out = dict(requests=n, scale=scale, paths=paths, seconds=t, paths_per_s=paths / t, variant=variant,
               p50_ms=float(np.percentile(done_ms, 50)), p99_ms=float(np.percentile(done_ms, 99)),
               launch="one persistent ms_render_batch launch, replayed from a CUDA graph (memsets + kernel)")
    if sequential:
        one = torch.zeros(max(r.width * r.height for r in reqs), dtype=torch.float64, device="cuda")
        ost = torch.zeros(ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for r in reqs:
            ms.ms_render(r, cset, one, ost, ws=ws)
        b.record()
        b.synchronize()
        out["sequential_seconds"] = a.elapsed_time(b) / 1e3
    return out


def _render_batch(reqs: list, cset, variant=0):
    reqs = [ms.render_params(dict(r, variant=variant)) for r in reqs]
    npx = sum(r.width * r.height for r in reqs)
    img = torch.zeros(npx, dtype=torch.float64, device="cuda")
    st = torch.zeros(len(reqs), ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
    ws = ms.workspace(ms.ms_render_workspace_size(reqs))
    learned = any(r.mode == ms.MS_SPHERE for r in reqs)
    ms.ms_render_batch(reqs, cset if learned else None, img, st, ws=ws)       # warm-up
    img.zero_()
    st.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    ms.ms_render_batch(reqs, cset if learned else None, img, st, ws=ws)
    b.record()
    b.synchronize()
    return img.cpu().numpy(), st.cpu().numpy(), a.elapsed_time(b) / 1e3


def absorption_sweep(sigma=64.0, res=256, spp=64, settings=6, cset=None, variant=0, opts=None):
    """Render time of both methods against absorption: RGB absorption (2e-3, 2e-4, 2e-3) x 2^i, i < settings."""
    cset, opts = _model_set(cset, opts)
    out = []
    for i in range(settings):
        absorb = [a * 2.0 ** i for a in (2e-3, 2e-4, 2e-3)]
        row = dict(absorption_rgb=absorb)
        for mode, name in ((ms.MS_SPHERE, "sphere"), (ms.MS_BRUTE, "brute")):
            reqs = [dict(synth.render_scene(sigma, width=res, height=res, spp=spp, mode=mode, seed=7, albedo=1.0 - a),
                         **opts) for a in absorb]
            img, st, t = _render_batch(reqs, cset, variant)
            paths = 3 * res * res * spp
            row[name] = dict(seconds=t, paths_per_s=paths / t, mean_rgb=[float(img[k * res * res:(k + 1) * res * res].mean()
                                                                            / spp) for k in range(3)],
                             steps_per_path=float(st[:, 4].sum() + st[:, 3].sum()) / paths)
        row["speedup"] = row["brute"]["seconds"] / row["sphere"]["seconds"]
        out.append(row)
    return out


def fallback_sweep(sigma=64.0, res=128, spp=256, ref_spp=8192, tau_mins=(0.5, 1.0, 2.0, 4.0, 8.0), cset=None,
                   variant=0, ref=None, opts=None, bf_variant=None):
    """Render time and RMSE against a brute-force reference for several minimum optical radii of a sphere step;
    ``ref``: the reference image (rendered here when None).  Each row's ``cost`` = time x RMSE^2, the work
    needed per unit of inverse squared error (lower is better)."""
    cset, opts = _model_set(cset, opts)
    base = dict(synth.render_scene(sigma, width=res, height=res, spp=ref_spp, mode=ms.MS_BRUTE, seed=101), **opts)
    bfv = variant if bf_variant is None else bf_variant
    if ref is None:
        ref, _ = _render(base, cset, bfv)
    out = []
    for tm in tau_mins:
        img, t = _render(dict(base, mode=ms.MS_SPHERE, spp=spp, seed=202, min_optical_radius=tm), cset, variant)
        e = float(np.sqrt(np.mean((img - ref) ** 2)))
        out.append(dict(tau_min=tm, seconds=t, rmse=e, cost=t * e * e))
    bf, t_bf = _render(dict(base, spp=spp, seed=303), cset, bfv)
    e = float(np.sqrt(np.mean((bf - ref) ** 2)))
    out.append(dict(tau_min=None, mode="brute force", seconds=t_bf, rmse=e, cost=t_bf * e * e))
    return out


def time_breakdown(sigmas=(64.0, 128.0), res=512, spp=64, cset=None, opts=None):
    """Where each method's time goes, per density: the instrumented render kernel (phase_timers) reports the
    warps' cycles by round kind (march, decoder, transition, refill) and counts the march steps of shadow rays
    apart from the path's own marches (camera, flight, re-entry).  The march cycles are split between the two in
    proportion to their steps (every march step runs the same loop body).  Counts are per entering path."""
    cset, opts = _model_set(cset, opts)
    out = []
    for s in sigmas:
        for mode, name in ((ms.MS_SPHERE, "sphere tracing"), (ms.MS_BRUTE, "brute force")):
            p = dict(synth.render_scene(s, width=res, height=res, spp=spp, mode=mode, seed=1), **opts)
            rp = ms.render_params(dict(p, phase_timers=1))
            img = torch.zeros(res * res, dtype=torch.float64, device="cuda")
            st = torch.zeros(ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
            ws = ms.workspace(ms.ms_render_workspace_size([rp]))
            ms.ms_render(rp, cset if mode == ms.MS_SPHERE else None, img, st, ws=ws)
            st = st.cpu().numpy().astype(np.float64)
            cyc = st[12:16]
            tot = max(cyc.sum(), 1.0)
            radius = st[3] + st[4] if mode == ms.MS_SPHERE else 0.0
            march_steps = st[8] - radius
            shadow = st[11]
            ent = max(st[1], 1.0)
            share = dict(march_own=cyc[0] / tot * (march_steps - shadow) / max(march_steps, 1.0),
                         march_shadow=cyc[0] / tot * shadow / max(march_steps, 1.0),
                         decoder=cyc[1] / tot, transition=cyc[2] / tot, refill=cyc[3] / tot)
            out.append(dict(sigma_t=s, method=name, res=res, spp=spp, time_share=share,
                            per_entering_path=dict(flights=st[2] / ent, sphere_steps=st[3] / ent,
                                                   brute_events=st[4] / ent, nee=st[7] / ent,
                                                   march_steps_own=(march_steps - shadow) / ent,
                                                   march_steps_shadow=shadow / ent)))
    return out


def fallback_policy(sigmas=(16.0, 32.0, 64.0, 128.0), res=128, spp=256, ref_spp=8192,
                    tau_mins=(0.5, 1.0, 2.0, 4.0, 8.0), cset=None, variant=0, refs=None, opts=None, bf_variant=None):
    """The thin-region threshold per density (Sec. 6): for each density the sweep above, and the minimum optical
    radius with the lowest cost (time x RMSE^2 against the brute-force reference at the same spp); beside it,
    what the library's per-density default (min_optical_radius = 0) picks."""
    cset, opts = _model_set(cset, opts)
    out = []
    for s in sigmas:
        rows = fallback_sweep(s, res, spp, ref_spp, tau_mins, cset, variant, None if refs is None else refs[s],
                              opts=opts, bf_variant=bf_variant)
        best = min((r for r in rows if r["tau_min"] is not None), key=lambda r: r["cost"])
        out.append(dict(sigma_t=s, best_tau_min=best["tau_min"],
                        library_default=float(ms.lib().ms_render_default_min_optical_radius(s)), sweep=rows))
    return out


def autotuned_variants(sigmas, res, spp, cset=None, opts=None):
    """(sphere-tracing variant, brute-force variant): each method's fastest renderer variant on one batch of the
    given densities at res x res px x spp (each method gets its own pick, as in the benchmark)."""
    cset, opts = _model_set(cset, opts)
    picks = []
    for mode in (ms.MS_SPHERE, ms.MS_BRUTE):
        reqs = [ms.render_params(dict(synth.render_scene(s, width=res, height=res, spp=spp, mode=mode), **opts))
                for s in sigmas]
        img = torch.zeros(len(reqs) * res * res, dtype=torch.float64, device="cuda")
        st = torch.zeros(len(reqs), ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
        best, _ = ms.ms_render_autotune(reqs, cset if mode == ms.MS_SPHERE else None, img, st)
        picks.append(best)
    return picks[0], picks[1]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--res", type=int, default=128)
    ap.add_argument("--ref-spp", type=int, default=8192)
    ap.add_argument("--st-spp", type=int, default=256)
    ap.add_argument("--sigmas", default="16,32,64,128", help="densities of the equal-RMSE comparison")
    ap.add_argument("--batched", action="store_true", help="run the 64-request batch instead")
    ap.add_argument("--scale", type=float, default=0.25)
    ap.add_argument("--absorption", action="store_true", help="run the absorption sweep instead")
    ap.add_argument("--fallback", action="store_true", help="run the fallback-threshold sweep instead")
    ap.add_argument("--policy", action="store_true", help="the fallback-threshold sweep at every density")
    ap.add_argument("--models", default=pipeline.RENDER_SET, choices=sorted(pipeline.MODEL_SETS),
                    help="the model set to render with")
    a = ap.parse_args(argv)
    cset, opts = pipeline.render_set(a.models)
    if a.batched:
        print(json.dumps(batched(scale=a.scale, cset=cset, opts=opts)))
        return
    if a.absorption:
        for r in absorption_sweep(cset=cset, opts=opts):
            print(json.dumps(r))
        return
    if a.fallback:
        for r in fallback_sweep(cset=cset, opts=opts):
            print(json.dumps(r))
        return
    if a.policy:
        sigmas = tuple(float(v) for v in a.sigmas.split(","))
        for r in fallback_policy(sigmas=sigmas, res=a.res, ref_spp=a.ref_spp, spp=a.st_spp, cset=cset, opts=opts):
            print(json.dumps(r))
        return
    sigmas = tuple(float(v) for v in a.sigmas.split(","))
    sv, bv = autotuned_variants(sigmas, a.res, max(1, a.st_spp // 16), cset, opts)
    for r in equal_rmse(sigmas=sigmas, res=a.res, ref_spp=a.ref_spp, st_spp=a.st_spp, cset=cset, opts=opts,
                        variant=sv, bf_variant=bv):
        print(json.dumps(dict(r, variant=sv, bf_variant=bv)))


if __name__ == "__main__":
    main()
