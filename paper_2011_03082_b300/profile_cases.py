"""Small, fixed invocations of each kernel for profiling (ncu) and quick timing.

``python -m paper_2011_03082_b300.profile_cases CASE [--repeat R]`` with CASE one of:
  walk      65,536 photons, optical radius 8, g 0.8, albedo 0.999, isotropic start (FP32); walk_sat: 2^24 of them
  walk24    2^24 walks with the training media (FP32, reservoir); walk22: 2^22 of them (ncu captures)
  records   the record transform (ms_training_records) of 2^24 such walks
  decoder   2^22 decoder queries, P_out 6 (FP32, Philox normals); decoder16: the same in FP16 (tensor cores)
  train     one training step of EventGen, batch 65,536
  render    one 128x128 px x 16 spp render at sigma_t 64, sphere tracing with the trained decoders
  brute     the same render in brute-force mode
  render512 / brute512   512x512 px x 64 spp at sigma_t 128 (sphere tracing / brute force)
  render512g             render512 with sphere radii also from a 128^3 voxel grid of conservative distances
  batch128 / batch256 / batch384 / batch512
                         the benchmark's launch (one ms_render_batch of sigma_t 16, 32, 64, 128, trained
                         decoders) at 128^2 .. 512^2 px x 16 spp, with L2 flushed before the launch (256 MB
                         write) as in the benchmark: small cases of the benchmark launch for ncu captures
Each case runs ``--repeat`` times (default 2) and prints the CUDA-event time of the last run.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import build, ms, pipeline, synth


def case_walk(n=65536, reservoir=0, media=None):
    w = synth.walk_cfg()
    if media is None:
        media = ms.media_tensor(w["optical_radius"], w["g"], w["albedo"], w["dir_in"], 1, 0)
    out = ms.walk_outputs(n, per_photon=reservoir > 0)
    ws = ms.workspace(256)
    return lambda: ms.ms_simulate_walks(media, n, out, seed=1, reservoir=reservoir, ws=ws)


def case_walk24(n=1 << 24):
    tau, g, phi = synth.training_media(1, n)
    media = ms.media_tensor(tau.astype(np.float32), g.astype(np.float32), phi.astype(np.float32), (0, 0, 1), 0, 1)
    return case_walk(n, 2, media)


def case_records(n=1 << 24):
    """The record transform of 2^24 training walks (the walks run once, untimed, when the case is built)."""
    tau, g, phi = synth.training_media(1, n)
    media = ms.media_tensor(tau.astype(np.float32), g.astype(np.float32), phi.astype(np.float32), (0, 0, 1), 0, 1)
    out = ms.walk_outputs(n)
    ms.ms_simulate_walks(media, n, out, seed=1, reservoir=2, precision=ms.MS_FP32, max_events=1 << 24)
    recs = {k: torch.empty(n, d, device="cuda") for k, d in
            (("cL", 2), ("xL", 1), ("cP", 3), ("xP", 3), ("cE", 7), ("xE", 6))}
    return lambda: ms.ms_training_records(n, out["n_events"], out["exit_pos"], out["exit_dir"], out["rep_pos"],
                                          out["rep_dir"], media, 1001, recs)


def case_decoder(n=1 << 22, p_out=6, precision=ms.MS_FP32):
    w = torch.from_numpy(synth.xavier_decoder(7, 4, p_out)).cuda()
    c = torch.from_numpy(synth.decoder_queries(7, n)).cuda()
    mlv = torch.empty(n, 2 * p_out, device="cuda")
    smp = torch.empty(n, p_out, device="cuda")
    d = ms.decoder_struct(w, 4, p_out, precision=precision)
    return lambda: ms.ms_cvae_infer(d, c, n, seed=7, out_mean_logvar=mlv, out_sample=smp)


def case_train(B=65536):
    p_in, p_out, latent, width = synth.MODEL_SHAPES["event"]
    shape = ms.cvae_shape(p_in, p_out, latent, width)
    p = torch.from_numpy(synth.xavier_cvae(1, p_in, p_out, latent, width)).cuda()
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    g = torch.Generator().manual_seed(0)
    x = torch.randn(B, p_out, generator=g).cuda()
    c = torch.randn(B, p_in, generator=g).cuda()
    ws = ms.workspace(ms.ms_cvae_workspace_size(shape, B))
    loss3 = torch.zeros(3, device="cuda")
    return lambda: ms.ms_cvae_train_step(shape, p, m, v, x, c, B, step=1, loss3=loss3, ws=ws)


def case_render(mode=ms.MS_SPHERE, res=128, spp=16, sigma=64.0, grid_n=0):
    """One render with the benchmark's model set; the returned callable exposes the per-request counters as
    ``.stats``."""
    cset, opts = pipeline.render_set()
    scene = dict(synth.render_scene(sigma, width=res, height=res, spp=spp, mode=mode), **opts)
    grid = None
    if grid_n:
        grid = ms.ms_sdf_grid_build(scene["disp_amp"], scene["disp_freq"], grid_n)
        scene.update(sdf_grid_n=grid_n, sdf_grid=grid.data_ptr())
    p = ms.render_params(scene)
    img = torch.zeros(res * res, dtype=torch.float64, device="cuda")
    st = torch.zeros(ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
    ws = ms.workspace(ms.ms_render_workspace_size([p]))

    def run():
        st.zero_()
        ms.ms_render(p, cset if mode == ms.MS_SPHERE else None, img, st, ws=ws)
    run.stats = st
    run.grid = grid          # keeps the grid alive with the case
    return run


def case_batch(res, spp=16, sigmas=(16.0, 32.0, 64.0, 128.0)):
    """The benchmark's four-density batch (and model set) at a reduced size, default renderer variant."""
    cset, opts = pipeline.render_set()
    reqs = [ms.render_params(dict(synth.render_scene(s, width=res, height=res, spp=spp, mode=ms.MS_SPHERE), **opts))
            for s in sigmas]
    img = torch.zeros(len(reqs) * res * res, dtype=torch.float64, device="cuda")
    st = torch.zeros(len(reqs), ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
    ws = ms.workspace(ms.ms_render_workspace_size(reqs))

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def run():
        img.zero_()
        st.zero_()
        flush.fill_(1)
        ms.ms_render_batch(reqs, cset, img, st, ws=ws)
    run.stats = st
    return run


CASES = {"records": case_records, "walk": case_walk, "walk_sat": lambda: case_walk(1 << 24), "walk24": case_walk24, "walk22": lambda: case_walk24(1 << 22), "decoder": case_decoder, "train": case_train,
         "decoder16": lambda: case_decoder(precision=ms.MS_FP16),
         "render": case_render, "brute": lambda: case_render(ms.MS_BRUTE),
         "render512": lambda: case_render(ms.MS_SPHERE, 512, 64, 128.0),
         "render512g": lambda: case_render(ms.MS_SPHERE, 512, 64, 128.0, grid_n=128),
         "brute512": lambda: case_render(ms.MS_BRUTE, 512, 64, 128.0),
         "batch128": lambda: case_batch(128), "batch256": lambda: case_batch(256),
         "batch384": lambda: case_batch(384), "batch512": lambda: case_batch(512)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--repeat", type=int, default=2)
    a = ap.parse_args(argv)
    build.build()
    fn = CASES[a.case]()
    ms_ = None
    for _ in range(a.repeat):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        e.synchronize()
        ms_ = s.elapsed_time(e)
    out = {"case": a.case, "ms": ms_}
    if hasattr(fn, "stats"):
        out["stats"] = fn.stats.cpu().tolist()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
