"""GPU parity of the renderer against the oracle where the method branches, with the trained decoders.

The trained LengthGen, PathGen and EventGen (``weights/cvae_set.npz``, Table 1 shapes) give the sphere steps
their realistic N and Lambda, unlike the untrained decoders of test_gpu_render.py.  Cases:
  * densities 16 and 64 with the benchmark scene (g 0.8, albedo 0.999);
  * albedo 1 (the Lambda = N branch, no absorption);
  * g -0.7 (backward scattering), 0 and 5e-5 (the isotropic branch of the HG sampler, |g| < 1e-4);
  * densities 256 and 512, and a sphere radius capped by the largest optical radius (tau_max 16 at sigma_t 64);
  * a heterogeneous batch shaped like the 64-request workload (resolution, spp, density, g, albedo and
    displacement frequency drawn per request), checked per request at sampled pixels;
  * the exact N = 1 step and centre event (exact_n1, exact_centre; alone and together) with the set trained
    for them (``weights/cvae_set_atoms.npz``).
Acceptance (oracle images O1 with seed 1 and O2 with seed 2, GPU image G2 with seed 2) — the single-precision
GPU path follows the FP64 oracle's paths except where a floating-point decision flips, which gives another
sample of the same distribution:
  * at least 98% of pixels coincide with O2 to 2 sigma_t (1 + A k) EPS relative (the march's boundary band);
  * whole image: |RMSE(G2, O1) / RMSE(O2, O1) - 1| <= 0.01 (image RMSE within 1% of the oracle's own noise);
  * path counters within 1%.
"""
import numpy as np
import pytest
import torch

from oracle import cvae
from paper_2011_03082_b300 import ms, pipeline, synth

pytestmark = pytest.mark.gpu

EPS = 1e-4


@pytest.fixture(scope="module")
def trained():
    models = pipeline.load()
    dec = {k: pipeline.decoder_part(k, models[k]["params"]) for k in pipeline.MODELS}
    dev = {k: (torch.from_numpy(dec[k]).cuda(), *synth.MODEL_SHAPES[k]) for k in pipeline.MODELS}
    return dict(np=dec, cset=ms.cvae_set(dev), models=models)


def _oracle_decs(t):
    return [(t["np"][k].astype(np.float64), *synth.MODEL_SHAPES[k]) for k in pipeline.MODELS]


def gpu_render(params, cset):
    img = torch.zeros(params["height"] * params["width"], dtype=torch.float64, device="cuda")
    st = torch.zeros(16, dtype=torch.int64, device="cuda")
    ms.ms_render(ms.render_params(params), cset if params["mode"] == 1 else None, img, st)
    torch.cuda.synchronize()
    return img.cpu().numpy().reshape(params["height"], params["width"]), st.cpu().numpy()


def rmse(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)))


CASES = {
    "sigma16": dict(sigma_t=16.0),
    "sigma64": dict(sigma_t=64.0),
    "albedo1_sigma64": dict(sigma_t=64.0, albedo=1.0),
    "g_neg0.7_sigma32": dict(sigma_t=32.0, g=-0.7),
    "g0_sigma32": dict(sigma_t=32.0, g=0.0),
    "g5e-5_sigma32": dict(sigma_t=32.0, g=5e-5),
    "sigma256": dict(sigma_t=256.0),
    "sigma512": dict(sigma_t=512.0),
    "taumax16_sigma64": dict(sigma_t=64.0, max_optical_radius=16.0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_trained_render_matches_oracle(trained, orc, case):
    over = CASES[case]
    p1 = dict(synth.render_scene(over["sigma_t"], width=32, height=32, spp=16, mode=1, seed=1),
              **{k: v for k, v in over.items() if k != "sigma_t"})
    p2 = dict(p1, seed=2)
    decs = _oracle_decs(trained)
    o1, _, _ = orc.render(p1, decs)
    o2, s2, _ = orc.render(p2, decs)
    g2, gs = gpu_render(p2, trained["cset"])
    sigma = p1["sigma_t"]
    tol = 2.0 * sigma * (1.0 + p1["disp_amp"] * p1["disp_freq"]) * EPS
    same = np.abs(g2 - o2) <= tol * np.abs(o2) + 1e-9
    assert same.mean() >= 0.98, same.mean()
    noise = rmse(o2, o1)
    assert noise > 0
    assert abs(rmse(g2, o1) / noise - 1.0) <= 0.01, (rmse(g2, o1), noise)
    assert gs[0] == s2[0] == 32 * 32 * 16 and gs[15] == 0
    assert gs[3] > 0, "no sphere step"
    for k in (1, 2, 3, 4, 5, 7):
        assert abs(int(gs[k]) - int(s2[k])) <= 0.01 * max(s2[k], 100), (k, gs[k], s2[k])


def test_trained_heterogeneous_batch_matches_oracle_per_request(trained, orc):
    """A batch shaped like the 64-request workload (seed 5; resolutions and spp scaled by 1/16; densities
    log-uniform in [8, 1024], g U[0.5, 0.95], albedo U[0.95, 1], displacement frequency U[2, 10]) in one
    persistent launch; the oracle renders 4 sampled pixels of every request on the same streams.  At least 95%
    of the sampled pixels coincide to the renderer's tolerance, and every other one differs from the oracle by
    no more than the oracle's own seed-to-seed spread over that request's sampled pixels."""
    reqs = synth.batch_requests(5, 64, scale=1 / 16)
    preqs = [ms.render_params(r) for r in reqs]
    npx = sum(r["width"] * r["height"] for r in reqs)
    images = torch.zeros(npx, dtype=torch.float64, device="cuda")
    stats = torch.zeros(len(reqs), 16, dtype=torch.int64, device="cuda")
    ms.ms_render_batch(preqs, trained["cset"], images, stats)
    torch.cuda.synchronize()
    img = images.cpu().numpy()
    st = stats.cpu().numpy()
    decs = _oracle_decs(trained)
    rng = np.random.default_rng(8)
    off, coincide, total = 0, 0, 0
    for i, r in enumerate(reqs):
        W, H, spp = r["width"], r["height"], r["spp"]
        assert st[i, 0] == W * H * spp
        pix = rng.integers(0, W * H, 4)
        o2, os2 = orc.render_pixels(r, pix, decs)
        o1, _ = orc.render_pixels(dict(r, seed=r["seed"] + 1), pix, decs)
        g = img[off + pix]
        tol = 2.0 * r["sigma_t"] * (1.0 + r["disp_amp"] * r["disp_freq"]) * EPS
        same = np.abs(g - o2) <= tol * np.abs(o2) + 1e-9
        spread = np.abs(o1 - o2).max()
        assert np.all(np.abs(g - o2)[~same] <= spread), (i, r["sigma_t"], g, o2, o1)
        coincide += int(same.sum())
        total += pix.size
        off += W * H
    assert coincide >= 0.95 * total, (coincide, total)


def test_eventgen_gradient_at_the_training_batch_matches_oracle():
    """EventGen (Table 1: p_in 7, p_out 6, latent 5, width 16) at the training batch of 65,536 samples (512 blocks
    of partials): loss terms and gradient against the FP64 oracle, kernel-drawn normals."""
    p_in, p_out, latent, width = synth.MODEL_SHAPES["event"]
    B = 65536
    rng = np.random.default_rng(12)
    p = (synth.xavier_cvae(12, p_in, p_out, latent, width) + 0.05 * rng.standard_normal(
        pipeline._n_params("event"))).astype(np.float32)
    x = rng.standard_normal((B, p_out)).astype(np.float32)
    c = rng.standard_normal((B, p_in)).astype(np.float32)
    e = rng.standard_normal((B, latent)).astype(np.float32)
    shape = ms.cvae_shape(p_in, p_out, latent, width)
    grad = torch.zeros(p.size, device="cuda")
    loss3 = torch.zeros(3, device="cuda")
    ms.ms_cvae_forward_backward(shape, torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda(),
                                torch.from_numpy(c).cuda(), B, eps_z=torch.from_numpy(e).cuda(), grad=grad,
                                loss3=loss3)
    torch.cuda.synchronize()
    loss, rec, kl, g = cvae.neg_elbo_grad(p.astype(np.float64), cvae.Shape(p_in, p_out, latent, width), x, c, e)
    assert np.allclose(loss3.cpu().numpy(), [loss, rec, kl], rtol=1e-4, atol=1e-5)
    gg = grad.cpu().numpy()
    assert np.abs(gg - g).max() <= 1e-4 * np.abs(g).max(), np.abs(gg - g).max() / np.abs(g).max()


def _round_matrices(w, shape, half):
    """The packed decoder weights with the three weight matrices rounded to FP16 or BF16 (nearest even) and the
    biases kept: the weights the renderer's half-precision decoders multiply with (FP32 accumulation, biases
    added in FP32)."""
    p_in, p_out, latent, width = shape
    k = p_in + latent
    sizes = [width * k, width, width * width, width, 2 * p_out * width, 2 * p_out]
    out, off = [], 0
    for i, n in enumerate(sizes):
        part = np.asarray(w[off:off + n], np.float32)
        if i % 2 == 0:
            part = part.astype(np.float16).astype(np.float32) if half == "fp16" else \
                cvae.round_bf16(part.astype(np.float64)).astype(np.float32)
        out.append(part)
        off += n
    assert off == len(w)
    return np.concatenate(out)


@pytest.mark.parametrize("half", ["fp16", "bf16"])
def test_half_precision_decoders_render_matches_oracle(trained, orc, half):
    """The precision form on the hot path: the renderer with FP16 or BF16 decoders (weights rounded once,
    activations carried as two halves, FP32 accumulation) against the FP64 oracle evaluating the same rounded
    weight matrices, with the same acceptance as the FP32 decoders (sigma_t 64, trained decoders)."""
    prec = ms.MS_FP16 if half == "fp16" else ms.MS_BF16
    rounded = {k: _round_matrices(trained["np"][k], synth.MODEL_SHAPES[k], half) for k in pipeline.MODELS}
    dev = {k: (torch.from_numpy(trained["np"][k]).cuda(), *synth.MODEL_SHAPES[k]) for k in pipeline.MODELS}
    cset = ms.cvae_set(dev, precision=prec)
    decs = [(rounded[k].astype(np.float64), *synth.MODEL_SHAPES[k]) for k in pipeline.MODELS]
    p1 = synth.render_scene(64.0, width=32, height=32, spp=16, mode=1, seed=1)
    p2 = dict(p1, seed=2)
    o1, _, _ = orc.render(p1, decs)
    o2, s2, _ = orc.render(p2, decs)
    g2, gs = gpu_render(p2, cset)
    tol = 2.0 * 64.0 * (1.0 + p1["disp_amp"] * p1["disp_freq"]) * EPS
    same = np.abs(g2 - o2) <= tol * np.abs(o2) + 1e-9
    assert same.mean() >= 0.98, same.mean()
    noise = rmse(o2, o1)
    assert abs(rmse(g2, o1) / noise - 1.0) <= 0.01, (rmse(g2, o1), noise)
    for k in (1, 2, 3, 4, 5, 7):
        assert abs(int(gs[k]) - int(s2[k])) <= 0.01 * max(s2[k], 100), (k, gs[k], s2[k])
    # the rounding's own effect, against the FP32 decoders on the same streams (reported, not bounded)
    g32, _ = gpu_render(p2, trained["cset"])
    print(f"{half}: rmse vs FP32-decoder image {rmse(g2, g32):.3e}, seed-to-seed noise {noise:.3e}")


def test_renderer_rejects_mixed_or_unknown_decoder_precision(trained):
    dev = {k: (torch.from_numpy(trained["np"][k]).cuda(), *synth.MODEL_SHAPES[k]) for k in pipeline.MODELS}
    cs = ms.cvae_set(dev, precision=ms.MS_FP16)
    cs.path.precision = ms.MS_FP32
    p = synth.render_scene(32.0, width=4, height=4, spp=1, mode=1)
    with pytest.raises(ms.MsError, match="share one precision"):
        gpu_render(p, cs)
    cs.path.precision = ms.MS_FP64
    with pytest.raises(ms.MsError, match="precision"):
        gpu_render(p, cs)


@pytest.fixture(scope="module")
def atoms():
    models = pipeline.load_set("atoms")
    dec = {k: pipeline.decoder_part(k, models[k]["params"]) for k in pipeline.MODELS}
    cs = ms.cvae_set({k: (torch.from_numpy(dec[k]).cuda(), *synth.MODEL_SHAPES[k]) for k in pipeline.MODELS})
    return dict(models=models, cset=cs, decs=[(dec[k].astype(np.float64), *synth.MODEL_SHAPES[k])
                                              for k in pipeline.MODELS])


def test_atoms_set_needs_its_options(atoms):
    assert pipeline.render_options(atoms["models"]) == dict(exact_n1=1, exact_centre=1)


@pytest.mark.parametrize("exact_n1,exact_centre", [(1, 1), (1, 0), (0, 1)])
def test_exact_atoms_render_matches_oracle(orc, atoms, exact_n1, exact_centre):
    """The exact N = 1 step (exact_n1: N = 1 with probability exp(-tau), then the exit along the centre event's
    HG direction, alpha = beta = 0, and the centre as the representative event) and the exact centre event
    (exact_centre: the first event with probability phi / Lambda), each alone and together: the renderer against
    the oracle with the same rules and the same decoders (the set trained for both), same acceptance as the other
    trained cases (sigma_t 16 and 64)."""
    opt = dict(exact_n1=exact_n1, exact_centre=exact_centre)
    for sigma in (16.0, 64.0):
        p1 = dict(synth.render_scene(sigma, width=32, height=32, spp=16, mode=1, seed=1), **opt)
        p2 = dict(p1, seed=2)
        o1, _, _ = orc.render(p1, atoms["decs"])
        o2, s2, _ = orc.render(p2, atoms["decs"])
        g2, gs = gpu_render(p2, atoms["cset"])
        tol = 2.0 * sigma * (1.0 + p1["disp_amp"] * p1["disp_freq"]) * EPS
        same = np.abs(g2 - o2) <= tol * np.abs(o2) + 1e-9
        assert same.mean() >= 0.98, (sigma, same.mean())
        noise = rmse(o2, o1)
        assert abs(rmse(g2, o1) / noise - 1.0) <= 0.01, (sigma, rmse(g2, o1), noise)
        for k in (1, 2, 3, 4, 5, 7):
            assert abs(int(gs[k]) - int(s2[k])) <= 0.01 * max(s2[k], 100), (sigma, k, gs[k], s2[k])
