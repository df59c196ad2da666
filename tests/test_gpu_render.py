"""GPU parity of ms_render / ms_render_batch against the oracle renderer (Sec. 3, 4.1, 4.3, Eq. 5).

The GPU renders in single precision on the same Philox stream as the FP64 oracle, so paths coincide except
where a decision taken in floating point flips: the sphere / brute-force choice at sigma_t r = tau_min, the
rounding of N, or which side of the EPS band a march stops on.  A flipped path is another sample of the same
distribution, and with the untrained test decoders (NEE weights Lambda up to ~1e3) one flipped path can
dominate a pixel, so the acceptance counts flips instead of letting one move the image RMSE.  With oracle
images O1 (seed 1) and O2 (seed 2) and the GPU image G2 (seed 2):
  * paths coincide: at least 99% of pixels agree with O2 to 2 sigma_t (1 + A k) EPS relative (a march may
    stop anywhere in the band |f| < (1 + A k) EPS, which moves a shadow ray's transmittance by up to about
    sigma_t (1 + A k) EPS relative, 1% at sigma_t = 64);
  * on those pixels, |RMSE(G2, O1) / RMSE(O2, O1) - 1| <= 0.01;
  * a pixel with a flipped path differs from O1 by no more than O2 differs from O1 anywhere;
  * the path counters agree within 1%."""
import numpy as np
import pytest
import torch

from paper_2011_03082_b300 import ms, synth

pytestmark = pytest.mark.gpu


def _models():
    out = {}
    for i, (name, shape) in enumerate(synth.MODEL_SHAPES.items()):
        out[name] = (synth.xavier_decoder(100 + i, *shape), *shape)
    return out


def gpu_render(params, models=None):
    img = torch.zeros(params["height"], params["width"], dtype=torch.float64, device="cuda")
    st = torch.zeros(16, dtype=torch.int64, device="cuda")
    cs = None
    keep = []
    if models is not None:
        dm = {}
        for k, (w, *shape) in models.items():
            t = torch.from_numpy(w).cuda()
            keep.append(t)
            dm[k] = (t, *shape)
        cs = ms.cvae_set(dm)
    ms.ms_render(ms.render_params(params), cs, img, st)
    torch.cuda.synchronize()
    return img.cpu().numpy(), st.cpu().numpy()


def oracle_render(orc, params, models=None):
    decs = None
    if models is not None:
        decs = [(models[k][0].astype(np.float64), *models[k][1:]) for k in ("length", "path", "event")]
    img, st, _ = orc.render(params, decs)
    return img, st


def rmse(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)))


CASES = [("brute_16", 16.0, 0), ("brute_64", 64.0, 0), ("sphere_64", 64.0, 1), ("sphere_16", 16.0, 1)]


@pytest.mark.parametrize("name,sigma,mode", CASES, ids=[c[0] for c in CASES])
def test_render_matches_oracle(orc, name, sigma, mode):
    models = _models() if mode == 1 else None
    p1 = synth.render_scene(sigma, width=32, height=32, spp=16, mode=mode, seed=1)
    p2 = dict(p1, seed=2)
    o1, _ = oracle_render(orc, p1, models)
    o2, s2 = oracle_render(orc, p2, models)
    g2, gs = gpu_render(p2, models)
    tol = 2.0 * sigma * (1.0 + p1["disp_amp"] * p1["disp_freq"]) * 1e-4
    same = np.abs(g2 - o2) <= tol * np.abs(o2) + 1e-9
    assert same.mean() >= 0.99, same.mean()
    noise = rmse(o2[same], o1[same])
    assert noise > 0
    assert abs(rmse(g2[same], o1[same]) / noise - 1.0) <= 0.01, (rmse(g2[same], o1[same]), noise)
    assert np.all(np.abs(g2 - o1)[~same] <= np.abs(o2 - o1).max())
    assert gs[0] == s2[0] == 32 * 32 * 16 and gs[15] == 0
    assert abs(int(gs[1]) - int(s2[1])) <= 0.002 * s2[1]
    for k in (2, 3, 4, 7, 8, 9):
        assert abs(int(gs[k]) - int(s2[k])) <= 0.01 * max(s2[k], 100), (k, gs[k], s2[k])


def test_zero_albedo_is_black():
    img, st = gpu_render(synth.render_scene(16.0, width=16, height=16, spp=4, mode=0, albedo=0.0))
    assert st[4] > 0 and np.all(img == 0.0)


def test_sample_offsets_and_batches_compose():
    models = _models()
    full = synth.render_scene(32.0, width=24, height=16, spp=8, mode=1, seed=3)
    a, sa = gpu_render(full, models)
    h1, s1 = gpu_render(dict(full, spp=4), models)
    h2, s2 = gpu_render(dict(full, spp=4, sample_offset=4), models)
    assert np.allclose(a, h1 + h2, rtol=1e-6, atol=1e-12) and np.array_equal(sa[:10], (s1 + s2)[:10])
    # three requests in one persistent launch equal the three single renders
    reqs = [full, synth.render_scene(8.0, width=8, height=8, spp=3, mode=0, seed=4),
            synth.render_scene(128.0, width=5, height=7, spp=2, mode=1, seed=5, disp_freq=3.0)]
    singles = [gpu_render(r, models) for r in reqs]
    npx = sum(r["width"] * r["height"] for r in reqs)
    imgs = torch.zeros(npx, dtype=torch.float64, device="cuda")
    st = torch.zeros(len(reqs), 16, dtype=torch.int64, device="cuda")
    dm = {k: (torch.from_numpy(w).cuda(), *shape) for k, (w, *shape) in models.items()}
    ms.ms_render_batch([ms.render_params(r) for r in reqs], ms.cvae_set(dm), imgs, st)
    torch.cuda.synchronize()
    off = 0
    for i, (r, (img, s)) in enumerate(zip(reqs, singles)):
        n = r["width"] * r["height"]
        assert np.allclose(imgs[off:off + n].cpu().numpy(), img.ravel(), rtol=1e-6, atol=1e-12)
        assert np.array_equal(st[i].cpu().numpy()[:10], s[:10])
        off += n


def test_full_size_render_properties():
    """512 x 512 pixels, 256 samples per pixel, sigma_t 64, sphere tracing with decoders."""
    p = synth.render_scene(64.0, mode=1)
    img, st = gpu_render(p, _models())
    assert st[0] == 512 * 512 * 256
    assert np.all(np.isfinite(img)) and np.all(img >= 0) and img.sum() > 0
    assert st[3] > 0 and st[7] <= st[3] + st[4] and st[15] == 0


def test_bad_requests_are_rejected():
    img = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = torch.zeros(16, dtype=torch.int64, device="cuda")
    for bad in (dict(sigma_t=0.0), dict(g=1.0), dict(albedo=1.5), dict(width=0), dict(mode=5)):
        p = dict(synth.render_scene(8.0, width=2, height=2, spp=1, mode=0), **bad)
        with pytest.raises(ms.MsError):
            ms.ms_render(ms.render_params(p), None, img, st)
    with pytest.raises(ms.MsError, match="decoders"):
        ms.ms_render(ms.render_params(synth.render_scene(8.0, width=2, height=2, spp=1, mode=1)), None, img, st)


def test_kernel_variants_agree_and_autotune():
    """Every scheduling variant traces the same paths (same counters, images equal up to the order of the
    per-pixel additions); the autotuner returns one of them."""
    models = _models()
    p = synth.render_scene(64.0, width=32, height=32, spp=8, mode=1, seed=9)
    ref_img, ref_st = None, None
    for v in range(ms.lib().ms_render_variants()):
        img, st = gpu_render(dict(p, variant=v), models)
        if ref_img is None:
            ref_img, ref_st = img, st
        assert np.array_equal(st[:10], ref_st[:10]), v
        assert np.allclose(img, ref_img, rtol=1e-6, atol=1e-12), v
    dm = {k: (torch.from_numpy(w).cuda(), *shape) for k, (w, *shape) in models.items()}
    imgs = torch.zeros(32 * 32, dtype=torch.float64, device="cuda")
    st = torch.zeros(ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
    best, times = ms.ms_render_autotune([ms.render_params(p)], ms.cvae_set(dm), imgs, st)
    assert 0 <= best < len(times) and min(times) == times[best] and all(t > 0 for t in times)
    with pytest.raises(ms.MsError, match="variant"):
        gpu_render(dict(p, variant=99), models)


def test_batch_in_a_cuda_graph_matches_direct_launch():
    """The batched renderer (a memset and one persistent kernel) captured in a CUDA graph and replayed gives
    the direct launch's images and counters; every request reports a completion time."""
    models = _models()
    reqs = [ms.render_params(r) for r in synth.batch_requests(5, 6, scale=1 / 32)]
    npx = sum(r.width * r.height for r in reqs)
    dm = {k: (torch.from_numpy(w).cuda(), *shape) for k, (w, *shape) in models.items()}
    cset = ms.cvae_set(dm)
    ws = ms.workspace(ms.ms_render_workspace_size(reqs))
    direct = torch.zeros(npx, dtype=torch.float64, device="cuda")
    dst = torch.zeros(len(reqs), 16, dtype=torch.int64, device="cuda")
    ms.ms_render_batch(reqs, cset, direct, dst, ws=ws)
    torch.cuda.synchronize()
    imgs = torch.zeros(npx, dtype=torch.float64, device="cuda")
    st = torch.zeros(len(reqs), 16, dtype=torch.int64, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g):
            imgs.zero_()
            st.zero_()
            ms.ms_render_batch(reqs, cset, imgs, st, ws=ws)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert np.allclose(imgs.cpu().numpy(), direct.cpu().numpy(), rtol=1e-6, atol=1e-12)
    assert np.array_equal(st.cpu().numpy()[:, :10], dst.cpu().numpy()[:, :10])
    assert np.all(st.cpu().numpy()[:, 10] > 0)


@pytest.mark.parametrize("A,k,n", [(0.1, 6.0, 64), (0.15, 10.0, 48)])
def test_sdf_grid_matches_oracle(orc, A, k, n):
    """The voxel grid of conservative distances: the GPU's (single-precision marking, integer distance
    transform) equals the oracle's, except in the rare voxels whose marking test is decided by rounding."""
    g = ms.ms_sdf_grid_build(A, k, n).cpu().numpy().astype(np.float64)
    ref, _, h = orc.sdf_grid(A, k, n)
    same = np.abs(g - ref) <= 1e-5 * (1.0 + ref)
    assert same.mean() >= 0.999, same.mean()
    assert np.abs(g - ref).max() <= 2.0 * h


def test_render_with_sdf_grid_matches_oracle(orc):
    """Sphere radii from the larger of the distance bound and the voxel grid: the image and counters agree with
    the oracle's (same acceptance as without the grid), and the larger spheres take fewer sphere steps."""
    models = _models()
    n = 64
    grid = ms.ms_sdf_grid_build(0.1, 6.0, n)
    p1 = synth.render_scene(64.0, width=32, height=32, spp=16, mode=1, seed=1)
    p2 = dict(p1, seed=2)
    og = dict(sdf_grid_n=n)
    o1, _ = oracle_render(orc, dict(p1, **og), models)
    o2, s2 = oracle_render(orc, dict(p2, **og), models)
    g2, gs = gpu_render(dict(p2, sdf_grid_n=n, sdf_grid=grid.data_ptr()), models)
    _, gs_plain = gpu_render(p2, models)
    tol = 2.0 * 64.0 * (1.0 + 0.6) * 1e-4
    same = np.abs(g2 - o2) <= tol * np.abs(o2) + 1e-9
    assert same.mean() >= 0.99, same.mean()
    noise = rmse(o2[same], o1[same])
    assert abs(rmse(g2[same], o1[same]) / noise - 1.0) <= 0.01
    for kk in (2, 3, 4, 7):
        assert abs(int(gs[kk]) - int(s2[kk])) <= 0.01 * max(s2[kk], 100), (kk, gs[kk], s2[kk])
    assert gs[3] + gs[4] < gs_plain[3] + gs_plain[4]     # fewer sphere steps plus events per path


def test_full_size_batch_sampled_pixels_match_oracle(orc):
    """The benchmark's launch at full size: one ms_render_batch of the four densities (sigma_t 16, 32, 64, 128),
    512 x 512 px x 256 spp each, sphere tracing with the default kernel variant, here with the synthetic
    decoders (the oracle takes no GPU-trained weights).  The oracle renders 16 sampled pixels per density one by
    one on the same streams (O2), and again on another sample range (O1, sample offset 256) for its own spread.
    With 256 paths per pixel a pixel holds a flipped path (see the module docstring) more often than at 16 spp,
    so: at least 95% of the sampled pixels coincide with O2 to 2 sigma_t (1 + A k) EPS relative (measured: all
    64, within 4e-5 relative), and every other pixel differs from O2 by no more than O1 differs from O2 on the
    sampled set; the batch's path counts are exact."""
    models = _models()
    sig = (16.0, 32.0, 64.0, 128.0)
    reqs = [synth.render_scene(s, mode=1, seed=1) for s in sig]
    W, H, spp = reqs[0]["width"], reqs[0]["height"], reqs[0]["spp"]
    assert (W, H, spp) == (512, 512, 256)
    dm, keep = {}, []
    for k, (w, *shape) in models.items():
        t = torch.from_numpy(w).cuda()
        keep.append(t)
        dm[k] = (t, *shape)
    cs = ms.cvae_set(dm)
    preqs = [ms.render_params(r) for r in reqs]
    images = torch.zeros(len(reqs) * W * H, dtype=torch.float64, device="cuda")
    stats = torch.zeros(len(reqs), 16, dtype=torch.int64, device="cuda")
    ms.ms_render_batch(preqs, cs, images, stats)
    torch.cuda.synchronize()
    g_all = images.cpu().numpy().reshape(len(reqs), H * W)
    st = stats.cpu().numpy()
    assert np.all(st[:, 0] == W * H * spp) and np.all(st[:, 15] == 0)
    decs = [(models[k][0].astype(np.float64), *models[k][1:]) for k in ("length", "path", "event")]
    rng = np.random.default_rng(42)
    coincide, total = 0, 0
    for i, (s, r) in enumerate(zip(sig, reqs)):
        px = rng.integers(128, 384, 16)
        py = rng.integers(128, 384, 16)
        pix = py * W + px
        o2, _ = orc.render_pixels(r, pix, decs)
        o1, _ = orc.render_pixels(dict(r, sample_offset=spp), pix, decs)
        g = g_all[i, pix]
        tol = 2.0 * s * (1.0 + r["disp_amp"] * r["disp_freq"]) * 1e-4
        same = np.abs(g - o2) <= tol * np.abs(o2) + 1e-9
        spread = np.abs(o1 - o2).max()
        assert np.all(np.abs(g - o2)[~same] <= spread), (s, np.abs(g - o2)[~same], spread)
        coincide += int(same.sum())
        total += pix.size
    assert coincide >= 0.95 * total, (coincide, total)


@pytest.mark.parametrize("mode", [0, 1])
def test_phase_timers_instrumentation_traces_the_same_paths(mode):
    """The instrumented kernel (phase_timers) traces the same paths as the timed one (same counters, image equal up
    to the order of the per-pixel additions), counts shadow-ray march steps (stats[11], fewer than all march
    steps) and reports positive warp cycles for the round kinds that ran (stats[12..15])."""
    models = _models() if mode == 1 else None
    p = synth.render_scene(64.0, width=24, height=24, spp=8, mode=mode, seed=6)
    img, st = gpu_render(p, models)
    img_t, st_t = gpu_render(dict(p, phase_timers=1), models)
    assert np.array_equal(st[:10], st_t[:10]) and np.all(st[11:] == 0)
    assert np.allclose(img, img_t, rtol=1e-6, atol=1e-12)
    assert 0 < st_t[11] < st_t[8]
    assert st_t[12] > 0 and st_t[14] > 0 and st_t[15] > 0
    assert (st_t[13] > 0) == (mode == 1)
