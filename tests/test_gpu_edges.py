"""Edge and degenerate cases of the boundary calls on the GPU: empty inputs, caps, a camera that misses the
object, the smallest image, vanishing density and the smallest voxel grid — each against the oracle or an
exact expectation."""
import numpy as np
import pytest
import torch

from paper_2011_03082_b300 import ms, synth

pytestmark = pytest.mark.gpu


def _models():
    return {name: (synth.xavier_decoder(100 + i, *shape), *shape) for i, (name, shape) in
            enumerate(synth.MODEL_SHAPES.items())}


def _gpu(params, models=None):
    img = torch.zeros(params["height"] * params["width"], dtype=torch.float64, device="cuda")
    st = torch.zeros(16, dtype=torch.int64, device="cuda")
    cs = None
    if models is not None:
        cs = ms.cvae_set({k: (torch.from_numpy(w).cuda(), *shape) for k, (w, *shape) in models.items()})
    ms.ms_render(ms.render_params(params), cs, img, st)
    torch.cuda.synchronize()
    return img.cpu().numpy().reshape(params["height"], params["width"]), st.cpu().numpy()


def _oracle(orc, params, models=None):
    decs = None if models is None else [(models[k][0].astype(np.float64), *models[k][1:])
                                        for k in ("length", "path", "event")]
    img, st, _ = orc.render(params, decs)
    return img, st


def test_empty_decoder_and_records_calls_are_no_ops():
    w = torch.from_numpy(synth.xavier_decoder(1, 4, 6)).cuda()
    out = torch.full((1, 6), 7.0, device="cuda")
    ms.ms_cvae_infer(ms.decoder_struct(w, 4, 6), torch.zeros(1, 4, device="cuda"), 0, out_sample=out)
    recs = {k: torch.full((1, d), 7.0, device="cuda") for k, d in
            (("cL", 2), ("xL", 1), ("cP", 3), ("xP", 3), ("cE", 7), ("xE", 6))}
    z1, z3 = torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros(1, 3, device="cuda")
    ms.ms_training_records(0, z1, z3, z3, z3, z3, ms.media_tensor(2.0, 0.5, 0.9), 1, recs)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0) and all(torch.all(v == 7.0) for v in recs.values())


@pytest.mark.parametrize("mode", [0, 1])
def test_segment_cap_truncates_like_the_oracle(orc, mode):
    """max_segments = 2: every path is cut after two flights; the GPU counts the same cut paths and draws the
    same image (paths coincide up to rounding)."""
    models = _models() if mode else None
    p = synth.render_scene(64.0, width=24, height=24, spp=8, mode=mode, seed=4, max_segments=2)
    g, gs = _gpu(p, models)
    o, os_ = _oracle(orc, p, models)
    assert os_[6] > 0
    for k in (0, 1, 2, 6, 7):
        assert abs(int(gs[k]) - int(os_[k])) <= 0.01 * max(int(os_[k]), 50), (k, gs[k], os_[k])
    same = np.abs(g - o) <= 0.02 * np.abs(o) + 1e-9
    assert same.mean() >= 0.98


def test_camera_that_misses_the_object_gives_black():
    p = synth.render_scene(32.0, width=16, height=16, spp=4, mode=0, seed=2)
    p.update(cam_pos=(0.0, 0.0, 3.0), cam_at=(0.0, 0.0, 6.0))       # looking away from the object
    img, st = _gpu(p)
    assert st[0] == 16 * 16 * 4 and st[1] == 0 and st[7] == 0 and np.all(img == 0.0)


@pytest.mark.parametrize("mode", [0, 1])
def test_one_pixel_one_sample(orc, mode):
    models = _models() if mode else None
    p = synth.render_scene(32.0, width=1, height=1, spp=1, mode=mode, seed=9)
    g, gs = _gpu(p, models)
    o, os_ = _oracle(orc, p, models)
    assert gs[0] == os_[0] == 1 and gs[1] == os_[1]
    assert abs(g[0, 0] - o[0, 0]) <= 1e-3 * abs(o[0, 0]) + 1e-9


def test_vanishing_density_matches_the_oracle(orc):
    """sigma_t = 1e-3: almost every path crosses the object without an event; the rare events give the same
    image and counters as the oracle."""
    p = synth.render_scene(1e-3, width=32, height=32, spp=8, mode=0, seed=3)
    g, gs = _gpu(p)
    o, os_ = _oracle(orc, p)
    for k in (0, 1, 2, 4, 7):
        assert gs[k] == os_[k], (k, gs[k], os_[k])
    assert np.allclose(g, o, rtol=1e-3, atol=1e-12)


def test_smallest_voxel_grid_renders_like_the_oracle(orc):
    """n = 4: every voxel is within one diagonal of a voxel that may hold surface, so the grid is all zeros and
    the radii fall back to the distance bound; images and counters are those without a grid."""
    models = _models()
    grid = ms.ms_sdf_grid_build(0.1, 6.0, 4)
    assert torch.all(grid == 0)
    p = synth.render_scene(32.0, width=16, height=16, spp=8, mode=1, seed=5)
    g0, s0 = _gpu(p, models)
    g4, s4 = _gpu(dict(p, sdf_grid_n=4, sdf_grid=grid.data_ptr()), models)
    assert np.array_equal(g0, g4) and np.array_equal(s0[:10], s4[:10])
