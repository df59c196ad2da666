"""What the trained networks gain over the same method without training (Sec. 5.3, Sec. 5.1).

* Distributions (the evaluation grid of Sec. 5.3: sigma_t in {1, 4, 20, 100}, g in {-0.7, 0, 0.4, 0.9},
  albedo 1, 10,000 paths from the centre of the unit sphere with incoming direction (0,0,1)): the two-sample
  KS statistic between decoder samples and oracle walks, for N (LengthGen) and for cos theta, alpha and beta
  given the walk's N (PathGen; the paper's Figs. 9-10 show the same four quantities), compared between the
  trained and the untrained (Glorot) weights.
* Rendering: a sphere-traced image with the trained decoders is much closer to a brute-force reference than
  the same render with untrained decoders; and with the set trained for the exact N = 1 step and centre event
  (both drawn exactly) the image mean matches brute force, where the paper-form set is several percent dark.
The absolute KS values are reported, not bounded: the paper prints no numbers for them (figures only)."""
import numpy as np
import pytest
import torch
from scipy import stats

from oracle import cvae
from paper_2011_03082_b300 import ms, pipeline, synth

pytestmark = pytest.mark.gpu

SIGMAS = (1.0, 4.0, 20.0, 100.0)
GS = (-0.7, 0.0, 0.4, 0.9)
N_SAMPLES = 10000


def _decoders(trained: bool):
    if trained:
        m = pipeline.load()
        return {k: pipeline.decoder_part(k, m[k]["params"]) for k in pipeline.MODELS}
    return {k: synth.xavier_decoder(500 + i, *synth.MODEL_SHAPES[k]) for i, k in enumerate(pipeline.MODELS)}


def _sample(wdec, name, cond, seed):
    p_in, p_out, latent, width = synth.MODEL_SHAPES[name]
    n = cond.shape[0]
    w = torch.from_numpy(wdec[name]).cuda()
    c = torch.from_numpy(np.ascontiguousarray(cond, np.float32)).cuda()
    out = torch.zeros(n, p_out, device="cuda")
    ms.ms_cvae_infer(ms.decoder_struct(w, p_in, p_out, latent, width), c, n, seed=seed, out_sample=out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def ground_truth(orc):
    gt = {}
    for s in SIGMAS:
        for g in GS:
            r = orc.walk(int(1000 * s + 10 * g) + 1, N_SAMPLES,
                         dict(optical_radius=s, g=float(np.float32(g)), albedo=1.0, dir_in=(0.0, 0.0, 1.0),
                              isotropic_start=0, first_event_at_origin=1))
            n = r["n_events"].size
            zero = np.zeros((n, 3))
            tg = cvae.training_targets(r["n_events"], r["exit_pos"], r["exit_dir"], zero, zero, np.full(n, s),
                                       np.full(n, g), np.ones(n), np.full(n, 0.5))
            gt[(s, g)] = (r["n_events"].astype(np.float64), tg["xP"][:, 0], tg["xP"][:, 1], tg["xP"][:, 2])
    return gt


def _ks_table(wdec, gt):
    out = {}
    for (s, g), (N, ct, al, be) in gt.items():
        cond = np.stack([np.full(N_SAMPLES, np.log(s)), np.full(N_SAMPLES, g)], 1)
        y = _sample(wdec, "length", cond, seed=11)[:, 0]
        Ns = np.maximum(1.0, np.floor(np.exp(np.minimum(y, 30.0)) + 0.5))
        condp = np.stack([cond[:, 0], cond[:, 1], np.log(N)], 1)
        pth = _sample(wdec, "path", condp, seed=12)
        ctp = np.clip(pth[:, 0], -1, 1)
        # (alpha, beta) as the renderer uses them: rescaled to unit length when longer
        ab = pth[:, 1:3] / np.maximum(1.0, np.sqrt((pth[:, 1:3] ** 2).sum(axis=1)))[:, None]
        out[(s, g)] = (stats.ks_2samp(np.log(Ns), np.log(N)).statistic, stats.ks_2samp(ctp, ct).statistic,
                       stats.ks_2samp(ab[:, 0], al).statistic, stats.ks_2samp(ab[:, 1], be).statistic)
    return out


def test_trained_decoders_beat_untrained_on_the_evaluation_grid(ground_truth, capsys):
    """Trained PathGen beats the untrained decoder everywhere on the grid; trained LengthGen beats it at every
    optical radius >= 4 and on the grid mean.  At optical radius 1 most photons leave after the event at the
    centre (N = 1): LengthGen's posterior collapses (KL ~ 0.05), so its decoder is one Gaussian in the
    dequantised ln N per condition and cannot form that spike; there its KS(N) is only required below 0.45
    (0.23-0.39 measured; the untrained decoder is near 0.35 by chance, and a broken model reaches 0.8-1)."""
    trained = _ks_table(_decoders(True), ground_truth)
    untrained = _ks_table(_decoders(False), ground_truth)
    with capsys.disabled():
        print("\nsigma_t  g    KS trained/untrained: N | cos theta given N | alpha given N | beta given N")
        for k in sorted(trained):
            print(f"{k[0]:6.0f} {k[1]:4.1f}   " + "   ".join(f"{trained[k][j]:.3f} / {untrained[k][j]:.3f}"
                                                          for j in range(4)))
    for k in trained:
        assert trained[k][1] < untrained[k][1], k
        if k[0] >= 4:
            assert trained[k][0] < untrained[k][0], k
        else:
            assert trained[k][0] < 0.45, k
    assert np.mean([v[0] for v in trained.values()]) < np.mean([v[0] for v in untrained.values()])
    for j in (2, 3):    # alpha and beta: better than untrained on the grid mean
        assert np.mean([v[j] for v in trained.values()]) < np.mean([v[j] for v in untrained.values()]), j


def test_trained_sphere_tracing_is_close_to_brute_force():
    """32 x 32 px at sigma_t 32: brute-force reference at 4,096 spp; sphere tracing at 512 spp with trained and
    with untrained decoders.  The trained image's error is far below the untrained one's."""
    def render(mode, spp, wdec=None, seed=1):
        p = synth.render_scene(32.0, width=32, height=32, spp=spp, mode=mode, seed=seed)
        img = torch.zeros(32 * 32, dtype=torch.float64, device="cuda")
        st = torch.zeros(ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
        cs = None
        if wdec is not None:
            cs = ms.cvae_set({k: (torch.from_numpy(wdec[k]).cuda(), *synth.MODEL_SHAPES[k]) for k in pipeline.MODELS})
        ms.ms_render(ms.render_params(p), cs, img, st)
        torch.cuda.synchronize()
        return img.cpu().numpy() / spp

    ref = render(ms.MS_BRUTE, 4096, seed=7)
    tr = render(ms.MS_SPHERE, 512, _decoders(True), seed=8)
    un = render(ms.MS_SPHERE, 512, _decoders(False), seed=8)
    e_tr = float(np.sqrt(np.mean((tr - ref) ** 2)))
    e_un = float(np.sqrt(np.mean((un - ref) ** 2)))
    assert e_tr < 0.5 * e_un, (e_tr, e_un)


@pytest.mark.parametrize("sigma", [64.0, 128.0])
def test_exact_point_masses_remove_the_learned_bias(sigma):
    """The model set trained for the exact N = 1 step and centre event, rendered with both drawn exactly, against
    the paper-form set (every model trained on every record): image mean over 128 x 128 px at 1,024 spp against
    a 4,096-spp brute-force reference of the benchmark scene.  The paper form is more than 3% too dark (the
    Gaussian decoders' fit to the two point masses degenerates); the exact form is within 1.5%."""
    def mean(models, mode, spp, seed):
        cs, opt = pipeline.render_set(models)
        p = dict(synth.render_scene(sigma, width=128, height=128, spp=spp, mode=mode, seed=seed), **opt)
        img = torch.zeros(128 * 128, dtype=torch.float64, device="cuda")
        st = torch.zeros(ms.MS_RENDER_STATS, dtype=torch.int64, device="cuda")
        ms.ms_render(ms.render_params(p), cs if mode == ms.MS_SPHERE else None, img, st)
        torch.cuda.synchronize()
        return float(img.sum().item()) / spp

    ref = mean("paper", ms.MS_BRUTE, 4096, seed=7)
    r_paper = mean("paper", ms.MS_SPHERE, 1024, seed=8) / ref
    r_atoms = mean("atoms", ms.MS_SPHERE, 1024, seed=8) / ref
    assert r_paper < 0.97, (r_paper, r_atoms)
    assert abs(r_atoms - 1.0) < 0.015, (r_paper, r_atoms)
