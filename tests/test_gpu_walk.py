"""GPU parity of ms_simulate_walks against the oracle walk (Sec. 3.1, Eq. 1, Sec. 4.3).

* MS_FP64: every integer output (scatter counts, status, representative index, all histogram bins and
  counters) equals the oracle's bit for bit, and the exit / representative vectors equal the oracle's FP64
  values rounded to float32.
* MS_FP32: same Philox stream as the oracle run with 24-bit uniforms; the paths coincide except where a
  single-precision decision flips, so >= 99% of photons have identical (N, status), and the distributions
  of N, exit cos(theta) and exit-direction cosine agree (two-sample KS < 0.01 at the 65,536-photon
  configuration).
"""
import numpy as np
import pytest
import torch
from scipy import stats

from paper_2011_03082_b300 import ms, synth

pytestmark = pytest.mark.gpu


def _media_np(n, sig, g, phi, iso, paper, dir_in=(0.0, 0.0, 1.0)):
    """float32-rounded media for both sides."""
    f = lambda v: np.asarray(np.broadcast_to(np.float32(v), (n,)) if np.ndim(v) == 0 else np.float32(v))
    return dict(optical_radius=f(sig).astype(np.float64), g=f(g).astype(np.float64),
                albedo=f(phi).astype(np.float64), dir_in=np.asarray(dir_in, np.float64),
                isotropic_start=iso, first_event_at_origin=paper)


def _gpu_walk(n, m, *, seed, precision, reservoir=0, max_events=1 << 20, offset=0, per_photon=True):
    per_media = np.ndim(m["optical_radius"]) > 0 and np.size(m["optical_radius"]) > 1
    media = ms.media_tensor(m["optical_radius"], m["g"], m["albedo"], m["dir_in"], m["isotropic_start"],
                            m["first_event_at_origin"], n=n if per_media else 1)
    out = ms.walk_outputs(n, per_photon)
    ms.ms_simulate_walks(media, n, out, seed=seed, photon_offset=offset, max_events=max_events,
                         reservoir=reservoir, precision=precision)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle_media(m, n):
    d = dict(m)
    for k in ("optical_radius", "g", "albedo"):
        v = np.asarray(d[k])
        d[k] = v if v.size > 1 else float(v.ravel()[0])
    return d


CASES = [
    # name, n, sigma, g, albedo, iso, paper, reservoir, max_events
    ("cfg1", 65536, 8.0, 0.8, 0.999, 1, 0, 0, 1 << 20),
    ("paper_reservoir", 5000, 3.0, 0.5, 0.9, 0, 1, 2, 1 << 20),
    ("uniform_reservoir_trunc", 3001, 12.0, 0.9, 0.97, 1, 1, 1, 40),
    ("albedo0", 4097, 2.0, 0.0, 0.0, 0, 0, 0, 1 << 20),
    ("single", 1, 5.0, -0.5, 0.95, 1, 0, 1, 1 << 20),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_walk_is_bit_exact(orc, case):
    _, n, sig, g, phi, iso, paper, res, mx = case
    m = _media_np(n, sig, g, phi, iso, paper)
    gpu = _gpu_walk(n, m, seed=1, precision=ms.MS_FP64, reservoir=res, max_events=mx)
    ref = orc.walk(1, n, _oracle_media(m, n), reservoir_mode=res, max_events=mx)
    for k in ("hist_n", "hist_pos", "hist_cos", "counters"):
        assert np.array_equal(gpu[k].astype(np.uint64).reshape(ref[k].shape), ref[k]), k
    for k in ("n_events", "status", "rep_index"):
        assert np.array_equal(gpu[k], ref[k].astype(gpu[k].dtype)), k
    for k in ("exit_pos", "exit_dir", "rep_pos", "rep_dir"):
        assert np.array_equal(gpu[k], ref[k].astype(np.float32)), k


def test_fp64_walk_per_photon_media_and_offset(orc):
    n = 6000
    tau, g, phi = synth.training_media(3, n)
    m = _media_np(n, tau.astype(np.float32), g.astype(np.float32), phi.astype(np.float32), 0, 1)
    m["optical_radius"] = np.minimum(m["optical_radius"], 40.0)  # keep the oracle fast
    gpu = _gpu_walk(n, m, seed=5, precision=ms.MS_FP64, reservoir=2, offset=12345)
    ref = orc.walk(5, n, _oracle_media(m, n), reservoir_mode=2, photon_offset=12345)
    for k in ("n_events", "status", "rep_index"):
        assert np.array_equal(gpu[k], ref[k].astype(gpu[k].dtype)), k
    for k in ("exit_pos", "exit_dir", "rep_pos", "rep_dir"):
        assert np.array_equal(gpu[k], ref[k].astype(np.float32)), k
    assert np.array_equal(gpu["counters"].astype(np.uint64), ref["counters"])


def test_empty_walk_is_a_no_op():
    out = ms.walk_outputs(0, False)
    media = ms.media_tensor(2.0, 0.5, 0.9)
    ms.ms_simulate_walks(media, 0, out, precision=ms.MS_FP32)
    torch.cuda.synchronize()
    assert int(out["counters"].sum()) == 0


def test_invalid_arguments_are_rejected():
    media = ms.media_tensor(2.0, 0.5, 0.9)
    out = ms.walk_outputs(4, False)
    with pytest.raises(ms.MsError, match="precision"):
        ms.ms_simulate_walks(media, 4, out, precision=7)
    with pytest.raises(ms.MsError, match="max_events"):
        ms.ms_simulate_walks(media, 4, out, max_events=0)
    with pytest.raises(ms.MsError, match="device pointer"):
        host = torch.zeros(32, dtype=torch.uint8).pin_memory()
        ms.lib().ms_simulate_walks  # noqa: B018 - library loaded
        p = ms.WalkParams(1, 0, 4, host.data_ptr(), 0, 10, 0, 0)
        o = ms.WalkOut()
        ws = ms.workspace(256)
        st = ms.lib().ms_simulate_walks(ms.C.byref(p), ms.C.byref(o), ms._ptr(ws), 256, ms._stream())
        ms._check(st, "ms_simulate_walks")


def _ks(a, b):
    return stats.ks_2samp(a, b).statistic


def test_fp32_walk_matches_oracle_stream(orc):
    """cfg1 (65,536 photons, optical radius 8, g 0.8, albedo 0.999, isotropic fly-first start)."""
    w = synth.walk_cfg()
    n = w["n_photons"]
    m = _media_np(n, w["optical_radius"], w["g"], w["albedo"], 1, 0)
    gpu = _gpu_walk(n, m, seed=w["seed"], precision=ms.MS_FP32, reservoir=1)
    ref = orc.walk(w["seed"], n, _oracle_media(m, n), uniform_bits=24, reservoir_mode=1)
    same = (gpu["n_events"] == ref["n_events"]) & (gpu["status"] == ref["status"])
    assert same.mean() >= 0.99, same.mean()
    esc_g, esc_r = gpu["status"] == 0, ref["status"] == 0
    assert _ks(gpu["n_events"], ref["n_events"]) < 0.01
    assert _ks(gpu["exit_pos"][esc_g, 2], ref["exit_pos"][esc_r, 2]) < 0.01
    mu_g = np.sum(gpu["exit_pos"][esc_g] * gpu["exit_dir"][esc_g], 1)
    mu_r = np.sum(ref["exit_pos"][esc_r] * ref["exit_dir"][esc_r], 1)
    assert _ks(mu_g, mu_r) < 0.01
    both = same & esc_g
    assert np.abs(gpu["exit_pos"][both] - ref["exit_pos"][both]).max() < 1e-3
    c = gpu["counters"]
    assert c[0] + c[1] + c[2] == n and c[3] == gpu["n_events"].astype(np.int64).sum()
    assert gpu["hist_pos"].sum() == c[0] and gpu["hist_n"].sum() == n


def test_fp32_walk_full_training_size_properties(orc):
    """2^24 walks with per-walk media (the training-data configuration): conservation at full size, and
    sampled photons recomputed one by one by the oracle."""
    n = 1 << 24
    tau, g, phi = synth.training_media(1, n)
    media = ms.media_tensor(tau.astype(np.float32), g.astype(np.float32), phi.astype(np.float32), (0, 0, 1), 0, 1)
    out = ms.walk_outputs(n)
    ms.ms_simulate_walks(media, n, out, seed=1, reservoir=2, precision=ms.MS_FP32)
    torch.cuda.synchronize()
    N = out["n_events"].cpu().numpy()
    st = out["status"].cpu().numpy()
    c = out["counters"].cpu().numpy()
    assert np.all(st == 0) and c[0] == n and c[3] == N.astype(np.int64).sum()
    k = out["rep_index"].cpu().numpy()
    assert np.all((k >= 1) & (k <= N))
    rng = np.random.default_rng(0)
    idx = rng.choice(n, 300, replace=False)
    idx = idx[tau[idx] < 60]
    agree = 0
    for i in idx:
        m = _media_np(1, np.float32(tau[i]), np.float32(g[i]), np.float32(phi[i]), 0, 1)
        r = orc.walk(1, 1, _oracle_media(m, 1), photon_offset=int(i), reservoir_mode=2, uniform_bits=24)
        agree += int(r["n_events"][0] == N[i])
    assert agree >= 0.97 * len(idx)
