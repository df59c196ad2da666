"""Pins of the oracle walk (Sec. 3.1) against what the paper and the mathematics fix (CPU only)."""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy import integrate, stats

from tests.test_oracle_rng_math import philox_py

Z = (0.0, 0.0, 1.0)


def medium(sigma, g=0.0, albedo=1.0, iso=0, paper=1, dir_in=Z):
    return dict(optical_radius=sigma, g=g, albedo=albedo, dir_in=dir_in, isotropic_start=iso,
                first_event_at_origin=paper)


def binom_ok(k, n, p, z=5.0):
    return abs(k / n - p) <= z * math.sqrt(p * (1 - p) / n) + 1.0 / n


@pytest.mark.parametrize("sigma", [0.5, 1.0, 2.0, 4.0])
def test_transmission_albedo_zero(orc, sigma):
    """Fly-first, albedo 0: a photon leaves only if its first free path reaches the sphere: exp(-sigma R)."""
    n = 1 << 16
    r = orc.walk(11, n, medium(sigma, 0.8, 0.0, paper=0))
    esc = int(r["counters"][0])
    assert binom_ok(esc, n, math.exp(-sigma))
    assert int(r["counters"][1]) == n - esc
    esc_mask = r["status"] == 0
    assert np.all(r["n_events"][esc_mask] == 0) and np.all(r["n_events"][~esc_mask] == 1)
    assert np.allclose(r["exit_pos"][esc_mask], Z, atol=1e-15)


@pytest.mark.parametrize("g", [0.0, 0.5, 0.9])
def test_single_event_escape_probability(orc, g):
    """Paper convention: after the event at the centre the sphere is at distance 1 in every direction, so
    P(N = 1) = exp(-sigma R) for every g."""
    n, sigma = 1 << 16, 1.5
    r = orc.walk(12, n, medium(sigma, g))
    assert binom_ok(int(np.sum(r["n_events"] == 1)), n, math.exp(-sigma))
    assert r["hist_n"][1] == np.sum(r["n_events"] == 1)


def test_two_event_probability_quadrature(orc):
    """g = 0: P(N = 2) = int_0^1 sigma e^{-sigma l} (1/2) int_{-1}^{1} e^{-sigma t(l, mu)} dmu dl with
    t(l, mu) = -l mu + sqrt(1 - l^2 (1 - mu^2)) the distance to the sphere from radius l."""
    n, sigma = 1 << 17, 1.5

    def inner(mu, l):
        t = -l * mu + math.sqrt(1.0 - l * l * (1.0 - mu * mu))
        return 0.5 * math.exp(-sigma * t)

    p2, _ = integrate.dblquad(lambda mu, l: sigma * math.exp(-sigma * l) * inner(mu, l), 0.0, 1.0, -1.0, 1.0,
                              epsabs=1e-12)
    r = orc.walk(13, n, medium(sigma, 0.0))
    assert binom_ok(int(np.sum(r["n_events"] == 2)), n, p2)


def test_free_path_is_exponential(orc):
    """First event position along +z (fly-first, albedo 0, uniform reservoir): truncated Exp(sigma)."""
    n, sigma = 1 << 15, 2.0
    r = orc.walk(14, n, medium(sigma, 0.0, 0.0, paper=0), reservoir_mode=1)
    ab = r["status"] == 1
    l = r["rep_pos"][ab, 2]
    assert np.allclose(r["rep_pos"][ab, :2], 0.0) and np.all(r["rep_index"][ab] == 1)
    cdf = lambda x: (1 - np.exp(-sigma * x)) / (1 - math.exp(-sigma))
    assert stats.kstest(l, cdf).pvalue > 1e-4
    assert np.allclose(r["rep_dir"][ab], Z)


def test_conservation_and_histograms(orc):
    n = 20000
    rng = np.random.default_rng(0)
    m = medium(rng.uniform(0.5, 20, n), rng.uniform(0, 0.95, n), rng.uniform(0.9, 1.0, n))
    r = orc.walk(15, n, m, max_events=200)
    c = r["counters"]
    assert c[0] + c[1] + c[2] == n and c[2] > 0
    assert c[3] == r["n_events"].astype(np.int64).sum()
    assert r["hist_n"].sum() == n and r["hist_pos"].sum() == c[0] and r["hist_cos"].sum() == c[0]
    assert np.all(r["n_events"] <= 200) and np.all(r["n_events"][r["status"] == 2] == 200)
    # quarter-octave bins of N, from their definition: [2^e (1 + m/4), 2^e (1 + (m+1)/4))
    N = r["n_events"].astype(np.int64)
    e = np.floor(np.log2(np.maximum(N, 1))).astype(np.int64)
    frac = (N - 2 ** e) * 4 // 2 ** e
    bins = np.where(N == 0, 0, np.minimum(63, 1 + 4 * e + frac))
    assert np.array_equal(np.bincount(bins, minlength=64), r["hist_n"].astype(np.int64))
    # exit-direction cosines are those of an outgoing crossing
    esc = r["status"] == 0
    mu = np.sum(r["exit_pos"][esc] * r["exit_dir"][esc], axis=1)
    assert mu.min() >= 0.0
    assert np.array_equal(np.bincount(np.minimum(63, (mu * 64).astype(int)), minlength=64),
                          r["hist_cos"].astype(np.int64))
    assert np.allclose(np.linalg.norm(r["exit_pos"][esc], axis=1), 1.0, atol=1e-14)


def test_isotropic_start_gives_uniform_exit_positions(orc):
    """Rotational invariance (Sec. 4.1): with an isotropic start the exit point is uniform on the sphere;
    the 32 x 64 (cos theta, phi) bins have equal area."""
    n = 1 << 16
    r = orc.walk(1, n, medium(8.0, 0.8, 0.999, iso=1, paper=0))
    h = r["hist_pos"].astype(np.float64).ravel()
    assert stats.chisquare(h).pvalue > 1e-4


def test_exact_absorption_identity(orc):
    """Roulette draws its own uniform, so an absorbing walk follows the albedo-1 walk until it is absorbed:
    N_phi = min(N_1, k_abs) with k_abs the first event whose roulette uniform is >= phi, and the absorbed
    fraction estimates E[1 - phi^N_1] (Sec. 3.2, q(N, phi) = 1 - phi^N)."""
    n, sigma, phi = 4096, 4.0, 0.9
    r1 = orc.walk(21, n, medium(sigma, 0.8, 1.0))
    rp = orc.walk(21, n, medium(sigma, 0.8, phi))
    kabs = np.full(n, 1 << 30)
    hi = [orc.philox_words(21, 0, n, s, 0)[:, 3] for s in range(int(r1["n_events"].max()))]
    lo = [orc.philox_words(21, 0, n, s, 2)[:, 3] for s in range(int(r1["n_events"].max()))]
    for s in range(len(hi) - 1, -1, -1):
        u3 = ((hi[s].astype(np.uint64) << np.uint64(21)) | (lo[s].astype(np.uint64) >> np.uint64(11))) * 2.0**-53
        kabs = np.where(u3 >= phi, s + 1, kabs)  # event k sits at step k-1 in the paper convention
    assert np.array_equal(rp["n_events"], np.minimum(r1["n_events"], kabs))
    esc = rp["status"] == 0
    assert np.array_equal(esc, r1["n_events"] < kabs)
    assert np.array_equal(rp["exit_pos"][esc], r1["exit_pos"][esc])
    assert np.array_equal(rp["exit_dir"][esc], r1["exit_dir"][esc])
    q = 1.0 - phi ** r1["n_events"].astype(np.float64)
    assert abs(np.mean(~esc) - q.mean()) < 5 * math.sqrt(q.mean() * (1 - q.mean()) / n)


def test_reservoir_selection_probabilities(orc):
    """Representative event k is chosen with probability phi^k / Lambda^(N) (Sec. 4.3); roulette off."""
    n, phi = 1 << 15, 0.7
    r = orc.walk(22, n, medium(2.5, 0.5, phi), reservoir_mode=2)
    assert np.all(r["status"] == 0)
    for N in (2, 3, 4):
        sel = r["n_events"] == N
        ks = r["rep_index"][sel]
        w = phi ** np.arange(1, N + 1)
        obs = np.bincount(ks, minlength=N + 1)[1:]
        assert stats.chisquare(obs, w / w.sum() * obs.sum()).pvalue > 1e-4
    # uniform mode at phi = 1
    r = orc.walk(23, n, medium(2.5, 0.5, 1.0), reservoir_mode=1)
    sel = r["n_events"] == 3
    assert stats.chisquare(np.bincount(r["rep_index"][sel], minlength=4)[1:]).pvalue > 1e-4


def test_photon_offset_shards_compose(orc):
    """Two shards by photon offset sum to the single run bit for bit."""
    m = medium(5.0, 0.6, 0.95, iso=1, paper=0)
    a = orc.walk(9, 3000, m)
    b1 = orc.walk(9, 1700, m)
    b2 = orc.walk(9, 1300, m, photon_offset=1700)
    for k in ("hist_n", "hist_pos", "hist_cos", "counters"):
        assert np.array_equal(a[k], b1[k] + b2[k])
    assert np.array_equal(a["n_events"], np.concatenate([b1["n_events"], b2["n_events"]]))


# ----------------------------------------------------------------------------------------------------------
# Tiny cases traced by a separate restatement of the step rules in 60-digit arithmetic (mpmath), on the
# same Philox words: every integer must agree, floats to 1e-12.

def _u53(seed, pid, step, tag):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    hi = philox_py([step, pid & 0xFFFFFFFF, pid >> 32, tag], key)
    lo = philox_py([step, pid & 0xFFFFFFFF, pid >> 32, tag + 2], key)
    return [mp.mpf((h << 21) | (l >> 11)) / mp.mpf(2) ** 53 for h, l in zip(hi, lo)]


def _u_reservoir(seed, pid, step):
    """The reservoir's uniform at a step: the low 11 bits of the tag 2 words 0..2, which the 53-bit uniforms
    leave unused, as a 33-bit fraction."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    lo = philox_py([step, pid & 0xFFFFFFFF, pid >> 32, 2], key)
    return mp.mpf(((lo[0] & 0x7FF) << 22) | ((lo[1] & 0x7FF) << 11) | (lo[2] & 0x7FF)) / mp.mpf(2) ** 33


def _trace(seed, pid, sigma, g, phi, iso, paper, res_mode, max_events=10**6):
    mp.mp.dps = 60
    if iso:
        u = _u53(seed, pid, 0, 1 if paper else 0)
        uz, uphi = (u[2], u[3]) if paper else (u[1], u[2])
        z = 1 - 2 * uz
        st = mp.sqrt(max(0, 1 - z * z))
        w = [st * mp.cos(2 * mp.pi * uphi), st * mp.sin(2 * mp.pi * uphi), z]
    else:
        w = [mp.mpf(0), mp.mpf(0), mp.mpf(1)]
    p = [mp.mpf(0)] * 3
    n, status, wsum, pw, rep_k = 0, 0, mp.mpf(0), mp.mpf(1), 0
    x = [mp.mpf(0)] * 3
    s = 0
    while True:
        u = _u53(seed, pid, s, 0)
        if s > 0 or paper:
            if n >= max_events:
                status = 2
                break
            n += 1
            if res_mode:
                a = _u_reservoir(seed, pid, s)
                wk = 1 if res_mode == 1 else pw * phi
                pw = wk if res_mode == 2 else pw
                wsum += wk
                if a * wsum < wk:
                    rep_k = n
            if res_mode != 2 and u[3] >= phi:
                status = 1
                break
            if abs(g) < 1e-4:
                mu = 2 * u[1] - 1
            else:
                t = (1 - g * g) / (1 - g + 2 * g * u[1])
                mu = min(1, max(-1, (1 + g * g - t * t) / (2 * g)))
            sgn = 1 if w[2] >= 0 else -1
            aa = -1 / (sgn + w[2])
            b = w[0] * w[1] * aa
            t1 = [1 + sgn * w[0] * w[0] * aa, sgn * b, -sgn * w[0]]
            t2 = [b, sgn + w[1] * w[1] * aa, -w[1]]
            sth = mp.sqrt(max(0, 1 - mu * mu))
            ph = 2 * mp.pi * u[2]
            w = [sth * mp.cos(ph) * t1[i] + sth * mp.sin(ph) * t2[i] + mu * w[i] for i in range(3)]
            nn = mp.sqrt(sum(v * v for v in w))
            w = [v / nn for v in w]
        l = -mp.log(1 - u[0]) / sigma
        b = sum(p[i] * w[i] for i in range(3))
        c = sum(v * v for v in p) - 1
        te = -b + mp.sqrt(max(0, b * b - c))
        if l >= te:
            x = [p[i] + te * w[i] for i in range(3)]
            nx = mp.sqrt(sum(v * v for v in x))
            x = [v / nx for v in x]
            break
        p = [p[i] + l * w[i] for i in range(3)]
        s += 1
    return n, status, [float(v) for v in x], [float(v) for v in w], rep_k


@pytest.mark.parametrize("iso,paper,res_mode,sigma,g,phi", [
    (0, 1, 2, 3.0, 0.8, 0.9), (1, 0, 0, 2.0, 0.0, 0.95), (1, 1, 1, 1.5, -0.5, 0.8), (0, 0, 0, 4.0, 0.95, 1.0)])
def test_tiny_cases_against_high_precision_restatement(orc, iso, paper, res_mode, sigma, g, phi):
    n = 6
    r = orc.walk(77, n, medium(sigma, g, phi, iso=iso, paper=paper), reservoir_mode=res_mode)
    for i in range(n):
        N, status, x, w, k = _trace(77, i, sigma, g, phi, iso, paper, res_mode)
        assert (N, status, k if res_mode else 0) == (int(r["n_events"][i]), int(r["status"][i]),
                                                     int(r["rep_index"][i]))
        if status == 0:
            assert np.allclose(r["exit_pos"][i], x, atol=1e-12)
            assert np.allclose(r["exit_dir"][i], w, atol=1e-12)


def test_spare_bit_uniforms_are_uniform_and_independent(orc):
    """The uniforms drawn from bits the main uniforms leave unused (the walk's reservoir uniform: low bytes of
    words 0..2 at 24 bits, low 11 bits of the tag 2 words at 53 bits; the sphere step's absorption and azimuth
    uniforms: low bytes of the tag 2 and tag 3 words) are uniform on [0, 1) and uncorrelated with the uniforms
    taken from the same words' other bits, over 200,000 counters.  (Taking bits the main uniforms use, such
    as a word's top byte, would correlate with them.)"""
    from scipy import stats
    n = 200_000
    hi = orc.philox_words(9, 0, n, 5, 0).astype(np.uint64)
    lo = orc.philox_words(9, 0, n, 5, 2).astype(np.uint64)
    spare24 = ((hi[:, 0] & 0xFF) << 16 | (hi[:, 1] & 0xFF) << 8 | (hi[:, 2] & 0xFF)) / 2.0 ** 24
    spare33 = ((lo[:, 0] & 0x7FF) << 22 | (lo[:, 1] & 0x7FF) << 11 | (lo[:, 2] & 0x7FF)) / 2.0 ** 33
    u24 = (hi >> 8) / 2.0 ** 24
    u53 = ((hi << 21) | (lo >> 11)).astype(np.float64) / 2.0 ** 53
    bound = 5.0 / np.sqrt(n)
    for spare, main in ((spare24, u24), (spare33, u53)):
        assert stats.kstest(spare, "uniform").pvalue > 1e-4
        for j in range(4):
            assert abs(np.corrcoef(spare, main[:, j])[0, 1]) < bound
    # a "spare" uniform from bits the main uniform uses (the top byte of word 0) is not independent of it
    bad = (hi[:, 0] >> 24) / 256.0
    assert abs(np.corrcoef(bad, u24[:, 0])[0, 1]) > 10 * bound
