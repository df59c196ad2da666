"""Pins of the oracle's random stream and deterministic math (CPU only).

The Philox4x32-10 stream is checked against a second, independent restatement of the published definition
(Python big integers instead of C uint32 arithmetic) and against statistical properties (uniformity,
bit balance, avalanche, serial independence).  Known-answer vectors of the reference distribution are not
available here.  The deterministic log / sincos / atan2 are checked against mpmath at high precision and the
C library.
"""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy import stats

M32 = 0xFFFFFFFF


def philox_py(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11) restated with Python integers."""
    x = list(ctr)
    k = list(key)
    for r in range(10):
        if r:
            k = [(k[0] + 0x9E3779B9) & M32, (k[1] + 0xBB67AE85) & M32]
        pa = 0xD2511F53 * x[0]
        pb = 0xCD9E8D57 * x[2]
        x = [((pb >> 32) ^ x[1] ^ k[0]) & M32, pb & M32, ((pa >> 32) ^ x[3] ^ k[1]) & M32, pa & M32]
    return x


def test_philox_matches_independent_restatement(orc):
    rng = np.random.default_rng(0)
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64)]
        key = [int(v) for v in rng.integers(0, 2**32, 2, dtype=np.uint64)]
        assert list(orc.philox(ctr, key)) == philox_py(ctr, key)
    # bulk words use counter (step, id_lo, id_hi, tag) and key (seed_lo, seed_hi)
    seed, id0 = 0x1234_5678_9ABC_DEF0, (7 << 32) + 5
    w = orc.philox_words(seed, id0, 3, 11, 9)
    for i in range(3):
        idv = id0 + i
        assert list(w[i]) == philox_py([11, idv & M32, idv >> 32, 9], [seed & M32, seed >> 32])


def test_philox_uniformity_and_bit_balance(orc):
    w = orc.philox_words(1, 0, 1 << 16, 0, 0).ravel()
    counts = np.bincount((w >> 24).astype(np.int64), minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4
    bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 32).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(w.size))
    u = orc.u24(w)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4


def test_philox_avalanche_and_independence(orc):
    rng = np.random.default_rng(3)
    flips = []
    for _ in range(400):
        ctr = [int(v) for v in rng.integers(0, 2**32, 4, dtype=np.uint64)]
        key = [1, 0]
        bit = int(rng.integers(0, 128))
        ctr2 = list(ctr)
        ctr2[bit // 32] ^= 1 << (bit % 32)
        a = np.array(orc.philox(ctr, key), np.uint32)
        b = np.array(orc.philox(ctr2, key), np.uint32)
        flips.append(np.unpackbits((a ^ b).view(np.uint8)).sum())
    assert abs(np.mean(flips) - 64.0) < 2.0
    # neighbouring ids and steps are uncorrelated
    u0 = orc.u24(orc.philox_words(5, 0, 1 << 15, 0, 0)[:, 0])
    u1 = orc.u24(orc.philox_words(5, 0, 1 << 15, 1, 0)[:, 0])
    assert abs(np.corrcoef(u0, u1)[0, 1]) < 5 / np.sqrt(u0.size)
    assert abs(np.corrcoef(u0[:-1], u0[1:])[0, 1]) < 5 / np.sqrt(u0.size)


def _ulp_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_det_log_accuracy(orc):
    rng = np.random.default_rng(1)
    x = np.concatenate([1.0 - rng.integers(0, 2**53, 3000) * 2.0**-53,
                        np.exp(rng.uniform(-700, 700, 1000)), [1.0, 0.5, 2.0**-53, 0.75, 1.5]])
    got = orc.det_log(x)
    mp.mp.prec = 120
    ref = np.array([float(mp.log(mp.mpf(float(v)))) for v in x])
    nz = ref != 0
    assert np.all(got[~nz] == 0.0)
    assert _ulp_err(got[nz], ref[nz]).max() <= 2.0


def test_det_sincos_turns_accuracy(orc):
    rng = np.random.default_rng(2)
    u = np.concatenate([rng.random(3000), [0.0, 0.125, 0.25, 0.5, 0.75, 1.0 - 2.0**-53]])
    sc = orc.det_sincos_turns(u)
    mp.mp.prec = 120
    s_ref = np.array([float(mp.sin(2 * mp.pi * mp.mpf(float(v)))) for v in u])
    c_ref = np.array([float(mp.cos(2 * mp.pi * mp.mpf(float(v)))) for v in u])
    assert np.abs(sc[:, 0] - s_ref).max() <= 4e-16
    assert np.abs(sc[:, 1] - c_ref).max() <= 4e-16
    assert np.all(sc[:, 0] ** 2 + sc[:, 1] ** 2 - 1.0 < 1e-15)


def test_det_atan2_accuracy(orc):
    rng = np.random.default_rng(4)
    y = rng.standard_normal(3000)
    x = rng.standard_normal(3000)
    y = np.concatenate([y, [0.0, 1.0, -1.0, 0.0, 1e-300]])
    x = np.concatenate([x, [1.0, 0.0, 0.0, -1.0, 1.0]])
    got = orc.det_atan2(y, x)
    mp.mp.prec = 120
    ref = np.array([float(mp.atan2(mp.mpf(float(a)), mp.mpf(float(b)))) for a, b in zip(y, x)])
    assert np.abs(got - ref).max() <= 4 * np.spacing(math.pi)


@pytest.mark.parametrize("g", [0.0, 0.3, 0.8, 0.95, -0.7])
def test_hg_inverse_cdf(orc, g):
    """The sampled cosine inverts the HG CDF of Eq. 1, whose mean is g and second moment (1+2g^2)/3."""
    n = 20000
    u = (np.arange(n) + 0.5) / n
    mu = orc.hg_cosine(u, g)
    if abs(g) > 1e-4:
        cdf = (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))
    else:
        cdf = (1 + mu) / 2
    # the sampler is the inverse of the CDF P(cos <= mu)
    assert np.abs(cdf - u).max() < 1e-12
    assert abs(mu.mean() - g) < 1e-3
    assert abs((mu * mu).mean() - (1 + 2 * g * g) / 3) < 1e-3


def test_scatter_rotation(orc):
    rng = np.random.default_rng(5)
    for _ in range(300):
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        mu, u = rng.uniform(-1, 1), rng.random()
        r = orc.scatter_dir(w, mu, u)
        assert abs(np.linalg.norm(r) - 1) < 1e-14
        assert abs(r @ w - mu) < 1e-13
    # about +z the basis is the coordinate frame: spherical coordinates exactly
    r = orc.scatter_dir([0.0, 0.0, 1.0], 0.3, 0.2)
    st = math.sqrt(1 - 0.09)
    assert np.allclose(r, [st * math.cos(0.4 * math.pi), st * math.sin(0.4 * math.pi), 0.3], atol=1e-15)
    # azimuths are uniform: the rotated vectors average to mu * w
    w = np.array([0.6, -0.0, 0.8])
    avg = np.mean([orc.scatter_dir(w, 0.5, (k + 0.5) / 64) for k in range(64)], axis=0)
    assert np.allclose(avg, 0.5 * w, atol=1e-12)


@pytest.mark.parametrize("count", [3, 5, 8, 10, 11])
def test_decoder_normals_are_independent_standard_normals(orc, count):
    """The decoder workload's normals (Box-Muller on 24-bit uniforms; with ten normals the last pair comes from
    the low bytes the first eight uniforms leave unused, so two Philox blocks serve instead of three): every
    column is standard normal (KS against N(0, 1), mean and variance within 5 standard errors) and no two columns
    correlate, over 100,000 queries.  Counts that fill whole blocks keep the plain layout: normals 4j..4j+3 from
    block j."""
    n = 100_000
    z = orc.decoder_normals(7, 0, n, count)
    assert z.shape == (n, count)
    se = 1.0 / np.sqrt(n)
    for j in range(count):
        assert stats.kstest(z[:, j], "norm").pvalue > 1e-4, j
        assert abs(z[:, j].mean()) < 5 * se and abs(z[:, j].var() - 1.0) < 5 * np.sqrt(2.0) * se, j
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(count)).max() < 5 * se
    # the first eight normals (and all of them when count is not 9 or 10) come from the blocks in order
    full = min(count, 8) if count in (9, 10) else count
    plain = np.concatenate([orc.normals_from_words(orc.philox_words(7, 0, n, j, 0xD0))
                            for j in range((full + 3) // 4)], axis=1)[:, :full]
    assert np.array_equal(z[:, :full], plain)
