"""Pins of the oracle's sphere-tracing step as a whole, and of its march, against what the paper's physics fixes.

* The exact-sampler pin (Sec. 3, Fig. 2b; Sec. 4.1, Eq. 3-4; Sec. 4.3, Eq. 5).  In the oracle's mode 2 each
  sphere step draws a brute-force walk record in the unit sphere at optical radius sigma_t r (the albedo-1
  physics, representative event with weights phi^k: exactly what the three CVAEs are trained to imitate), turns
  it into the models' outputs, and puts those through the same code as the learned samplers' outputs: the
  Eq. 4 frame R^CVAE R_psi, the exit direction from (alpha, beta) in (e_n, e_b, e_t), the representative event
  scaled by r, NEE with weight Lambda^(N) = sum_{i=1..N} phi^i, then absorption with probability 1 - phi^N.
  With an exact sampler the sphere step only reorganises the random walk, so the image must equal the
  brute-force image in expectation.  Mistakes planted in that composition fail the pin.
* The Lambda-weighted representative NEE is unbiased (Sec. 4.3, Eq. 5): on the same walks, Lambda^(N) times
  the representative event's term has the mean of the per-event NEE sum; with the paper's printed
  sum over i = 0..N (N + 1 terms) it does not.
* The centre event (exact_centre): in a training record the representative event is the first one — at the
  sphere's centre, with the incoming direction — exactly when its position is the centre, and given N that
  happens with probability phi / Lambda^(N) (Sec. 4.3, k = 1), the probability the renderer draws it with.
* The N = 1 step (exact_n1): with probability exp(-tau) the first free path leaves the sphere; such a record
  exits radially (exit direction = exit position, so alpha = beta = 0) along one HG scattering of the incoming
  direction, and its representative event is the centre: what the renderer draws for that step.
* The march (sphere tracing, Hart 1996): a plain Lipschitz-only march (step |f| / (1 + A k)) finds the same
  boundary crossings as the three-bound march, up to the boundary band, and renders the same image.
"""
import numpy as np
import pytest

from paper_2011_03082_b300 import synth

EPS = 1e-4      # the march's boundary band, in units of the distance bound (oracle/render.c R_EPS)


def _batches(orc, params, k):
    """k images on disjoint sample ranges (per-pixel means over each batch's spp)."""
    s = params["spp"]
    return np.array([orc.render(dict(params, sample_offset=b * s))[0] / s for b in range(k)])


def _z(a, b):
    """z statistics of mean(b) - mean(a) over batches: of the image sums, and per pixel (pixels where both
    batch sets vary)."""
    k = a.shape[0]
    ta, tb = a.sum((1, 2)), b.sum((1, 2))
    z_tot = (tb.mean() - ta.mean()) / np.sqrt(ta.var(ddof=1) / k + tb.var(ddof=1) / k)
    va, vb = a.var(0, ddof=1) / k, b.var(0, ddof=1) / k
    ok = (va + vb) > 0
    z_pix = (b.mean(0) - a.mean(0))[ok] / np.sqrt(va + vb)[ok]
    return float(z_tot), z_pix


# sigma_t, albedo, g, minimum optical radius of a sphere step
EXACT_CASES = [(s, phi, g, 1.0) for s in (16.0, 64.0) for phi in (0.99, 1.0) for g in (0.8, -0.5)] + [
    (64.0, 0.9, 0.8, 0.01), (16.0, 1.0, -0.5, 0.01)]


@pytest.mark.parametrize("sigma,phi,g,tau_min", EXACT_CASES,
                         ids=[f"s{int(c[0])}_a{c[1]}_g{c[2]}_t{c[3]}" for c in EXACT_CASES])
def test_exact_sampler_sphere_step_matches_brute_force(orc, sigma, phi, g, tau_min):
    """Sphere tracing with the exact sampler equals brute-force path tracing within Monte Carlo error, on the
    whole image (|z| <= 4) and per pixel (|z| <= 5), 16 batches of 8 x 8 px x 128 spp each (independent
    streams: the brute-force and sphere-traced images use different seeds)."""
    base = synth.render_scene(sigma, width=8, height=8, spp=128, mode=0, g=g, albedo=phi, seed=11)
    bf = _batches(orc, base, 16)
    ex = _batches(orc, dict(base, mode=2, seed=12, min_optical_radius=tau_min), 16)
    z_tot, z_pix = _z(bf, ex)
    assert abs(z_tot) <= 4.0, z_tot
    assert np.abs(z_pix).max() <= 5.0, np.abs(z_pix).max()
    # the sphere steps are exercised
    _, st, _ = orc.render(dict(base, mode=2, seed=12, min_optical_radius=tau_min))
    assert st[3] > 0.05 * st[2], st


@pytest.mark.parametrize("plant,what", [(1, "Lambda over i = 0..N"), (2, "e_t negated"),
                                        (3, "no NEE on an absorbing step"), (4, "event not scaled by r")])
def test_exact_sampler_pin_catches_planted_mistakes(orc, plant, what):
    """Each plausible mistake planted in the oracle's sphere step moves the image sum by more than 5 standard
    errors from brute force (sigma_t 64, albedo 0.9, g 0.8, sphere steps down to optical radius 0.01), where the
    unplanted step stays within 3."""
    base = synth.render_scene(64.0, width=8, height=8, spp=256, mode=0, g=0.8, albedo=0.9, seed=21)
    bf = _batches(orc, base, 16)
    st_params = dict(base, mode=2, seed=22, min_optical_radius=0.01)
    try:
        orc.set_plant(plant)
        bad = _batches(orc, st_params, 16)
    finally:
        orc.set_plant(0)
    good = _batches(orc, st_params, 16)
    assert abs(_z(bf, good)[0]) <= 3.0
    assert abs(_z(bf, bad)[0]) > 5.0, (what, _z(bf, bad)[0])


def _event_term(X, W, light, tau, g):
    """rho_g(W . w_L) exp(-tau d) / |x_L - X|^2 for events X inside the unit sphere (d: distance from X to the
    sphere toward the light)."""
    dl = light[None, :] - X
    d2 = np.sum(dl * dl, axis=1)
    wl = dl / np.sqrt(d2)[:, None]
    b = np.sum(X * wl, axis=1)
    d = -b + np.sqrt(np.maximum(b * b - (np.sum(X * X, axis=1) - 1.0), 0.0))
    mu = np.sum(W * wl, axis=1)
    rho = (1.0 - g * g) / (4.0 * np.pi * (1.0 + g * g - 2.0 * g * mu) ** 1.5)
    return rho * np.exp(-tau * d) / d2


@pytest.mark.parametrize("tau,g,phi,power", [(4.0, 0.8, 0.9, True), (16.0, 0.8, 0.99, False),
                                             (8.0, -0.5, 0.95, False), (2.0, -0.5, 0.95, True),
                                             (4.0, 0.0, 1.0, True)])
def test_lambda_weighted_representative_nee_is_unbiased(orc, tau, g, phi, power):
    """Sec. 4.3: choosing event k with probability phi^k / Lambda and weighting its NEE term by
    Lambda = sum_{i=1..N} phi^i reproduces the mean of the per-event NEE sum sum_k phi^k term_k (the brute-force
    estimate, Eq. 5), on the same walks (paired, |z| <= 4).  The paper's printed Lambda = sum_{i=0..N} phi^i adds
    one extra term per walk, a bias of E[term_k] that the same test rejects (|z| > 8) where that term is not
    negligible (it is where the light reaches few of the events: optical radius 8 and more)."""
    n = 200_000
    light = np.array([0.3, 1.2, 1.5])
    r = orc.walk_nee(5, n, tau, g, phi, light)
    N = r["n_events"].astype(np.float64)
    assert np.all(r["rep_index"] >= 1) and np.all(r["rep_index"] <= r["n_events"])
    lam = N if phi == 1.0 else phi * (1.0 - phi ** N) / (1.0 - phi)
    term = _event_term(r["rep_pos"], r["rep_dir"], light, tau, g)
    d = lam * term - r["nee_sum"]
    z = d.mean() / (d.std(ddof=1) / np.sqrt(n))
    assert abs(z) <= 4.0, z
    if power:
        d_paper = (lam + 1.0) * term - r["nee_sum"]
        z_paper = d_paper.mean() / (d_paper.std(ddof=1) / np.sqrt(n))
        assert z_paper > 8.0, z_paper


@pytest.mark.parametrize("tau,g,phi,power", [(2.0, 0.8, 0.9, True), (6.0, -0.5, 0.97, True),
                                             (3.0, 0.0, 1.0, False)])
def test_centre_event_probability(orc, tau, g, phi, power):
    """The representative event is the first one exactly when it sits at the centre (0, 0, 0), and then its
    direction is the incoming (0, 0, 1); later events never sit at the centre.  Given N, the first event is
    picked with probability phi / Lambda^(N), Lambda^(N) = phi (1 - phi^N) / (1 - phi) (N at phi = 1): the count
    over 200,000 walks against the sum of those probabilities (|z| <= 4).  Taking the uniform 1 / N instead (a
    plausible slip: the walks' events are equally likely only at phi = 1) fails the same count (|z| > 8)."""
    n = 200_000
    r = orc.walk_nee(9, n, tau, g, phi, np.array([0.3, 1.2, 1.5]))
    N = r["n_events"].astype(np.float64)
    first = r["rep_index"] == 1
    at_centre = np.all(r["rep_pos"] == 0.0, axis=1)
    assert np.array_equal(first, at_centre)
    assert np.all(r["rep_dir"][first] == np.array([0.0, 0.0, 1.0]))
    lam = N if phi == 1.0 else phi * (1.0 - phi ** N) / (1.0 - phi)

    def z_of(p):
        return (first.sum() - p.sum()) / np.sqrt(np.sum(p * (1.0 - p)) + 1e-300)

    assert abs(z_of(phi / lam)) <= 4.0, z_of(phi / lam)
    if power:
        assert abs(z_of(1.0 / N)) > 8.0, z_of(1.0 / N)


@pytest.mark.parametrize("tau,g", [(0.7, 0.8), (1.5, -0.5), (1.0, 0.0)])
def test_single_event_step_is_exact(orc, tau, g):
    """A record with N = 1 has probability exp(-tau) (binomial |z| <= 4); its exit direction equals its exit
    position (alpha = beta = 0 in the model frame), cos theta = x_z follows the HG law of cosines with
    parameter g (KS against the closed-form CDF F(mu) = (1 - g^2) / (2g) [(1 + g^2 - 2 g mu)^(-1/2) - 1 / (1 + g)],
    uniform at g = 0), and its representative event is the centre with the incoming direction (0, 0, 1)."""
    from scipy import stats
    n, phi = 200_000, 0.95
    r = orc.walk(31, n, dict(optical_radius=tau, g=g, albedo=phi, dir_in=(0.0, 0.0, 1.0), isotropic_start=0,
                             first_event_at_origin=1), reservoir_mode=2)
    one = r["n_events"] == 1
    p1 = np.exp(-tau)
    assert abs(one.sum() - n * p1) <= 4.0 * np.sqrt(n * p1 * (1.0 - p1))
    x, w = r["exit_pos"][one], r["exit_dir"][one]
    assert np.max(np.abs(x - w)) < 1e-12
    assert np.all(r["rep_index"][one] == 1)
    assert np.all(r["rep_pos"][one] == 0.0) and np.all(r["rep_dir"][one] == np.array([0.0, 0.0, 1.0]))
    if g == 0.0:
        cdf = lambda mu: (mu + 1.0) / 2.0
    else:
        cdf = lambda mu: (1.0 - g * g) / (2.0 * g) * (1.0 / np.sqrt(1.0 + g * g - 2.0 * g * mu) - 1.0 / (1.0 + g))
    assert stats.kstest(x[:, 2], cdf).pvalue > 1e-3


def _f(A, k, q):
    q = np.atleast_2d(q)
    return np.sqrt(np.sum(q * q, axis=1)) - 1.0 - A * np.sin(k * q[:, 0]) * np.sin(k * q[:, 1]) * np.sin(k * q[:, 2])


@pytest.mark.parametrize("A,k", [(0.1, 6.0), (0.2, 6.0), (0.15, 10.0), (0.3, 5.0)])
def test_plain_lipschitz_march_finds_the_same_crossings(orc, A, k):
    """The three-bound march and plain sphere tracing (the Lipschitz step alone) agree on 1,000 rays from
    inside and outside: the same outcome (crossing or escape), and crossings that lie in one connected piece of
    the boundary band |f| <= (1 + A k) EPS (f sampled every 1e-6 between the two stopping points stays in the
    band), so they are the same crossing."""
    lip = 1.0 + A * k
    rng = np.random.default_rng(17)
    crossings = 0
    for i in range(1000):
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        p = rng.uniform(-0.6, 0.6, 3) if i % 2 else -2.5 * w + rng.uniform(-0.8, 0.8, 3)
        r0, t0 = orc.ray_crossing(A, k, p, w)
        r1, t1 = orc.ray_crossing(A, k, p, w, plain=True)
        assert r0 == r1, (i, r0, r1)
        if r0 != 1:
            continue
        crossings += 1
        lo, hi = min(t0, t1), max(t0, t1)
        s = np.linspace(lo, hi, max(2, int((hi - lo) / 1e-6) + 1))
        assert np.abs(_f(A, k, p[None, :] + s[:, None] * w[None, :])).max() <= lip * EPS * 1.01, (i, t0, t1)
    assert crossings >= 900


@pytest.mark.parametrize("sigma,mode", [(16.0, 0), (64.0, 0), (16.0, 2), (64.0, 2)])
def test_plain_lipschitz_march_renders_the_same_image(orc, sigma, mode):
    """Whole images with the plain Lipschitz march equal the three-bound march's up to the boundary band.
    Paths coincide except where a march stops elsewhere in the band and a later decision flips, so the paired
    image difference is far below the seed-to-seed noise (RMSE ratio <= 0.5).  Where in the band a march stops
    moves a shadow ray's inside length by up to about (1 + A k) EPS per crossing, i.e. its transmittance by up
    to sigma_t (1 + A k) EPS relative (the plain march stops at the band's far edge, the three-bound march near
    the surface), so over 8 batches the image sums agree to 2 sigma_t (1 + A k) EPS relative plus 4 paired
    standard errors."""
    p = synth.render_scene(sigma, width=16, height=16, spp=16, mode=mode, seed=5)
    a = _batches(orc, p, 8)
    b = _batches(orc, dict(p, march_mode=1, max_march=1 << 20), 8)
    c = _batches(orc, dict(p, seed=6), 8)
    rm = lambda x, y: float(np.sqrt(np.mean((x - y) ** 2)))
    assert rm(a, b) <= 0.5 * rm(a, c), (rm(a, b), rm(a, c))
    sa, sb = a.sum((1, 2)), b.sum((1, 2))
    d = sb - sa
    band = 2.0 * sigma * (1.0 + p["disp_amp"] * p["disp_freq"]) * EPS * sa.mean()
    assert abs(d.mean()) <= band + 4.0 * d.std(ddof=1) / np.sqrt(d.size), (d.mean(), band)
