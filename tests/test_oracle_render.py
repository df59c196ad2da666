"""Pins of the oracle renderer (Sec. 3, 4.1, 4.3; Eq. 1 and 5), CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2011_03082_b300 import synth


def test_inside_length_undisplaced_sphere_is_the_chord(orc):
    rng = np.random.default_rng(0)
    xl = np.array([2.0, 2.0, 3.0])
    for _ in range(200):
        X = rng.uniform(-0.55, 0.55, 3)
        w = (xl - X) / np.linalg.norm(xl - X)
        b, c = X @ w, X @ X - 1
        chord = -b + math.sqrt(b * b - c)
        assert abs(orc.inside_length(0.0, 6.0, X, xl) - chord) < 2e-4


@pytest.mark.parametrize("A,k", [(0.1, 6.0), (0.1, 10.0), (0.15, 10.0)])
def test_inside_length_displaced_sphere_against_dense_sampling(orc, A, k):
    """Inside length of a segment against dense sampling of f.  A march stops where |f| / (1 + A k) < 1e-4,
    which at a grazing crossing (|df/dt| small) lies up to about 2e-4 / |df/dt| from the crossing, so segments
    with a crossing slope below 0.2 are skipped."""
    rng = np.random.default_rng(1)
    f = _disp_sdf(A, k)
    checked = 0
    for _ in range(60):
        X = rng.uniform(-0.8, 0.8, 3)
        if f(X) > -0.02:
            continue
        xl = rng.uniform(-3, 3, 3) * np.array([1, 1, 0]) + np.array([0, 0, 3.0])
        t = np.linspace(0, 1, 400001)
        D = np.linalg.norm(xl - X)
        fv = f(X + t[:, None] * (xl - X))
        inside = fv < 0
        ch = np.nonzero(inside[1:] != inside[:-1])[0]
        if np.any(np.abs(fv[ch + 1] - fv[ch]) / ((t[1] - t[0]) * D) < 0.2):
            continue
        ref = inside[:-1].mean() * D
        assert abs(orc.inside_length(A, k, X, xl) - ref) < 1e-3
        checked += 1
    assert checked > 20


def _disp_sdf(A, k):
    return lambda p: (np.linalg.norm(p, axis=-1) - 1
                      - A * np.sin(k * p[..., 0]) * np.sin(k * p[..., 1]) * np.sin(k * p[..., 2]))


@pytest.mark.parametrize("A,k", [(0.1, 2.0), (0.1, 6.0), (0.1, 10.0), (0.3, 4.0), (0.15, 10.0)])
def test_ray_crossing_against_dense_sampling(orc, A, k):
    """The march (sphere tracing with the radial-plus-Lipschitz step, including its early escape) finds the
    first sign change of f along the ray, found here by sampling f every 4e-5 (A k from 0.2 to 1.5, so the
    step's quadratic has positive, zero and negative leading coefficient).  Grazing crossings and near misses,
    which sampling cannot resolve, are skipped."""
    f = _disp_sdf(A, k)
    rng = np.random.default_rng(int(100 * A + k))
    t = np.linspace(0.0, 8.0, 200001)
    dt = t[1] - t[0]
    n_hit = n_escape = n_inside = 0
    for _ in range(150):
        if rng.random() < 0.6:          # from outside, aimed near the object
            p = rng.standard_normal(3)
            p *= rng.uniform(1.25, 3.0) / np.linalg.norm(p)
            w = rng.uniform(-1.3, 1.3, 3) - p
        else:                           # from inside
            p = rng.uniform(-0.85, 0.85, 3)
            if f(p) > -0.01:
                continue
            w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        fv = f(p + t[:, None] * w)
        outside = fv[0] > 0
        change = np.nonzero((fv[1:] > 0) != outside)[0]
        status, tc = orc.ray_crossing(A, k, p, w)
        if change.size == 0:
            if np.min(np.abs(fv)) < 2e-3:
                continue                # near miss
            assert outside and status == 0, (p, w, status)
            n_escape += 1
            continue
        i = change[0]
        slope = abs(fv[i + 1] - fv[i]) / dt
        if slope < 0.05 or (outside and np.min(fv[:i + 1]) < 2e-3 and np.argmin(fv[:i + 1]) < i - 50):
            continue                    # grazing crossing, or a near miss before the crossing
        assert status == 1, (p, w, status)
        # the march stops where |f| / (1 + A k) < 1e-4, i.e. up to (1 + A k) 1e-4 / slope before the crossing
        assert abs(tc - t[i]) < 1.2 * (1 + A * k) * 1e-4 / slope + 2 * dt, (p, w, tc, t[i])
        n_inside += not outside
        n_hit += outside
    assert n_hit > 15 and n_escape > 5 and n_inside > 15, (n_hit, n_escape, n_inside)


def _render(orc, **kw):
    decoders = kw.pop("decoders", None)
    p = synth.render_scene(kw.pop("sigma_t", 8.0), width=kw.pop("width", 16), height=kw.pop("height", 16),
                           spp=kw.pop("spp", 4), mode=kw.pop("mode", 0))
    p.update(kw)
    return orc.render(p, decoders)


def test_zero_albedo_gives_black_image(orc):
    img, st, _ = _render(orc, albedo=0.0)
    assert st[4] > 0 and np.all(img == 0.0)


def test_vanishing_density_gives_black_image(orc):
    img, st, _ = _render(orc, sigma_t=1e-9)
    assert st[1] > 0 and st[4] == 0 and np.all(img == 0.0)


def test_light_intensity_is_linear(orc):
    a, _, _ = _render(orc, light_I=10.0)
    b, _, _ = _render(orc, light_I=20.0)
    assert np.allclose(b, 2 * a, rtol=1e-14, atol=0) and a.sum() > 0


def test_sphere_mode_without_spheres_equals_brute_force(orc):
    """With a minimum optical radius no sphere reaches, the sphere tracer takes the thin-region fallback at
    every collision and consumes the same random numbers as brute force."""
    a, sa, _ = _render(orc, mode=0)
    b, sb, _ = _render(orc, mode=1, min_optical_radius=1e30)
    assert np.array_equal(a, b) and np.array_equal(sa[:8], sb[:8])
    assert sb[8] == sa[8] + sb[4]      # plus one distance evaluation per collision for the sphere radius


def test_single_scattering_limit_matches_quadrature(orc):
    """Undisplaced sphere, tiny albedo: only the first event's NEE survives (O(phi^2) corrections).  The pixel
    value is phi * int_0^2 sigma e^{-sigma s} rho_g(cos) e^{-sigma d_in(s)} I / d(s)^2 ds along the central
    camera ray entering at (0,0,1) going -z (Eq. 2 transmittance, Eq. 1 phase function, Eq. 5 term)."""
    sigma, g, phi, I = 2.0, 0.6, 1e-3, 10.0
    xl = np.array([2.0, 2.0, 3.0])
    W = np.array([0.0, 0.0, -1.0])

    def integrand(s):
        X = np.array([0.0, 0.0, 1.0 - s])
        dl = xl - X
        d = np.linalg.norm(dl)
        wl = dl / d
        cosang = W @ wl
        rho = (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * cosang) ** 1.5)
        b, c = X @ wl, X @ X - 1
        din = -b + math.sqrt(b * b - c)
        return sigma * math.exp(-sigma * s) * rho * math.exp(-sigma * din) * I / (d * d)

    ref = phi * integrate.quad(integrand, 0.0, 2.0, epsabs=1e-14, limit=200)[0]
    spp = 40000
    p = synth.render_scene(sigma, width=1, height=1, spp=spp, mode=0, g=g, albedo=phi, disp_amp=0.0)
    p["fov_y_deg"] = 1e-4
    img, st, _ = orc.render(p)
    est = img[0, 0] / spp
    # per-path standard error from the same integrand: second moment by quadrature
    m2 = phi * phi * integrate.quad(lambda s: integrand(s) ** 2 / (sigma * math.exp(-sigma * s)), 0, 2)[0]
    se = math.sqrt(max(m2 - ref * ref, 0) / spp)
    assert abs(est - ref) < 5 * se + 2e-3 * ref, (est, ref, se)


def test_sphere_mode_runs_with_models(orc):
    decs = []
    for i, (name, shape) in enumerate(synth.MODEL_SHAPES.items()):
        decs.append((synth.xavier_decoder(100 + i, *shape).astype(np.float64), *shape))
    img, st, _ = _render(orc, mode=1, sigma_t=64.0, decoders=decs)
    assert st[3] > 0 and np.all(np.isfinite(img)) and np.all(img >= 0)


def _surface_points(A, k, n_dir, seed):
    """Points of the displaced sphere: along each unit direction u the surface is the root of
    t - 1 - A sin(k t u_x) sin(k t u_y) sin(k t u_z) (unique: its t-derivative is at least 1 - A k > 0)."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n_dir, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    lo, hi = np.full(n_dir, 1.0 - A), np.full(n_dir, 1.0 + A)
    g = lambda t: t - 1 - A * np.prod(np.sin(k * t[:, None] * u), axis=1)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        pos = g(mid) > 0
        hi = np.where(pos, mid, hi)
        lo = np.where(pos, lo, mid)
    return 0.5 * (lo + hi)[:, None] * u


def test_sdf_grid_distance_transform_against_brute_force(orc):
    """On a 14^3 grid the values are (e - sqrt(3)) h with e the Euclidean distance between the voxel's centre and
    the nearest centre of a voxel that may hold surface, found here by brute force over all pairs."""
    A, k, n = 0.12, 7.0, 14
    grid, b, h = orc.sdf_grid(A, k, n)
    c = -b + (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    f = np.sqrt(x * x + y * y + z * z) - 1 - A * np.sin(k * x) * np.sin(k * y) * np.sin(k * z)
    marked = np.argwhere(np.abs(f) <= (1 + A * k) * np.sqrt(3) / 2 * h)
    assert 0 < len(marked) < n ** 3
    idx = np.argwhere(np.ones((n, n, n), bool))
    e = np.sqrt(((idx[:, None, :] - marked[None, :, :]) ** 2).sum(axis=2).min(axis=1)).reshape(n, n, n)
    assert np.allclose(grid, np.maximum(e - np.sqrt(3), 0) * h, rtol=0, atol=1e-12)


@pytest.mark.parametrize("A,k,n", [(0.1, 6.0, 32), (0.15, 10.0, 48), (0.1, 6.0, 96)])
def test_sdf_grid_is_conservative_and_useful(orc, A, k, n):
    """Every voxel value is at most the distance from any point of the voxel to the surface (checked at random
    points against the nearest of 100,000 surface points, an upper bound of the true distance), and deep inside
    it is above the global Lipschitz bound (the grid's reason to exist)."""
    grid, b, h = orc.sdf_grid(A, k, n)
    assert grid.shape == (n, n, n) and np.all(grid >= 0)
    surf = _surface_points(A, k, 100_000, 3)
    rng = np.random.default_rng(int(1000 * A + k))
    pts = rng.uniform(-1.0 - A, 1.0 + A, (1500, 3))
    idx = np.clip(np.floor((pts + b) / h).astype(int), 0, n - 1)
    gv = grid[idx[:, 2], idx[:, 1], idx[:, 0]]
    for i in range(0, len(pts), 250):
        p = pts[i:i + 250]
        d = np.sqrt(((p[:, None, :] - surf[None, :, :]) ** 2).sum(-1)).min(axis=1)
        assert np.all(gv[i:i + 250] <= d + 1e-12), (gv[i:i + 250] - d).max()
    c = np.clip(np.floor((np.zeros(3) + b) / h).astype(int), 0, n - 1)
    assert grid[c[2], c[1], c[0]] > (1.0 - A) / (1.0 + A * k)


def _radial_surface_points(f, n, rng):
    """n points on the displaced sphere: radial bisection of f along random directions."""
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    lo, hi = np.full(n, 0.5), np.full(n, 1.6)
    for _ in range(60):
        m = 0.5 * (lo + hi)
        neg = f(m[:, None] * u) < 0
        lo = np.where(neg, m, lo)
        hi = np.where(neg, hi, m)
    return lo[:, None] * u


def _disp_grad(A, k, p):
    s, c = np.sin(k * p), np.cos(k * p)
    return p / np.linalg.norm(p) - A * k * np.array([c[0] * s[1] * s[2], s[0] * c[1] * s[2], s[0] * s[1] * c[2]])


@pytest.mark.parametrize("A,k", [(0.1, 6.0), (0.2, 4.0), (0.05, 10.0)])
def test_band_step_never_crosses_and_is_tight(orc, A, k):
    """The march's step off the boundary band (a second-order bound on f along the ray) against dense sampling
    of f: from surface points, along directions that leave the surface at shallow angles on either side, the
    surface is never met within the step, and for the worst-curved of them the step reaches most of the way
    to where the ray does meet it again (at least 60 %).  A curvature bound too small by a third lets some rays
    cross; one three times too large keeps every step below 30 % of that distance."""
    rng = np.random.default_rng(int(10 * k))
    f = _disp_sdf(A, k)
    pts = _radial_surface_points(f, 1500, rng)
    best, checked = 0.0, 0
    for p in pts:
        n = _disp_grad(A, k, p)
        n /= np.linalg.norm(n)
        t = rng.standard_normal(3)
        t -= (t @ n) * n
        t /= np.linalg.norm(t)
        side = rng.choice([-1.0, 1.0])
        c = rng.uniform(0.01, 0.3)
        w = t * math.sqrt(1 - c * c) + side * c * n
        p0 = p + side * 1e-9 * n                     # on the chosen side of the surface, inside the band
        s = orc.band_step(A, k, p0, w)
        assert s >= 1e-4, (p0, w, s)
        tt = np.linspace(0.0, 3.0 * s, 6001)[1:]
        h = side * f(p0 + tt[:, None] * w)
        neg = np.nonzero(h < -1e-12)[0]
        if neg.size:
            assert tt[neg[0]] > s, (p0, w, s, tt[neg[0]])
            best = max(best, s / tt[neg[0]])
        checked += 1
    assert checked == len(pts)
    assert best > 0.6, best


def test_band_step_on_the_sphere(orc):
    """A = 0 (the unit sphere): outside, a ray leaving the sphere never returns, and the step is the cap (4);
    inside, a ray leaving the surface at cos theta to the inward normal meets it again after the chord
    2 cos theta, and the step stays within it and reaches at least a quarter of it (below the cap |p| / 2);
    a ray moving toward the surface reports a crossing (-1)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        t = rng.standard_normal(3)
        t -= (t @ u) * u
        t /= np.linalg.norm(t)
        c = rng.uniform(0.02, 1.0)
        w_out = c * u + math.sqrt(1 - c * c) * t
        assert orc.band_step(0.0, 6.0, (1 + 1e-9) * u, w_out) == 4.0
        w_in = -c * u + math.sqrt(1 - c * c) * t
        s = orc.band_step(0.0, 6.0, (1 - 1e-9) * u, w_in)
        assert s <= 2 * c and s >= min(0.5 * c, 0.5) - 1e-12, (c, s)
        assert orc.band_step(0.0, 6.0, (1 - 1e-9) * u, w_out) == -1.0


@pytest.mark.parametrize("A,k", [(0.1, 6.0), (0.2, 4.0), (0.05, 10.0)])
def test_march_step_never_crosses_and_closes_in(orc, A, k):
    """One march step (the largest of the Lipschitz, radial-plus-Lipschitz and curvature steps) against dense
    sampling of f, from points inside and outside at distances 1e-3 .. 0.3 from the surface in random
    directions: the surface is never met within the step.  Aimed at the surface along its normal from close
    by, the step covers nearly all of the gap (at least 90 % from 1e-3 .. 1e-2 away): the curvature step
    converges quadratically where the Lipschitz step alone would cover 1 / (1 + A k) of it."""
    rng = np.random.default_rng(int(7 * k))
    f = _disp_sdf(A, k)
    surf = _radial_surface_points(f, 600, rng)
    checked = 0
    for p in surf:
        n = _disp_grad(A, k, p)
        n /= np.linalg.norm(n)
        side = rng.choice([-1.0, 1.0])
        gap = 10 ** rng.uniform(-3, math.log10(0.3))
        x = p + side * gap * n
        if side * f(x) < 2e-4:
            continue                                    # not on the chosen side at that distance
        w = rng.standard_normal(3)
        w /= np.linalg.norm(w)
        s = orc.march_step(A, k, x, w)
        if s == math.inf:
            assert side > 0                             # escape: outside only, and never meets the surface
            tt = np.linspace(0.0, 6.0, 60001)[1:]
            assert np.all(f(x + tt[:, None] * w) > -1e-12), (x, w)
            continue
        assert s > 0, (x, w, s)
        tt = np.linspace(0.0, s, 4001)[1:]
        assert np.all(side * f(x + tt[:, None] * w) > -1e-12), (x, w, s)
        checked += 1
    assert checked > 300
    ratios = []
    for p in surf[:200]:
        n = _disp_grad(A, k, p)
        n /= np.linalg.norm(n)
        for side in (-1.0, 1.0):
            x = p + side * rng.uniform(1e-3, 1e-2) * n
            w = -side * n
            tt = np.linspace(0.0, 0.05, 50001)
            h = side * f(x + tt[:, None] * w)
            cross = tt[np.nonzero(h < 0)[0][0]]
            ratios.append(orc.march_step(A, k, x, w) / cross)
    ratios = np.array(ratios)
    assert ratios.max() < 1.0 and np.median(ratios) > 0.9, (ratios.max(), np.median(ratios))


@pytest.mark.parametrize("mode", [0, 1])
def test_render_pixels_equal_the_whole_image(orc, mode):
    """Rendering selected pixels one by one uses exactly the whole image's streams: the values equal the full
    render's pixels bit for bit, in both modes (the check of full-size renders at sampled pixels rests on it)."""
    decs = None
    if mode:
        decs = [(synth.xavier_decoder(100 + i, *shape).astype(np.float64), *shape)
                for i, shape in enumerate(synth.MODEL_SHAPES.values())]
    p = synth.render_scene(48.0, width=20, height=14, spp=3, mode=mode, seed=5)
    img, _, _ = orc.render(p, decs)
    pix = np.array([0, 7, 131, 139, 150, 279])
    v, _ = orc.render_pixels(p, pix, decs)
    assert np.array_equal(v, img.reshape(-1)[pix])
