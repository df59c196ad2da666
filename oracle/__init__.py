"""CPU oracle of the learned sphere-tracing method — TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 restatement of what the CUDA library computes, written from the paper and sharing no
code with the library:

* ``rng.c``      Philox4x32-10 counter generator (published definition)
* ``detmath.c``  log / sincos / atan2 from IEEE basic operations (bit-reproducible walk decisions)
* ``walk.c``     brute-force HG random walk in the unit sphere (Sec. 3.1, Sec. 4.3 reservoir)
* ``render.c``   sphere-traced and brute-force rendering with next-event estimation (Sec. 3, 4.1, 4.3)
* ``cvae.py``    CVAE decoder, negative ELBO, analytic backward, Adam, training targets (Sec. 3.2, 4.1)

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
LIB_PATH = HERE / "libms_oracle.so"
SOURCES = ["rng.c", "detmath.c", "walk.c", "render.c"]

_lib = None


def build(force: bool = False) -> Path:
    """Compile the C part of the oracle (no FMA contraction, so the FP64 walk is bit-reproducible)."""
    srcs = [HERE / s for s in SOURCES]
    newest = max(s.stat().st_mtime for s in srcs + [HERE / "oracle.h"])
    if not force and LIB_PATH.exists() and LIB_PATH.stat().st_mtime >= newest:
        return LIB_PATH
    tmp = LIB_PATH.with_suffix(f".so.tmp{os.getpid()}")
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
           "-o", str(tmp)] + [str(s) for s in srcs] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Medium(C.Structure):
    _fields_ = [("optical_radius", C.c_double), ("g", C.c_double), ("albedo", C.c_double),
                ("dir_in", C.c_double * 3), ("isotropic_start", C.c_int32),
                ("first_event_at_origin", C.c_int32)]


MEDIUM_DTYPE = np.dtype([("optical_radius", "<f8"), ("g", "<f8"), ("albedo", "<f8"), ("dir_in", "<f8", (3,)),
                         ("isotropic_start", "<i4"), ("first_event_at_origin", "<i4")])
assert MEDIUM_DTYPE.itemsize == C.sizeof(Medium)


class Decoder(C.Structure):
    _fields_ = [("p_in", C.c_int32), ("latent", C.c_int32), ("width", C.c_int32), ("p_out", C.c_int32),
                ("w", C.POINTER(C.c_double))]


class RenderParams(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_uint32), ("max_segments", C.c_uint32),
                ("cam_pos", C.c_double * 3), ("cam_at", C.c_double * 3), ("fov_y_deg", C.c_double),
                ("light_pos", C.c_double * 3), ("light_I", C.c_double),
                ("sigma_t", C.c_double), ("g", C.c_double), ("albedo", C.c_double),
                ("disp_amp", C.c_double), ("disp_freq", C.c_double),
                ("mode", C.c_int32), ("sdf_grid_n", C.c_int32), ("march_mode", C.c_int32),
                ("max_march", C.c_int32), ("exact_n1", C.c_int32), ("exact_centre", C.c_int32),
                ("min_optical_radius", C.c_double), ("max_optical_radius", C.c_double),
                ("seed", C.c_uint64), ("sample_offset", C.c_uint64), ("sdf_grid", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(LIB_PATH))
        P = C.c_void_p
        L.om_philox.argtypes = [P, P, P]
        L.om_philox_words.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, P]
        L.om_log.argtypes = [C.c_double]
        L.om_log.restype = C.c_double
        L.om_sincos_turns.argtypes = [C.c_double, P, P]
        L.om_atan2.argtypes = [C.c_double, C.c_double]
        L.om_atan2.restype = C.c_double
        L.om_walk.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, P, C.c_int, C.c_uint32, C.c_int, C.c_int,
                              P, P, P, P, P, P, P, P, P, P, P, C.c_int]
        L.om_walk.restype = C.c_int
        L.om_render.argtypes = [P, P, P, P, C.c_int]
        L.om_render.restype = C.c_int
        L.om_render_pixels.argtypes = [P, P, P, C.c_int, P, P, C.c_int]
        L.om_render_pixels.restype = C.c_int
        L.om_decoder_sample.argtypes = [P, P, P, P, P]
        L.om_hg_cosine.argtypes = [C.c_double, C.c_double]
        L.om_hg_cosine.restype = C.c_double
        L.om_scatter_dir.argtypes = [P, C.c_double, C.c_double, P]
        L.om_inside_length.argtypes = [C.c_double, C.c_double, P, P]
        L.om_inside_length.restype = C.c_double
        L.om_ray_crossing.argtypes = [C.c_double, C.c_double, P, P, P, C.c_int]
        L.om_ray_crossing.restype = C.c_int
        L.om_band_step.argtypes = [C.c_double, C.c_double, P, P]
        L.om_band_step.restype = C.c_double
        L.om_march_step.argtypes = [C.c_double, C.c_double, P, P]
        L.om_march_step.restype = C.c_double
        L.om_walk_nee.argtypes = [C.c_uint64, C.c_uint64, C.c_double, C.c_double, C.c_double, P, P, P, P, P, P,
                                  C.c_int]
        L.om_walk_nee.restype = C.c_int
        L.om_set_plant.argtypes = [C.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- RNG and deterministic math

def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().om_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_words(seed, id0, n, step, tag):
    out = np.zeros((n, 4), np.uint32)
    lib().om_philox_words(seed, id0, n, step, tag, _ptr(out))
    return out


def u24(words):
    return (np.asarray(words, np.uint32) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24


def det_log(x):
    return np.array([lib().om_log(float(v)) for v in np.ravel(x)])


def det_sincos_turns(u):
    s, c = C.c_double(), C.c_double()
    out = []
    for v in np.ravel(u):
        lib().om_sincos_turns(float(v), C.byref(s), C.byref(c))
        out.append((s.value, c.value))
    return np.array(out)


def det_atan2(y, x):
    return np.array([lib().om_atan2(float(a), float(b)) for a, b in zip(np.ravel(y), np.ravel(x))])


def hg_cosine(u, g):
    return np.array([lib().om_hg_cosine(float(v), float(g)) for v in np.ravel(u)])


def scatter_dir(w, mu, u):
    w = np.ascontiguousarray(w, np.float64)
    out = np.zeros(3)
    lib().om_scatter_dir(_ptr(w), float(mu), float(u), _ptr(out))
    return out


def normals_from_words(words):
    """Box-Muller on 24-bit uniforms: word pairs (w0,w1), (w2,w3) -> four normals per row."""
    u = u24(words)
    out = np.empty_like(u)
    for pair in range(2):
        ua, ub = u[:, 2 * pair], u[:, 2 * pair + 1]
        r = np.sqrt(-2.0 * np.log(1.0 - ua))
        out[:, 2 * pair] = r * np.cos(2.0 * np.pi * ub)
        out[:, 2 * pair + 1] = r * np.sin(2.0 * np.pi * ub)
    return out


def decoder_normals(seed, offset, n, count):
    """Latent and posterior normals of the decoder queries offset..offset+n-1 (the input layout of the decoder
    workload, stated in include/ms.h): B Philox blocks, counter (j, id_lo, id_hi, 0xD0) for j < B, where B is the
    fewest blocks whose 4B words give 2 ceil(count/2) uniforms when every word gives a 24-bit uniform from its
    top bits and every three words give one more from their low bytes.  Uniforms in order: the top bits of words
    0..4B-1, then the low bytes of words (0,1,2), (3,4,5), ...; normals 2m, 2m+1 are Box-Muller on uniforms 2m,
    2m+1.  Returns [n][count]."""
    need = count + (count & 1)
    nb = 1
    while 4 * nb + (4 * nb) // 3 < need:
        nb += 1
    words = np.concatenate([philox_words(seed, offset, n, j, 0xD0) for j in range(nb)], axis=1)   # [n][4B]
    top = u24(words)
    low = (words & np.uint32(0xFF)).astype(np.uint64)
    spare = [((low[:, 3 * i] << 16) | (low[:, 3 * i + 1] << 8) | low[:, 3 * i + 2]).astype(np.float64) * 2.0 ** -24
             for i in range((4 * nb) // 3)]
    u = np.concatenate([top] + [s[:, None] for s in spare], axis=1)[:, :need]
    out = np.empty((n, need))
    for m in range(need // 2):
        ua, ub = u[:, 2 * m], u[:, 2 * m + 1]
        r = np.sqrt(-2.0 * np.log(1.0 - ua))
        out[:, 2 * m] = r * np.cos(2.0 * np.pi * ub)
        out[:, 2 * m + 1] = r * np.sin(2.0 * np.pi * ub)
    return out[:, :count]


# ---------------------------------------------------------------- walk

def walk(seed, n_photons, media, *, photon_offset=0, max_events=1 << 20, reservoir_mode=0, uniform_bits=53,
         per_photon=True, n_threads=0):
    """Run the oracle walk.  ``media`` is a dict of scalars or of length-n arrays with keys optical_radius,
    g, albedo, dir_in ([3] or [n][3]), isotropic_start, first_event_at_origin."""
    per_media = any(np.ndim(media[k]) > (1 if k == "dir_in" else 0) for k in media)
    n_media = n_photons if per_media else 1
    arr = np.zeros(max(n_media, 1), dtype=MEDIUM_DTYPE)
    for k in ("optical_radius", "g", "albedo", "isotropic_start", "first_event_at_origin"):
        arr[k] = np.broadcast_to(np.asarray(media[k]), (n_media,))
    arr["dir_in"] = np.broadcast_to(np.asarray(media["dir_in"], np.float64), (n_media, 3))
    out = dict(hist_n=np.zeros(64, np.uint64), hist_pos=np.zeros((32, 64), np.uint64),
               hist_cos=np.zeros(64, np.uint64), counters=np.zeros(8, np.uint64))
    if per_photon:
        out.update(n_events=np.zeros(n_photons, np.int32), status=np.zeros(n_photons, np.uint8),
                   exit_pos=np.zeros((n_photons, 3)), exit_dir=np.zeros((n_photons, 3)),
                   rep_pos=np.zeros((n_photons, 3)), rep_dir=np.zeros((n_photons, 3)),
                   rep_index=np.zeros(n_photons, np.int32))
    g = out.get
    out["threads"] = lib().om_walk(
        seed, photon_offset, n_photons, _ptr(arr), int(per_media), max_events,
        reservoir_mode, uniform_bits, _ptr(g("n_events")), _ptr(g("status")), _ptr(g("exit_pos")),
        _ptr(g("exit_dir")), _ptr(g("rep_pos")), _ptr(g("rep_dir")), _ptr(g("rep_index")), _ptr(out["hist_n"]),
        _ptr(out["hist_pos"]), _ptr(out["hist_cos"]), _ptr(out["counters"]), n_threads)
    return out


def walk_nee(seed, n_photons, tau, g, phi, light, n_threads=0):
    """Training-record walks (paper convention, w_in = (0,0,1), albedo-1 physics, representative event with
    weights phi^k) with, per photon, the brute-force next-event sum over all events toward a point light at
    ``light`` (outside the unit sphere): sum_k phi^k rho_g(W_k . w_L) exp(-tau d_k) / |x_L - X_k|^2.  Returns
    dict(n_events, rep_pos, rep_dir, rep_index, nee_sum)."""
    xl = np.ascontiguousarray(light, np.float64)
    out = dict(n_events=np.zeros(n_photons, np.int32), rep_pos=np.zeros((n_photons, 3)),
               rep_dir=np.zeros((n_photons, 3)), rep_index=np.zeros(n_photons, np.int32),
               nee_sum=np.zeros(n_photons))
    lib().om_walk_nee(seed, n_photons, tau, g, phi, _ptr(xl), _ptr(out["n_events"]), _ptr(out["rep_pos"]),
                      _ptr(out["rep_dir"]), _ptr(out["rep_index"]), _ptr(out["nee_sum"]), n_threads)
    return out


def set_plant(k: int):
    """Test hook: plant a deliberate mistake in the renderer's sphere step (0 removes it); see render.c."""
    lib().om_set_plant(int(k))


# ---------------------------------------------------------------- renderer

def _decoder_struct(wvec, p_in, p_out, latent=4, width=16):
    w = np.ascontiguousarray(np.asarray(wvec, np.float64))
    return Decoder(p_in, latent, width, p_out, w.ctypes.data_as(C.POINTER(C.c_double))), w


def _render_setup(params: dict, decoders):
    """RenderParams and decoder structs for ``params`` (keys follow RenderParams) and ``decoders``; the arrays
    in the returned list must outlive the call."""
    P = RenderParams()
    for k, v in params.items():
        if k == "sdf_grid":
            continue            # the oracle builds its own grid (sdf_grid_n); never take a device pointer
        if isinstance(getattr(P, k), C.Array):
            setattr(P, k, type(getattr(P, k))(*[float(t) for t in v]))
        else:
            setattr(P, k, v)
    keep = []
    if params.get("sdf_grid_n", 0) and params.get("mode", 0) != 0:
        g, _, _ = sdf_grid(P.disp_amp, P.disp_freq, int(params["sdf_grid_n"]))
        g = np.ascontiguousarray(g)
        keep.append(g)
        P.sdf_grid = g.ctypes.data
    decs = (Decoder * 3)()
    if decoders is not None:
        for i, dd in enumerate(decoders):
            d, arr = _decoder_struct(*dd)
            decs[i] = d
            keep.append(arr)
    return P, decs, keep


def render(params: dict, decoders=None, n_threads=0):
    """Render; ``params`` keys follow RenderParams; ``decoders`` is a list of three (weights, p_in, p_out) or
    (weights, p_in, p_out, latent, width) for LengthGen, PathGen, EventGen (latent 4, width 16 when not given).
    mode 0 is brute force, 1 sphere tracing with the decoders, 2 sphere tracing with the exact sampler (a walk
    in the sphere in place of the decoders; no decoders needed); march_mode 1 marches with the Lipschitz step
    alone (give a larger max_march).
    Returns (image_sum[h][w], stats[16], threads)."""
    P, decs, keep = _render_setup(params, decoders)
    image = np.zeros((P.height, P.width), np.float64)
    stats = np.zeros(16, np.uint64)
    nt = lib().om_render(C.byref(P), C.cast(decs, C.c_void_p), _ptr(image), _ptr(stats), n_threads)
    if nt < 0:
        raise ValueError("om_render: the decoders need more than 24 normals per sphere step, or are too wide")
    return image, stats, nt


def render_pixels(params: dict, pixels, decoders=None, n_threads=0):
    """The same render restricted to the pixels with flat indices ``pixels`` (py * width + px): returns
    (their sums over the spp samples, stats[16] of those paths), on the streams the whole image uses."""
    P, decs, keep = _render_setup(params, decoders)
    pix = np.ascontiguousarray(pixels, np.int64)
    values = np.zeros(pix.size, np.float64)
    stats = np.zeros(16, np.uint64)
    nt = lib().om_render_pixels(C.byref(P), C.cast(decs, C.c_void_p), _ptr(pix), int(pix.size), _ptr(values),
                                _ptr(stats), n_threads)
    if nt < 0:
        raise ValueError("om_render_pixels: bad pixel index or decoders")
    return values, stats


def decoder_sample_one(wvec, p_in, p_out, c, z, eps):
    d, arr = _decoder_struct(wvec, p_in, p_out)
    c = np.ascontiguousarray(c, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    e = np.ascontiguousarray(eps, np.float64)
    x = np.zeros(p_out)
    lib().om_decoder_sample(C.byref(d), _ptr(c), _ptr(z), _ptr(e), _ptr(x))
    return x


def inside_length(A, k, X, xl):
    X = np.ascontiguousarray(X, np.float64)
    xl = np.ascontiguousarray(xl, np.float64)
    return lib().om_inside_length(A, k, _ptr(X), _ptr(xl))


def sdf_grid(A, k, n):
    """Voxel grid of conservative distances to the displaced sphere (Sec. 3: the bounding volume voxelised in a
    pre-process, each voxel holding a conservative shortest distance to the surface).  The cube [-b, b]^3,
    h = 2 (1 + A) / (n - 2), b = 1 + A + h, in n^3 voxels (index [iz][iy][ix]):
      1. a voxel may hold surface if |f(c)| <= (1 + A k) h sqrt(3) / 2 at its centre c (f's Lipschitz constant
         is 1 + A k, and no point of the voxel is farther than h sqrt(3) / 2 from c);
      2. e = the Euclidean distance, in voxels, from each voxel's centre to the nearest such voxel's centre
         (scipy's exact Euclidean distance transform);
      3. value = (e - sqrt(3)) h, at least 0 (points of two voxels are at most one diagonal nearer than their
         centres).
    Returns (grid, b, h)."""
    from scipy import ndimage
    h = 2.0 * (1.0 + A) / (n - 2)
    b = 1.0 + A + h
    c = -b + (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    f = np.sqrt(x * x + y * y + z * z) - 1.0 - A * np.sin(k * x) * np.sin(k * y) * np.sin(k * z)
    may_hold = np.abs(f) <= (1.0 + A * k) * (np.sqrt(3.0) / 2.0) * h
    e = ndimage.distance_transform_edt(~may_hold)
    return np.maximum(0.0, (e - np.sqrt(3.0)) * h), b, h


def band_step(A, k, p, w):
    """The march's step from a point p of the boundary band along w, on the side of f(p); -1 when the ray
    moves toward the surface (a crossing)."""
    p = np.ascontiguousarray(p, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    return float(lib().om_band_step(A, k, _ptr(p), _ptr(w)))


def march_step(A, k, p, w):
    """One step of the march from p along w on the side of f(p): -1 for a crossing of the boundary band,
    inf when the surface cannot be reached (outside)."""
    p = np.ascontiguousarray(p, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    return float(lib().om_march_step(A, k, _ptr(p), _ptr(w)))


def ray_crossing(A, k, p, w, plain=False):
    """First boundary crossing along p + t w of the displaced sphere: (status, t) with status 1 crossing,
    0 escape (outside rays only), 2 step cap; ``plain`` marches with the Lipschitz step alone."""
    p = np.ascontiguousarray(p, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    t = np.zeros(1)
    r = lib().om_ray_crossing(A, k, _ptr(p), _ptr(w), _ptr(t), int(bool(plain)))
    return r, float(t[0])
