"""Seeded synthetic inputs shared by the CUDA path's callers and by the oracle's tests.

This module only draws inputs (media, decoder queries, initial weights, scene parameters) from numpy
generators; it contains none of the method's arithmetic.  The random numbers the method itself draws
(free paths, roulette, HG sampling, latent and posterior normals) come from the counter-based Philox
stream that each side implements on its own.

Workloads (the shapes of the paper's experiments, Sec. 5, with synthetic stand-ins for its meshes):
* ``walk_cfg``        65,536 photons, optical radius 8, g 0.8, albedo 0.999, isotropic start, seed 1
* ``decoder_queries`` condition (log optical radius U[0,6], g U[0,0.95], albedo U[0.9,1], cosine U[-1,1])
* ``training_media``  optical radius log-uniform in [1,256], g U[-1,1), albedo U[0.9,1]
* ``render_scene``    displaced unit sphere 0.1 sin(6x) sin(6y) sin(6z), point light, g 0.8, albedo 0.999
* ``batch_requests``  heterogeneous render requests (resolution, spp, density, g, albedo, frequency)
"""
from __future__ import annotations

import numpy as np

# Model shapes (P_in, P_out) of the three learned samplers (Eq. 3): LengthGen, PathGen, EventGen.
# (p_in, p_out, latent, width) of the three CVAEs: the final settings of Table 1 (D = 2 hidden layers)
MODEL_SHAPES = {"length": (2, 1, 2, 8), "path": (3, 3, 5, 16), "event": (7, 6, 5, 16)}
# defaults of the generic helpers (and of the decoder benchmark's condition-4 decoders)
LATENT = 4
WIDTH = 16


def xavier_mlp(rng: np.random.Generator, n_in: int, width: int, n_out: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases, packed W1,b1,W2,b2,W3,b3 (row-major [out][in]) as float32."""
    parts = []
    for fi, fo in ((n_in, width), (width, width), (width, n_out)):
        a = np.sqrt(6.0 / (fi + fo))
        parts.append(rng.uniform(-a, a, size=(fo, fi)).ravel())
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def xavier_decoder(seed: int, p_in: int, p_out: int, latent: int = LATENT, width: int = WIDTH) -> np.ndarray:
    return xavier_mlp(np.random.default_rng(seed), p_in + latent, width, 2 * p_out)


def xavier_cvae(seed: int, p_in: int, p_out: int, latent: int = LATENT, width: int = WIDTH) -> np.ndarray:
    """Encoder block (input [x;c], output 2L) followed by the decoder block (input [c;z], output 2P_out)."""
    rng = np.random.default_rng(seed)
    enc = xavier_mlp(rng, p_out + p_in, width, 2 * latent)
    dec = xavier_mlp(rng, p_in + latent, width, 2 * p_out)
    return np.concatenate([enc, dec])


def decoder_queries(seed: int, n: int) -> np.ndarray:
    """[n][4] float32 conditions: log optical radius U[0,6], g U[0,0.95], albedo U[0.9,1], cosine U[-1,1]."""
    rng = np.random.default_rng(seed)
    c = np.empty((n, 4), np.float32)
    c[:, 0] = rng.uniform(0.0, 6.0, n)
    c[:, 1] = rng.uniform(0.0, 0.95, n)
    c[:, 2] = rng.uniform(0.9, 1.0, n)
    c[:, 3] = rng.uniform(-1.0, 1.0, n)
    return c


def standard_normals(seed: int, shape) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape).astype(np.float32)


def walk_cfg() -> dict:
    return dict(seed=1, n_photons=65536, optical_radius=8.0, g=0.8, albedo=0.999,
                dir_in=(0.0, 0.0, 1.0), isotropic_start=1, first_event_at_origin=0)


def training_media(seed: int, n: int):
    """Per-walk media: optical radius log-uniform in [1,256], g U[-1,1) (the anisotropy range of the paper's
    training set, Sec. 5), albedo U[0.9,1]."""
    rng = np.random.default_rng(seed)
    tau = np.exp(rng.uniform(0.0, np.log(256.0), n))
    g = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.9, 1.0, n)
    return tau, g, phi


def render_scene(sigma_t: float, *, width=512, height=512, spp=256, mode=1, seed=1, sample_offset=0,
                 g=0.8, albedo=0.999, disp_amp=0.1, disp_freq=6.0, max_segments=1 << 20) -> dict:
    """Displaced-sphere scene: camera at (0,0,3) looking at the origin, 40 degree vertical field of view,
    point light of intensity 10 at (2,2,3)."""
    return dict(width=width, height=height, spp=spp, max_segments=max_segments,
                cam_pos=(0.0, 0.0, 3.0), cam_at=(0.0, 0.0, 0.0), fov_y_deg=40.0,
                light_pos=(2.0, 2.0, 3.0), light_I=10.0, sigma_t=float(sigma_t), g=g, albedo=albedo,
                disp_amp=disp_amp, disp_freq=disp_freq, mode=mode,
                min_optical_radius=1.0, max_optical_radius=256.0, seed=seed, sample_offset=sample_offset)


def batch_requests(seed: int, n: int = 64, scale: float = 1.0) -> list:
    """Heterogeneous requests: resolution from {128,256,512,1024}^2, spp from {64,256,1024}, sigma_t
    log-uniform in [8,1024], g U[0.5,0.95], albedo U[0.95,1], displacement frequency U[2,10].
    ``scale`` < 1 shrinks resolutions and spp for tests."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        res = int(rng.choice([128, 256, 512, 1024]))
        spp = int(rng.choice([64, 256, 1024]))
        res = max(4, int(res * scale))
        spp = max(1, int(spp * scale))
        out.append(render_scene(float(np.exp(rng.uniform(np.log(8.0), np.log(1024.0)))), width=res, height=res,
                                spp=spp, g=float(rng.uniform(0.5, 0.95)), albedo=float(rng.uniform(0.95, 1.0)),
                                disp_freq=float(rng.uniform(2.0, 10.0)), seed=int(rng.integers(1, 2**31))))
    return out
