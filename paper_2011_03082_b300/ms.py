"""Thin Python binding of the C ABI in ``include/ms.h`` (libms.so).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.  Tensors are
PyTorch CUDA tensors (PyTorch provides device memory and streams); the functions pass their device pointers
and the current CUDA stream to the library.  There is no CPU fallback: if ``libms.so`` cannot be loaded the
functions raise.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np
import torch

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "libms.so"

MS_FP32, MS_FP64, MS_FP16, MS_BF16 = 0, 1, 2, 3
MS_BRUTE, MS_SPHERE = 0, 1
MS_ESCAPED, MS_ABSORBED, MS_TRUNCATED = 0, 1, 2
MS_RENDER_STATS = 16

# the C ABI's exported symbols (checked by the tests against include/ms.h)
EXPORTS = ("ms_last_error", "ms_version", "ms_walk_workspace_size", "ms_simulate_walks", "ms_cvae_infer",
           "ms_cvae_num_params", "ms_cvae_workspace_size", "ms_cvae_forward", "ms_cvae_forward_backward",
           "ms_adam_step", "ms_cvae_train_step", "ms_cvae_train_step_dev_workspace_size", "ms_cvae_train_step_dev",
           "ms_cvae_static_scratch_bytes", "ms_cvae_train_step_static", "ms_training_records",
           "ms_render_workspace_size", "ms_render", "ms_render_batch", "ms_render_default_min_optical_radius",
           "ms_render_variants", "ms_render_variant_info", "ms_render_autotune", "ms_sdf_grid_workspace_size",
           "ms_sdf_grid_build", "ms_alu_peaks_scratch_bytes", "ms_alu_peaks")
PEAK_NAMES = ("ffma", "ex2", "lg2", "sin", "rsqrt", "imad", "lop3", "imulhi")


class MsError(RuntimeError):
    pass


class Medium(C.Structure):
    _fields_ = [("optical_radius", C.c_float), ("g", C.c_float), ("albedo", C.c_float), ("dir_in", C.c_float * 3),
                ("isotropic_start", C.c_int32), ("first_event_at_origin", C.c_int32)]


MEDIUM_DTYPE = np.dtype([("optical_radius", "<f4"), ("g", "<f4"), ("albedo", "<f4"), ("dir_in", "<f4", (3,)),
                         ("isotropic_start", "<i4"), ("first_event_at_origin", "<i4")])
assert MEDIUM_DTYPE.itemsize == C.sizeof(Medium) == 32


class WalkParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("photon_offset", C.c_uint64), ("n_photons", C.c_uint64),
                ("media", C.c_void_p), ("per_photon_media", C.c_int32), ("max_events", C.c_uint32),
                ("reservoir", C.c_int32), ("precision", C.c_int32)]


class WalkOut(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("n_events", "status", "exit_pos", "exit_dir", "rep_pos", "rep_dir",
                                          "rep_index", "hist_n", "hist_pos", "hist_cos", "counters")]


class Decoder(C.Structure):
    _fields_ = [("p_in", C.c_int32), ("latent", C.c_int32), ("width", C.c_int32), ("p_out", C.c_int32),
                ("precision", C.c_int32), ("weights", C.c_void_p)]


class CvaeShape(C.Structure):
    _fields_ = [("p_in", C.c_int32), ("p_out", C.c_int32), ("latent", C.c_int32), ("width", C.c_int32),
                ("precision", C.c_int32)]


class RenderParams(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("spp", C.c_uint32), ("max_segments", C.c_uint32),
                ("cam_pos", C.c_float * 3), ("cam_at", C.c_float * 3), ("fov_y_deg", C.c_float),
                ("light_pos", C.c_float * 3), ("light_I", C.c_float),
                ("sigma_t", C.c_float), ("g", C.c_float), ("albedo", C.c_float),
                ("disp_amp", C.c_float), ("disp_freq", C.c_float), ("mode", C.c_int32),
                ("min_optical_radius", C.c_float), ("max_optical_radius", C.c_float),
                ("seed", C.c_uint64), ("sample_offset", C.c_uint64), ("variant", C.c_int32),
                ("sdf_grid_n", C.c_int32), ("sdf_grid", C.c_void_p), ("exact_n1", C.c_int32),
                ("phase_timers", C.c_int32), ("exact_centre", C.c_int32)]


class CvaeSet(C.Structure):
    _fields_ = [("length", Decoder), ("path", Decoder), ("event", Decoder)]


_lib = None


def lib():
    """Load libms.so (raises MsError if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise MsError(f"{LIB_PATH} is missing; build it with paper_2011_03082_b300.build.build()")
    L = C.CDLL(str(LIB_PATH))
    P, U64, I32, F = C.c_void_p, C.c_uint64, C.c_int32, C.c_float
    sig = {
        "ms_last_error": ([], C.c_char_p),
        "ms_version": ([], C.c_int),
        "ms_walk_workspace_size": ([P], C.c_size_t),
        "ms_simulate_walks": ([P, P, P, C.c_size_t, P], C.c_int),
        "ms_cvae_infer": ([P, P, P, U64, U64, U64, P, P, P], C.c_int),
        "ms_cvae_num_params": ([P], C.c_size_t),
        "ms_cvae_workspace_size": ([P, U64], C.c_size_t),
        "ms_cvae_forward": ([P, P, P, P, P, U64, U64, U64, P, P, C.c_size_t, P], C.c_int),
        "ms_cvae_forward_backward": ([P, P, P, P, P, U64, U64, U64, P, P, P, C.c_size_t, P], C.c_int),
        "ms_adam_step": ([P, P, P, P, U64, U64, F, F, F, F, F, P], C.c_int),
        "ms_cvae_train_step": ([P, P, P, P, P, P, P, U64, U64, U64, F, F, P, P, C.c_size_t, P], C.c_int),
        "ms_cvae_train_step_dev_workspace_size": ([P, U64], C.c_size_t),
        "ms_cvae_train_step_dev": ([P, P, P, P, P, P, U64, U64, U64, P, F, F, P, P, C.c_size_t, P], C.c_int),
        "ms_cvae_static_scratch_bytes": ([], C.c_size_t),
        "ms_cvae_train_step_static": ([P, P, P, P, P, P, P, U64, U64, U64, F, F, P, P], C.c_int),
        "ms_training_records": ([U64, P, P, P, P, P, P, I32, U64, P, P, P, P, P, P, P], C.c_int),
        "ms_render_workspace_size": ([P, C.c_int], C.c_size_t),
        "ms_sdf_grid_workspace_size": ([I32], C.c_size_t),
        "ms_sdf_grid_build": ([C.c_float, C.c_float, I32, P, P, C.c_size_t, P], C.c_int),
        "ms_render": ([P, P, P, P, P, C.c_size_t, P], C.c_int),
        "ms_render_batch": ([P, C.c_int, P, P, P, P, C.c_size_t, P], C.c_int),
        "ms_render_default_min_optical_radius": ([C.c_float], C.c_float),
        "ms_render_variants": ([], C.c_int),
        "ms_render_variant_info": ([C.c_int, P, P, P, P], C.c_int),
        "ms_render_autotune": ([P, C.c_int, P, P, P, P, C.c_size_t, C.c_int, P, P, P], C.c_int),
        "ms_alu_peaks_scratch_bytes": ([], C.c_size_t),
        "ms_alu_peaks": ([P, P, C.c_size_t, P], C.c_int),
    }
    for name, (args, res) in sig.items():
        if not hasattr(L, name):
            continue
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status: int, what: str):
    if status < 0:
        raise MsError(f"{what} failed ({status}): {lib().ms_last_error().decode()}")
    return status


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise MsError("device tensor expected")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Caller-owned scratch (256-byte aligned by the CUDA caching allocator)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


# ------------------------------------------------------------------------------------------------ walks

def media_tensor(optical_radius, g, albedo, dir_in=(0.0, 0.0, 1.0), isotropic_start=0, first_event_at_origin=1,
                 n=None, device="cuda") -> torch.Tensor:
    """Pack media (scalars or arrays) into a device array of ms_medium (32 bytes each)."""
    scal = [np.ndim(v) == 0 for v in (optical_radius, g, albedo, isotropic_start, first_event_at_origin)]
    if n is None:
        n = 1 if all(scal) and np.ndim(dir_in) == 1 else max(
            len(np.atleast_1d(v)) for v in (optical_radius, g, albedo))
    a = np.zeros(n, MEDIUM_DTYPE)
    a["optical_radius"], a["g"], a["albedo"] = optical_radius, g, albedo
    a["dir_in"] = np.broadcast_to(np.asarray(dir_in, np.float32), (n, 3))
    a["isotropic_start"], a["first_event_at_origin"] = isotropic_start, first_event_at_origin
    return torch.from_numpy(a.view(np.uint8).copy()).to(device)


def walk_outputs(n: int, per_photon: bool = True, device="cuda") -> dict:
    z = lambda *s, dt=torch.float32: torch.zeros(*s, dtype=dt, device=device)
    out = dict(hist_n=z(64, dt=torch.int64), hist_pos=z(32, 64, dt=torch.int64), hist_cos=z(64, dt=torch.int64),
               counters=z(8, dt=torch.int64))
    if per_photon:
        out.update(n_events=z(n, dt=torch.int32), status=z(n, dt=torch.uint8), exit_pos=z(n, 3), exit_dir=z(n, 3),
                   rep_pos=z(n, 3), rep_dir=z(n, 3), rep_index=z(n, dt=torch.int32))
    return out


def ms_simulate_walks(media: torch.Tensor, n_photons: int, out: dict, *, seed=1, photon_offset=0,
                      max_events=1 << 20, reservoir=0, precision=MS_FP32, ws=None, stream=None):
    n_media = media.numel() // 32
    p = WalkParams(seed, photon_offset, n_photons, _ptr(media).value, int(n_media > 1), max_events, reservoir,
                   precision)
    o = WalkOut(*[_ptr(out.get(k)).value if out.get(k) is not None else None for k, _ in WalkOut._fields_])
    if ws is None:
        ws = workspace(lib().ms_walk_workspace_size(C.byref(p)), media.device)
    return _check(lib().ms_simulate_walks(C.byref(p), C.byref(o), _ptr(ws), ws.numel(), _stream(stream)),
                  "ms_simulate_walks")


# ------------------------------------------------------------------------------------------------ decoders

def decoder_struct(weights: torch.Tensor, p_in, p_out, latent=4, width=16, precision=MS_FP32) -> Decoder:
    d = Decoder(p_in, latent, width, p_out, precision, _ptr(weights).value)
    d._owned = weights
    return d


def ms_cvae_infer(dec: Decoder, cond: torch.Tensor, n: int, *, z_eps=None, seed=7, offset=0, out_mean_logvar=None,
                  out_sample=None, stream=None):
    return _check(lib().ms_cvae_infer(C.byref(dec), _ptr(cond), _ptr(z_eps), seed, offset, n, _ptr(out_mean_logvar),
                                      _ptr(out_sample), _stream(stream)), "ms_cvae_infer")


# ------------------------------------------------------------------------------------------------ training

def cvae_shape(p_in, p_out, latent=4, width=16, precision=MS_FP32) -> CvaeShape:
    return CvaeShape(p_in, p_out, latent, width, precision)


def ms_cvae_num_params(shape: CvaeShape) -> int:
    return int(lib().ms_cvae_num_params(C.byref(shape)))


def ms_cvae_workspace_size(shape: CvaeShape, batch: int) -> int:
    return int(lib().ms_cvae_workspace_size(C.byref(shape), batch))


def ms_cvae_forward_backward(shape, params, x, c, B, *, eps_z=None, seed=1, step=0, grad=None, loss3=None, ws=None,
                             stream=None):
    if ws is None:
        ws = workspace(ms_cvae_workspace_size(shape, B), params.device)
    return _check(lib().ms_cvae_forward_backward(C.byref(shape), _ptr(params), _ptr(x), _ptr(c), _ptr(eps_z), B, seed,
                                                 step, _ptr(grad), _ptr(loss3), _ptr(ws), ws.numel(),
                                                 _stream(stream)), "ms_cvae_forward_backward")


def ms_cvae_forward(shape, params, x, c, B, *, eps_z=None, seed=1, step=0, loss3=None, ws=None, stream=None):
    if ws is None:
        ws = workspace(ms_cvae_workspace_size(shape, B), params.device)
    return _check(lib().ms_cvae_forward(C.byref(shape), _ptr(params), _ptr(x), _ptr(c), _ptr(eps_z), B, seed, step,
                                        _ptr(loss3), _ptr(ws), ws.numel(), _stream(stream)), "ms_cvae_forward")


def ms_adam_step(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
    return _check(lib().ms_adam_step(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), params.numel(), t, lr, beta1, beta2,
                                     eps, weight_decay, _stream(stream)), "ms_adam_step")


def ms_cvae_train_step(shape, params, m, v, x, c, B, *, eps_z=None, seed=1, step=1, lr=1e-3, weight_decay=0.0,
                       loss3=None, ws=None, stream=None):
    if ws is None:
        ws = workspace(ms_cvae_workspace_size(shape, B), params.device)
    return _check(lib().ms_cvae_train_step(C.byref(shape), _ptr(params), _ptr(m), _ptr(v), _ptr(x), _ptr(c),
                                           _ptr(eps_z), B, seed, step, lr, weight_decay, _ptr(loss3), _ptr(ws),
                                           ws.numel(), _stream(stream)), "ms_cvae_train_step")


def ms_cvae_train_step_dev(shape, params, m, v, x_all, c_all, n_records, B, step_dev, *, seed=1, lr=1e-3,
                           weight_decay=0.0, loss3=None, ws=None, stream=None):
    """One graph-replayable training step: batch sampling, normals and Adam's t all on the device; step_dev is
    a one-element int64 device tensor holding t (incremented by the call's kernels)."""
    if ws is None:
        ws = workspace(int(lib().ms_cvae_train_step_dev_workspace_size(C.byref(shape), B)), params.device)
    return _check(lib().ms_cvae_train_step_dev(C.byref(shape), _ptr(params), _ptr(m), _ptr(v), _ptr(x_all),
                                               _ptr(c_all), n_records, B, seed, _ptr(step_dev), lr, weight_decay,
                                               _ptr(loss3), _ptr(ws), ws.numel(), _stream(stream)),
                  "ms_cvae_train_step_dev")


def ms_cvae_train_step_static(shape, params, m, v, x, c, B, *, eps_z=None, seed=1, step=1, lr=1e-3,
                              weight_decay=0.0, loss3=None, stream=None):
    """ms_cvae_train_step without a workspace: the scratch is a fixed array inside the library (for callers
    that may not allocate device memory).  Calls overlapping on the GPU race on that array."""
    return _check(lib().ms_cvae_train_step_static(C.byref(shape), _ptr(params), _ptr(m), _ptr(v), _ptr(x), _ptr(c),
                                                  _ptr(eps_z), B, seed, step, lr, weight_decay, _ptr(loss3),
                                                  _stream(stream)), "ms_cvae_train_step_static")


def ms_sdf_grid_build(disp_amp, disp_freq, n, device="cuda", stream=None) -> torch.Tensor:
    """The n^3 voxel grid of conservative distances for a request's displaced sphere (device float32 [n][n][n]);
    pass it as ``sdf_grid=grid.data_ptr(), sdf_grid_n=n`` in the render parameters (and keep it alive)."""
    g = torch.empty(n, n, n, dtype=torch.float32, device=device)
    nb = int(lib().ms_sdf_grid_workspace_size(n))
    ws = torch.empty(nb // 4 + 4, dtype=torch.int32, device=device)
    _check(lib().ms_sdf_grid_build(disp_amp, disp_freq, n, _ptr(g), _ptr(ws), nb, _stream(stream)),
           "ms_sdf_grid_build")
    if stream is not None:
        ws.record_stream(stream)     # the scratch stays reserved until that stream's work is done
    return g


def ms_training_records(n, n_events, exit_pos, exit_dir, rep_pos, rep_dir, media, seed, outs: dict, stream=None):
    per = int(media.numel() // 32 > 1)
    return _check(lib().ms_training_records(n, _ptr(n_events), _ptr(exit_pos), _ptr(exit_dir), _ptr(rep_pos),
                                            _ptr(rep_dir), _ptr(media), per, seed, _ptr(outs["cL"]),
                                            _ptr(outs["xL"]), _ptr(outs["cP"]), _ptr(outs["xP"]),
                                            _ptr(outs["cE"]), _ptr(outs["xE"]), _stream(stream)),
                  "ms_training_records")


# ------------------------------------------------------------------------------------------------ rendering

def render_params(d: dict) -> RenderParams:
    P = RenderParams()
    for k, v in d.items():
        cur = getattr(P, k)
        if isinstance(cur, C.Array):
            setattr(P, k, type(cur)(*[float(t) for t in v]))
        else:
            setattr(P, k, v)
    return P


def cvae_set(models: dict, precision=MS_FP32) -> CvaeSet:
    """models: {"length": (weights, p_in, p_out, latent, width), "path": ..., "event": ...} with device float32
    weights (latent 4 and width 16 when a tuple has three entries).  The returned struct keeps the weight
    tensors alive (it holds only their device pointers otherwise)."""
    s = CvaeSet()
    for k in ("length", "path", "event"):
        w, p_in, p_out, *lw = models[k]
        latent, width = lw if lw else (4, 16)
        setattr(s, k, decoder_struct(w, p_in, p_out, latent, width, precision=precision))
    s._owned = {k: models[k][0] for k in ("length", "path", "event")}
    return s


def ms_render_workspace_size(reqs) -> int:
    arr = (RenderParams * len(reqs))(*reqs)
    return int(lib().ms_render_workspace_size(arr, len(reqs)))


def ms_render(p: RenderParams, models: CvaeSet | None, image, stats, ws=None, stream=None):
    if ws is None:
        ws = workspace(ms_render_workspace_size([p]), image.device)
    return _check(lib().ms_render(C.byref(p), C.byref(models) if models is not None else None, _ptr(image),
                                  _ptr(stats), _ptr(ws), ws.numel(), _stream(stream)), "ms_render")


def ms_render_batch(reqs, models: CvaeSet | None, images, stats, ws=None, stream=None):
    arr = (RenderParams * len(reqs))(*reqs)
    if ws is None:
        ws = workspace(ms_render_workspace_size(reqs), images.device)
    return _check(lib().ms_render_batch(arr, len(reqs), C.byref(models) if models is not None else None,
                                        _ptr(images), _ptr(stats), _ptr(ws), ws.numel(), _stream(stream)),
                  "ms_render_batch")


def ms_render_autotune(reqs, models: CvaeSet | None, images, stats, repeats=1, ws=None, stream=None):
    """Time every renderer variant on ``reqs`` and return (best variant, per-variant milliseconds)."""
    arr = (RenderParams * len(reqs))(*reqs)
    if ws is None:
        ws = workspace(ms_render_workspace_size(reqs), images.device)
    nv = int(lib().ms_render_variants())
    times = (C.c_float * nv)()
    best = C.c_int(-1)
    _check(lib().ms_render_autotune(arr, len(reqs), C.byref(models) if models is not None else None, _ptr(images),
                                    _ptr(stats), _ptr(ws), ws.numel(), repeats, C.byref(best), times,
                                    _stream(stream)), "ms_render_autotune")
    return best.value, list(times)


def ms_render_variant_info(i):
    vals = [C.c_int() for _ in range(4)]
    _check(lib().ms_render_variant_info(i, *[C.byref(v) for v in vals]), "ms_render_variant_info")
    return dict(zip(("decode_batch", "trans_batch", "steps", "min_blocks"), (v.value for v in vals)))


# ------------------------------------------------------------------------------------------------ peaks

def ms_alu_peaks(device=None, stream=None) -> dict:
    """Measured whole-GPU issue rates (operations per second) of FFMA, the special-function unit (ex2, lg2, sin,
    rsqrt) and integer multiply-add, logic and high multiply; waits for the stream."""
    n = int(lib().ms_alu_peaks_scratch_bytes())
    ws = workspace(n, device)
    out = (C.c_double * len(PEAK_NAMES))()
    _check(lib().ms_alu_peaks(out, _ptr(ws), ws.numel(), _stream(stream)), "ms_alu_peaks")
    return dict(zip(PEAK_NAMES, list(out)))
