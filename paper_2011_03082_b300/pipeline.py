"""Training pipeline of the three learned samplers (Sec. 3.1-3.2, Sec. 4.1, Eq. 3), on the GPU.

1. ``generate_records``: brute-force HG walks from the centre of the unit sphere in the paper's convention
   (first event at the centre, incoming direction (0,0,1)) with per-walk media drawn like the training set
   (optical radius log-uniform in [1,256], g U[-1,1), albedo U[0.9,1]); the path follows the albedo-1
   physics and the representative event is chosen with weights albedo^k (``reservoir=2``); the records are
   turned into the conditions and targets of LengthGen, PathGen and EventGen by ``ms_training_records``.
2. ``train``: each CVAE is trained with the library's kernels: one step (mini-batch drawn on the device,
   forward, backward, deterministic reduction, Adam) is captured in a CUDA graph and replayed
   (``ms_cvae_train_step_dev``).
3. ``save`` / ``load``: a versioned ``.npz`` with the packed float32 parameters (encoder then decoder), each
   model's shape (p_in, p_out, latent, width: the final settings of Table 1) and the training log.
4. Checkpoint and resume (``--checkpoint-dir``, ``--checkpoint-every``): each model's full training state
   (master weights, Adam moments, step, draw key) is written every few steps with a CRC (``checkpoint.py``); a
   run started again with the same directory continues each model from its last checkpoint and ends with the
   same parameters, bit for bit, as a run that was never interrupted.

With ``--exact-n1`` the three models are trained on the records with N >= 2 only: a renderer using such a set
draws N = 1 with its exact probability exp(-tau) (the first free path from the centre leaves the sphere,
Sec. 3.1) and then the whole step exactly (the path leaves radially along the centre event's HG scattering of
the incoming direction, so alpha = beta = 0: a point mass of PathGen's output that a Gaussian decoder cannot
form; the centre is the representative event), and samples N >= 2 steps from the models (``render_options``).
The paper's form trains every model on every record.

With ``--exact-centre`` EventGen is trained on the records whose representative event is not the first one:
the first event sits at the centre with the incoming direction, and the weights phi^k / Lambda of Sec. 4.3
pick it with probability phi / Lambda (every record with N = 1, about 1/N of the others), a point mass of
(X~, W~) = (0, 0, 0, 0, 0, 1) that a Gaussian decoder cannot form: fitting it drives the decoder's variances
towards zero and pulls the continuous part of the law toward the centre.  A renderer using such a set draws
the centre event with its exact probability and samples the later events from EventGen.

Run as ``python -m paper_2011_03082_b300.pipeline [--walks N] [--steps S] [--out PATH] [--precision bf16]``.
"""
from __future__ import annotations

import argparse
import json
import time
from pathlib import Path

import numpy as np
import torch

from . import checkpoint as ckpt
from . import ms, synth

FORMAT = 2
WEIGHTS_DIR = Path(__file__).resolve().parent / "weights"
DEFAULT_WEIGHTS = WEIGHTS_DIR / "cvae_set.npz"
# committed model sets: the paper's form (every model trained on every record), the same in BF16 training
# arithmetic, and the set trained for the exact N = 1 step and centre event (--exact-n1 --exact-centre)
MODEL_SETS = {"paper": "cvae_set.npz", "bf16": "cvae_set_bf16.npz", "atoms": "cvae_set_atoms.npz"}
RENDER_SET = "atoms"        # the set the experiments and the benchmark render with
MODELS = ("length", "path", "event")
RECORD_KEYS = {"length": ("cL", "xL"), "path": ("cP", "xP"), "event": ("cE", "xE")}


def generate_records(n_walks: int, seed: int = 1, device="cuda") -> dict:
    tau, g, phi = synth.training_media(seed, n_walks)
    media = ms.media_tensor(tau.astype(np.float32), g.astype(np.float32), phi.astype(np.float32), (0.0, 0.0, 1.0),
                            0, 1, device=device)
    out = ms.walk_outputs(n_walks, device=device)
    ms.ms_simulate_walks(media, n_walks, out, seed=seed, reservoir=2, precision=ms.MS_FP32, max_events=1 << 24)
    recs = {k: torch.empty(n_walks, d, device=device) for k, d in
            (("cL", 2), ("xL", 1), ("cP", 3), ("xP", 3), ("cE", 7), ("xE", 6))}
    ms.ms_training_records(n_walks, out["n_events"], out["exit_pos"], out["exit_dir"], out["rep_pos"],
                           out["rep_dir"], media, seed + 1000, recs)
    recs["counters"] = out["counters"]
    return recs


def train_one(name: str, c: torch.Tensor, x: torch.Tensor, *, steps: int, batch: int, lr: float, seed: int,
              log_every: int = 100, precision: int = ms.MS_FP32, checkpoint=None, checkpoint_every: int = 0,
              resume: bool = False):
    """Train one CVAE: one training step (device-side batch sampling, forward, backward, deterministic
    reduction, Adam with its step counter on the device) is captured in a CUDA graph and replayed.
    ``precision``: MS_FP32, or MS_BF16 (BF16 products with FP32 accumulation and FP32 master weights).
    ``checkpoint``: a file the training state is written to every ``checkpoint_every`` steps and after the last
    step; with ``resume`` and an existing file, training continues after the step it holds (its model, shape,
    arithmetic, draw key, batch and learning rate must match)."""
    p_in, p_out, latent, width = synth.MODEL_SHAPES[name]
    shape = ms.cvae_shape(p_in, p_out, latent, width, precision=precision)
    dev = c.device
    params = torch.from_numpy(synth.xavier_cvae(seed, p_in, p_out, latent, width)).to(dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    step = torch.ones(1, dtype=torch.int64, device=dev)
    t_first, log = 1, []
    if resume and checkpoint is not None and Path(checkpoint).exists():
        st = ckpt.read(checkpoint)
        want = dict(name=name, shape=[p_in, p_out, latent, width], precision=int(precision), seed=int(seed),
                    batch=int(batch), lr=float(lr))
        bad = {k: (st[k], v_) for k, v_ in want.items() if st[k] != v_}
        if bad:
            raise ckpt.CheckpointError(f"{checkpoint}: does not match this run: {bad}")
        params.copy_(torch.from_numpy(st["params"]))
        m.copy_(torch.from_numpy(st["m"]))
        v.copy_(torch.from_numpy(st["v"]))
        step.fill_(int(st["step"]) + 1)
        t_first = int(st["step"]) + 1
        log = [tuple(r) for r in st["extra"].get("log", [])]

    def save_state(t):
        torch.cuda.synchronize(dev)
        ckpt.write(checkpoint, name=name, shape=(p_in, p_out, latent, width), precision=precision, step=t,
                   seed=seed, lr=lr, batch=batch, params=params.cpu().numpy(), m=m.cpu().numpy(),
                   v=v.cpu().numpy(), extra=dict(log=[list(r) for r in log]))
    loss3 = torch.zeros(3, device=dev)
    ws = ms.workspace(int(ms.lib().ms_cvae_train_step_dev_workspace_size(ms.C.byref(shape), batch)), dev)
    x = x.contiguous()
    c = c.contiguous()
    n = c.shape[0]
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph):
            ms.ms_cvae_train_step_dev(shape, params, m, v, x, c, n, batch, step, seed=seed, lr=lr, loss3=loss3, ws=ws)
    for t in range(t_first, steps + 1):
        graph.replay()
        if t % log_every == 0 or t == 1 or t == steps:
            log.append((t, *[float(v_) for v_ in loss3.tolist()]))
        if checkpoint is not None and ((checkpoint_every and t % checkpoint_every == 0) or t == steps):
            save_state(t)
    return params, log


def train(records: dict, *, steps=20000, batch=65536, lr=1e-3, seed=1, log_every=100,
          precision: int = ms.MS_FP32, exact_n1: bool = False, exact_centre: bool = False,
          checkpoint_dir=None, checkpoint_every: int = 0) -> dict:
    """Train the three CVAEs; with ``checkpoint_dir``, each model's state goes to ``<dir>/<model>.ckpt`` every
    ``checkpoint_every`` steps and at its end, and a model whose file exists continues from it (a finished
    model is not trained again)."""
    models = {}
    for i, name in enumerate(MODELS):
        ck, xk = RECORD_KEYS[name]
        c, x = records[ck], records[xk]
        if exact_n1:
            # the records with N >= 2: LengthGen's dequantised y = ln(N - 1/2 + u) is >= ln(3/2) exactly for
            # those; PathGen's and EventGen's conditions hold ln N (>= ln 2 = 0.69 for those, 0 for N = 1)
            keep = x[:, 0] >= float(np.log(1.5)) if name == "length" else c[:, -1] > 0.5
            c, x = c[keep].contiguous(), x[keep].contiguous()
        if name == "event" and exact_centre:
            # the records whose representative event is a later one: the first event's X~ is exactly zero
            keep = (x[:, :3] != 0.0).any(dim=1)
            c, x = c[keep].contiguous(), x[keep].contiguous()
        path = None if checkpoint_dir is None else Path(checkpoint_dir) / f"{name}.ckpt"
        params, log = train_one(name, c, x, steps=steps, batch=batch, lr=lr, seed=seed + 17 * i,
                                log_every=log_every, precision=precision, checkpoint=path,
                                checkpoint_every=checkpoint_every, resume=path is not None)
        models[name] = dict(params=params.cpu().numpy(), log=log)
    return models


def render_options(models: dict) -> dict:
    """Render-request fields that a model set needs: ``exact_n1`` when its LengthGen was trained on N >= 2,
    ``exact_centre`` when its EventGen was trained without the records whose representative event is the first."""
    meta = models.get("meta", {})
    return dict(exact_n1=int(bool(meta.get("exact_n1", False))),
                exact_centre=int(bool(meta.get("exact_centre", False))))


def load_set(name: str) -> dict:
    """A committed model set by name (``MODEL_SETS``)."""
    return load(WEIGHTS_DIR / MODEL_SETS[name])


def render_set(models=None, device="cuda", precision=None):
    """(the ms.cvae_set of a model set's decoders on ``device``, the render-request fields the set needs).
    ``models``: a loaded set, a name of ``MODEL_SETS``, or None for ``RENDER_SET``; ``precision``: the decoders'
    arithmetic (ms.MS_FP32 when None)."""
    if models is None or isinstance(models, str):
        models = load_set(models or RENDER_SET)
    dm = device_decoders(models, device)
    cset = ms.cvae_set(dm) if precision is None else ms.cvae_set(dm, precision=precision)
    return cset, render_options(models)


def decoder_part(name: str, params: np.ndarray) -> np.ndarray:
    """The decoder block of a packed CVAE parameter vector (what the renderer evaluates)."""
    p_in, p_out, L, W = synth.MODEL_SHAPES[name]
    n_enc = W * (p_out + p_in) + W + W * W + W + 2 * L * W + 2 * L
    return np.ascontiguousarray(params[n_enc:], dtype=np.float32)


def save(path, models: dict, meta: dict):
    path = Path(path)
    path.parent.mkdir(parents=True, exist_ok=True)
    arrays = {f"{k}_params": v["params"].astype(np.float32) for k, v in models.items()}
    arrays.update({f"{k}_log": np.asarray(v["log"], np.float64) for k, v in models.items()})
    arrays.update({f"{k}_shape": np.asarray(synth.MODEL_SHAPES[k], np.int64) for k in models})
    np.savez(path, format=np.int64(FORMAT), meta=json.dumps(meta), **arrays)


def load(path=DEFAULT_WEIGHTS) -> dict:
    z = np.load(path, allow_pickle=False)
    if int(z["format"]) != FORMAT:
        raise ValueError(f"{path}: unsupported weights format {int(z['format'])}")
    for k in MODELS:
        shape = tuple(int(v) for v in z[f"{k}_shape"])
        if shape != tuple(synth.MODEL_SHAPES[k]) or z[f"{k}_params"].size != _n_params(k):
            raise ValueError(f"{path}: {k} has shape {shape}, expected {synth.MODEL_SHAPES[k]}")
    return {k: dict(params=z[f"{k}_params"], log=z[f"{k}_log"]) for k in MODELS} | {
        "meta": json.loads(str(z["meta"]))}


def _n_params(name: str) -> int:
    p_in, p_out, L, W = synth.MODEL_SHAPES[name]
    enc = W * (p_out + p_in) + W + W * W + W + 2 * L * W + 2 * L
    dec = W * (p_in + L) + W + W * W + W + 2 * p_out * W + 2 * p_out
    return enc + dec


def device_decoders(models: dict, device="cuda") -> dict:
    """{name: (decoder weights on the device, p_in, p_out, latent, width)} as ms.cvae_set expects."""
    out = {}
    for name in MODELS:
        out[name] = (torch.from_numpy(decoder_part(name, models[name]["params"])).to(device), *synth.MODEL_SHAPES[name])
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--walks", type=int, default=1 << 24)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=str(DEFAULT_WEIGHTS))
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="fp32",
                    help="training arithmetic (bf16: BF16 products, FP32 accumulation and master weights)")
    ap.add_argument("--exact-n1", action="store_true",
                    help="train the models on the N >= 2 records (the N = 1 step is then drawn exactly)")
    ap.add_argument("--exact-centre", action="store_true",
                    help="train EventGen without the centre-event records (that event is then drawn exactly)")
    ap.add_argument("--checkpoint-dir", default=None,
                    help="write each model's training state here, and continue from it when it exists")
    ap.add_argument("--checkpoint-every", type=int, default=1000)
    a = ap.parse_args(argv)
    prec = ms.MS_BF16 if a.precision == "bf16" else ms.MS_FP32
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    recs = generate_records(a.walks, a.seed)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    models = train(recs, steps=a.steps, batch=a.batch, lr=a.lr, seed=a.seed, precision=prec, exact_n1=a.exact_n1,
                   exact_centre=a.exact_centre, checkpoint_dir=a.checkpoint_dir,
                   checkpoint_every=a.checkpoint_every)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    c = recs["counters"].cpu().tolist()
    meta = dict(walks=a.walks, steps=a.steps, batch=a.batch, lr=a.lr, seed=a.seed, precision=a.precision,
                exact_n1=bool(a.exact_n1), exact_centre=bool(a.exact_centre),
                walk_seconds=t1 - t0,
                train_seconds=t2 - t1, walk_counters=c,
                final_loss={k: v["log"][-1][1] for k, v in models.items()})
    save(a.out, models, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
