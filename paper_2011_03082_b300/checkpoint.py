"""Checkpoint and resume of a CVAE's training state.

A checkpoint holds everything a training run needs to continue as if it had not stopped: the FP32 master
parameters, Adam's first and second moments, the step counter, the key of the mini-batch and latent draws, the
learning rate, batch size, arithmetic and the model's shape.  Because the mini-batch indices and latent normals
of step t come from the counter-based generator keyed by (seed, t), and the gradient reduction runs in a fixed
order, a resumed run reproduces the uninterrupted run bit for bit.

File layout (little endian):

    magic    8 bytes  b"MSCVAECK"
    version  u32      1
    header   u32      length H of the JSON header
    payload  u64      length P of the payload
    crc32    u32      zlib CRC-32 of header || payload
    header   H bytes  JSON: name, shape (p_in, p_out, latent, width), precision, step, seed, lr, batch, n_params,
                      weight_decay, extra (caller's dict)
    payload  P bytes  params, m, v as float32 arrays of n_params each

``read`` checks the magic, version, lengths and CRC and raises ``CheckpointError`` on any mismatch, so a
truncated or corrupted file is never resumed from.  Files are written to a temporary name and renamed, so an
interrupted write leaves the previous checkpoint intact.
"""
from __future__ import annotations

import json
import os
import struct
import zlib
from pathlib import Path

import numpy as np

MAGIC = b"MSCVAECK"
VERSION = 1
_FIXED = struct.Struct("<8sIIQI")


class CheckpointError(ValueError):
    pass


def write(path, *, name: str, shape, precision: int, step: int, seed: int, lr: float, batch: int,
          params, m, v, weight_decay: float = 0.0, extra: dict | None = None) -> Path:
    """Write a checkpoint of the state after ``step`` completed steps.  ``params``, ``m`` and ``v``: float32
    arrays (numpy or CPU-convertible) of the same length."""
    arrs = [np.ascontiguousarray(np.asarray(a), dtype=np.float32).ravel() for a in (params, m, v)]
    n = arrs[0].size
    if any(a.size != n for a in arrs):
        raise CheckpointError("params, m and v must have the same length")
    header = json.dumps(dict(name=name, shape=[int(s) for s in shape], precision=int(precision), step=int(step),
                             seed=int(seed), lr=float(lr), batch=int(batch), n_params=int(n),
                             weight_decay=float(weight_decay), extra=extra or {}), sort_keys=True).encode()
    payload = b"".join(a.tobytes() for a in arrs)
    crc = zlib.crc32(payload, zlib.crc32(header)) & 0xFFFFFFFF
    path = Path(path)
    path.parent.mkdir(parents=True, exist_ok=True)
    tmp = path.with_name(path.name + f".tmp{os.getpid()}")
    with open(tmp, "wb") as f:
        f.write(_FIXED.pack(MAGIC, VERSION, len(header), len(payload), crc))
        f.write(header)
        f.write(payload)
    os.replace(tmp, path)
    return path


def read(path) -> dict:
    """The checkpoint at ``path`` as a dict of the header's fields plus ``params``, ``m``, ``v`` (float32)."""
    data = Path(path).read_bytes()
    if len(data) < _FIXED.size:
        raise CheckpointError(f"{path}: truncated (no header)")
    magic, version, hlen, plen, crc = _FIXED.unpack_from(data, 0)
    if magic != MAGIC:
        raise CheckpointError(f"{path}: not a CVAE checkpoint")
    if version != VERSION:
        raise CheckpointError(f"{path}: unsupported checkpoint version {version}")
    if len(data) != _FIXED.size + hlen + plen:
        raise CheckpointError(f"{path}: truncated or padded ({len(data)} bytes, expected "
                              f"{_FIXED.size + hlen + plen})")
    header = data[_FIXED.size:_FIXED.size + hlen]
    payload = data[_FIXED.size + hlen:]
    if zlib.crc32(payload, zlib.crc32(header)) & 0xFFFFFFFF != crc:
        raise CheckpointError(f"{path}: CRC mismatch (corrupted)")
    meta = json.loads(header)
    n = int(meta["n_params"])
    if plen != 3 * 4 * n:
        raise CheckpointError(f"{path}: payload of {plen} bytes does not hold 3 x {n} float32")
    arr = np.frombuffer(payload, dtype=np.float32)
    meta.update(params=arr[:n].copy(), m=arr[n:2 * n].copy(), v=arr[2 * n:].copy())
    return meta
