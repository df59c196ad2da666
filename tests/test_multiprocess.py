"""Sharding across processes (CPU, gloo, world size 2).

Photons and pixel samples are independent and keyed by offsets in the counter-based stream, so the work
shards across ranks with no collective on the data path; summing the ranks' integer histograms / counters
(one all-reduce, as a multi-GPU job would do once at the end) reproduces the single-process result bit for
bit, and summed images match to rounding.  The benchmark's multi-rank mode uses the same offsets
(sample_offset = rank * spp)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


MEDIUM = dict(optical_radius=6.0, g=0.7, albedo=0.98, dir_in=(0.0, 0.0, 1.0), isotropic_start=1,
              first_event_at_origin=0)
N = 6000


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2011_03082_b300 import synth
    # walk shard: photons [rank * N / world, (rank + 1) * N / world)
    lo, hi = rank * N // world, (rank + 1) * N // world
    r = oracle.walk(3, hi - lo, MEDIUM, photon_offset=lo, per_photon=False)
    h = torch.from_numpy(np.concatenate([r["hist_n"], r["hist_pos"].ravel(), r["hist_cos"], r["counters"]])
                         .astype(np.int64))
    dist.all_reduce(h)
    # render shard: samples [rank * spp, (rank + 1) * spp)
    p = synth.render_scene(16.0, width=12, height=10, spp=4, mode=0, seed=5, sample_offset=rank * 4)
    img, st, _ = oracle.render(p)
    t = torch.from_numpy(img.ravel().copy())
    s = torch.from_numpy(st.astype(np.int64))
    dist.all_reduce(t)
    dist.all_reduce(s)
    if rank == 0:
        q.put((h.numpy(), t.numpy(), s.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_sum_to_the_single_run(orc):
    from paper_2011_03082_b300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    h, img, st = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r = orc.walk(3, N, MEDIUM, per_photon=False)
    ref = np.concatenate([r["hist_n"], r["hist_pos"].ravel(), r["hist_cos"], r["counters"]]).astype(np.int64)
    assert np.array_equal(h, ref)
    full, fst, _ = orc.render(synth.render_scene(16.0, width=12, height=10, spp=8, mode=0, seed=5))
    assert np.allclose(img, full.ravel(), rtol=1e-12, atol=0)
    assert np.array_equal(st[:10], fst[:10].astype(np.int64))
