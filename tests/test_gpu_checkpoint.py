"""Resume from a checkpoint reproduces the uninterrupted training run bit for bit (the mini-batch and latent draws
of step t are keyed by (seed, t), the gradient reduction runs in a fixed order, and the checkpoint holds the
master weights, Adam moments and step).  A checkpoint of a different run is refused."""
import numpy as np
import pytest
import torch

from paper_2011_03082_b300 import checkpoint as ck
from paper_2011_03082_b300 import pipeline, synth

pytestmark = pytest.mark.gpu


def _records(name, n=20000):
    p_in, p_out, _, _ = synth.MODEL_SHAPES[name]
    rng = np.random.default_rng(21)
    c = torch.from_numpy(rng.standard_normal((n, p_in)).astype(np.float32)).cuda()
    x = torch.from_numpy(rng.standard_normal((n, p_out)).astype(np.float32)).cuda()
    return c, x


@pytest.mark.parametrize("name", ["length", "event"])
def test_resume_is_bit_exact(tmp_path, name):
    c, x = _records(name)
    kw = dict(batch=4096, lr=1e-3, seed=9, log_every=5)
    full, log_full = pipeline.train_one(name, c, x, steps=30, **kw)
    path = tmp_path / f"{name}.ckpt"
    part, _ = pipeline.train_one(name, c, x, steps=12, checkpoint=path, checkpoint_every=5, **kw)
    assert ck.read(path)["step"] == 12
    resumed, log_res = pipeline.train_one(name, c, x, steps=30, checkpoint=path, checkpoint_every=5, resume=True,
                                          **kw)
    torch.cuda.synchronize()
    assert torch.equal(resumed, full)
    # the resumed log holds every entry of the uninterrupted one, equal, and the interrupted run's last step
    by_step = {r[0]: r for r in log_res}
    assert set(by_step) == {r[0] for r in log_full} | {12}
    assert all(np.array_equal(np.asarray(by_step[r[0]]), np.asarray(r)) for r in log_full)
    st = ck.read(path)
    assert st["step"] == 30 and np.array_equal(st["params"], full.cpu().numpy())


def test_resume_refuses_another_run(tmp_path):
    c, x = _records("length")
    path = tmp_path / "length.ckpt"
    pipeline.train_one("length", c, x, steps=3, batch=1024, lr=1e-3, seed=9, checkpoint=path)
    with pytest.raises(ck.CheckpointError, match="does not match"):
        pipeline.train_one("length", c, x, steps=6, batch=1024, lr=2e-3, seed=9, checkpoint=path, resume=True)
