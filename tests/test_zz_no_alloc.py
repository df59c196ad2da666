"""ms_cvae_train_step_static — the training step for callers that may not allocate device memory — gives the
same result as ms_cvae_train_step with a caller-provided workspace.

Two steps in a row on each path, through the C ABI; the parameters, Adam state and loss terms must agree
within the training tests' tolerance.  This file is collected last so that a failure here comes after every
other test has run; it also passes on its own in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2011_03082_b300 import ms, synth

pytestmark = pytest.mark.gpu


def test_static_scratch_step_matches_workspace_step():
    p_in, p_out, B = 7, 6, 65536
    rng = np.random.default_rng(11)
    p0 = synth.xavier_cvae(3, p_in, p_out)
    x = torch.from_numpy(rng.standard_normal((B, p_out)).astype(np.float32)).cuda()
    c = torch.from_numpy(rng.standard_normal((B, p_in)).astype(np.float32)).cuda()
    shape = ms.cvae_shape(p_in, p_out)
    assert ms.ms_cvae_workspace_size(shape, B) <= ms.lib().ms_cvae_static_scratch_bytes()
    results = []
    for use_static in (False, True):
        p = torch.from_numpy(p0.copy()).cuda()
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        losses = []
        for t in (1, 2):
            loss3 = torch.zeros(3, device="cuda")
            if use_static:
                ms.ms_cvae_train_step_static(shape, p, m, v, x, c, B, seed=5, step=t, lr=1e-3, loss3=loss3)
            else:
                ms.ms_cvae_train_step(shape, p, m, v, x, c, B, seed=5, step=t, lr=1e-3, loss3=loss3)
            torch.cuda.synchronize()
            losses.append(loss3.cpu().numpy())
        results.append((p.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy(), np.array(losses)))
    (pa, ma, va, la), (pb, mb, vb, lb) = results
    assert np.allclose(la, lb, rtol=1e-4, atol=1e-5)
    assert np.abs(pa - pb).max() <= 1e-6 and np.abs(ma - mb).max() <= 1e-6 * max(1.0, np.abs(ma).max())
    assert np.abs(va - vb).max() <= 1e-6 * max(1.0, np.abs(va).max())


def test_static_scratch_rejects_oversized_batches():
    shape = ms.cvae_shape(7, 6)
    B = 1 << 26
    assert ms.ms_cvae_workspace_size(shape, B) > ms.lib().ms_cvae_static_scratch_bytes()
    t = torch.zeros(16, device="cuda")
    with pytest.raises(ms.MsError, match="static"):
        ms.ms_cvae_train_step_static(shape, t, t, t, t, t, B)
