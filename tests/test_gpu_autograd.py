"""The CVAE loss as a torch.autograd.Function (Sec. 3.2: the models are trained through PyTorch), with forward
and backward in the library's kernels: its loss and parameter gradient against the FP64 oracle, the
forward-only entry point (ms_cvae_forward) against the fused one, and a torch.optim.Adam step on its gradient
against the library's own training step."""
import numpy as np
import pytest
import torch

from oracle import cvae
from paper_2011_03082_b300 import autograd, ms, synth

pytestmark = pytest.mark.gpu


def _data(p_in, p_out, latent, width, B, seed):
    rng = np.random.default_rng(seed)
    p = synth.xavier_cvae(seed, p_in, p_out, latent, width)
    p = (p + 0.05 * rng.standard_normal(p.size)).astype(np.float32)
    x = rng.standard_normal((B, p_out)).astype(np.float32)
    c = rng.standard_normal((B, p_in)).astype(np.float32)
    e = rng.standard_normal((B, latent)).astype(np.float32)
    return p, x, c, e


@pytest.mark.parametrize("name", list(synth.MODEL_SHAPES))
@pytest.mark.parametrize("B", [7, 4096])
def test_autograd_gradient_matches_oracle(name, B):
    p_in, p_out, latent, width = synth.MODEL_SHAPES[name]
    p, x, c, e = _data(p_in, p_out, latent, width, B, 3)
    shape = ms.cvae_shape(p_in, p_out, latent, width)
    params = torch.from_numpy(p).cuda().requires_grad_(True)
    loss, rec, kl = autograd.cvae_loss(params, torch.from_numpy(x).cuda(), torch.from_numpy(c).cuda(), shape,
                                       eps_z=torch.from_numpy(e).cuda())
    assert loss.requires_grad and not rec.requires_grad and not kl.requires_grad
    (2.0 * loss).backward()
    ref_loss, ref_rec, ref_kl, ref_g = cvae.neg_elbo_grad(p.astype(np.float64), cvae.Shape(p_in, p_out, latent, width),
                                                          x, c, e)
    got = np.array([loss.item(), rec.item(), kl.item()])
    assert np.allclose(got, [ref_loss, ref_rec, ref_kl], rtol=1e-4, atol=1e-5)
    g = params.grad.cpu().numpy()
    assert np.abs(g - 2.0 * ref_g).max() <= 1e-4 * np.abs(2.0 * ref_g).max()


@pytest.mark.parametrize("precision", [ms.MS_FP32, ms.MS_BF16])
def test_forward_only_equals_fused_loss(precision):
    """ms_cvae_forward (no backward pass) gives the fused call's loss terms bit for bit, with given and with
    kernel-drawn normals; with no gradient requested the autograd.Function takes that path."""
    p_in, p_out, latent, width = synth.MODEL_SHAPES["event"]
    B = 65536 + 37
    p, x, c, e = _data(p_in, p_out, latent, width, B, 4)
    shape = ms.cvae_shape(p_in, p_out, latent, width, precision=precision)
    P, X, Cc, E = (torch.from_numpy(a).cuda() for a in (p, x, c, e))
    for eps in (E, None):
        l_fused = torch.zeros(3, device="cuda")
        l_fwd = torch.full((3,), float("nan"), device="cuda")
        ms.ms_cvae_forward_backward(shape, P, X, Cc, B, eps_z=eps, seed=9, step=4, grad=torch.zeros_like(P),
                                    loss3=l_fused)
        ms.ms_cvae_forward(shape, P, X, Cc, B, eps_z=eps, seed=9, step=4, loss3=l_fwd)
        torch.cuda.synchronize()
        assert torch.equal(l_fused, l_fwd), (l_fused, l_fwd)
    with torch.no_grad():
        loss, rec, kl = autograd.cvae_loss(P, X, Cc, shape, eps_z=E, seed=9, step=4)
    ms.ms_cvae_forward_backward(shape, P, X, Cc, B, eps_z=E, seed=9, step=4, grad=torch.zeros_like(P), loss3=l_fused)
    torch.cuda.synchronize()
    assert torch.equal(torch.stack([loss, rec, kl]), l_fused)


def test_forward_rejects_bad_arguments():
    shape = ms.cvae_shape(7, 6, 5, 16)
    t = torch.zeros(16, device="cuda")
    with pytest.raises(ms.MsError, match="workspace"):
        ms.ms_cvae_forward(shape, t, t, t, 1 << 20, loss3=t, ws=ms.workspace(256))
    with pytest.raises(ms.MsError, match="not built"):
        ms.ms_cvae_forward(ms.cvae_shape(5, 5, 5, 16), t, t, t, 4, loss3=t)


def test_torch_adam_on_the_autograd_gradient_equals_the_library_step():
    """One torch.optim.Adam step on the autograd.Function's gradient equals ms_cvae_train_step (same bias-corrected
    Adam, beta 0.9 / 0.999, eps 1e-8), and the loss goes down over a few such steps."""
    p_in, p_out, latent, width = synth.MODEL_SHAPES["path"]
    B = 8192
    p, x, c, e = _data(p_in, p_out, latent, width, B, 5)
    shape = ms.cvae_shape(p_in, p_out, latent, width)
    X, Cc, E = (torch.from_numpy(a).cuda() for a in (x, c, e))
    params = torch.from_numpy(p).cuda().requires_grad_(True)
    opt = torch.optim.Adam([params], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    losses = []
    for _ in range(5):
        opt.zero_grad()
        loss, _, _ = autograd.cvae_loss(params, X, Cc, shape, eps_z=E)
        loss.backward()
        opt.step()
        losses.append(loss.item())
        if len(losses) == 1:
            after_one = params.detach().clone()
    lib_p = torch.from_numpy(p).cuda()
    m, v = torch.zeros_like(lib_p), torch.zeros_like(lib_p)
    ms.ms_cvae_train_step(shape, lib_p, m, v, X, Cc, B, eps_z=E, step=1, lr=1e-3, loss3=torch.zeros(3, device="cuda"))
    torch.cuda.synchronize()
    assert torch.allclose(after_one, lib_p, rtol=0, atol=1e-6)
    assert losses[-1] < losses[0]
