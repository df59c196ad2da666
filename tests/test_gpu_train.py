"""GPU parity of the hand-written CVAE training (Sec. 3.2) against the FP64 oracle: loss terms, gradients,
Adam, determinism, and the loss curve of 20 steps."""
import numpy as np
import pytest
import torch

from oracle import cvae
from paper_2011_03082_b300 import ms, synth

pytestmark = pytest.mark.gpu

# (p_in, p_out, latent, width): the uniform latent-4 / width-16 set and the final Table 1 shapes
SHAPES = [(2, 1, 4, 16), (3, 3, 4, 16), (7, 6, 4, 16), (4, 6, 4, 16)] + list(synth.MODEL_SHAPES.values())


def _data(p_in, p_out, B, seed, latent=4, width=16):
    rng = np.random.default_rng(seed)
    p = synth.xavier_cvae(seed, p_in, p_out, latent, width)
    p = (p + 0.05 * rng.standard_normal(p.size)).astype(np.float32)
    x = rng.standard_normal((B, p_out)).astype(np.float32)
    c = rng.standard_normal((B, p_in)).astype(np.float32)
    e = rng.standard_normal((B, latent)).astype(np.float32)
    return p, x, c, e


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("p_in,p_out,latent,width", SHAPES)
@pytest.mark.parametrize("B", [1, 300, 4096])
def test_loss_and_gradient_match_oracle(p_in, p_out, latent, width, B):
    p, x, c, e = _data(p_in, p_out, B, 1, latent, width)
    shape = ms.cvae_shape(p_in, p_out, latent, width)
    grad = torch.zeros(p.size, device="cuda")
    loss3 = torch.zeros(3, device="cuda")
    ms.ms_cvae_forward_backward(shape, _dev(p), _dev(x), _dev(c), B, eps_z=_dev(e), grad=grad, loss3=loss3)
    torch.cuda.synchronize()
    loss, rec, kl, g = cvae.neg_elbo_grad(p.astype(np.float64), cvae.Shape(p_in, p_out, latent, width), x, c, e)
    l3 = loss3.cpu().numpy()
    assert np.allclose(l3, [loss, rec, kl], rtol=1e-4, atol=1e-5)
    gg = grad.cpu().numpy()
    scale = np.abs(g).max()
    assert np.abs(gg - g).max() <= 1e-4 * scale, np.abs(gg - g).max() / scale


def test_gradient_is_deterministic():
    p_in, p_out, B = 7, 6, 65536
    p, x, c, _ = _data(p_in, p_out, B, 2)
    shape = ms.cvae_shape(p_in, p_out)
    outs = []
    for _ in range(2):
        grad = torch.zeros(p.size, device="cuda")
        loss3 = torch.zeros(3, device="cuda")
        ms.ms_cvae_forward_backward(shape, _dev(p), _dev(x), _dev(c), B, seed=3, step=5, grad=grad, loss3=loss3)
        torch.cuda.synchronize()
        outs.append((grad.cpu().numpy(), loss3.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("p_in,p_out,latent,width", [(3, 3, 4, 16), (7, 6, 5, 16), (2, 1, 2, 8)])
def test_philox_eps_matches_oracle_normals(orc, p_in, p_out, latent, width):
    B, step = 2000, 9
    p, x, c, _ = _data(p_in, p_out, B, 4, latent, width)
    shape = ms.cvae_shape(p_in, p_out, latent, width)
    grad = torch.zeros(p.size, device="cuda")
    loss3 = torch.zeros(3, device="cuda")
    ms.ms_cvae_forward_backward(shape, _dev(p), _dev(x), _dev(c), B, seed=11, step=step, grad=grad, loss3=loss3)
    torch.cuda.synchronize()
    # normals 4j..4j+3 of sample b: counter (j, b, step, 0xE0), id = (step << 32) | b
    e = np.concatenate([orc.normals_from_words(orc.philox_words(11, step << 32, B, j, 0xE0))
                        for j in range((latent + 3) // 4)], axis=1)[:, :latent]
    loss, rec, kl, g = cvae.neg_elbo_grad(p.astype(np.float64), cvae.Shape(p_in, p_out, latent, width), x, c, e)
    assert np.allclose(loss3.cpu().numpy(), [loss, rec, kl], rtol=1e-4, atol=1e-5)
    assert np.abs(grad.cpu().numpy() - g).max() <= 1e-3 * np.abs(g).max()


@pytest.mark.parametrize("wd", [0.0, 0.01])
def test_adam_matches_oracle(wd):
    rng = np.random.default_rng(5)
    n = 1300
    p0 = rng.standard_normal(n).astype(np.float32)
    pt, mt, vt = _dev(p0.copy()), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    p, m, v = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 6):
        g = rng.standard_normal(n).astype(np.float32)
        ms.ms_adam_step(pt, mt, vt, _dev(g), t, 1e-3, weight_decay=wd)
        p, m, v = cvae.adam_step(p, m, v, g.astype(np.float64), t, 1e-3, weight_decay=wd)
    torch.cuda.synchronize()
    assert np.abs(pt.cpu().numpy() - p).max() <= 1e-6


def test_training_loss_curve_matches_oracle():
    """20 Adam steps on a 1,024-sample batch with given eps: the GPU and oracle loss curves agree."""
    p_in, p_out, B = 3, 3, 1024
    p, x, c, _ = _data(p_in, p_out, B, 6)
    rng = np.random.default_rng(7)
    shape = ms.cvae_shape(p_in, p_out)
    pt, mt, vt = _dev(p.copy()), torch.zeros(p.size, device="cuda"), torch.zeros(p.size, device="cuda")
    po, mo, vo = p.astype(np.float64), np.zeros(p.size), np.zeros(p.size)
    loss3 = torch.zeros(3, device="cuda")
    gl, ol = [], []
    for t in range(1, 21):
        e = rng.standard_normal((B, 4)).astype(np.float32)
        ms.ms_cvae_train_step(shape, pt, mt, vt, _dev(x), _dev(c), B, eps_z=_dev(e), step=t, lr=1e-2, loss3=loss3)
        gl.append(float(loss3[0]))
        loss, _, _, g = cvae.neg_elbo_grad(po, cvae.Shape(p_in, p_out), x, c, e)
        po, mo, vo = cvae.adam_step(po, mo, vo, g, t, 1e-2)
        ol.append(loss)
    assert np.allclose(gl, ol, rtol=2e-3), (gl, ol)
    assert gl[-1] < gl[0]


def test_unsupported_shape_is_rejected():
    shape = ms.cvae_shape(5, 5)
    with pytest.raises(ms.MsError, match="not built"):
        ms.ms_cvae_forward_backward(shape, torch.zeros(10, device="cuda"), torch.zeros(10, device="cuda"),
                                    torch.zeros(10, device="cuda"), 2, ws=ms.workspace(1 << 20))


def _dev_step_reference(orc, p0, xa, ca, shape, B, seed, steps, lr):
    """Oracle training with the device-step sampling rule: record (w * n) >> 32 with w = word 0 of counter
    (0, t, b, 0xB0), latent normals 4j..4j+3 from counter (j, b, t, 0xE0)."""
    n = xa.shape[0]
    p, m, v = p0.astype(np.float64), np.zeros(p0.size), np.zeros(p0.size)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for t in range(1, steps + 1):
        idx = np.array([(int(orc.philox([0, t, b, 0xB0], key)[0]) * n) >> 32 for b in range(B)])
        eps = np.concatenate([orc.normals_from_words(orc.philox_words(seed, t << 32, B, j, 0xE0))
                              for j in range((shape.latent + 3) // 4)], axis=1)[:, :shape.latent]
        _, _, _, g = cvae.neg_elbo_grad(p, shape, xa[idx], ca[idx], eps)
        p, m, v = cvae.adam_step(p, m, v, g, t, lr)
    return p


@pytest.mark.parametrize("latent,width", [(4, 16), (5, 16)])
def test_device_step_training_matches_oracle_and_replays_in_a_graph(orc, latent, width):
    p_in, p_out, n, B, steps, seed, lr = 3, 3, 5000, 1024, 5, 21, 1e-2
    p0, xa, ca, _ = _data(p_in, p_out, n, 8, latent, width)
    shape = ms.cvae_shape(p_in, p_out, latent, width)
    ref = _dev_step_reference(orc, p0, xa, ca, cvae.Shape(p_in, p_out, latent, width), B, seed, steps, lr)

    def run(graph: bool):
        p, m, v = _dev(p0.copy()), torch.zeros(p0.size, device="cuda"), torch.zeros(p0.size, device="cuda")
        step = torch.ones(1, dtype=torch.int64, device="cuda")
        loss3 = torch.zeros(3, device="cuda")
        ws = ms.workspace(ms.lib().ms_cvae_train_step_dev_workspace_size(ms.C.byref(shape), B))
        x, c = _dev(xa), _dev(ca)
        if not graph:
            for _ in range(steps):
                ms.ms_cvae_train_step_dev(shape, p, m, v, x, c, n, B, step, seed=seed, lr=lr, loss3=loss3, ws=ws)
        else:
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                with torch.cuda.graph(g):
                    ms.ms_cvae_train_step_dev(shape, p, m, v, x, c, n, B, step, seed=seed, lr=lr, loss3=loss3, ws=ws)
            for _ in range(steps):
                g.replay()
        torch.cuda.synchronize()
        assert int(step.item()) == steps + 1
        return p.cpu().numpy()

    direct, replayed = run(False), run(True)
    assert np.array_equal(direct, replayed)
    assert np.abs(direct - ref).max() <= 2e-4 * max(1.0, np.abs(ref).max()), np.abs(direct - ref).max()


@pytest.mark.parametrize("p_in,p_out,latent,width", [(3, 3, 4, 16), (7, 6, 4, 16), (7, 6, 5, 16), (2, 1, 2, 8)])
def test_bf16_training_matches_oracle(p_in, p_out, latent, width):
    """BF16 numerics (weight matrices and layer inputs rounded to BF16, FP32 accumulation and master weights)
    against the oracle with the same rounding: loss and gradient within 2e-2 of the largest component."""
    B = 4096
    p, x, c, e = _data(p_in, p_out, B, 12, latent, width)
    shape = ms.cvae_shape(p_in, p_out, latent, width, precision=ms.MS_BF16)
    grad = torch.zeros(p.size, device="cuda")
    loss3 = torch.zeros(3, device="cuda")
    ms.ms_cvae_forward_backward(shape, _dev(p), _dev(x), _dev(c), B, eps_z=_dev(e), grad=grad, loss3=loss3)
    torch.cuda.synchronize()
    sh = cvae.Shape(p_in, p_out, latent, width)
    loss, rec, kl, g = cvae.neg_elbo_grad(p.astype(np.float64), sh, x, c, e, bf16=True)
    assert np.allclose(loss3.cpu().numpy(), [loss, rec, kl], rtol=2e-3, atol=2e-3)
    assert np.abs(grad.cpu().numpy() - g).max() <= 2e-2 * np.abs(g).max()
    _, _, _, g32 = cvae.neg_elbo_grad(p.astype(np.float64), sh, x, c, e)
    assert np.abs(grad.cpu().numpy() - g).max() < np.abs(g32 - g).max()   # closer to its own precision
