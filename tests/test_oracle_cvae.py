"""Pins of the oracle CVAE (Sec. 3.2) and training-target transform (Sec. 4.1), CPU only."""
import math

import numpy as np
import pytest
import torch
from scipy import integrate, stats

from oracle import cvae
from paper_2011_03082_b300 import synth

SHAPES = [cvae.Shape(2, 1), cvae.Shape(3, 3), cvae.Shape(7, 6), cvae.Shape(4, 6)]


def _batch(shape, B, seed):
    rng = np.random.default_rng(seed)
    p = synth.xavier_cvae(seed, shape.p_in, shape.p_out).astype(np.float64)
    p += 0.05 * rng.standard_normal(p.size)       # nonzero biases
    x = rng.standard_normal((B, shape.p_out))
    c = rng.standard_normal((B, shape.p_in))
    eps = rng.standard_normal((B, shape.latent))
    return p, x, c, eps


@pytest.mark.parametrize("shape", SHAPES)
def test_decoder_matches_torch(shape):
    p, _, c, z = _batch(shape, 64, 1)
    _, dec = cvae.split_cvae(p, shape)
    wdec = p[shape.n_enc:]
    mu, lv = cvae.decoder_forward(wdec, shape, c, z)
    F = torch.nn.functional
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    h = F.softplus(F.linear(t(np.concatenate([c, z], 1)), t(dec["D1"]), t(dec["d1"])))
    h = F.softplus(F.linear(h, t(dec["D2"]), t(dec["d2"])))
    y = F.linear(h, t(dec["D3"]), t(dec["d3"])).numpy()
    assert np.allclose(mu, y[:, :shape.p_out], rtol=1e-13, atol=1e-13)
    assert np.allclose(lv, y[:, shape.p_out:], rtol=1e-13, atol=1e-13)


def test_decoder_closed_forms():
    shape = cvae.Shape(4, 6)
    w = np.zeros(shape.n_dec)
    n_in, W = 8, 16
    off_b3 = shape.n_dec - 12
    w[off_b3:] = np.arange(12) * 0.1
    mu, lv = cvae.decoder_forward(w, shape, np.ones((3, 4)), np.ones((3, 4)))
    assert np.allclose(np.concatenate([mu, lv], 1), w[off_b3:])            # zero weights: output = b3
    off_W3 = off_b3 - 12 * W
    w[off_W3:off_b3] = 1.0                                                   # Softplus(0) = ln 2 per unit
    mu, lv = cvae.decoder_forward(w, shape, np.zeros((1, 4)), np.zeros((1, 4)))
    assert np.allclose(mu[0], 16 * math.log(2) + w[off_b3:off_b3 + 6], atol=1e-14)
    x = cvae.decoder_sample(w, shape, np.zeros((1, 4)), np.zeros((1, 4)), np.ones((1, 6)))
    assert np.allclose(x[0], mu[0] + np.exp(0.5 * lv[0]), atol=1e-14)
    assert n_in * W + W + W * W + W + 12 * W + 12 == shape.n_dec


def test_elbo_terms_against_scipy():
    """Reconstruction = -log N(x; mu, Sigma) (scipy), KL(N(mu,Sigma) || N(0,I)) by numerical quadrature."""
    shape = cvae.Shape(3, 3)
    p, x, c, eps = _batch(shape, 5, 2)
    loss, rec, kl, C = cvae.neg_elbo(p, shape, x, c, eps)
    enc, dec = C["enc"], C["dec"]
    mu_e, lv_e = C["mu_e"], C["lv_e"]
    z = mu_e + np.exp(0.5 * lv_e) * eps
    mu_d, lv_d = cvae.decoder_forward(p[shape.n_enc:], shape, c, z)
    rec_ref = -stats.norm.logpdf(x, mu_d, np.exp(0.5 * lv_d)).sum(axis=1).mean()
    assert abs(rec - rec_ref) < 1e-12
    kl_ref = 0.0
    for b in range(5):
        for l in range(shape.latent):
            m, s = mu_e[b, l], math.exp(0.5 * lv_e[b, l])
            f = lambda t: stats.norm.pdf(t, m, s) * (stats.norm.logpdf(t, m, s) - stats.norm.logpdf(t))
            kl_ref += integrate.quad(f, m - 30 * s, m + 30 * s, epsabs=1e-13, limit=200)[0]
    assert abs(kl - kl_ref / 5) < 1e-9
    assert abs(loss - (rec + kl)) < 1e-12


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_gradient_against_central_differences(shape):
    p, x, c, eps = _batch(shape, 7, 3)
    _, _, _, g = cvae.neg_elbo_grad(p, shape, x, c, eps)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(shape.n_enc, 40, replace=False),
                          shape.n_enc + rng.choice(shape.n_dec, 40, replace=False)])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (cvae.neg_elbo(pp, shape, x, c, eps)[0] - cvae.neg_elbo(pm, shape, x, c, eps)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_adam_first_step_and_torch_agreement():
    rng = np.random.default_rng(5)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(6)]
    lr = 1e-3
    p, m, v = cvae.adam_step(p0, np.zeros(50), np.zeros(50), grads[0], 1, lr)
    assert np.allclose(p0 - p, lr * grads[0] / (np.abs(grads[0]) + 1e-8), rtol=1e-12, atol=0)
    for wd, opt_cls in ((0.0, torch.optim.Adam), (0.01, torch.optim.AdamW)):
        tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
        opt = opt_cls([tp], lr=lr, betas=(0.9, 0.999), eps=1e-8, weight_decay=wd)
        p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
        for t, gr in enumerate(grads, 1):
            tp.grad = torch.tensor(gr, dtype=torch.float64)
            opt.step()
            p, m, v = cvae.adam_step(p, m, v, gr, t, lr, weight_decay=wd)
        assert np.allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_training_targets_invert_eq4():
    """Applying Eq. 4 and the exit frame of Sec. 4.1 to the targets with the record's psi gives back the
    recorded exit point, exit direction and representative event."""
    rng = np.random.default_rng(6)
    n = 500
    x = rng.standard_normal((n, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    w = rng.standard_normal((n, 3)) + x * 2
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    X = rng.uniform(-0.5, 0.5, (n, 3))
    W = rng.standard_normal((n, 3))
    W /= np.linalg.norm(W, axis=1, keepdims=True)
    N = rng.integers(1, 1000, n)
    u = rng.random(n)
    t = cvae.training_targets(N, x, w, X, W, np.full(n, 3.0), np.full(n, 0.5), np.full(n, 0.95), u)
    ct, al, be = t["xP"].T
    st = np.sqrt(1 - ct * ct)
    nrm = np.sqrt(np.maximum(0, 1 - al * al - be * be))
    # exit direction in the CVAE frame: alpha e_b + beta e_t + n e_n, e_b=(0,1,0), e_t=(ct,0,-st), e_n=(st,0,ct)
    wt = np.stack([be * ct + nrm * st, al, -be * st + nrm * ct], 1)
    xt = np.stack([st, np.zeros(n), ct], 1)
    psi = np.arctan2(x[:, 1], x[:, 0])
    R = lambda v: np.stack([np.cos(psi) * v[:, 0] - np.sin(psi) * v[:, 1],
                            np.sin(psi) * v[:, 0] + np.cos(psi) * v[:, 1], v[:, 2]], 1)
    assert np.allclose(R(xt), x, atol=1e-12)
    outward = np.sum(w * x, 1) > 0
    assert np.allclose(R(wt)[outward], w[outward], atol=1e-9)
    assert np.allclose(R(t["xE"][:, :3]), X, atol=1e-12) and np.allclose(R(t["xE"][:, 3:]), W, atol=1e-12)
    Nb = np.floor(np.exp(t["xL"][:, 0]) + 0.5)
    assert np.array_equal(Nb, N) and np.allclose(t["cP"][:, 2], np.log(N))
    assert np.allclose(t["cE"][:, 3:6], t["xP"])


def test_bf16_rounding_and_variant():
    """round_bf16 is round-to-nearest-even (checked against torch's bfloat16 cast); the BF16 variant's loss and
    analytic gradient equal torch autograd through a float64 CVAE that rounds the same tensors with a
    straight-through cast (value rounded, derivative 1); and it differs from the FP64 gradient by a
    BF16-sized amount."""
    rng = np.random.default_rng(9)
    a = rng.standard_normal(10000) * 10 ** rng.uniform(-3, 3, 10000)
    ref = torch.tensor(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cvae.round_bf16(a), ref)
    shape = cvae.Shape(3, 3)
    p, x, c, eps = _batch(shape, 64, 10)
    _, _, _, g32 = cvae.neg_elbo_grad(p, shape, x, c, eps)
    loss16, _, _, g16 = cvae.neg_elbo_grad(p, shape, x, c, eps, bf16=True)
    rel = np.abs(g16 - g32).max() / np.abs(g32).max()
    assert 1e-5 < rel < 5e-2

    F = torch.nn.functional
    q = lambda t: t + (t.to(torch.float32).to(torch.bfloat16).to(torch.float64) - t).detach()
    tp = torch.tensor(p, requires_grad=True)
    sizes = shape.enc_sizes() + shape.dec_sizes()
    parts, off = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        parts[name] = tp[off:off + n].reshape(shp)
        off += n
    T = lambda v: torch.tensor(v, dtype=torch.float64)

    def net(P, k, inp):
        h = F.softplus(F.linear(q(inp), q(P[k + "1"]), P[k.lower() + "1"]))
        h = F.softplus(F.linear(q(h), q(P[k + "2"]), P[k.lower() + "2"]))
        return F.linear(q(h), q(P[k + "3"]), P[k.lower() + "3"])

    L, Po = shape.latent, shape.p_out
    eo = net(parts, "E", torch.cat([T(x), T(c)], 1))
    mu_e, lv_e = eo[:, :L], eo[:, L:]
    z = mu_e + torch.exp(0.5 * lv_e) * T(eps)
    do = net(parts, "D", torch.cat([T(c), z], 1))
    nll = -torch.distributions.Normal(do[:, :Po], torch.exp(0.5 * do[:, Po:])).log_prob(T(x)).sum(1)
    kl = torch.distributions.kl_divergence(torch.distributions.Normal(mu_e, torch.exp(0.5 * lv_e)),
                                           torch.distributions.Normal(0.0, 1.0)).sum(1)
    loss = (nll + kl).mean()
    loss.backward()
    assert abs(loss.item() - loss16) < 1e-12
    assert np.allclose(tp.grad.numpy(), g16, rtol=1e-10, atol=1e-13)
