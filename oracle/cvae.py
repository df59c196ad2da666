"""Oracle: conditional VAE decoder, ELBO, backward pass and Adam in FP64 numpy — TEST INFRASTRUCTURE ONLY.

Plain restatement of Sec. 3.2 of the paper ("Model architectures and inference"):

* Encoder Enc(x, c) and decoder Dec(z, c) are MLPs with Softplus between hidden layers and linear outputs
  giving a mean and the log of a diagonal covariance (the paper predicts log Sigma).
* Training maximises the ELBO  -KL(q_Enc(z|x,c) || N(0, I)) + <log p_Dec(x|z,c)>; this module returns the
  negative ELBO averaged over the batch, with one reparameterised latent sample z = mu + sqrt(Sigma) eps.
* Inference draws z ~ N(0, I) and returns x = sqrt(Sigma_Dec) eps + mu_Dec.
* The optimiser is Adam (AdamW's decoupled weight decay is a flag), as named in Sec. 3.2.
* A BF16 training variant (not in the paper; a precision choice of the training step): weight matrices and
  every layer's input are rounded to bfloat16 (nearest even), everything else stays FP64 here; the gradient
  with respect to the master weights is the gradient with respect to the rounded ones.

Parameter packing (float arrays, row-major [out][in] matrices):
  encoder  E1[W][P_out+P_in] e1[W] E2[W][W] e2[W] E3[2L][W] e3[2L]     input order [x ; c]
  decoder  D1[W][P_in+L]     d1[W] D2[W][W] d2[W] D3[2P_out][W] d3[2P_out]  input order [c ; z]
A CVAE's parameter vector is the encoder block followed by the decoder block.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import this module.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

LOG_2PI = float(np.log(2.0 * np.pi))


@dataclass(frozen=True)
class Shape:
    p_in: int
    p_out: int
    latent: int = 4
    width: int = 16

    def enc_sizes(self):
        W, L = self.width, self.latent
        return [("E1", (W, self.p_out + self.p_in)), ("e1", (W,)), ("E2", (W, W)), ("e2", (W,)),
                ("E3", (2 * L, W)), ("e3", (2 * L,))]

    def dec_sizes(self):
        W, L = self.width, self.latent
        return [("D1", (W, self.p_in + L)), ("d1", (W,)), ("D2", (W, W)), ("d2", (W,)),
                ("D3", (2 * self.p_out, W)), ("d3", (2 * self.p_out,))]

    @property
    def n_dec(self) -> int:
        return sum(int(np.prod(s)) for _, s in self.dec_sizes())

    @property
    def n_enc(self) -> int:
        return sum(int(np.prod(s)) for _, s in self.enc_sizes())

    @property
    def n_params(self) -> int:
        return self.n_enc + self.n_dec


def unpack(vec, sizes):
    out, off = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = np.asarray(vec[off:off + n], dtype=np.float64).reshape(shp)
        off += n
    return out, off


def split_cvae(params, shape: Shape):
    enc, n = unpack(params, shape.enc_sizes())
    dec, _ = unpack(params[n:], shape.dec_sizes())
    return enc, dec


def softplus(a):
    return np.logaddexp(0.0, a)


def sigmoid(a):
    return 0.5 * (1.0 + np.tanh(0.5 * a))


def round_bf16(a):
    """Round to bfloat16, nearest even (through float32, whose top 16 bits are bfloat16)."""
    b = np.asarray(a, np.float64).astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _q(a, bf16):
    return round_bf16(a) if bf16 else a


def mlp3(Wa, ba, Wb, bb, Wc, bc, inp, bf16=False):
    """Three weight layers with Softplus after the first two (Sec. 3.2, Fig. 3b)."""
    inp = _q(inp, bf16)
    a1 = inp @ _q(Wa, bf16).T + ba
    h1 = _q(softplus(a1), bf16)
    a2 = h1 @ _q(Wb, bf16).T + bb
    h2 = _q(softplus(a2), bf16)
    out = h2 @ _q(Wc, bf16).T + bc
    return out, (inp, a1, h1, a2, h2)


def decoder_forward(dec_params, shape: Shape, c, z):
    """Decoder of Sec. 3.2: returns (mu_Dec, log Sigma_Dec), each [n][P_out]."""
    d, _ = unpack(np.asarray(dec_params, dtype=np.float64), shape.dec_sizes())
    inp = np.concatenate([np.asarray(c, np.float64), np.asarray(z, np.float64)], axis=1)
    out, _ = mlp3(d["D1"], d["d1"], d["D2"], d["d2"], d["D3"], d["d3"], inp)
    return out[:, :shape.p_out], out[:, shape.p_out:]


def decoder_sample(dec_params, shape: Shape, c, z, eps):
    """x = sqrt(Sigma_Dec) eps + mu_Dec (reparameterisation, Sec. 3.2)."""
    mu, lv = decoder_forward(dec_params, shape, c, z)
    return mu + np.exp(0.5 * lv) * np.asarray(eps, np.float64)


def neg_elbo(params, shape: Shape, x, c, eps_z, bf16=False):
    """Negative ELBO averaged over the batch; returns (loss, rec, kl, cache)."""
    enc, dec = split_cvae(np.asarray(params, np.float64), shape)
    x = np.asarray(x, np.float64)
    c = np.asarray(c, np.float64)
    eps_z = np.asarray(eps_z, np.float64)
    L, P = shape.latent, shape.p_out
    eo, ecache = mlp3(enc["E1"], enc["e1"], enc["E2"], enc["e2"], enc["E3"], enc["e3"],
                      np.concatenate([x, c], axis=1), bf16)
    mu_e, lv_e = eo[:, :L], eo[:, L:]
    sd_e = np.exp(0.5 * lv_e)
    z = mu_e + sd_e * eps_z
    do, dcache = mlp3(dec["D1"], dec["d1"], dec["D2"], dec["d2"], dec["D3"], dec["d3"],
                      np.concatenate([c, z], axis=1), bf16)
    mu_d, lv_d = do[:, :P], do[:, P:]
    r = x - mu_d
    inv_var = np.exp(-lv_d)
    rec = 0.5 * np.sum(lv_d + r * r * inv_var + LOG_2PI, axis=1)
    kl = 0.5 * np.sum(mu_e * mu_e + np.exp(lv_e) - lv_e - 1.0, axis=1)
    cache = dict(enc=enc, dec=dec, ecache=ecache, dcache=dcache, mu_e=mu_e, lv_e=lv_e, sd_e=sd_e,
                 r=r, inv_var=inv_var, eps_z=eps_z, bf16=bf16)
    return float(np.mean(rec + kl)), float(np.mean(rec)), float(np.mean(kl)), cache


def _mlp3_backward(Wa, Wb, Wc, cache, dout):
    inp, a1, h1, a2, h2 = cache
    gWc = dout.T @ h2
    gbc = dout.sum(axis=0)
    dh2 = dout @ Wc
    da2 = dh2 * sigmoid(a2)
    gWb = da2.T @ h1
    gbb = da2.sum(axis=0)
    dh1 = da2 @ Wb
    da1 = dh1 * sigmoid(a1)
    gWa = da1.T @ inp
    gba = da1.sum(axis=0)
    dinp = da1 @ Wa
    return (gWa, gba, gWb, gbb, gWc, gbc), dinp


def neg_elbo_grad(params, shape: Shape, x, c, eps_z, bf16=False):
    """Analytic gradient of neg_elbo with respect to the packed parameters; returns (loss, rec, kl, grad)."""
    loss, rec, kl, C = neg_elbo(params, shape, x, c, eps_z, bf16)
    qw = lambda W: _q(W, bf16)
    B = x.shape[0]
    L = shape.latent
    enc, dec = C["enc"], C["dec"]
    dmu_d = -C["r"] * C["inv_var"] / B
    dlv_d = 0.5 * (1.0 - C["r"] * C["r"] * C["inv_var"]) / B
    gdec, dinp = _mlp3_backward(qw(dec["D1"]), qw(dec["D2"]), qw(dec["D3"]), C["dcache"],
                                np.concatenate([dmu_d, dlv_d], 1))
    dz = dinp[:, shape.p_in:]
    dmu_e = dz + C["mu_e"] / B
    dlv_e = dz * C["eps_z"] * 0.5 * C["sd_e"] + 0.5 * (np.exp(C["lv_e"]) - 1.0) / B
    genc, _ = _mlp3_backward(qw(enc["E1"]), qw(enc["E2"]), qw(enc["E3"]), C["ecache"],
                             np.concatenate([dmu_e, dlv_e], 1))
    grad = np.concatenate([g.ravel() for g in genc] + [g.ravel() for g in gdec])
    assert grad.size == shape.n_params and L == shape.latent
    return loss, rec, kl, grad


def adam_step(params, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0):
    """One Adam step (Kingma & Ba), bias-corrected, t = 1, 2, ...; AdamW decoupled decay when weight_decay > 0.
    Returns new (params, m, v)."""
    p = np.asarray(params, np.float64).copy()
    if weight_decay:
        p = p - lr * weight_decay * p
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    p = p - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


def training_targets(n_events, exit_pos, exit_dir, rep_pos, rep_dir, optical_radius, g, albedo, u_deq):
    """Walk records -> conditions and targets of LengthGen, PathGen and EventGen (Sec. 4.1, Eq. 3).

    Each record is rotated about the reference direction (0,0,1) by -psi, psi = atan2(x_y, x_x), so that the
    exit point lies in the x-z half-plane with x >= 0, i.e. x~ = (sin theta, 0, cos theta) of Eq. 4.  In that
    frame e_b = (0,1,0) and e_t = (cos theta, 0, -sin theta), so alpha = w~_y and
    beta = w~_x cos theta - w~_z sin theta.  The scatter count is dequantised as y = ln(N - 1/2 + u).
    Returns dict of float64 arrays: cL[n,2], xL[n,1], cP[n,3], xP[n,3], cE[n,7], xE[n,6].
    """
    N = np.asarray(n_events, np.float64)
    xp = np.asarray(exit_pos, np.float64).reshape(-1, 3)
    wp = np.asarray(exit_dir, np.float64).reshape(-1, 3)
    Xp = np.asarray(rep_pos, np.float64).reshape(-1, 3)
    Wp = np.asarray(rep_dir, np.float64).reshape(-1, 3)
    psi = np.arctan2(xp[:, 1], xp[:, 0])
    cs, sn = np.cos(psi), np.sin(psi)

    def rot(v):
        return np.stack([cs * v[:, 0] + sn * v[:, 1], -sn * v[:, 0] + cs * v[:, 1], v[:, 2]], axis=1)

    xr, wr, Xr, Wr = rot(xp), rot(wp), rot(Xp), rot(Wp)
    ct = xr[:, 2]
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    alpha = wr[:, 1]
    beta = wr[:, 0] * ct - wr[:, 2] * st
    ltau = np.log(np.asarray(optical_radius, np.float64))
    g = np.asarray(g, np.float64)
    phi = np.asarray(albedo, np.float64)
    lnN = np.log(N)
    yN = np.log(N - 0.5 + np.asarray(u_deq, np.float64))
    return dict(
        cL=np.stack([ltau, g], 1), xL=yN[:, None],
        cP=np.stack([ltau, g, lnN], 1), xP=np.stack([ct, alpha, beta], 1),
        cE=np.stack([ltau, g, phi, ct, alpha, beta, lnN], 1), xE=np.concatenate([Xr, Wr], 1),
    )
