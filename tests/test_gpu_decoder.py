"""GPU parity of ms_cvae_infer (Sec. 3.2 decoder) against the FP64 oracle decoder.

Tolerances: FP32 max |error| <= 1e-5 on the decoder outputs when z and eps are given (the arithmetic of the
kernel alone); <= 1e-4 when the kernel draws z and eps from its Philox stream (single-precision Box-Muller
against the oracle's double-precision Box-Muller on the same words)."""
import numpy as np
import pytest
import torch

from oracle import cvae
from paper_2011_03082_b300 import ms, synth

pytestmark = pytest.mark.gpu

# (p_in, p_out, latent, width): latent-4 / width-16 shapes, the final Table 1 shapes, and width 8 with P_out 6
SHAPES = [(4, 1, 4, 16), (4, 6, 4, 16), (2, 1, 4, 16), (3, 3, 4, 16), (7, 6, 4, 16), (1, 8, 4, 16),
          (12, 2, 4, 16), (2, 1, 2, 8), (3, 3, 5, 16), (7, 6, 5, 16), (4, 6, 4, 8)]


def _run(w, p_in, p_out, cond, n, z_eps=None, seed=7, offset=0, latent=4, width=16):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    wt, ct = dev(w), dev(cond)
    ze = dev(z_eps) if z_eps is not None else None
    mlv = torch.zeros(n, 2 * p_out, device="cuda")
    smp = torch.zeros(n, p_out, device="cuda")
    d = ms.decoder_struct(wt, p_in, p_out, latent=latent, width=width)
    ms.ms_cvae_infer(d, ct, n, z_eps=ze, seed=seed, offset=offset, out_mean_logvar=mlv, out_sample=smp)
    torch.cuda.synchronize()
    return mlv.cpu().numpy(), smp.cpu().numpy()


@pytest.mark.parametrize("p_in,p_out,latent,width", SHAPES)
@pytest.mark.parametrize("n", [1, 1000, 65539])
def test_decoder_given_normals(p_in, p_out, latent, width, n):
    shape = cvae.Shape(p_in, p_out, latent, width)
    w = synth.xavier_decoder(7, p_in, p_out, latent, width)
    w = w + np.float32(0.05) * synth.standard_normals(8, w.shape)   # nonzero biases too
    rng = np.random.default_rng(1)
    cond = rng.uniform(-1, 2, (n, p_in)).astype(np.float32)
    ze = synth.standard_normals(2, (n, latent + p_out))
    mlv, smp = _run(w, p_in, p_out, cond, n, ze, latent=latent, width=width)
    mu, lv = cvae.decoder_forward(w.astype(np.float64), shape, cond, ze[:, :latent])
    assert np.abs(mlv[:, :p_out] - mu).max() <= 1e-5
    assert np.abs(mlv[:, p_out:] - lv).max() <= 1e-5
    ref = mu + np.exp(0.5 * lv) * ze[:, latent:]
    assert np.abs(smp - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("p_in,p_out,latent,width", [(4, 1, 4, 16), (4, 6, 4, 16), (2, 1, 2, 8), (7, 6, 5, 16),
                                                     (3, 3, 5, 16), (5, 2, 3, 16)])
def test_decoder_philox_normals(orc, p_in, p_out, latent, width):
    n, offset = 5000, 123456
    w = synth.xavier_decoder(7, p_in, p_out, latent, width)
    cond = np.random.default_rng(4).uniform(-1, 2, (n, p_in)).astype(np.float32)
    mlv, smp = _run(w, p_in, p_out, cond, n, None, seed=7, offset=offset, latent=latent, width=width)
    nz = orc.decoder_normals(7, offset, n, latent + p_out)
    shape = cvae.Shape(p_in, p_out, latent, width)
    mu, lv = cvae.decoder_forward(w.astype(np.float64), shape, cond, nz[:, :latent])
    assert np.abs(mlv[:, :p_out] - mu).max() <= 1e-4
    ref = mu + np.exp(0.5 * lv) * nz[:, latent:]
    assert np.abs(smp - ref).max() <= 1e-4


@pytest.mark.parametrize("prec", [ms.MS_FP32, ms.MS_FP16])
@pytest.mark.parametrize("p_in,p_out,latent,width", [(4, 6, 4, 16), (7, 6, 5, 16), (2, 1, 2, 8)])
def test_unaligned_rows_take_the_general_path_with_equal_results(p_in, p_out, latent, width, prec):
    """Row pointers that are not 16-byte aligned go to the runtime-shaped kernels; they compute the same
    arithmetic as the shape-specialised ones, so the outputs are bit-identical."""
    n = 3000
    w = torch.from_numpy(synth.xavier_decoder(7, p_in, p_out, latent, width)).cuda()
    cond = np.random.default_rng(5).uniform(-1, 2, (n, p_in)).astype(np.float32)
    d = ms.decoder_struct(w, p_in, p_out, latent, width, precision=prec)
    outs = []
    for shift in (0, 1):                       # shift 1: every pointer 4 bytes past a 16-byte boundary
        cbuf = torch.zeros(n * p_in + 4, device="cuda")
        cbuf[shift:shift + n * p_in] = torch.from_numpy(cond.ravel()).cuda()
        mbuf = torch.zeros(n * 2 * p_out + 4, device="cuda")
        sbuf = torch.zeros(n * p_out + 4, device="cuda")
        c = cbuf[shift:shift + n * p_in].view(n, p_in)
        mlv = mbuf[shift:shift + n * 2 * p_out].view(n, 2 * p_out)
        smp = sbuf[shift:shift + n * p_out].view(n, p_out)
        ms.ms_cvae_infer(d, c, n, seed=3, offset=9, out_mean_logvar=mlv, out_sample=smp)
        torch.cuda.synchronize()
        outs.append((mlv.cpu().numpy().copy(), smp.cpu().numpy().copy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_decoder_full_size_sampled(orc):
    """The 2^22-query configuration (condition [log tau, g, albedo, cos] + z of dim 4, P_out 6): sampled
    queries recomputed by the oracle."""
    n, p_in, p_out = 1 << 22, 4, 6
    w = synth.xavier_decoder(7, p_in, p_out)
    cond = synth.decoder_queries(7, n)
    mlv, smp = _run(w, p_in, p_out, cond, n, None, seed=7)
    idx = np.random.default_rng(3).choice(n, 2000, replace=False)
    idx.sort()
    nz = np.concatenate([orc.decoder_normals(7, int(i), 1, 10) for i in idx])
    mu, lv = cvae.decoder_forward(w.astype(np.float64), cvae.Shape(p_in, p_out), cond[idx], nz[:, :4])
    assert np.abs(mlv[idx, :p_out] - mu).max() <= 1e-4
    assert np.all(np.isfinite(smp))


def test_decoder_rejects_bad_shapes():
    w = torch.zeros(1000, device="cuda")
    c = torch.zeros(4, 4, device="cuda")
    out = torch.zeros(4, 2, device="cuda")
    for kw in (dict(p_in=4, p_out=9), dict(p_in=13, p_out=1), dict(p_in=4, p_out=1, width=12)):
        d = ms.decoder_struct(w, kw["p_in"], kw["p_out"], width=kw.get("width", 16))
        with pytest.raises(ms.MsError):
            ms.ms_cvae_infer(d, c, 4, out_mean_logvar=out)


def _round_bf16(a):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    b = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("p_in,p_out,latent,width", [(4, 1, 4, 16), (4, 6, 4, 16), (7, 6, 4, 16), (3, 3, 4, 16),
                                                     (2, 1, 2, 8), (3, 3, 5, 16), (7, 6, 5, 16), (4, 6, 4, 8)])
def test_half_precision_decoder(p_in, p_out, latent, width, prec):
    """Tensor-core decoder (FP16 or BF16 weights and activations, FP32 accumulation): max |error| <= 3e-3
    against the FP64 oracle given the same rounded weights; the error against the FP32 weights is bounded
    too (rounding of the weights themselves)."""
    n = 40000
    w = synth.xavier_decoder(7, p_in, p_out, latent, width)
    cond = synth.decoder_queries(7, n)[:, :p_in] if p_in <= 4 else \
        np.random.default_rng(2).uniform(-1, 2, (n, p_in)).astype(np.float32)
    ze = synth.standard_normals(3, (n, latent + p_out))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    mlv = torch.zeros(n, 2 * p_out, device="cuda")
    smp = torch.zeros(n, p_out, device="cuda")
    d = ms.decoder_struct(dev(w), p_in, p_out, latent, width, precision=ms.MS_FP16 if prec == "fp16" else ms.MS_BF16)
    ms.ms_cvae_infer(d, dev(cond), n, z_eps=dev(ze), out_mean_logvar=mlv, out_sample=smp)
    torch.cuda.synchronize()
    wq = w.astype(np.float16).astype(np.float64) if prec == "fp16" else _round_bf16(w)
    shape = cvae.Shape(p_in, p_out, latent, width)
    mu, lv = cvae.decoder_forward(wq, shape, cond, ze[:, :latent])
    got = mlv.cpu().numpy()
    assert np.abs(got[:, :p_out] - mu).max() <= 3e-3
    assert np.abs(got[:, p_out:] - lv).max() <= 3e-3
    mu32, _ = cvae.decoder_forward(w.astype(np.float64), shape, cond, ze[:, :latent])
    assert np.abs(got[:, :p_out] - mu32).max() <= (2e-2 if prec == "bf16" else 3e-3)
    assert np.allclose(smp.cpu().numpy(), mu + np.exp(0.5 * lv) * ze[:, latent:], atol=1e-2)


def test_decoder_error_report_on_the_benchmark_queries(capsys):
    """The decoder workload's queries (condition (log tau, g, albedo, cos) + latent 4, width 16, P_out 1 and 6;
    65,536 queries with given normals) in each precision: max |error| of (mu, log Sigma) against the FP64 oracle
    with the weights the kernel multiplies (the kernel's arithmetic; <= 1e-5 FP32, <= 3e-3 FP16 / BF16) and
    against the unrounded weights (the total error of the half-precision forms), printed as a table."""
    n = 65536
    cond = synth.decoder_queries(7, n)
    rows = []
    for p_out in (1, 6):
        w = synth.xavier_decoder(7, 4, p_out)
        ze = synth.standard_normals(5, (n, 4 + p_out))
        shape = cvae.Shape(4, p_out, 4, 16)
        mu64, lv64 = cvae.decoder_forward(w.astype(np.float64), shape, cond, ze[:, :4])
        ref = np.concatenate([mu64, lv64], axis=1)
        for prec, code in (("fp32", ms.MS_FP32), ("fp16", ms.MS_FP16), ("bf16", ms.MS_BF16)):
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
            mlv = torch.zeros(n, 2 * p_out, device="cuda")
            d = ms.decoder_struct(dev(w), 4, p_out, 4, 16, precision=code)
            ms.ms_cvae_infer(d, dev(cond), n, z_eps=dev(ze), out_mean_logvar=mlv)
            torch.cuda.synchronize()
            got = mlv.cpu().numpy()
            if prec == "fp32":
                err_k = np.abs(got - ref).max()
            else:
                wq = w.astype(np.float16).astype(np.float64) if prec == "fp16" else _round_bf16(w)
                mq, lq = cvae.decoder_forward(wq, shape, cond, ze[:, :4])
                err_k = np.abs(got - np.concatenate([mq, lq], axis=1)).max()
            err_t = np.abs(got - ref).max()
            rows.append((p_out, prec, err_k, err_t))
            assert err_k <= (1e-5 if prec == "fp32" else 3e-3), (p_out, prec, err_k)
    with capsys.disabled():
        print("\nP_out  precision  max|err| kernel arithmetic   max|err| total (vs FP32 weights)")
        for p_out, prec, ek, et in rows:
            print(f"{p_out:5d}  {prec:9s}  {ek:.2e}                  {et:.2e}")
