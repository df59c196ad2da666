"""The measured ALU peaks that the benchmark's roofline divides by, and the renderer's per-density fallback
default (a request with min_optical_radius <= 0)."""
import numpy as np
import pytest
import torch

from paper_2011_03082_b300 import ms, synth

pytestmark = pytest.mark.gpu


def test_alu_peaks_are_measured_and_consistent():
    """Every unit's rate is positive and below a per-SM-per-clock bound at the maximum clock (148 SMs,
    2,032 MHz, 10% margin): 128 FFMA; 32 for 2^x, which this GPU issues at twice the rate of the special-function
    unit's other functions (16: log2, sin, rsqrt); 64 integer multiply-add or logic; 32 high-half multiplies.
    FFMA issues several times faster than the special-function unit."""
    r = ms.ms_alu_peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    clk = 2.032e9 * 1.1
    assert all(v > 0 for v in r.values()), r
    bound = dict(ffma=128, ex2=32, lg2=16, sin=16, rsqrt=16, imad=64, lop3=64, imulhi=32)
    for k, lanes in bound.items():
        assert r[k] <= n_sm * lanes * clk, (k, r[k])
    assert 3.0 <= r["ffma"] / r["sin"] <= 20.0, r
    assert r["lop3"] >= r["ex2"], r


def test_default_min_optical_radius_is_the_policy_value():
    """min_optical_radius = 0 renders exactly as the explicit per-density default."""
    from paper_2011_03082_b300 import pipeline
    cs = ms.cvae_set(pipeline.device_decoders(pipeline.load()))
    for sigma in (24.0, 100.0):
        tau = float(ms.lib().ms_render_default_min_optical_radius(sigma))
        outs = []
        for tm in (0.0, tau):
            p = synth.render_scene(sigma, width=16, height=16, spp=8, mode=ms.MS_SPHERE, seed=4)
            p["min_optical_radius"] = tm
            img = torch.zeros(256, dtype=torch.float64, device="cuda")
            st = torch.zeros(16, dtype=torch.int64, device="cuda")
            ms.ms_render(ms.render_params(p), cs, img, st)
            torch.cuda.synchronize()
            outs.append((img.cpu().numpy(), st.cpu().numpy()))
        assert np.array_equal(outs[0][1][:10], outs[1][1][:10])
        assert np.allclose(outs[0][0], outs[1][0], rtol=1e-6, atol=1e-12)
