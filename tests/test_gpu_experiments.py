"""The absorption and fallback studies (Sec. 5, Fig. 8; Sec. 6 thin-region fallback) on small images: what
their images must show independently of timing."""
import numpy as np
import pytest

from paper_2011_03082_b300 import experiments

pytestmark = pytest.mark.gpu


def test_absorption_sweep_darkens_with_absorption():
    """RGB absorption (2e-3, 2e-4, 2e-3) x 2^i: every channel gets darker as absorption doubles, in both
    methods, and the channel with ten times less absorption (green) stays the brightest."""
    rows = experiments.absorption_sweep(sigma=32.0, res=48, spp=32, settings=3)
    for name in ("sphere", "brute"):
        means = np.array([r[name]["mean_rgb"] for r in rows])
        assert np.all(np.diff(means[:, 0]) < 0) and np.all(np.diff(means[:, 2]) < 0), means
        assert np.all(means[:, 1] > means[:, 0]), means
        assert all(r[name]["seconds"] > 0 for r in rows)


def test_fallback_sweep_runs_and_reports_errors():
    rows = experiments.fallback_sweep(sigma=32.0, res=32, spp=16, ref_spp=256, tau_mins=(1.0, 4.0))
    assert len(rows) == 3 and rows[-1]["mode"] == "brute force"
    assert all(np.isfinite(r["rmse"]) and r["rmse"] > 0 and r["seconds"] > 0 for r in rows)
