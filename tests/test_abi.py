"""The C ABI library builds, loads and exports every entry point that include/ms.h declares (CPU only: no
compute call is made)."""
import ctypes
import re
from pathlib import Path

from paper_2011_03082_b300 import build, ms

ROOT = Path(__file__).resolve().parent.parent


def declared_entry_points():
    text = (ROOT / "include" / "ms.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ms_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    build.build()
    lib = ctypes.CDLL(str(ms.LIB_PATH))
    names = declared_entry_points()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(ms.EXPORTS) <= set(names)


def test_host_only_queries():
    L = ms.lib()
    assert L.ms_version() >= 10000
    shape = ms.cvae_shape(7, 6)
    assert ms.ms_cvae_num_params(shape) == (16 * 13 + 16 + 256 + 16 + 8 * 16 + 8) + (16 * 11 + 16 + 256 + 16 + 12 * 16 + 12)
    assert ms.ms_cvae_workspace_size(shape, 65536) > 0


def test_fallback_policy_is_a_host_function_of_the_density():
    """The per-density thin-region threshold (ms_render_default_min_optical_radius) is positive, held constant
    beyond the measured densities, and between two neighbouring knots lies between their values."""
    f = lambda s: float(ms.lib().ms_render_default_min_optical_radius(s))
    knots = [16.0, 32.0, 64.0, 128.0]
    vals = [f(s) for s in knots]
    assert all(v > 0 for v in vals)
    assert f(1.0) == vals[0] and f(1e6) == vals[-1]
    for (a, va), (b, vb) in zip(zip(knots, vals), zip(knots[1:], vals[1:])):
        mid = f((a * b) ** 0.5)
        assert min(va, vb) - 1e-6 <= mid <= max(va, vb) + 1e-6
