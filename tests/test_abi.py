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
