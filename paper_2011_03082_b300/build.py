"""Builds the CUDA library ``libms.so`` in-tree for sm_103a with nvcc.

Every ``csrc/*.cu`` file is compiled to an object (in parallel) and linked into one shared library with
the C ABI of ``include/ms.h``.  Translation units listed in ``NO_FMA`` are compiled with ``--fmad=false``
(the bit-reproducible double-precision walk).  Rebuilds only when a source or header is newer than the
library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = ROOT / "_build"
LIB = PKG / "libms.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NO_FMA = {"walk_f64.cu"}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libms.so")


def _flags(src: Path) -> list:
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=default",
         "--expt-relaxed-constexpr", "-I", str(ROOT / "include"), "-I", str(CSRC)] + ARCH
    if src.name in NO_FMA:
        f.append("--fmad=false")
    return f


def sources() -> list:
    return sorted(CSRC.glob("*.cu"))


def _stale() -> bool:
    if not LIB.exists():
        return True
    deps = list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh")) + list((ROOT / "include").glob("*.h")) + [
        Path(__file__)]
    return max(p.stat().st_mtime for p in deps) > LIB.stat().st_mtime


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> Path:
    if not force and not ptxas_info and not _stale():
        return LIB
    BUILD.mkdir(exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(src: Path):
        obj = BUILD / (src.stem + ".o")
        cmd = [cc, "-c", str(src), "-o", str(obj)] + _flags(src)
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for obj, log in ex.map(compile_one, sources()):
            objs.append(obj)
            if verbose or ptxas_info:
                sys.stderr.write(log)
    tmp = LIB.with_name(f"libms.so.tmp{os.getpid()}")
    cmd = [cc, "-shared", "-o", str(tmp)] + [str(o) for o in objs] + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
