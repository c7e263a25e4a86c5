"""Builds libfuse.so (the CUDA library behind include/fuse.h) in-tree with nvcc for sm_103a.

The library is compiled into paper_2210_04184_gb300/_build/libfuse.so; it links the CUDA
runtime statically so the only runtime dependency is the NVIDIA driver."""
from __future__ import annotations

import os
import pathlib
import shutil
import subprocess

PKG = pathlib.Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT = PKG / "_build" / "libfuse.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources() -> list[pathlib.Path]:
    return sorted(CSRC.glob("*.cu"))


def _stale() -> bool:
    if not OUT.exists():
        return True
    t = OUT.stat().st_mtime
    deps = list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh")) + list((ROOT / "include").glob("*.h"))
    return any(p.stat().st_mtime > t for p in deps)


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(force: bool = False, verbose: bool = False) -> pathlib.Path:
    if not force and not _stale():
        return OUT
    OUT.parent.mkdir(exist_ok=True)
    objs = []
    procs = []
    for src in sources():
        obj = OUT.parent / (src.stem + ".o")
        cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               f"-I{ROOT / 'include'}", f"-I{CSRC}", "-c", str(src), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(obj)
    for p, cmd in procs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = OUT.with_name(f"libfuse.{os.getpid()}.so")
    subprocess.run([nvcc(), ARCH, "-shared", "--cudart", "static", *map(str, objs), "-o", str(tmp)],
                   check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
