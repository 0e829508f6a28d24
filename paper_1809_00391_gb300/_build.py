"""Build libmbt.so in-tree with nvcc for sm_103a (GB300).

Each CUDA translation unit is compiled in parallel, then linked into
``paper_1809_00391_gb300/_build/libmbt.so`` (CUDA runtime linked statically).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = BUILD / "libmbt.so"
INCLUDE = PKG.parent / "include"
SOURCES = ["k_push.cu", "k_post.cu", "k_resident.cu", "api.cu", "serve.cu", "sharded.cu", "k_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code is built without floating-point contraction so that it rounds the
# same on x86-64 and aarch64 (gcc fuses a*b+c into an FMA by default on Arm).
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I", str(INCLUDE)]
# extra nvcc flags for tuning experiments (e.g. "-DMBT_PUSH_STAGES=2"); part of the staleness key
EXTRA = os.environ.get("MBT_NVCC_EXTRA", "").split()


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmbt")


def _stale() -> bool:
    if not LIB.exists():
        return True
    stamp = BUILD / "flags.txt"
    if not stamp.exists() or stamp.read_text() != " ".join(FLAGS + EXTRA):
        return True
    t = LIB.stat().st_mtime
    deps = [Path(__file__)] + list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) + list(INCLUDE.glob("*.h"))
    return any(p.stat().st_mtime > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    """Compile every CUDA source and link libmbt.so; returns its path."""
    if not force and not _stale():
        return LIB
    BUILD.mkdir(exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = BUILD / (Path(src).stem + ".o")
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *EXTRA, "-c", str(CSRC / src), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            print(out)
        if p.returncode != 0:
            failed.append((" ".join(cmd), out))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"$ {c}\n{o}" for c, o in failed))
    tmp = BUILD / f"libmbt.{os.getpid()}.so"
    link = [nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout)
    os.replace(tmp, LIB)
    (BUILD / "flags.txt").write_text(" ".join(FLAGS + EXTRA))
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
