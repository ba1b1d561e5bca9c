"""Builds the CUDA library libsq_gb300.so in-tree for sm_103a (nvcc, no cmake).

    python -m paper_2006_03697_gb300.build          # or build() from Python

Each .cu translation unit is compiled in parallel, then linked into one shared object
under paper_2006_03697_gb300/_lib/. The ABI it exports is include/sq_api.h.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
SRC = PKG / "csrc"
OUT_DIR = PKG / "_lib"
LIB = OUT_DIR / "libsq_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["sq_api.cu", "sq_setup.cu", "sq_sweep.cu", "sq_step_tma.cu", "sq_reduce.cu", "sq_lanczos.cu", "sq_noalloc.cu", "sq_batch.cu", "sq_serve.cu", "sq_gk.cu", "sq_gauss.cu"]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or "/usr/local/cuda/bin/nvcc"
    return cand if Path(cand).exists() else "nvcc"


def build(verbose: bool = False, force: bool = False) -> Path:
    OUT_DIR.mkdir(exist_ok=True)
    srcs = [SRC / s for s in SOURCES]
    deps = srcs + list(SRC.glob("*.h")) + list(SRC.glob("*.cuh")) + [ROOT / "include" / "sq_api.h"]
    if LIB.exists() and not force:
        newest = max(p.stat().st_mtime for p in deps)
        if LIB.stat().st_mtime > newest:
            return LIB
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(ROOT / "include"),
                    "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
    objs = []
    procs = []
    for s in srcs:
        o = OUT_DIR / (s.stem + ".o")
        objs.append(o)
        cmd = [nvcc()] + flags + ["-c", str(s), "-o", str(o)]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        txt = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(" ".join(cmd) + "\n" + txt)
        elif verbose and txt.strip():
            print(txt)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [nvcc()] + ARCH + ["-shared", "-o", str(tmp)] + [str(o) for o in objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
