"""Build libnrto.so in-tree for sm_103a with nvcc (no JIT cache, no torch extension machinery)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libnrto.so")
SOURCES = ["api.cu", "mlp.cu", "solver_uni.cu", "solver_quad.cu", "solver_arm.cu"]
FLAGS = ["-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-lineinfo",
         "-gencode", "arch=compute_103a,code=sm_103a", "--expt-relaxed-constexpr"]


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    out.append(os.path.join(HERE, "..", "include", "nrto.h"))
    out.append(os.path.abspath(__file__))
    return out


def _stale() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    return any(os.path.getmtime(d) > t for d in _deps() if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the sources (host API and outer-loop kernels, warm-start network, one solver-kernel
    unit per dynamics kind) into libnrto.so if stale; the units compile in parallel processes."""
    if not force and not _stale():
        return OUT
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    compile_flags = [f for f in FLAGS if f != "-shared"]
    procs = []
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = ["nvcc", *compile_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    failed = False
    for src, obj, pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            failed = True
            sys.stderr.write(f"--- {src}\n{out}{err}")
        elif verbose:
            sys.stderr.write(f"--- {src}\n{err}")
    if failed:
        raise RuntimeError("nvcc failed building libnrto.so")
    link = ["nvcc", "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", OUT + ".tmp",
            *[obj for _, obj, _ in procs]]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking libnrto.so")
    os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(OUT)
