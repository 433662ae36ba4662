"""Build ``libef.so`` (the C-ABI library of include/ef.h) in-tree with nvcc for sm_103a.

Objects go to ``_build/`` beside this file; the translation units compile in parallel.  A stamp
of the sources and flags skips the rebuild when nothing changed.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libef.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC] + ARCH
UNITS = ["ef_plan.cpp", "ef_moments.cu", "ef_noalloc.cu", "ef_mlp.cu", "ef_surrogate.cu", "ef_collide_f32_3d.cu", "ef_collide_rg_f32.cu", "ef_collide_tm_f32.cu", "ef_collide_f64_3d.cu",
         "ef_collide_f32_2d.cu", "ef_collide_f64_2d.cu", "ef_features_f32.cu", "ef_features_f64.cu", "ef_step.cu", "ef_stream.cpp",
         "ef_transport.cu", "ef_classical.cu", "ef_kernelg.cu", "ef_galerkin.cu"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stamp() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode() + f.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = _stamp()
    stamp_file = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(OUT) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read() == stamp:
                return OUT
    nvcc = _nvcc()
    procs = []
    objs = []
    for u in UNITS:
        obj = os.path.join(BUILD, u + ".o")
        objs.append(obj)
        cmd = [nvcc] + NVCC_FLAGS + ["-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for u, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((u, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join("%s:\n%s" % f for f in failed))
    tmp = OUT + ".tmp.%d" % os.getpid()
    cmd = [nvcc, "-shared"] + ARCH + ["-o", tmp] + objs + ["-lpthread", "-ldl", "-lrt"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
