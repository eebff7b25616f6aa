"""Build of the CUDA library (in-tree, sm_103a only).

Generates the selection-network header and compiles ``csrc/*.cu`` into
``_build/libcrb.so`` with nvcc. No torch extension machinery is involved.
"""

from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
GEN = os.path.join(CSRC, "_gen")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libcrb.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cuh", ".cpp", ".h"))] + [os.path.join(ROOT, "include", "crb.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(GEN, exist_ok=True)
    os.makedirs(OUT, exist_ok=True)
    net = os.path.join(GEN, "networks.cuh")
    gen = os.path.join(CSRC, "gen_networks.py")
    if force or _stale(net, [gen]):
        subprocess.run([sys.executable, gen, net + ".tmp", "--quick"], check=True)
        os.replace(net + ".tmp", net)
    if force or _stale(LIB, _sources() + [net]):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
               "-I", os.path.join(ROOT, "include"), "-I", GEN,
               os.path.join(CSRC, "crb.cu"), os.path.join(CSRC, "noalloc.cu"), os.path.join(CSRC, "serve.cu"),
               os.path.join(CSRC, "poisson.cu"),
               "-o", tmp]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
