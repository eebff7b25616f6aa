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
        units = ["crb.cu", "noalloc.cu", "serve.cu", "poisson.cu", "partition.cu"]
        common = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                  "-I", os.path.join(ROOT, "include"), "-I", GEN]
        if verbose:
            common.insert(1, "-Xptxas=-v")
        # the translation units compile in parallel, then link into one shared library
        procs = []
        for u in units:
            obj = os.path.join(OUT, u + f".{os.getpid()}.o")
            procs.append((obj, subprocess.Popen(common + ["-c", os.path.join(CSRC, u), "-o", obj],
                                                stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        log, failed = "", False
        for obj, pr in procs:
            out, _ = pr.communicate()
            log += out
            failed |= pr.returncode != 0
        if failed:
            raise RuntimeError("nvcc failed:\n" + log)
        if verbose:
            print(log)
        tmp = LIB + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp] + [o for o, _ in procs], capture_output=True,
                           text=True)
        for o, _ in procs:
            os.remove(o)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
