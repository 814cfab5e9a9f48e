"""Builds libfe.so in-tree for sm_103a: runs the local-kernel generator, then nvcc per
translation unit (in parallel) and links a shared library with the static CUDA runtime.

    python -m paper_1501_01809_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
GEN = os.path.join(CSRC, "generated", "fe_local.cuh")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libfe.so")
SOURCES = ["fe_api.cpp", "fe_sparsity.cu", "fe_assemble.cu", "fe_asm_f64_push.cu", "fe_asm_f64_pull.cu",
           "fe_asm_dd2.cu", "fe_asm_dd3_push.cu", "fe_asm_dd3_pull.cu", "fe_asm_fused_f64.cu", "fe_asm_fused_dd.cu", "fe_asm_f32.cu", "fe_asm_tc.cu", "fe_batch.cu", "fe_solve.cu", "fe_serve.cpp", "fe_serve_asm.cu", "fe_global.cu", "fe_wave.cu",
           "fe_noalloc.cu", "fe_stored_f64.cu", "fe_stored_dd.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfe")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    from . import codegen
    os.makedirs(os.path.dirname(GEN), exist_ok=True)
    codegen.main(["codegen", GEN])
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers += [GEN, os.path.join(ROOT, "include", "fe.h")]
    cc = nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src + ".o")
        if force or _stale(o, [s] + headers):
            cmd = [cc] + _flags() + ["-c", s, "-o", o + ".tmp"]
            jobs.append((cmd, o))

    def run(job):
        cmd, o = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {o}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(o + ".tmp", o)
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return o

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(OUT_DIR, s + ".o") for s in SOURCES]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
