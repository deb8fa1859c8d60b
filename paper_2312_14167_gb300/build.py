"""Build libfr.so (the FR hot path for sm_103a) in-tree with nvcc.

Translation units are compiled in parallel, one -gencode (sm_103a), then
linked into ``paper_2312_14167_gb300/libfr.so``.  Used by
``__graft_entry__.build()`` and by ``python -m paper_2312_14167_gb300.build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfr.so")

SOURCES = ["fr_mesh.cpp", "fr_api.cu", "fr_k2_f32.cu", "fr_k2_f64.cu",
           "fr_k3_f32.cu", "fr_k3_f64.cu", "fr_peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _flags(debug=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                "--expt-relaxed-constexpr", "-Xptxas", "-O3"]
    if os.environ.get("FR_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    # tuning knobs for sweeps: minimum CTAs per SM asked of the register
    # allocator for the 2-D FP32 stage kernels
    for knob in ("FR_MINB_FLUX_2D_F32", "FR_MINB_GRAD_2D_F32", "FR_MINB_FLUX_3D_F32",
                 "FR_MINB_GRAD_3D_F32"):
        if os.environ.get(knob):
            f += [f"-D{knob}={int(os.environ[knob])}"]
    return f


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(CSRC, "fr_kernels.cuh"), os.path.join(CSRC, "fr_internal.h"),
            os.path.join(ROOT, "include", "fr.h")]
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        if force or _stale(o, s):
            cmd = [nvcc] + _flags() + ["-c", s, "-o", o]
            if src.endswith("_f32.cu") and os.environ.get("FR_F32_FAST", "1") == "1":
                # FP32 kernels: approximate division / square root (a few ulp)
                # and flush-to-zero; the FP32 parity tests bound the result
                cmd = cmd[:1] + ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"] + cmd[1:]
            if src == "fr_api.cu":
                cmd = cmd[:1] + ["-Xcompiler", "-fopenmp"] + cmd[1:]
            if src.endswith(".cpp"):
                cmd = [nvcc, "-x", "cu"] + _flags() + ["-Xcompiler", "-fopenmp", "-c", s, "-o", o]
            jobs.append((src, cmd))

    def run(job):
        src, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r.returncode, r.stdout + r.stderr

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for src, rc, out in ex.map(run, jobs):
                if verbose or rc != 0 or os.environ.get("FR_PTXAS_VERBOSE"):
                    sys.stderr.write(out)
                if rc != 0:
                    raise RuntimeError(f"nvcc failed on {src}")
    objs = [os.path.join(BUILD, s + ".o") for s in SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fopenmp", "-o", tmp] + objs + ["-lcudart", "-lgomp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
