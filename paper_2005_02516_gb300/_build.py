"""Compile the CUDA library libesdg.so in-tree for sm_103a.

Translation units compile in parallel (one per polynomial degree, volume
rule and inverse-mass kind, one per rule for the ensemble kernel, plus the
C-ABI, the host builder and the request server) and link into paper_2005_02516_gb300/libesdg.so.
"""

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libesdg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources():
    cu = (["esdg_api.cu", "esdg_ensemble.cu", "esdg_ensemble_s.cu", "esdg_volume.cu", "esdg_sbp_f32.cu",
           "esdg_sbp_f64.cu", "esdg_selftest.cu", "esdg_diag.cu"] + ["esdg_kernels_n%d.cu" % n for n in range(1, 6)]
          + ["esdg_kernels_s%d.cu" % n for n in range(1, 6)]
          + ["esdg_kernels_w%s%d.cu" % (r, n) for r in "ns" for n in range(1, 6)]
          + ["esdg_kernels_tn%d.cu" % n for n in range(1, 4)] + ["esdg_kernels_ts%d.cu" % n for n in range(1, 5)])
    return cu, ["host_build.cpp", "esdg_server.cpp"]


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build failed: %s\n%s" % (" ".join(cmd), p.stdout))
    return p.stdout


def build(verbose=False, extra_nvcc=()):
    os.makedirs(BUILD, exist_ok=True)
    cu, cpp = _sources()
    inc = ["-I", CSRC, "-I", os.path.join(os.path.dirname(HERE), "include")]
    jobs = []
    for f in cu:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append([nvcc(), "-c", os.path.join(CSRC, f), "-o", obj, "-O3", "-std=c++17", "-lineinfo",
                     "-Xcompiler", "-fPIC", *ARCH, *inc, *extra_nvcc])
    for f in cpp:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append([nvcc(), "-x", "c++", "-c", os.path.join(CSRC, f), "-o", obj, "-O2", "-std=c++17",
                     "-Xcompiler", "-fPIC", *inc])
    with ThreadPoolExecutor(max_workers=min(os.cpu_count() or 8, 16, len(jobs))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [os.path.join(BUILD, f + ".o") for f in cu + cpp]
    tmp = LIB + ".tmp"
    _run([nvcc(), "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
