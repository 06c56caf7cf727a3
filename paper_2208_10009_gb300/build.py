"""Build the CUDA library (libsbr.so) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel; the shared library links the CUDA runtime
statically.  The output lives in ``paper_2208_10009_gb300/_lib/`` (git-ignored) and is
rebuilt when any source or header is newer than it.  A second variant,
``libsbr_checked.so``, is compiled with -DSBR_CHECKED: device bounds checks on traversal
stacks and face ids that report through the launch's status word (SBR_ECHECK) instead of
faulting.  ``libsbr_probe.so`` holds the FP32 FMA microbenchmark the benchmark's roofline
divides by (a measurement utility; the SBR library does not link it).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib")
SO = os.path.join(OUT, "libsbr.so")
SO_CHECKED = os.path.join(OUT, "libsbr_checked.so")
SO_PROBE = os.path.join(OUT, "libsbr_probe.so")   # FP32 peak microbenchmark (measurement only)
SOURCES = ["capi.cu", "host_geometry.cpp", "host_wedges.cpp", "host_faces.cpp", "kernels_trace.cu", "kernels_diffract.cu",
           "kernels_paths.cu", "kernels_refine.cu", "kernels_unfold.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
VARIANTS = {SO: [], SO_CHECKED: ["-DSBR_CHECKED"], SO_PROBE: []}
VARIANT_SOURCES = {SO: SOURCES, SO_CHECKED: SOURCES, SO_PROBE: ["probe_fp32.cu"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include"),
                   "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def _stale(so: str) -> bool:
    if not os.path.exists(so):
        return True
    t = os.path.getmtime(so)
    deps = glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "sbr.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Compile every translation unit of each stale variant (the checked one too unless
    checked=False) in one parallel pass and link the libraries; returns libsbr.so's path."""
    todo = [so for so in VARIANTS if (so == SO or checked) and (force or _stale(so))]
    if not todo:
        return SO
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()

    def compile_one(job):
        so, src = job
        sub = {SO_CHECKED: os.path.join(OUT, "checked"), SO_PROBE: os.path.join(OUT, "probe")}.get(so, OUT)
        os.makedirs(sub, exist_ok=True)
        obj = os.path.join(sub, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + _flags() + VARIANTS[so] + (["-x", "cu"] if src.endswith(".cpp") else []) + \
            ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return so, obj

    jobs = [(so, src) for so in todo for src in VARIANT_SOURCES[so]]
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), max(os.cpu_count() or 4, 4))) as ex:
        done = list(ex.map(compile_one, jobs))
    for so in todo:
        objs = [o for s, o in done if s == so]
        tmp = so + ".tmp"
        r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread", "-ldl"], capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, so)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose=True))
