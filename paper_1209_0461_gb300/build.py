"""Build libnupm.so (sm_103a) in-tree with nvcc.

Each .cu translation unit is compiled in parallel; the CUDA runtime is linked
statically so the library also loads on hosts without a GPU.  The output is
``paper_1209_0461_gb300/libnupm.so``; objects go to ``_build/`` beside it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libnupm.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["grid_f32.cu", "grid_f64.cu", "nu_response.cu", "pm_api.cu", "bins_static.cu", "sort.cu", "mlp.cu",
           "peaks.cu", "batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "--expt-relaxed-constexpr", "-lineinfo", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fvisibility=hidden"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, force: bool = False, ptxas_log: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "nupm.h"))
    nv = nvcc()
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or not _newer(o, [s] + headers):
            cmd = [nv] + ARCH + FLAGS + ["-c", s, "-o", o]
            if ptxas_log:
                cmd += ["-Xptxas", "-v"]
            jobs.append((src, cmd))

    def run(job):
        name, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True, cwd=CSRC)
        if ptxas_log:
            with open(os.path.join(BUILD, name + ".ptxas.log"), "w") as f:
                f.write(r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{r.stderr[-4000:]}")
        return name

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for name in ex.map(run, jobs):
            if verbose:
                print("compiled", name, file=sys.stderr)
    if force or jobs or not _newer(OUT, objs):
        cmd = [nv] + ARCH + ["-shared", "-cudart", "static", "-o", OUT] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    return OUT


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, ptxas_log="--ptxas" in sys.argv))
