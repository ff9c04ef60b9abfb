"""Builds the AIRPF CUDA library in-tree: paper_2312_06484_gb300/_build/libairpf.so.

sm_103a only (one -gencode), translation units compiled in parallel, no cmake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libairpf.so")
SOURCES = ["airpf_step.cu", "airpf_api.cu", "airpf_pmmh.cu", "airpf_static.cu", "airpf_group.cu", "airpf_grad.cu"]
# the step kernels: airpf_launch_inst.cu compiled once per precision, model and
# particles per thread
INST_SOURCE = "airpf_launch_inst.cu"
INST_UNITS = [(r, model, ppt) for r in ("float", "double") for model in ("AR1", "SV", "NGM", "LGSSM", "TOY", "CP")
              for ppt in (2, 4)] + [("float", "SV", 8), ("float", "NGM", 8)]
HEADERS = ["airpf_device.cuh", "airpf_exp_table.h", "airpf_log_table.h", "airpf_sincos_table.h", "airpf_internal.h", "airpf_step_impl.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    include = os.path.join(os.path.dirname(HERE), "include")
    deps_common = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(include, "airpf.h")]
    objs = []
    jobs = []
    units = [(src, src.replace(".cu", ".o"), []) for src in SOURCES]
    units += [(INST_SOURCE, f"airpf_launch_{'f32' if r == 'float' else 'f64'}_{model.lower()}_ppt{ppt}.o",
               [f"-DAIRPF_INST_R={r}", f"-DAIRPF_INST_MODEL={model}", f"-DAIRPF_INST_PPT={ppt}"])
              for r, model, ppt in INST_UNITS]
    for src, obj, defs in units:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, obj)
        objs.append(o)
        if force or _stale(o, [s] + deps_common):
            cmd = [_nvcc(), *ARCH, *FLAGS, *extra_flags, *defs, "-I", include, "-c", s, "-o", o]
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose or r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
