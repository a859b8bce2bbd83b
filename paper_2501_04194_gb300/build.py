"""Build libstl.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into a shared library with the
static CUDA runtime.  The library exports only the extern "C" ABI of include/stl.h.
"""
from __future__ import annotations

import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstl.so")
SOURCES = [f"stl_kern_{nt}_{d}{m}{r}.cu" for nt in (64, 256, 512) for d in "fb" for m in "hs" for r in ("", "_r")] + ["stl_kernels.cu", "stl_capi.cu", "stl_noalloc.cu", "stl_plan.cu", "stl_gemm.cu", "stl_mining.cu", "stl_fk.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
            "-I", os.path.join(ROOT, "include"), "-I", BUILD, "--expt-relaxed-constexpr", *extra]


FK_DEV = os.path.join(CSRC, "stl_fk_dev.cuh")
FK_INC = os.path.join(BUILD, "stl_fk_src.inc")


def _embed_fk_source():
    """The device building blocks of the formula-compiled kernels, as a C++ raw string (NVRTC
    compiles them at run time together with the generated code)."""
    with open(FK_DEV) as fh:
        src = fh.read()
    assert ")FKSRC" not in src
    text = 'R"FKSRC(' + src + ')FKSRC"\n'
    if not os.path.exists(FK_INC) or open(FK_INC).read() != text:
        with open(FK_INC, "w") as fh:
            fh.write(text)


def _stale(obj, srcs):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    # objects built on another host architecture (x86 here, aarch64 on the GPU machine) are stale
    stamp = os.path.join(BUILD, "ARCH")
    arch = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != arch or not os.path.exists(LIB):
        force = True
    with open(stamp, "w") as fh:
        fh.write(arch)
    _embed_fk_source()
    fk_only = {"stl_fk_dev.cuh", "stl_fk.h"}   # only the compiled-kernel units depend on these
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")) and f not in fk_only]
    headers.append(os.path.join(ROOT, "include", "stl.h"))
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        deps = [s, *headers]
        if src in ("stl_fk.cu", "stl_capi.cu"):
            deps += [os.path.join(CSRC, "stl_fk.h"), FK_INC]
        if force or _stale(o, deps):
            extra = ["-Xptxas", "-v"] if ptxas_info else []
            jobs.append([nvcc(), *_flags(extra), "-c", s, "-o", o])
    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        for l in logs:
            sys.stdout.write(l)
    objs = [os.path.join(BUILD, s + ".o") for s in SOURCES]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-ldl"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
