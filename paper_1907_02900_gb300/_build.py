"""Compile libhg.so (and the GPU input generator libhg_datagen.so) for sm_103a.

Translation units are compiled in parallel with nvcc and linked into shared
libraries under paper_1907_02900_gb300/lib/.  No CMake; a rebuild happens
only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
           "--expt-relaxed-constexpr", "-I", INCLUDE]

LIBS = {
    "libhg.so": ["hg_build.cu", "hg_probe.cu", "hg_join.cu", "hg_learned.cu", "hg_batch.cu", "hg_trace.cu", "hg_static.cu", "hg_api.cu"],
    "libhg_datagen.so": ["hg_datagen.cu"],
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    return glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> dict[str, str]:
    os.makedirs(LIBDIR, exist_ok=True)
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    deps = _deps()
    out = {}
    jobs = []
    for lib, srcs in LIBS.items():
        srcs = [s for s in srcs if os.path.exists(os.path.join(CSRC, s))]
        if not srcs:
            continue
        target = os.path.join(LIBDIR, lib)
        out[lib] = target
        if not force and not _stale(target, deps):
            continue
        jobs.append((lib, srcs, target))
    if not jobs:
        return out
    cc = nvcc()
    flags = NVFLAGS + (extra or [])

    def compile_one(src: str) -> str:
        obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        cmd = [cc] + ARCH + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, flush=True)
        return obj

    all_srcs = sorted({s for _, srcs, _ in jobs for s in srcs})
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = dict(zip(all_srcs, ex.map(compile_one, all_srcs)))
    for lib, srcs, target in jobs:
        tmp = target + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [objs[s] for s in srcs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {lib} failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, target)
    return out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
