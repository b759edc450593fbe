"""Builds libhologen.so in-tree with nvcc for sm_103a (no CMake, no torch extension machinery).

Each FFT length with a compiled instance is one translation unit (csrc/hg_len.cu with -DHG_LEN=N);
the generic kernels of every other {2,3,5}-smooth length are csrc/hg_gen.cu; the C ABI is
csrc/hg_api.cu.  Objects go to paper_2006_10509_gb300/_build/, the library to
paper_2006_10509_gb300/libhologen.so.  Translation units compile in parallel and are rebuilt only
when a source or header is newer than the object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhologen.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def lengths() -> list[int]:
    with open(os.path.join(CSRC, "hg_launch.h")) as f:
        text = f.read()
    m = re.search(r"#define HG_FOR_EACH_LENGTH\(X\)(.*?)\n\n", text, re.S)
    return [int(x) for x in re.findall(r"X\((\d+)\)", m.group(1))]


def _deps() -> float:
    newest = 0.0
    for d in (CSRC, INCLUDE):
        for name in os.listdir(d):
            if name.endswith((".cu", ".cuh", ".h")):
                newest = max(newest, os.path.getmtime(os.path.join(d, name)))
    return max(newest, os.path.getmtime(__file__))


def _compile(src: str, obj: str, defines: list[str], verbose: bool) -> str:
    cmd = [nvcc(), *ARCH, *CFLAGS, *defines, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr}")
    return r.stderr


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compiles (incrementally) and links libhologen.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    newest = _deps()
    units = [(os.path.join(CSRC, "hg_len.cu"), os.path.join(BUILD, f"hg_len_{n}.o"), [f"-DHG_LEN={n}"]) for n in lengths()]
    units.append((os.path.join(CSRC, "hg_api.cu"), os.path.join(BUILD, "hg_api.o"), []))
    units.append((os.path.join(CSRC, "hg_noalloc.cu"), os.path.join(BUILD, "hg_noalloc.o"), []))
    units.append((os.path.join(CSRC, "hg_dbs.cu"), os.path.join(BUILD, "hg_dbs.o"), []))
    units.append((os.path.join(CSRC, "hg_gen.cu"), os.path.join(BUILD, "hg_gen.o"), []))
    todo = [u for u in units if not os.path.exists(u[1]) or os.path.getmtime(u[1]) < newest]
    jobs = jobs or max(1, min(len(todo), os.cpu_count() or 4))
    logs = []
    if todo:
        with cf.ThreadPoolExecutor(jobs) as ex:
            futs = [ex.submit(_compile, s, o, d, verbose) for s, o, d in todo]
            for f in futs:
                logs.append(f.result())
    objs = [u[1] for u in units]
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        sys.stderr.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
