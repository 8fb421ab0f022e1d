"""Build the CUDA library libmls.so in-tree (nvcc, sm_103a only).

Each translation unit is compiled in parallel, then linked into
``paper_1408_0677_gb300/_build/libmls.so``.  Rebuilds only what changed.

Variants (separate objects and library, same sources):
  checked=True   -> _build/libmls_checked.so: -DMLS_CHECKED, every bin, tile,
                    cell and list index of the kernels tested against its
                    array (a bad one is recorded in the device error word,
                    which mls_sync reports, and clamped; no trap)
  sanitize=True  -> _build/libmls_asan.so: host code under AddressSanitizer
                    and UndefinedBehaviorSanitizer (load it with the
                    sanitizer runtime preloaded)
The binding loads the library named by MLS_LIBRARY, else libmls.so.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libmls.so")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = ["mls_api.cu", "prep.cu", "prepass.cu", "plain.cu", "handover.cu", "tc.cu", "tc64.cu",
           "bands_noalloc.cu", "variant.cu", "space_map.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _headers_mtime() -> float:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "mls.h"))
    return max(os.path.getmtime(h) for h in hs)


CHECKED_LIB = os.path.join(OUT, "libmls_checked.so")
ASAN_LIB = os.path.join(OUT, "libmls_asan.so")
# one -Xcompiler per flag: nvcc splits an -Xcompiler argument at its commas
SAN_FLAGS = ["-Xcompiler=-fsanitize=address", "-Xcompiler=-fsanitize=undefined", "-Xcompiler=-fno-omit-frame-pointer",
             "-Xcompiler=-fno-sanitize-recover=all"]


def build(force: bool = False, verbose: bool = False, checked: bool = False, sanitize: bool = False) -> str:
    odir = os.path.join(OUT, "checked" if checked else "asan" if sanitize else "")
    lib = CHECKED_LIB if checked else ASAN_LIB if sanitize else LIB
    extra = (["-DMLS_CHECKED"] if checked else []) + (SAN_FLAGS if sanitize else [])
    os.makedirs(odir, exist_ok=True)
    hdr = _headers_mtime()
    nvcc = _nvcc()

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(odir, src.replace(".cu", ".o"))
        if not force and os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), hdr):
            return o, False
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        os.replace(o + ".tmp", o)
        return o, True

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    changed = any(c for _, c in results)
    if force or changed or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", *ARCH, *(SAN_FLAGS if sanitize else []), "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
