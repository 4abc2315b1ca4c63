"""Build libdmas.so (the C-ABI library) in-tree with nvcc for sm_103a.

    python -m paper_2511_09165_b300.build [--force] [--verbose] [--ptxas-v]
                                          [--checked | --both]

Each translation unit compiles in its own nvcc process (in parallel); the
objects are linked into paper_2511_09165_b300/_lib/libdmas.so.  --checked
builds the host-checked variant instead (DMAS_CHECKED: every kernel index
tested before its access), libdmas_checked.so; --both builds the two.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
OBJ_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libdmas.so")
CHECKED_LIB = os.path.join(OUT_DIR, "libdmas_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    out = [os.path.join(CSRC, "dmas_api.cu"), os.path.join(CSRC, "dmas_plan.cpp"),
           os.path.join(CSRC, "dmas_server.cpp")]
    out += [os.path.join(CSRC, f"beam_o{n}.cu") for n in range(1, 9)]
    extra = sorted(f for f in os.listdir(CSRC)
                   if f.endswith(".cu") and not f.startswith(("beam_o", "dmas_api")))
    out += [os.path.join(CSRC, f) for f in extra]
    return out


def _headers() -> list[str]:
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose: bool, ptxas_v: bool, checked: bool = False) -> str:
    obj = os.path.join(OBJ_DIR, ("checked_" if checked else "") + os.path.basename(src) + ".o")
    if not ptxas_v and not _stale(obj, [src] + _headers()):
        return obj
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "-I" + INCLUDE, "-I" + CSRC, "-x", "c++", "-c", src, "-o", obj]
    else:
        cmd = [_nvcc()] + ARCH + NVCC_FLAGS + (["-DDMAS_CHECKED"] if checked else []) + \
            ["-c", src, "-o", obj]
        if ptxas_v:
            cmd.insert(1, "-Xptxas=-v")
    if verbose:
        print(" ".join(cmd), flush=True)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    if ptxas_v:
        sys.stdout.write(res.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False,
          checked: bool = False) -> str:
    """Compile and link libdmas.so (checked: libdmas_checked.so)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    srcs = sources()
    lib = CHECKED_LIB if checked else LIB
    pre = "checked_" if checked else ""
    if force:
        for s in srcs:
            obj = os.path.join(OBJ_DIR, pre + os.path.basename(s) + ".o")
            if os.path.exists(obj):
                os.remove(obj)
    workers = min(len(srcs), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, ptxas_v, checked), srcs))
    if force or _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, lib)
    return lib


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true", help="print register/smem usage")
    ap.add_argument("--checked", action="store_true", help="build libdmas_checked.so only")
    ap.add_argument("--both", action="store_true", help="build libdmas.so and libdmas_checked.so")
    a = ap.parse_args()
    if not a.checked:
        print(build(force=a.force, verbose=a.verbose, ptxas_v=a.ptxas_v))
    if a.checked or a.both:
        print(build(force=a.force, verbose=a.verbose, ptxas_v=a.ptxas_v, checked=True))


if __name__ == "__main__":
    main()
