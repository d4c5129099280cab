"""Build libdns.so (the C-ABI library) in-tree for sm_103a.

One translation unit per supported mesh size (dns_inst.cu with -DDNS_N=n)
plus the API unit, compiled in parallel and linked into
paper_1607_00850_gb300/libdns.so.  Object files go to _build/ beside this
file.  Only nvcc is needed (no cmake).

build(checked=True) makes the index-checked library libdns_checked.so
instead (-DDNS_CHECKED; objects in _build/checked/): the mesh sizes of
CHECKED_SIZES get kernels, the others an empty entry, so that it builds in
about half the time."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdns.so")
LIB_CHECKED = os.path.join(HERE, "libdns_checked.so")

SIZES = (6, 8, 12, 16, 18, 24, 32, 36, 48, 54, 64, 72, 96, 108, 128, 144, 162,
         192, 216, 256, 288, 324, 384, 432, 486, 512, 576, 648, 768, 864, 972, 1024)
CHECKED_SIZES = (16, 24, 36, 64, 96, 128, 256, 512, 1024)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdns")
    return cand


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, *extra]


def _sources_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "dns.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, obj: str, defines=()) -> str:
    cmd = [nvcc(), *_flags(defines), "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr}")
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, checked: bool = False) -> str:
    """Compile and link libdns.so (or, checked=True, libdns_checked.so) if
    any source is newer than it."""
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _sources_mtime():
        return lib
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(bdir, exist_ok=True)
    common = ("-DDNS_CHECKED",) if checked else ()
    units = [(os.path.join(CSRC, "dns_api.cu"), os.path.join(bdir, "dns_api.o"), common),
             (os.path.join(CSRC, "dns_noalloc.cu"), os.path.join(bdir, "dns_noalloc.o"), common),
             (os.path.join(CSRC, "dns_les.cu"), os.path.join(bdir, "dns_les.o"), common),
             (os.path.join(CSRC, "dns_peak.cu"), os.path.join(bdir, "dns_peak.o"), common)]
    # the largest meshes' units take longest: start them first, so that the
    # pool's last wave holds small units
    for n in sorted(SIZES, reverse=True):
        stub = ("-DDNS_STUB",) if checked and n not in CHECKED_SIZES else ()
        units.append((os.path.join(CSRC, "dns_inst.cu"), os.path.join(bdir, f"dns_inst_{n}.o"),
                      (f"-DDNS_N={n}", *common, *stub)))
    jobs = jobs or min(len(units), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda u: _compile(*u), units))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
