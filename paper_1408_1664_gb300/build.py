"""Build the CUDA library for sm_103a with nvcc.

The translation units compile in parallel and link into two shared libraries
with a plain C ABI (``include/bnedge.h``): ``_build/libbnedge.so`` (the
release build) and ``_build/libbnedge_testing.so``, the same objects plus the
test hooks of the header's BN_TESTING section (the runtime unit compiled a
second time with BN_TESTING defined).  ``_build/libbnpeaks.so`` holds the
arithmetic-rate probes the benchmark uses for its ALU rooflines.
``build_checked`` makes a debug library on request,
``_build/libbnedge_checked.so``: every unit compiled with BN_CHECK_BOUNDS
(the kernels check the offsets they form; bn_device.cuh) and the test hooks;
``build_asan`` makes ``_build/libbnedge_asan.so``, the host code built with
AddressSanitizer and UndefinedBehaviorSanitizer.
No torch headers are involved.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUTDIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUTDIR, "libbnedge.so")
LIB_TESTING = os.path.join(OUTDIR, "libbnedge_testing.so")
LIB_PEAKS = os.path.join(OUTDIR, "libbnpeaks.so")
LIB_CHECKED = os.path.join(OUTDIR, "libbnedge_checked.so")
LIB_ASAN = os.path.join(OUTDIR, "libbnedge_asan.so")
SOURCES = ["bn_kernels.cu", "bn_tile13.cu", "bn_levels.cu", "bn_runtime.cu", "bn_noalloc.cu",
           "bn_mega.cu"]
# extra nvcc flags per translation unit
UNIT_FLAGS: dict = {}
PEAKS_SOURCE = "bn_peaks.cu"
# (source, object, extra flags) of the second compile of the runtime unit
TESTING_UNIT = ("bn_runtime.cu", "bn_runtime_testing.o", ["-DBN_TESTING"])
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "bnedge.h"))
    return files


def _stale() -> bool:
    libs = (LIB, LIB_TESTING, LIB_PEAKS)
    if not all(os.path.exists(x) for x in libs):
        return True
    t = min(os.path.getmtime(x) for x in libs)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    """Compile (if needed) and return the path of the shared library."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUTDIR, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"] + (extra or [])

    def one(unit):
        src, obj, more = unit
        obj = os.path.join(OUTDIR, obj)
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags + more
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)
        return obj

    units = ([(src, src.replace(".cu", ".o"), UNIT_FLAGS.get(src, [])) for src in SOURCES] + [TESTING_UNIT]
             + [(PEAKS_SOURCE, PEAKS_SOURCE.replace(".cu", ".o"), [])])
    with cf.ThreadPoolExecutor(len(units)) as ex:
        objs = list(ex.map(one, units))
    release = objs[:len(SOURCES)]
    testing = [o for o in release if not o.endswith("bn_runtime.o")] + [objs[-2]]
    for out, parts in ((LIB, release), (LIB_TESTING, testing), (LIB_PEAKS, [objs[-1]])):
        tmp = out + ".tmp"
        cmd = [nvcc(), "-shared", "-o", tmp] + parts + ARCH + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
    return LIB


def _build_variant(out: str, subdir: str, flags_extra: list, link_extra: list, force: bool,
                   verbose: bool) -> str:
    """Every unit compiled once more with flags_extra (the runtime unit also
    with BN_TESTING) and linked into `out`."""
    if (not force and os.path.exists(out)
            and all(os.path.getmtime(f) <= os.path.getmtime(out) for f in _inputs())):
        return out
    odir = os.path.join(OUTDIR, subdir)
    os.makedirs(odir, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "-I", CSRC, "--expt-relaxed-constexpr"] + flags_extra

    def one(src):
        obj = os.path.join(odir, src.replace(".cu", ".o"))
        more = UNIT_FLAGS.get(src, []) + (["-DBN_TESTING"] if src == TESTING_UNIT[0] else [])
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags + more
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(one, SOURCES))
    tmp = out + ".tmp"
    r = subprocess.run([nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"] + link_extra,
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of the BN_CHECK_BOUNDS debug
    library (with the BN_TESTING hooks)."""
    return _build_variant(LIB_CHECKED, "checked", ["-DBN_CHECK_BOUNDS"], [], force, verbose)


# one flag per sanitizer: nvcc splits -Xcompiler arguments at commas
SANITIZE = ["-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer",
            "-fno-sanitize-recover=all"]


def build_asan(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of the library whose host code
    is built with AddressSanitizer and UndefinedBehaviorSanitizer (and the
    BN_TESTING hooks).  A process loading it must preload the sanitizer
    runtimes (LD_PRELOAD of libasan and libubsan)."""
    flags = []
    for f in SANITIZE:
        flags += ["-Xcompiler", f]
    link = []
    for f in SANITIZE[:2]:
        link += ["-Xcompiler", f]
    return _build_variant(LIB_ASAN, "asan", flags + ["-g"], link, force, verbose)


if __name__ == "__main__":
    print(build(force=True, verbose=True))
