"""Builds libhx.so in-tree from csrc/*.cu with nvcc for sm_103a (and
libhx_probe.so, the benchmark's FMA peak probe, from probe/alu_peaks.cu).

Translation units compile in parallel; the shared library links the CUDA
runtime statically.  Rebuilds only when a source or header is newer than the
library (or when force=True).  checked=True builds libhx_checked.so instead:
the same library with every computed node offset range-checked (HX_BOUNDS;
a violation is reported as HX_ERR_BOUNDS), for tests.
"""
import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "hx")
LIB = os.path.join(HERE, "libhx.so")
LIB_CHECKED = os.path.join(HERE, "libhx_checked.so")
# the benchmark's measurement support (FP64 / FP32 FMA peaks), include/hx_probe.h
PROBE_SRC = os.path.join(HERE, "probe", "alu_peaks.cu")
LIB_PROBE = os.path.join(HERE, "libhx_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build_probe(force=False):
    """libhx_probe.so: the FMA peak probe of include/hx_probe.h."""
    if not force and os.path.exists(LIB_PROBE) and os.path.getmtime(LIB_PROBE) >= max(
            os.path.getmtime(PROBE_SRC), os.path.getmtime(os.path.join(INCLUDE, "hx_probe.h"))):
        return LIB_PROBE
    tmp = LIB_PROBE + ".tmp%d" % os.getpid()
    cmd = [_nvcc()] + FLAGS + ARCH + ["-shared", "-o", tmp, PROBE_SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (PROBE_SRC, r.stdout, r.stderr))
    os.replace(tmp, LIB_PROBE)
    return LIB_PROBE


def build(force=False, verbose=False, ptxas_info=False, checked=False):
    if not checked:
        build_probe(force)
    lib = LIB_CHECKED if checked else LIB
    bdir = BUILD + "_checked" if checked else BUILD
    if not force and not stale(lib):
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DHX_BOUNDS"] if checked else [])

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + FLAGS + ARCH + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose or ptxas_info:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc, "-shared"] + ARCH + ["-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
