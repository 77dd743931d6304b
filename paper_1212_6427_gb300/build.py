"""Compile libicm.so in-tree for sm_103a (GB300).

Each .cu translation unit is compiled by nvcc in parallel, then linked into
paper_1212_6427_gb300/libicm.so.  Nothing is installed outside the package.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libicm.so")
# The checked build: device-side index checks on the blob stencils and the FFT tiles
# (-DICM_INDEX_CHECKS=1) raise an error bit (ICM_EINDEX at the next icm_sync) and skip
# the access instead of faulting.  Off by default; a library of its own.
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libicm_checked.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
# (source, object name, extra flags): the FFT file is compiled as six shards in
# parallel (x forward / y-z / x inverse passes, FP32 / FP64), the largest unit otherwise.
SOURCES = [("icm_api.cu", "icm_api", ()), ("icm_grid.cu", "icm_grid", ()), ("icm_blob.cu", "icm_blob", ()),
           ("icm_static.cu", "icm_static", ())] + [
    ("icm_fft.cu", "icm_fft_%d" % k, ("-DICM_FFT_SHARD=%d" % k,)) for k in range(6)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


def _nvcc():
    cand = shutil.which("nvcc")
    if cand:
        return cand
    for root in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        path = os.path.join(root, "bin", "nvcc")
        if root and os.path.exists(path):
            return path
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "icm.h"), __file__]
    return files


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build_library(force=False, verbose=False, extra_flags=(), checked=False):
    """Build libicm.so (or, with checked=True, libicm_checked.so with the device-side
    index checks) unless it is newer than every source.  Returns its path."""
    lib_out = LIB_CHECKED if checked else LIB
    build_dir = BUILD_CHECKED if checked else BUILD
    if checked:
        extra_flags = tuple(extra_flags) + ("-DICM_INDEX_CHECKS=1",)
    if not force and up_to_date(lib_out):
        return lib_out
    nvcc = _nvcc()
    os.makedirs(build_dir, exist_ok=True)

    def compile_one(unit):
        src, name, defs = unit
        obj = os.path.join(build_dir, name + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *defs, *extra_flags, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), res.stderr[-6000:]))
        if verbose:
            print(res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_out + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), res.stderr[-4000:]))
    os.replace(tmp, lib_out)
    return lib_out


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
