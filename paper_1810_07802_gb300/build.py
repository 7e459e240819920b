"""Build the CUDA library (sm_103a) into paper_1810_07802_gb300/_build/.

nvcc compiles each translation unit in parallel, then links one shared
library that exports the C ABI of include/dugks.h.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libdugks_gb300.so"
LIB_PATH = os.path.join(BUILD_DIR, LIB_NAME)
SOURCES = ["dugks_capi.cu", "dugks_fp64.cu", "dugks_fp32.cu", "dugks_static.cu", "dugks_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out.append(os.path.join(INCLUDE, "dugks.h"))
    out.append(os.path.abspath(__file__))
    return out


CHECKED_DIR = os.path.join(BUILD_DIR, "checked")
CHECKED_LIB_PATH = os.path.join(CHECKED_DIR, LIB_NAME)


def _stale(path):
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force=False, verbose_ptxas=False, checked=False):
    """Compile (if stale) and return the path of the shared library.
    checked=True builds the bounds-checked variant (DUGKS_BOUNDS_CHECK=1, every
    step-kernel index checked before use, violations reported as
    DUGKS_ERR_BOUNDS) into _build/checked/; it is not part of build()'s default
    output."""
    out_dir = CHECKED_DIR if checked else BUILD_DIR
    lib_path = CHECKED_LIB_PATH if checked else LIB_PATH
    if not force and not _stale(lib_path):
        return lib_path
    os.makedirs(out_dir, exist_ok=True)
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC] + ARCH
    if checked:
        flags += ["-DDUGKS_BOUNDS_CHECK=1"]
    if verbose_ptxas:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose_ptxas:
        for _, log in results:
            print(log)
    tmp = lib_path + ".tmp.%d" % os.getpid()
    cmd = [nvcc(), "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-cudart", "shared"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
