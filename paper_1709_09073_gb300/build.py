"""Build the in-tree CUDA library librlbm.so for sm_103a (GB300) with nvcc.

Translation units are compiled in parallel and linked into one shared library
under paper_1709_09073_gb300/_build/. No CMake, no torch extension machinery.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librlbm.so")
# the mixed-precision kernels are split by storage format so that they compile in parallel
UNITS = ["rlbm_api.cu", "rlbm_f64.cu", "rlbm_mixed.cu", "rlbm_mixed_f32.cu", "rlbm_mixed_f32dev.cu",
         "rlbm_mixed_bf16.cu", "rlbm_mixed_f16.cu", "rlbm_noalloc.cu", "rlbm_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + CSRC, "-I" + INCLUDE]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librlbm")
    return exe


def _sources_mtime():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "rlbm.h")]
    return max(os.path.getmtime(p) for p in paths)


def build(force=False, verbose=False, defines=(), build_dir=None):
    """Compile (if stale) and return the path of librlbm.so. `defines` adds -D
    options (tuning variants); `build_dir` places the result elsewhere."""
    bdir = build_dir or BUILD
    lib = os.path.join(bdir, "librlbm.so")
    os.makedirs(bdir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _sources_mtime():
        return lib
    exe = nvcc()

    def compile_unit(u):
        obj = os.path.join(bdir, u.replace(".cu", ".o"))
        cmd = [exe] + ARCH + FLAGS + ["-D" + d for d in defines] + ["-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (u, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_unit, UNITS))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
