"""Build libfdcgks.so for sm_103a in-tree (paper_2606_17772_gb300/_build/).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library.  No torch or Python types cross the library boundary.
The benchmark's FMA-pipe peak measurement (csrc/pipe_peak.cu) is built as a
separate small library, libpipepeak.so, beside it.
"""
import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfdcgks.so")
SOURCES = ["fdcgks_api.cu", "fdcgks_fp64.cu", "fdcgks_mixed.cu", "fdcgks_noalloc.cu", "fdcgks_ensemble.cu", "fdcgks_adjoint.cu",
           "fdcgks_line.cu"]
HEADERS = ["fdcgks_math.cuh", "fdcgks_internal.cuh", "fdcgks_kernels.cuh", "fdcgks_reverse.cuh"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    paths = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "fdcgks.h"))
    return paths


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force=False, verbose=False, out_dir=None, defines=()):
    """Compile the library if needed; returns the path of the .so.

    out_dir / defines build a variant elsewhere (tuning of the -D knobs
    documented in csrc/fdcgks_kernels.cuh); the default build uses neither.
    """
    out = out_dir or OUT
    lib = os.path.join(out, "libfdcgks.so")
    if not force and out_dir is None and up_to_date():
        return LIB
    os.makedirs(out, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(out, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + ["-D" + d for d in defines] + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


PEAK_SRC = os.path.join(CSRC, "pipe_peak.cu")
PEAK_LIB = os.path.join(OUT, "libpipepeak.so")


def build_pipe_peak(force=False):
    """Compile the FMA-pipe peak measurement used by the benchmark."""
    if not force and os.path.exists(PEAK_LIB) and os.path.getmtime(PEAK_LIB) >= os.path.getmtime(PEAK_SRC):
        return PEAK_LIB
    os.makedirs(OUT, exist_ok=True)
    tmp = PEAK_LIB + ".tmp.%d" % os.getpid()
    cmd = [_nvcc()] + NVCC_FLAGS + ["-shared", PEAK_SRC, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for pipe_peak.cu:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build_pipe_peak(force=True))
