"""In-tree build of the CUDA library libcraneplan.so for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into a shared library
with the CUDA runtime linked statically. No CMake, no torch extension machinery.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libcraneplan.so")
SOURCES = ["api.cu", "k_eval.cu", "k_init.cu", "k_sample.cu", "k_update.cu", "k_noalloc.cu", "k_grid.cu", "k_smooth.cu",
           "k_peaks.cu", "k_ik.cu", "k_sample_elites.cu", "k_hulls.cu", "k_finalize.cu", "k_traj.cu", "k_metrics.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcraneplan")
    return path


def _flags(verbose: bool):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--fmad=true", "-Xcompiler", "-fno-strict-aliasing"] + ARCH
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "craneplan.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, defines=(), lib_path=None,
          src_dir=None) -> str:
    """Compile and link libcraneplan.so if it is missing or older than its sources.

    `defines` (e.g. ["CP_EVAL_MIN_BLOCKS=2"]), `lib_path` and `src_dir` (a copy of csrc/)
    build a variant elsewhere."""
    lib = lib_path or LIB
    csrc = src_dir or CSRC
    if not force and not defines and lib_path is None and src_dir is None and not _stale():
        return LIB
    out_dir = os.path.dirname(os.path.abspath(lib))
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    tag = "" if not defines else "_" + "_".join(d.replace("=", "") for d in defines)
    objs = [os.path.join(out_dir, s.replace(".cu", tag + ".o")) for s in SOURCES
            if os.path.exists(os.path.join(csrc, s))]
    dflags = ["-D" + d for d in defines]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [cc, "-c", os.path.join(csrc, src), "-o", obj] + _flags(verbose) + dflags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        return r.stdout + r.stderr

    srcs = [s for s in SOURCES if os.path.exists(os.path.join(csrc, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    if verbose:
        print("".join(logs))
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
