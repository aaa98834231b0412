"""Build libcapt.so in-tree: host C++ (g++) and sm_103a CUDA kernels (nvcc), linked with
the static CUDA runtime.  Objects are compiled in parallel and rebuilt only when a
source or header is newer than the library."""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUTDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcapt.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-warn-spills"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", "-fno-fast-math", "-Wall"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CAPT library needs the CUDA toolkit to build")


def _cuda_include(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu"))) + sorted(glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


# Test-only variants: the same sources with extra preprocessor definitions, built into
# their own directory and library (never loaded unless a caller names the file).
VARIANTS = {
    # every first wait on a bulk copy into shared memory gives up at once (the copies
    # still complete and are drained): exercises the CAPT_E_TIMEOUT fallback paths
    "stage_timeout": ["-DCAPT_STAGE_POLLS=0u"],
}


def variant_lib(name: str) -> str:
    return os.path.join(HERE, f"libcapt_{name}.so")


def build(force: bool = False, verbose: bool = False, variant: str | None = None) -> str:
    """Compile every translation unit for sm_103a and link libcapt.so next to this file
    (or, for a test variant, libcapt_<variant>.so from its own build directory)."""
    lib = LIB if variant is None else variant_lib(variant)
    outdir = OUTDIR if variant is None else OUTDIR + "_" + variant
    defines = [] if variant is None else VARIANTS[variant]
    if not force and not _stale(lib):
        return lib
    nvcc = _nvcc()
    os.makedirs(outdir, exist_ok=True)
    inc = ["-I", INCLUDE, "-I", CSRC]

    def compile_one(src):
        obj = os.path.join(outdir, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            extra = os.environ.get("CAPT_NVCC_EXTRA", "").split()
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defines, *extra, *inc, "-c", src, "-o", obj]
        else:
            cmd = [os.environ.get("CXX", "g++"), *CXX_FLAGS, *defines, *inc, "-I", _cuda_include(nvcc), "-c", src,
                   "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
