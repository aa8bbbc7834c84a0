"""Build the CUDA library libocto_fmm.so in-tree (paper_2101_08226_gb300/_build/) for sm_103a."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libocto_fmm.so")
LIB_BC = os.path.join(OUT_DIR, "libocto_fmm_bc.so")  # index checks on (FMM_BOUNDS_CHECK)
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["fmm.cu", "tree.cpp", "peaks.cu", "scf.cu"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files


def _up_to_date(lib: str) -> bool:
    return os.path.exists(lib) and all(os.path.getmtime(lib) >= os.path.getmtime(f) for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds libocto_fmm.so and, from the same sources with -DFMM_BOUNDS_CHECK, the index-checked
    libocto_fmm_bc.so (used by its own tests), compiling every translation unit of both in
    parallel.  Returns the path of libocto_fmm.so."""
    if not force and _up_to_date(LIB) and _up_to_date(LIB_BC):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]

    def compile_one(job):
        src, checked = job
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ("_bc" if checked else "") + ".o")
        cmd = [nvcc] + common + (["-DFMM_BOUNDS_CHECK"] if checked else []) + \
            ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-c",
                   os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        return obj

    # the host-only tree code is shared; the CUDA sources are compiled twice
    jobs = [(src, False) for src in SOURCES] + [(src, True) for src in SOURCES if src.endswith(".cu")]
    with ThreadPoolExecutor(len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    plain = objs[:len(SOURCES)]
    checked = objs[len(SOURCES):] + [o for o, (src, _) in zip(plain, jobs) if src.endswith(".cpp")]
    for lib, parts in ((LIB, plain), (LIB_BC, checked)):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + parts, check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
