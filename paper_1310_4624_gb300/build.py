"""Build libpfarna.so (the CUDA library behind include/pfarna.h) with nvcc.

Compiles each translation unit for sm_103a only (``-gencode
arch=compute_103a,code=sm_103a``) in parallel, then links a shared library
in-tree at ``paper_1310_4624_gb300/_build/libpfarna.so``.  No CMake.

``build(debug=True)`` makes the PF_DEBUG variant in ``_build_debug/``: the
same kernels with explicit index checks that report into the device error
word (ERR_DEBUG) instead of touching memory out of bounds.  The binding loads
it when ``PFARNA_DEBUG=1``.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpfarna.so")
OUT_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DEBUG, "libpfarna.so")
SOURCES = ["pf_kernels.cu", "pf_api.cu", "pf_noalloc.cu", "pf_adjoint.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-v",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "pfarna.h"))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libpfarna.so (the PF_DEBUG variant if `debug`) if
    needed; return its path."""
    out, lib = (OUT_DEBUG, LIB_DEBUG) if debug else (OUT, LIB)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    flags = FLAGS + (["-DPF_DEBUG=1"] if debug else [])

    def compile_one(src):
        obj = os.path.join(out, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    with open(os.path.join(out, "ptxas.log"), "w") as f:
        for _, log in results:
            f.write(log)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
