"""Build librp.so in-tree with nvcc for sm_103a (no CMake, one -gencode)."""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librp.so")
SOURCES = ["rp_fill_xo.cu", "rp_fill_xss.cu", "rp_fill_pcg.cu", "rp_fill_ph.cu", "rp_fill_ph64.cu", "rp_kernels.cu", "rp_grad.cu", "rp_mvn.cu", "rp_static_scratch.cu", "rp_host.cpp"]
DEPS = SOURCES + ["rp_device.cuh", "rp_gamma.cuh", "rp_fill_impl.cuh", "rp_lean.cuh", "rp_rej.cuh", "rp_internal.h", "zig_tables.inc", "log_table.inc"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
          "-I", os.path.join(HERE, "..", "include")]
# No FMA contraction anywhere a value must equal the serial definition bit for
# bit; the gradients' bar is 1e-12 relative, so their file may contract.
FMAD = {"rp_grad.cu": "-fmad=true"}


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, f) for f in DEPS] + [os.path.join(HERE, "..", "include", "rp.h")]
    return any(os.path.getmtime(f) > t for f in srcs)


def build(force=False, verbose=False):
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nvcc] + ARCH + COMMON + [FMAD.get(src, "-fmad=false"), "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    build(force=True, verbose="-v" in sys.argv)
    print("built", LIB)
