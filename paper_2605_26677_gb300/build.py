"""Build the CUDA library liblbm_gb300.so for sm_103a, in-tree.

Each .cu under csrc/ is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically (so the library loads
without a GPU and exports only the C ABI of include/lbm.h).
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUTDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUTDIR, "liblbm_gb300.so")
SOURCES = ["lbm_api.cu", "lbm_step.cu", "lbm_step_f64.cu", "lbm_step_f32.cu", "lbm_step_bf16.cu", "lbm_step_f16.cu",
           "lbm_aux.cu", "lbm_noalloc.cu", "lbm_batch.cu", "lbm_batch_k64.cu", "lbm_batch_k32.cu", "lbm_batch_k16.cu",
           "lbm_batch_kf16.cu", "lbm_adjoint.cu",
           "lbm_adjoint_kernels.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbm.h"), __file__]
    return [f for f in files if os.path.isfile(f)]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link if the library is missing or older than a source."""
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in _deps()):
        return LIB
    os.makedirs(OUTDIR, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(src):
        obj = os.path.join(OUTDIR, src.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
