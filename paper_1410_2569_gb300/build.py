"""Build liblbm.so (the CUDA library behind include/lbm.h) in-tree.

nvcc for sm_103a only; translation units compiled in parallel, then linked
into paper_1410_2569_gb300/liblbm.so against the CUDA runtime.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liblbm.so")
# the checked build: every index of the step kernels tested against its
# buffer, a bad one latched as an error (LBM_ERR_STATE at the next
# synchronising call) instead of an access
LIB_CHECK = os.path.join(PKG, "liblbm_check.so")
CHECK_FLAGS = ["-DLBM_BOUNDS_CHECK"]
SOURCES = ["lbm_kernels.cu", "lbm_diag.cu", "lbm_adjoint.cu", "lbm_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC] + list(extra)


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbm.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force=False, verbose=False, extra=(), checked=True):
    """Build liblbm.so and (checked=True) liblbm_check.so, all translation
    units of both compiled in parallel; returns the path of liblbm.so."""
    targets = [(LIB, list(extra), "")]
    if checked:
        targets.append((LIB_CHECK, list(extra) + CHECK_FLAGS, "_check"))
    todo = [t for t in targets
            if force or not os.path.exists(t[0]) or os.path.getmtime(t[0]) < _deps()]
    if not todo:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()

    def compile_one(job):
        src, flags, tag = job
        obj = os.path.join(BUILD, src.replace(".cu", tag + ".o"))
        cmd = [nv] + _flags(flags) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    jobs = [(src, flags, tag) for _, flags, tag in todo for src in SOURCES]
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    for k, (lib, _, _) in enumerate(todo):
        mine = objs[k * len(SOURCES):(k + 1) * len(SOURCES)]
        tmp = lib + ".tmp"
        cmd = [nv] + ARCH + ["-shared", "-o", tmp] + mine + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if v else []
    print(build(force=True, verbose=v, extra=extra))
