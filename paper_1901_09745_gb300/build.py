"""Build the CUDA library (sm_103a) in-tree: paper_1901_09745_gb300/_lib/libpsc_lbm.so.

Each .cu file under csrc/ is compiled by its own nvcc process (in parallel), then linked
into one shared library with a plain C ABI (include/psc_lbm.h). Only the sm_103a target is
built.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libpsc_lbm.so")
# the bounds-checked variant (-DPSC_CHECKED, see psc_internal.h): its own objects and library
OBJ_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(LIBDIR, "libpsc_lbm_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code without FP contraction, so the __host__ __device__ helpers that the CPU tests
# call through testing.cu round as written on both machines (x86 and Arm)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-Wall", "-Xcompiler", "-Wno-unused-function", "-Xcompiler", "-ffp-contract=off"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers_mtime():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(os.path.dirname(HERE), "include", "psc_lbm.h"))
    hs.append(os.path.join(os.path.dirname(HERE), "include", "psc_testing.h"))
    return max(os.path.getmtime(h) for h in hs if os.path.exists(h))


def build(force=False, verbose=False, extra=(), checked=False):
    """Compile what is stale and link the library; with checked=True the bounds-checked
    variant (libpsc_lbm_checked.so)."""
    obj_dir, lib = (OBJ_CHECKED, LIB_CHECKED) if checked else (OBJ, LIB)
    if checked:
        extra = tuple(extra) + ("-DPSC_CHECKED",)
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    hdr = _headers_mtime()
    jobs = []
    for s in sources():
        src = os.path.join(CSRC, s)
        obj = os.path.join(obj_dir, s[:-3] + ".o")
        stale = force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr)
        jobs.append((src, obj, stale))
    cmds = [[cc] + ARCH + FLAGS + list(extra) + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
            for src, obj, stale in jobs if stale]
    if cmds:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), cmds))
        for c, r in zip(cmds, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(c))
    objs = [o for _, o, _ in jobs]
    if cmds or force or not os.path.exists(lib):
        link = [cc] + ARCH + ["-shared", "-o", lib + ".tmp"] + objs
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
