"""Build the CUDA library (sm_103a) in-tree: paper_2504_06408_gb300/_build/libspgemm.so.

Each translation unit under csrc/ is compiled in parallel with nvcc, then
linked into one shared library with a C ABI (include/spgemm.h).

Variant "checks" (_build_checks/libspgemm_checks.so) is the same library
compiled with -DSPG_CHECKS: every call validates its input matrices on the
device before queuing product kernels, numeric calls check C's row pointers
against the symbolic call's count, and the rank-indexed accumulation checks
each product's rank; a failure is reported as an SPG_ERR_* status.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libspgemm.so")
VARIANTS = {"": (OUT, LIB, []),
            "checks": (os.path.join(HERE, "_build_checks"),
                       os.path.join(HERE, "_build_checks", "libspgemm_checks.so"),
                       ["-DSPG_CHECKS"])}
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + [os.path.join(ROOT, "include", "spgemm.h"),
                                                 os.path.abspath(__file__)]


def up_to_date(variant: str = "") -> bool:
    lib = VARIANTS[variant][1]
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), variants=("",)) -> str:
    """Compile the given variants ("" = the library, "checks" = the checked
    build), all translation units in parallel; returns the first one's path."""
    todo = [v for v in variants if force or not up_to_date(v)]
    if todo:
        jobs = [(v, src) for v in todo for src in _sources()]
        for v in todo:
            os.makedirs(VARIANTS[v][0], exist_ok=True)
        with cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
            objs = list(ex.map(lambda j: _compile(j[0], j[1], verbose, extra), jobs))
        for v in todo:
            _link(v, [o for (vv, _), o in zip(jobs, objs) if vv == v])
    return VARIANTS[variants[0]][1]


def _compile(variant, src, verbose, extra):
    out, _, vflags = VARIANTS[variant]
    obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, *vflags, *extra, "-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        print(r.stderr, file=sys.stderr)
    return obj


def _link(variant, objs):
    lib = VARIANTS[variant][1]
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-cudart=static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


if __name__ == "__main__":
    extra = [a for a in sys.argv[1:] if a.startswith("-")]
    print(build(force=True, verbose=True, extra=extra, variants=("", "checks")))
