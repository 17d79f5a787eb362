"""Builds libdctgb.so (the C-ABI library) in-tree for sm_103a with nvcc.

Each translation unit compiles in parallel to ``_build/*.o``; the objects
link into ``_lib/libdctgb.so``.  The same sources also build at other CORDIC
iteration counts than the spec file's (``VARIANT_N``, compiled with
-DDCTGB_CORDIC_N=n into ``_lib/n<n>/libdctgb.so``), the spec's accuracy /
integer-work trade-off.  A library is rebuilt when a source or header is
newer than it.
"""
import concurrent.futures as cf
import glob
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libdctgb.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
              "-I" + INCLUDE, "-I" + CSRC]

# CORDIC iteration counts built besides the spec file's
VARIANT_N = (4, 5)


def spec_n():
    """The CORDIC iteration count of include/dctgb_spec.json."""
    with open(os.path.join(INCLUDE, "dctgb_spec.json")) as f:
        return int(json.load(f)["N_cordic_iterations"])


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def lib_path(n=None):
    """Path of the library at CORDIC iteration count n (None or the spec's: the default library)."""
    if n is None or n == spec_n():
        return LIB
    return os.path.join(LIBDIR, "n%d" % n, "libdctgb.so")


def _dirs(n):
    if n is None or n == spec_n():
        return BUILD, LIB, []
    return os.path.join(BUILD, "n%d" % n), lib_path(n), ["-DDCTGB_CORDIC_N=%d" % n]


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(INCLUDE, "dctgb.h"), os.path.join(INCLUDE, "dctgb_spec.json"), os.path.abspath(__file__)]


def up_to_date(n=None):
    lib = lib_path(n)
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src, verbose, flags, build_dir):
    obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
    cmd = [_nvcc()] + ARCH + NVCC_FLAGS + flags + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def _link(objs, lib):
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)


def build_many(ns, force=False, verbose=False, jobs=None):
    """Builds the libraries for the CORDIC counts in ns (None: the spec's)
    with one pool of parallel nvcc jobs over all their translation units.
    Returns their paths."""
    todo = [n for n in ns if force or not up_to_date(n)]
    srcs = sources()
    tasks = []
    for n in todo:
        build_dir, lib, flags = _dirs(n)
        os.makedirs(build_dir, exist_ok=True)
        os.makedirs(os.path.dirname(lib), exist_ok=True)
        tasks += [(n, src, flags, build_dir) for src in srcs]
    if tasks:
        jobs = jobs or min(len(tasks), max(2, os.cpu_count() or 2))
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            results = list(ex.map(lambda t: (t[0], _compile(t[1], verbose, t[2], t[3])), tasks))
        for n in todo:
            objs = [o for k, (o, log) in results if k == n]
            if verbose:
                for k, (o, log) in results:
                    if k == n:
                        sys.stderr.write(log)
            _link(objs, _dirs(n)[1])
    return [lib_path(n) for n in ns]


def build(force=False, verbose=False, jobs=None, n=None):
    """Compiles every .cu under csrc/ and links the library at CORDIC count
    n (None: the spec's, the default libdctgb.so).  Returns its path."""
    return build_many([n], force=force, verbose=verbose, jobs=jobs)[0]


if __name__ == "__main__":
    if "--all" in sys.argv:
        print(build_many([None] + list(VARIANT_N), force="--force" in sys.argv, verbose="-v" in sys.argv))
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
