"""Build the CUDA library ``libsj.so`` in-tree with nvcc for sm_103a.

Every ``csrc/*.cu`` is compiled in parallel to an object file and linked
into ``_build/libsj.so`` against the shared CUDA runtime (the one PyTorch
loads as well).  No fast-math: the cell function and all comparisons are
exact IEEE float32, denormals are kept (-ftz=false).

``build(check=True)`` makes the debug build ``_build_check/libsj.so``
(``-DSJ_CHECK=1``): the same library with bounds checks on the kernels'
data-dependent indexes; a failed check makes the call return SJ_EINTERNAL
with the site in its message (it stands in for compute-sanitizer).
"""
from __future__ import annotations

import glob
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsj.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "libsj.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-ftz=false",
    "-prec-div=true", "-prec-sqrt=true", "--expt-relaxed-constexpr",
    "-I", CSRC, "-I", INCLUDE,
]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _stamp(flags) -> str:
    h = hashlib.sha256()
    for f in _sources() + _headers() + [__file__]:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(flags).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, check: bool = False) -> str:
    """Compile and link; returns the library path.  Skips work when the
    sources, headers and flags are unchanged since the last build.  With
    check=True: the debug build with bounds checks (its own folder)."""
    out_dir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    flags = NVFLAGS + (["-DSJ_CHECK=1"] if check else [])
    os.makedirs(out_dir, exist_ok=True)
    stamp_file = os.path.join(out_dir, "stamp")
    stamp = _stamp(flags)
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        if open(stamp_file).read().strip() == stamp:
            return lib
    cc = nvcc()
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmd = [cc, *flags, "-c", src, "-o", obj]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose or ptxas_info:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(os.path.basename(f) for f in failed))
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.check_call([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                ptxas_info="--ptxas" in sys.argv, check="--check" in sys.argv))
