"""Builds libmagnus.so in-tree from csrc/*.cu for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel),
then the objects are linked into one shared library.  Plain nvcc, no cmake,
no -march flags: the same command builds on x86 and on Arm hosts.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libmagnus.so")
# input generators (no SpGEMM code): a library of their own
CSRC_INPUTS = os.path.join(HERE, "csrc_inputs")
OUT_INPUTS = os.path.join(HERE, "libmagnus_inputs.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _build_lib(src_dir: str, out: str, objdir: str, force: bool, verbose: bool) -> str:
    srcs = sorted(glob.glob(os.path.join(src_dir, "*.cu")))
    hdrs = sorted(glob.glob(os.path.join(src_dir, "*.cuh")) + glob.glob(os.path.join(src_dir, "*.h"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))
    if not force and not _stale(out, srcs + hdrs + [os.path.abspath(__file__)]):
        return out
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = out + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath", "-Xlinker", "/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, out)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds libmagnus.so and libmagnus_inputs.so (in parallel); returns
    the path of libmagnus.so."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        main = ex.submit(_build_lib, CSRC, OUT, os.path.join(HERE, "_build"), force, verbose)
        gen = ex.submit(_build_lib, CSRC_INPUTS, OUT_INPUTS, os.path.join(HERE, "_build_inputs"),
                        force, verbose)
        gen.result()
        return main.result()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
