"""Build the channelizer's CUDA library (sm_103a) in-tree with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libvspec.so")
# the same sources with bounds checks into a device status word (-DVSPEC_DEBUG)
LIB_DEBUG = os.path.join(PKG, "libvspec_debug.so")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
    "--expt-relaxed-constexpr",
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = True) -> str:
    """Compile every .cu under csrc/ into libvspec.so (one -gencode, sm_103a)
    and, with debug=True, also into libvspec_debug.so with the bounds checks
    of -DVSPEC_DEBUG; all translation units compile in parallel. Returns the
    release library's path."""
    variants = [(LIB, "_build", [])]
    if debug:
        variants.append((LIB_DEBUG, os.path.join("_build", "debug"), ["-DVSPEC_DEBUG"]))
    variants = [v for v in variants if force or _stale(v[0])]
    if not variants:
        return LIB
    nvcc = _nvcc()
    procs, links = [], []
    for lib, sub, defs in variants:
        objdir = os.path.join(PKG, sub)
        os.makedirs(objdir, exist_ok=True)
        objs = []
        for src in sources():
            obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
            cmd = [nvcc, *NVCC_FLAGS, *defs, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
            objs.append(obj)
        links.append((lib, objs))
    failed = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode != 0:
            sys.stderr.write(out)
        if pr.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    for lib, objs in links:
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs],
                       check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
