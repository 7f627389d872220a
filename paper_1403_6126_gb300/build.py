"""Builds the in-tree CUDA library ``librt_gb300.so`` for sm_103a.

nvcc compiles each translation unit in parallel (one -gencode, -lineinfo)
and links them into a shared library next to this file.  The build is
skipped when the library is newer than every source and header.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "librt_gb300.so")
# The index-checking build (RT_BOUNDS_CHECK): every shared- and global-memory
# index of the float step's per-tile code is range checked and a violation
# is reported as a step failure; for tests, not for measurement.
LIB_CHECK = os.path.join(HERE, "librt_gb300_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
# Units that instantiate the float step kernels (rt_step_quad.cuh, and the
# pair kernel of rt_step_pair.cuh for bf16 storage).  Their per-angle
# arithmetic spells out every fused multiply-add it wants; these units are
# compiled without implicit contraction so that the per-cell code rounds the
# same way wherever it is inlined: the single-problem, batch and
# allocation-free kernels then give bitwise equal results.
NO_CONTRACT = {"rt_step_f3.cu", "rt_step_f12.cu", "rt_step_b16.cu", "rt_batch_k512.cu", "rt_batch_k256.cu", "rt_batch_k128.cu",
               "rt_noalloc.cu"}


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _inputs():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force=False, verbose=False, check=False):
    """Compile and link; returns the library path (the index-checking build
    when check is set)."""
    lib = LIB_CHECK if check else LIB
    if not force and up_to_date(lib):
        return lib
    objdir = os.path.join(HERE, "_build_check" if check else "_build")
    os.makedirs(objdir, exist_ok=True)
    procs = []
    for src in _sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [NVCC] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                               "-c", src, "-o", obj]
        if os.path.basename(src) in NO_CONTRACT:
            cmd += ["-fmad=false"]
        if check:
            cmd += ["-DRT_BOUNDS_CHECK"]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-warn-spills"] if verbose else []
        procs.append((src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    objs, errors = [], []
    for src, obj, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append("%s:\n%s" % (src, out.decode(errors="replace")))
        elif verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
        objs.append(obj)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib + ".%d.tmp" % os.getpid()
    subprocess.check_call([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, check="--check" in sys.argv))
