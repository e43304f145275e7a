"""Build the channel library ``libchan.so`` in-tree for sm_103a.

Host set-up (quad-precision coefficient systems) is compiled with g++, the
kernels and the C ABI with nvcc; the shared object lands next to this file
so that it travels with the source tree.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libchan.so")
CU = ["chan_api.cu", "kernels_y.cu", "kernels_fft.cu", "kernels_misc.cu", "kernels_persist.cu", "noalloc.cu"]
CPP = ["setup_host.cpp"]
HEADERS = ["chan_internal.cuh", "chan_host.h", "df.cuh", "y_bodies.cuh", "fft_bodies.cuh"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(obj, srcs):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(verbose=False, force=False):
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "chan.h")]
    objs, jobs = [], []
    for f in CPP + CU:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        if force or _stale(obj, [src] + hdrs):
            if f in CPP:
                jobs.append(["g++", "-O2", "-fPIC", "-std=c++17", "-c", src, "-o", obj])
            else:
                jobs.append([_nvcc()] + NVCC_FLAGS + ["-c", src, "-o", obj])
        objs.append(obj)
    _run_all(jobs, verbose)   # the units compile concurrently
    if force or _stale(LIB, objs):
        cmd = [_nvcc(), "-shared", "-o", LIB] + objs + ["-lquadmath", "-lcudart"]
        _run(cmd, verbose)
    return LIB


def _run_all(cmds, verbose):
    procs = []
    for cmd in cmds:
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = None
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 and failed is None:
            sys.stderr.write(out)
            failed = cmd
    if failed:
        raise RuntimeError("build step failed: " + " ".join(failed))


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("build step failed: " + " ".join(cmd))


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
