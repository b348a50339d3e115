"""Builds libphasorpic.so in-tree for sm_103a with nvcc.

Flags: -gencode arch=compute_103a,code=sm_103a -lineinfo -O3.  The
particle-step sources (the fused FP32 kernel, the plain FP64 form and the
split-merge pass) are compiled with --fmad=false: their cell crossings, absorptions and collision
decisions then round exactly like the oracle's float32 / float64
instantiations, and the arithmetic that decides nothing (deposit weights,
moments, power tallies) is fused explicitly with fma intrinsics.  Every other
source (field solves, period end, MLP) lets the compiler contract.  Sources
compile in parallel to objects under _build/ and link into one library.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libphasorpic.so")
SOURCES = ["pp_capi.cu", "pp_setup.cu", "pp_fields.cu", "pp_pcg.cu", "pp_particles.cu", "pp_plain.cu", "pp_mlp.cu",
           "pp_mlp_train.cu", "pp_period.cu", "pp_control.cu"]
NO_CONTRACT = {"pp_particles.cu", "pp_plain.cu", "pp_control.cu"}
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
        [os.path.join(HERE, "..", "include", "phasorpic.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _compile(src, verbose):
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc(), "-O3", "-std=c++17"] + ARCH + ["-lineinfo", "-Xcompiler", "-fPIC", "-c"]
    if src in NO_CONTRACT:
        cmd += ["--fmad=false"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += ["-o", obj, os.path.join(CSRC, src)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r


def build(force=False, verbose=False):
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda f: _compile(f, verbose), SOURCES))
    for src, _, r in results:
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed compiling %s" % src)
        if verbose:
            sys.stderr.write(r.stderr)
    cmd = [nvcc()] + ARCH + ["-shared", "-Xlinker", "-z", "-Xlinker", "defs", "-o", LIB + ".tmp"]
    cmd += [obj for _, obj, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking libphasorpic.so")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
