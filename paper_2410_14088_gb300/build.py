"""Builds libqsim.so in-tree for sm_103a with nvcc (no cmake, no torch
extension machinery): each translation unit is compiled in parallel, then
linked into one shared library with the CUDA runtime linked statically."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqsim.so")
SOURCES = ["codec.cu", "gates.cu", "engine.cu", "mlp.cu", "persistent.cu", "noalloc.cu", "planner.cpp", "autotune.cpp"]
HEADERS = ["codec.cuh", "codec_dev.cuh", "gates.cuh", "gates_dev.cuh", "mlp.cuh", "persistent.cuh", "device_common.cuh",
           "qsim_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "qsim.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    import platform
    stamp = os.path.join(BUILD, "arch.txt")
    arch = platform.machine()
    if not os.path.exists(LIB) or not os.path.exists(stamp) or open(stamp).read() != arch:
        force = True  # objects from another machine (or a half build) are not reused
    with open(stamp, "w") as f:
        f.write(arch)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "-I" + CSRC]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, s):
            if src.endswith(".cu"):
                cmd = [cc] + ARCH + common + ["-Xptxas", "-v" if verbose else "-O3", "-c", s, "-o", o]
            else:
                cmd = [cc] + common + ["-x", "c++", "-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static", "-lpthread", "-ldl", "-lrt"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
