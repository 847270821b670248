"""In-tree build of liblm.so (CUDA kernels for sm_103a + the C-ABI host code).

Compiles csrc/*.cu with nvcc (-gencode arch=compute_103a,code=sm_103a) and
csrc/*.cpp with g++, in parallel, and links them into _build/liblm.so.  A
stamp of the sources' content avoids rebuilding unchanged code."""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _sources():
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp", ".h", ".cuh")))
    return [os.path.join(CSRC, f) for f in srcs] + [os.path.join(INCLUDE, "lm.h")]


def _stamp() -> str:
    h = hashlib.sha256()
    for p in _sources():
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH).encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False) -> str:
    """Build liblm.so if needed; returns its path.  Raises on failure."""
    os.makedirs(BUILD, exist_ok=True)
    stamp_file = os.path.join(BUILD, "stamp")
    st = _stamp()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == st:
                return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + os.path.join(cuda, "include"), "-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    objs = []
    for f in sorted(os.listdir(CSRC)):
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        if f.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc, "-c", src, "-o", obj]
        elif f.endswith(".cpp"):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-pthread", *inc, "-c", src, "-o", obj]
        else:
            continue
        objs.append(obj)
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errs = []
    for cmd, p in jobs:
        out = p.communicate()[0].decode(errors="replace")
        if p.returncode != 0:
            errs.append(" ".join(cmd) + "\n" + out)
        elif verbose and out.strip():
            print(out)
    if errs:
        raise RuntimeError("liblm build failed:\n" + "\n".join(errs))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared", "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("liblm link failed:\n" + " ".join(link) + "\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(st)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
