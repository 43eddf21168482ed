"""Build the CUDA library in-tree: paper_1210_0800_gb300/lib/libmgs_ddqd.so (sm_103a).

Translation units compile in parallel with nvcc, then link into one shared library
with the CUDA runtime linked statically.  No PyTorch extension machinery is involved:
the library has a plain C ABI (include/mgs_ddqd.h).
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIBRARY = os.path.join(LIBDIR, "libmgs_ddqd.so")
HOST_LIBRARY = os.path.join(LIBDIR, "libddqd_host.so")
SOURCES = ["api.cu", "mgs_d.cu", "mgs_dd.cu", "mgs_qd.cu", "noalloc.cu", "batched.cu", "newton.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--fmad=false"]
# extra nvcc flags for experiments; empty by default
EXTRA = os.environ.get("MGS_EXTRA_NVCC_FLAGS", "").split()
# the phase-trace variant (kernels record global-timer stamps; see trace.py)
TRACE_LIBRARY = os.path.join(LIBDIR, "trace", "libmgs_ddqd.so")


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _stale(library) -> bool:
    if not os.path.exists(library):
        return True
    t = os.path.getmtime(library)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "mgs_ddqd.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, trace: bool = False) -> str:
    """Compile the library (trace=True: the phase-trace variant, in lib/trace/)."""
    library = TRACE_LIBRARY if trace else LIBRARY
    libdir = os.path.dirname(library)
    os.makedirs(libdir, exist_ok=True)
    objdir = os.path.join(libdir, "_obj")
    os.makedirs(objdir, exist_ok=True)
    objs = [os.path.join(objdir, s.replace(".cu", ".o")) for s in SOURCES]
    if not force and not _stale(library):
        return library
    cc = nvcc()
    extra = EXTRA + (["-DMGS_TRACE=1"] if trace else [])
    procs = []
    for src, obj in zip(SOURCES, objs):
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s" % (" ".join(cmd), out.decode(errors="replace")))
        if verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
    tmp = library + ".tmp"
    link = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    subprocess.check_call(link)
    os.replace(tmp, library)
    return library


def build_host(force: bool = False) -> str:
    """Host build of the device arithmetic (csrc/ddqd.cuh as plain C++) for the CPU tests."""
    os.makedirs(LIBDIR, exist_ok=True)
    src = os.path.join(CSRC, "ddqd_host.cpp")
    deps = [src, os.path.join(CSRC, "ddqd.cuh")]
    if not force and os.path.exists(HOST_LIBRARY) and all(
            os.path.getmtime(d) <= os.path.getmtime(HOST_LIBRARY) for d in deps):
        return HOST_LIBRARY
    tmp = HOST_LIBRARY + ".tmp"
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-fPIC", "-shared",
                           "-Wno-unknown-pragmas", "-o", tmp, src])
    os.replace(tmp, HOST_LIBRARY)
    return HOST_LIBRARY


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print(build_host(force="--force" in sys.argv))
