"""Build the in-tree CUDA library libstokes_mg.so for sm_103a.

Host setup code is compiled with g++, the kernels and the C ABI with nvcc
(-gencode arch=compute_103a,code=sm_103a), each translation unit in
parallel, then linked into a shared library next to this file.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstokes_mg.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

SOURCES = [
    ("setup.cpp", ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-Wall", "-Wno-unused-variable"]),
    ("cutcell.cpp", ["g++", "-O3", "-std=c++17", "-fPIC", "-Wall"]),
    ("cutsetup.cpp", ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-Wall"]),
    ("kernels.cu", ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "--expt-relaxed-constexpr"]),
    ("api.cu", ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]),
    ("noalloc.cu", ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]),
    ("generic.cu", ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]),
    ("learn.cu", ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]),
    ("persist.cu", ["nvcc", ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "--expt-relaxed-constexpr"]),
]


def _nvcc_include():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    return ["-I" + os.path.join(cuda, "include")]


def build(verbose=False, force=False):
    """Compile every translation unit and link libstokes_mg.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    objs, procs = [], []
    newest_src = max(os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC))
    newest_src = max(newest_src, os.path.getmtime(os.path.join(HERE, "..", "include", "stokes_mg.h")))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) > newest_src:
        return LIB
    for src, cmd in SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        full = cmd + ["-c", os.path.join(CSRC, src), "-o", obj, "-I" + CSRC] + _nvcc_include()
        if verbose:
            print(" ".join(full), file=sys.stderr)
        procs.append((src, subprocess.Popen(full, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("compilation failed: " + ", ".join(failed))
    link = ["nvcc", ARCH, "-shared", "-o", LIB] + objs + ["-lcudart", "-lpthread", "-ldl"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        sys.stderr.write(r.stdout.decode(errors="replace"))
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force=True))
