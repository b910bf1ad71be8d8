"""Build the C-ABI shared library liboctgrav.so (host C++ + sm_103a CUDA) in-tree.

    python -m paper_1005_5384_gb300.build        # or build() from Python

nvcc compiles the kernels for sm_103a only (the GPU tree build with
-fmad=false); g++ compiles the host library with -ffp-contract=off (the octree
definition relies on uncontracted FP64 ops, and the two builds must agree to the
bit). The translation units compile in parallel; the result lands in
paper_1005_5384_gb300/_build/liboctgrav.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboctgrav.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cpp", ".h"))] + [os.path.join(INCLUDE, "octgrav.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    ko = os.path.join(BUILD, "octgrav_kernels.o")
    mo = os.path.join(BUILD, "octgrav_mlp.o")
    bo = os.path.join(BUILD, "octgrav_build.o")
    so = os.path.join(BUILD, "octgrav_sim.o")
    do = os.path.join(BUILD, "octgrav_direct.o")
    host_srcs = ("octgrav_host.cpp", "octgrav_host_build.cpp", "octgrav_host_mlp.cpp")
    host_objs = [os.path.join(BUILD, h.replace(".cpp", ".o")) for h in host_srcs]

    def nv(src, obj, *extra):
        return [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-v" if verbose else "-O3",
                "-Xcompiler", "-fPIC,-O2,-ffp-contract=off", *extra, "-I", INCLUDE,
                "-c", os.path.join(CSRC, src), "-o", obj]
    k_cmd = nv("octgrav_kernels.cu", ko)
    m_cmd = nv("octgrav_mlp.cu", mo)
    b_cmd = nv("octgrav_build.cu", bo, "-fmad=false")
    s_cmd = nv("octgrav_sim.cu", so, "-fmad=false")
    d_cmd = nv("octgrav_direct.cu", do)
    h_cmds = [["g++", "-O3", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-pthread",
               "-I", os.path.join(cuda, "include"), "-I", INCLUDE,
               "-c", os.path.join(CSRC, h), "-o", o] for h, o in zip(host_srcs, host_objs)]
    cmds = (k_cmd, m_cmd, b_cmd, s_cmd, d_cmd, *h_cmds)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    outs = [p.communicate()[0] for p in procs]
    for p, o, c in zip(procs, outs, cmds):
        if p.returncode != 0:
            raise RuntimeError("build failed: %s\n%s" % (" ".join(c), o))
        if verbose and o:
            print(o)
    tmp = LIB + ".%d.tmp" % os.getpid()
    link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, ko, mo, bo, so, do, *host_objs, "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(link), r.stdout))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
