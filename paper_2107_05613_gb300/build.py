"""In-tree builds of the native libraries.

libamge.so            the C-ABI solve library (CUDA, sm_103a only; it also holds the
                      host hierarchy generator, for the problem-level setup entry)
libamge_hierarchy.so  the host FP64 hierarchy generator (input data)

Both are compiled with explicit nvcc / g++ command lines, in parallel, into the
package directory (git-ignored).
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
AMGE_SO = os.path.join(PKG, "libamge.so")
HIER_SO = os.path.join(PKG, "inputs", "libamge_hierarchy.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CUDA_SOURCES = ["amge_api.cu", "amge_kernels.cu", "amge_kernels_mm.cu", "amge_server.cu", "amge_host_setup.cpp",
                "amge_noalloc.cu", "amge_setup.cpp", "amge_probe.cu", "amge_update.cu", "../inputs/amge_hierarchy.cpp"]
INPUTS = os.path.join(PKG, "inputs")


def _run(cmds):
    procs = [(c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for c in cmds]
    failed = []
    for c, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((c, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("native build failed:\n" + msg)


def build_hierarchy_lib():
    src = os.path.join(PKG, "inputs", "amge_hierarchy.cpp")
    tmp = HIER_SO + ".tmp"
    _run([["g++", "-O3", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src]])
    os.replace(tmp, HIER_SO)
    return HIER_SO


def build_amge_lib(verbose_ptxas=False):
    objdir = os.path.join(PKG, "_build")
    os.makedirs(objdir, exist_ok=True)
    cmds, objs = [], []
    for s in CUDA_SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(objdir, os.path.basename(s) + ".o")
        objs.append(obj)
        cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-O3,-fopenmp,-ffp-contract=off",
               "-I", INCLUDE, "-I", CSRC, "-I", INPUTS, "-c", src, "-o", obj]
        if verbose_ptxas and s.endswith(".cu"):
            cmd.insert(1, "-Xptxas=-v")
        cmds.append(cmd)
    _run(cmds)
    tmp = AMGE_SO + ".tmp"
    _run([[NVCC, *ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-fopenmp", "-o", tmp, *objs, "-lgomp"]])
    os.replace(tmp, AMGE_SO)
    return AMGE_SO


def build_all():
    """Build both libraries concurrently."""
    import threading

    errs = []

    def go(f):
        try:
            f()
        except Exception as e:  # noqa: BLE001
            errs.append(e)

    ts = [threading.Thread(target=go, args=(f,)) for f in (build_hierarchy_lib, build_amge_lib)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]


if __name__ == "__main__":
    build_all()
    print("built", AMGE_SO, HIER_SO, file=sys.stderr)
