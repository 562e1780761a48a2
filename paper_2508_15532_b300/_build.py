"""Build librt_b300.so in-tree for sm_103a (B300) with nvcc.

The library is the product: the CUDA kernels and the C ABI of include/rt.h.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["grid.cu", "geometry.cu", "stage.cu", "stage_flat.cu", "moments.cu", "adjoint.cu", "api.cu"]
LIB = os.path.join(HERE, "librt_b300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# stage.cu holds the general stage kernel, instantiated for several brick
# shapes; the compiler's choice of which multiply-adds to fuse differs between
# instances, so with contraction the results would depend on the brick shape
# (and an x3 slab, whose brick may differ from the whole box's, would not
# reproduce the whole box bit for bit).  Its fused multiply-adds are explicit.
EXTRA = {"stage.cu": ["-fmad=false"]}


def _deps():
    out = [os.path.join(CSRC, s) for s in SOURCES]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    out.append(os.path.join(ROOT, "include", "rt.h"))
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(d) for d in _deps()):
        return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    headers = [d for d in _deps() if not d.endswith(".cu")]
    newest_header = max(os.path.getmtime(h) for h in headers)
    objs = []
    procs = []
    for s in SOURCES:
        o = os.path.join(objdir, s.replace(".cu", ".o"))
        objs.append(o)
        src = os.path.join(CSRC, s)
        if (not force and os.path.exists(o)
                and os.path.getmtime(o) >= max(os.path.getmtime(src), newest_header)):
            continue
        cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-rdc=false",
               *EXTRA.get(s, []), "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, s), "-o", o]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), s))
    failed = []
    for p, s in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode())
        if p.returncode:
            failed.append(s)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.run(["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
