"""Builds libfw.so (the C-ABI library) for sm_103a with nvcc, in-tree.

    python -m paper_2205_03532_b300.csrc.build [--force]
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
ROOT = os.path.dirname(PKG)
SOURCES = ["fw_api.cu", "fw_bake.cu", "fw_detect.cu", "fw_solve.cu", "fw_diff.cu", "fw_probe.cu"]
HEADERS = ["fw_internal.h", "fw_device.cuh"]
LIB = os.path.join(PKG, "libfw.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]
# The solve flushes subnormal float32 values to zero: its reciprocal square root then needs no
# subnormal handling on the serial per-row chain.  Values that small (< 1.2e-38) carry no
# physical meaning in any of its quantities (velocities, impulses, effective masses).
# The adjoint's serial sweeps divide and take square roots on their dependency chain (the
# friction-disk projection and its reverse): the approximate forms (a few ulp) replace the
# correctly rounded library sequences there, which made up about half of the adjoint's
# time; the adjoint is checked against FP64 finite differences and the FP64 oracle with
# tolerances far above that.
FILE_FLAGS = {"fw_solve.cu": ["--ftz=true"], "fw_diff.cu": ["-prec-div=false", "-prec-sqrt=false"]}


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(HERE, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "fw.h"),
                                                                 os.path.abspath(__file__)]   # flags
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every source for sm_103a and links libfw.so next to the package."""
    if not force and not _stale():
        return LIB
    bdir = os.path.join(PKG, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs, cmds = [], []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmds.append([NVCC, *ARCH, *FLAGS, *FILE_FLAGS.get(src, []), "-I", os.path.join(ROOT, "include"), "-c",
                     os.path.join(HERE, src), "-o", obj])
        objs.append(obj)
    if verbose:
        for cmd in cmds:
            print(" ".join(cmd), file=sys.stderr)
    # the translation units are independent: compile them at the same time
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as ex:
        for f in [ex.submit(subprocess.check_call, c) for c in cmds]:
            f.result()
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp, "-cudart", "shared",
                           "-Xlinker", "-rpath=/usr/local/cuda/lib64"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
