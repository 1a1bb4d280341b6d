"""Build libddsp.so (the C-ABI CUDA library) in-tree for sm_103a.

    python -m paper_2605_03531_b300.build [--force] [--verbose]

Each .cu under csrc/ is compiled to an object with nvcc (``-gencode
arch=compute_103a,code=sm_103a -lineinfo -O3``) and linked into
``paper_2605_03531_b300/libddsp.so`` with the CUDA runtime linked
statically, so the library needs nothing but the driver at run time.
"""
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libddsp.so")
BUILD = os.path.join(PKG, "_build")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(INCLUDE, "ddsp.h"), os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


# The bounds-checked build (tests only): every checked access records the
# first violation in one device variable the translation units share, which
# takes relocatable device code.
BOUNDS_LIB = os.path.join(PKG, "libddsp_bounds.so")
BOUNDS_DEFINES = ("DDSP_BOUNDS_CHECK",)


def _compile(src, obj, verbose, extra):
    cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)


def build(force: bool = False, verbose: bool = False, lib: str = LIB,
          defines=()) -> str:
    """Compile every .cu (in parallel; an object is rebuilt when it is older
    than any source or header) and link `lib`.  `defines` adds -D flags (a
    build with other flags keeps its objects in a folder of its own)."""
    if not force and lib == LIB and not defines and up_to_date():
        return LIB
    extra = [f"-D{d}" for d in defines]
    if "DDSP_BOUNDS_CHECK" in defines:
        extra.append("-rdc=true")
    bdir = BUILD if not defines else BUILD + "_" + "_".join(
        d.lower() for d in defines)
    os.makedirs(bdir, exist_ok=True)
    newest = max(os.path.getmtime(d) for d in _deps())
    jobs = []
    objs = []
    for src in _sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < newest:
            jobs.append((src, obj))
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(_compile, s_, o_, verbose, extra) for s_, o_ in jobs]:
            f.result()
    tmp = lib + ".tmp"
    rdc = ["-rdc=true"] if "DDSP_BOUNDS_CHECK" in defines else []
    subprocess.run([NVCC, *ARCH, *rdc, "-shared", "-cudart", "static", "-o",
                    tmp, *objs], check=True)
    os.replace(tmp, lib)
    return lib


def build_bounds(force: bool = False) -> str:
    """The bounds-checked library (tests only), beside the normal one."""
    return build(force=force, lib=BOUNDS_LIB, defines=BOUNDS_DEFINES)


if __name__ == "__main__":
    if "--bounds" in sys.argv:
        print(build_bounds(force="--force" in sys.argv))
    else:
        print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
