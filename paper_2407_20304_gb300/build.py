"""Build the in-tree CUDA library libholo.so for sm_103a (GB300).

Each translation unit under csrc/ is compiled by its own nvcc process (in parallel), then
linked into paper_2407_20304_gb300/_build/libholo.so.  No CMake, no torch extension
machinery: the library exposes only the C ABI declared in include/holo.h.  bounds_check=True
builds the variant with HOLO_BOUNDS_CHECK defined (device checks of table-driven indices that
report HOLO_ERR_BOUNDS instead of faulting) into _build_bc/, which the binding loads when the
environment has HOLO_BOUNDS_CHECK=1.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libholo.so")
OUT_BC = os.path.join(HERE, "_build_bc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(ROOT, "include", "holo.h")]


def _compile(src, extra, force=False, out=OUT):
    obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
    dep_mtime = max(os.path.getmtime(p) for p in headers() + [src, __file__])
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= dep_mtime:
        return obj, None
    cmd = [nvcc(), "-c", src, "-o", obj, "-std=c++17", "-O3", "-lineinfo", *ARCH,
           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return obj, "$ " + " ".join(cmd) + "\n" + r.stdout + r.stderr
    return obj, (r.stdout + r.stderr) if "-Xptxas=-v" in extra else None


def compile_flags(bounds_check=False, ptxas_info=False):
    """Extra nvcc flags of a build variant."""
    return (["-DHOLO_BOUNDS_CHECK"] if bounds_check else []) + (["-Xptxas=-v"] if ptxas_info else [])


def build(verbose=False, ptxas_info=False, force=False, bounds_check=False):
    """Compile and link libholo.so if any source changed; returns the library path."""
    out = OUT_BC if bounds_check else OUT
    lib = os.path.join(out, "libholo.so")
    os.makedirs(out, exist_ok=True)
    extra = compile_flags(bounds_check, ptxas_info)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, force, out), srcs))
    errs = [e for _, e in results if e and "error" in e.lower()]
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    if verbose or ptxas_info:
        for _, e in results:
            if e:
                print(e)
    objs = [o for o, _ in results]
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc(), "-shared", "-o", lib, *objs, *ARCH]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n$ " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv, force="--force" in sys.argv,
                bounds_check="--bounds-check" in sys.argv))
