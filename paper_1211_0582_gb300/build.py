"""Build libdgmx.so in-tree with nvcc for sm_103a (GB300).

Every translation unit under csrc/ is compiled in parallel into
_build/*.o and linked into paper_1211_0582_gb300/_build/libdgmx.so. Objects
are rebuilt when their source or any header changed. `defines` and `out_dir`
make a separate build with extra preprocessor macros (the timing build of
stage_timing.py: -DDGMX_STAGE_TIMING into _build_timing/).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdgmx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def build(verbose: bool = False, jobs: int | None = None, defines=(), out_dir: str = OUT_DIR) -> str:
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libdgmx.so")
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr_time = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                     "-Xptxas", "-warn-spills"] + [f"-D{d}" for d in defines]

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time):
            return obj, ""
        cmd = [nvcc] + common + ["-c", src, "-o", obj + ".tmp"]
        if src.endswith(".cpp"):
            cmd = [nvcc] + common + ["-x", "cu", "-c", src, "-o", obj + ".tmp"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{p.stderr}")
        os.replace(obj + ".tmp", obj)
        return obj, p.stderr

    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, srcs))
    objs = [o for o, _ in results]
    if verbose:
        for o, log in results:
            if log.strip():
                print(os.path.basename(o), log, file=sys.stderr)
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
