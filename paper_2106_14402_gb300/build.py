"""Build libcb.so (the CUDA SpGEMM library) in-tree with nvcc for sm_103a.

Each .cu under csrc/ is compiled to an object in parallel, then linked into
paper_2106_14402_gb300/_build/libcb.so; the same sources compiled with
-DCB_CHECK give the bounds-checking debug library _build/libcb_check.so.
Objects are rebuilt when their source or any header is newer.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
GSRC = os.path.join(HERE, "csrc_gen")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcb.so")
OUT_CHECK = os.path.join(OUT, "check")
LIB_CHECK = os.path.join(OUT, "libcb_check.so")
GENLIB = os.path.join(OUT, "libcbgen.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcb.so")


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _lib_jobs(cc, out_dir, lib, extra, force, hdr):
    """(compile commands still needed, object files, link needed) of one library."""
    os.makedirs(out_dir, exist_ok=True)
    jobs, objs = [], []
    for s in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        o = os.path.join(out_dir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            jobs.append([cc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o])
    return jobs, objs, bool(jobs) or not os.path.exists(lib)


def _run(cmd, verbose=False):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout + r.stderr)


def build(verbose: bool = False, force: bool = False, extra_flags=(), check: bool | None = False) -> str:
    """Build libcb.so (check=False), the bounds-checking debug library
    libcb_check.so (check=True, -DCB_CHECK) or both (check=None; every
    translation unit of both compiled in one pool).  Returns the path of
    libcb.so, or of libcb_check.so when check=True."""
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    hdr = _headers_mtime()
    variants = {False: (OUT, LIB, list(extra_flags)),
                True: (OUT_CHECK, LIB_CHECK, list(extra_flags) + ["-DCB_CHECK"])}
    chosen = [False, True] if check is None else [bool(check)]
    plans = {v: _lib_jobs(cc, variants[v][0], variants[v][1], variants[v][2], force, hdr) for v in chosen}
    jobs = [j for v in chosen for j in plans[v][0]]
    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(lambda c: _run(c, verbose), jobs))
    for v in chosen:
        _, objs, link = plans[v]
        lib = variants[v][1]
        if link:
            tmp = lib + f".tmp{os.getpid()}"
            _run([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
                  "-Xlinker", "-rpath,/usr/local/cuda/lib64"], verbose)
            os.replace(tmp, lib)
    # the device-side input generator is a library of its own
    gsrc = os.path.join(GSRC, "cbgen.cu")
    if force or not os.path.exists(GENLIB) or os.path.getmtime(GENLIB) < os.path.getmtime(gsrc):
        tmp = GENLIB + f".tmp{os.getpid()}"
        _run([cc, *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
              "-o", tmp, gsrc, "-Xlinker", "-rpath,/usr/local/cuda/lib64"], verbose)
        os.replace(tmp, GENLIB)
    return LIB_CHECK if check is True else LIB


if __name__ == "__main__":
    print(build(verbose=True))
