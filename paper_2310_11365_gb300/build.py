"""In-tree build of libmmp.so for sm_103a (nvcc, one job per translation unit).

    python -m paper_2310_11365_gb300.build            # build if out of date
    python -m paper_2310_11365_gb300.build --force    # rebuild

The library links the shared CUDA runtime, so a process that already loaded
it (e.g. through PyTorch) shares one runtime and one primary context.
"""
from __future__ import annotations

import argparse
import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(HERE, "lib", "obj")
LIB = os.path.join(LIBDIR, "libmmp.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -ftz=true: FP32 subnormals flush to zero in every translation unit, so the
# hardware log2/rsqrt/sin/cos of the FP32 Box-Muller need no subnormal fix-up
# code, and the forward, batched and adjoint kernels round identically.
# Particle values, uniforms (>= 2^-24) and moments stay far above 1e-38.
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler", "-fPIC", "-Xcompiler",
          "-fvisibility=default", "-I", INCLUDE]


# Per-file flags.  driver.cu: no multiply-add contraction, so the FP64
# driver body rounds identically whether it is inlined into the per-problem
# or the batched driver kernel (contraction choices can depend on context).
FILE_FLAGS = {"driver.cu": ["-fmad=false"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "mmp.h")]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ and link lib/libmmp.so; returns its path."""
    if not force and not _stale(LIB, _deps() + [__file__]):
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    cc = nvcc()
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "mmp.h")]

    def compile_one(src: str) -> str:
        obj = os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src, __file__] + headers):
            # -Xptxas=-v only reports (registers, stack, spills); its report
            # is kept beside the object for resource_usage()
            cmd = [cc, "-Xptxas=-v", *ARCH, *CFLAGS, *FILE_FLAGS.get(os.path.basename(src), []), "-c", src,
                   "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            with open(obj[:-2] + ".ptxas.txt", "w") as fh:
                fh.write(r.stderr)
            if verbose:
                sys.stderr.write(r.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def resource_usage() -> dict[str, dict]:
    """Per kernel (mangled name), what ptxas reported when the library was
    last compiled: registers, stack frame bytes, spill store and load bytes."""
    import re

    out: dict[str, dict] = {}
    for log in sorted(glob.glob(os.path.join(OBJDIR, "*.ptxas.txt"))):
        props: dict[str, tuple[int, int, int]] = {}
        current = None   # the function whose properties come next
        entry = None     # the entry whose register count comes next
        for line in open(log):
            m = re.search(r"Function properties for (\S+)", line)
            if m:
                current = m.group(1)
                continue
            m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
            if m and current is not None:
                props[current] = tuple(int(g) for g in m.groups())
                current = None
                continue
            m = re.search(r"Compiling entry function '(\S+)'", line)
            if m:
                entry = m.group(1)
                continue
            m = re.search(r"Used (\d+) registers", line)
            if m and entry is not None:
                out[entry] = {"registers": int(m.group(1)), "file": os.path.basename(log)[: -len(".ptxas.txt")]}
                entry = None
        for name, rec in out.items():
            if name in props:
                rec["stack"], rec["spill_stores"], rec["spill_loads"] = props[name]
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", "--verbose", action="store_true")
    args = ap.parse_args()
    print(build(force=args.force, verbose=args.verbose))
