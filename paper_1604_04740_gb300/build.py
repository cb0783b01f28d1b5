"""Compile the CUDA library libne.so in-tree for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel to an object, then linked into
one shared library next to this file.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libne.so")
PROBE = os.path.join(HERE, "probe")
PROBE_LIB = os.path.join(PROBE, "libne_probe.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def _deps_mtime() -> float:
    hdrs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max([os.path.getmtime(h) for h in hdrs] + [0.0])


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
    deps = max(_deps_mtime(), max([os.path.getmtime(h) for h in glob.glob(os.path.join(PROBE, "*.h"))] + [0.0]))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), deps):
        return obj
    cmd = [NVCC, *ARCH, *FLAGS, "-I", PROBE, "-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def _link(lib: str, objs) -> None:
    newest = max(os.path.getmtime(o) for o in objs)
    manifest = os.path.join(OBJDIR, os.path.basename(lib) + ".objs")
    listed = open(manifest).read() if os.path.exists(manifest) else ""
    if not os.path.exists(lib) or os.path.getmtime(lib) < newest or listed != "\n".join(objs):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
        with open(manifest, "w") as f:
            f.write("\n".join(objs))


def build(verbose: bool = False) -> str:
    """Builds libne.so (the library) and probe/libne_probe.so (the benchmark's
    throughput probes, not part of the library's ABI); returns libne.so."""
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    psrcs = sorted(glob.glob(os.path.join(PROBE, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), srcs + psrcs))
    _link(LIB, objs[:len(srcs)])
    _link(PROBE_LIB, objs[len(srcs):])
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
