"""In-tree build of libles.so for sm_103a (nvcc, no cmake).

Each .cu translation unit is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_2212_12365_gb300/_build/libles.so`` (static CUDA runtime)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libles.so")
SOURCES = ["les_kernels.cu", "les_stage.cu", "les_fused.cu", "les_api.cu", "les_noalloc.cu", "les_peak.cu", "les_fwh.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


BOUNDS_BUILD = os.path.join(HERE, "_build_bounds")
BOUNDS_LIB = os.path.join(BOUNDS_BUILD, "libles.so")


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "les.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(build_dir: str, lib: str, extra: list[str]) -> list:
    """Start the nvcc processes of one library; returns (src, process, obj)."""
    os.makedirs(build_dir, exist_ok=True)
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", *ARCH,
             "-I", os.path.join(ROOT, "include"), "-I", CSRC] + extra
    procs = []
    for src in SOURCES:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + flags
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), obj))
    return procs


def _link(lib: str, procs: list, verbose: bool) -> None:
    failed = []
    for src, p, _ in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"[{s}]\n{o}" for s, o in failed))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([nvcc(), "-shared", *ARCH, "-o", tmp, *[o for _, _, o in procs], "-cudart", "static"],
                   check=True)
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          bounds: bool = False) -> str:
    """libles.so (bounds=False) or its index-bounds-checked debug build
    (-DLES_BOUNDS_CHECK, _build_bounds/libles.so); returns the library path."""
    build_dir, lib = (BOUNDS_BUILD, BOUNDS_LIB) if bounds else (BUILD, LIB)
    if not force and not _stale(lib):
        return lib
    _link(lib, _compile(build_dir, lib, (["-DLES_BOUNDS_CHECK"] if bounds else []) + (extra or [])), verbose)
    return lib


def build_all(force: bool = False, verbose: bool = False) -> tuple[str, str]:
    """Both libraries, compiled in parallel."""
    jobs = []
    for bounds, (build_dir, lib) in ((False, (BUILD, LIB)), (True, (BOUNDS_BUILD, BOUNDS_LIB))):
        if force or _stale(lib):
            jobs.append((lib, _compile(build_dir, lib, ["-DLES_BOUNDS_CHECK"] if bounds else [])))
    for lib, procs in jobs:
        _link(lib, procs, verbose)
    return LIB, BOUNDS_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
