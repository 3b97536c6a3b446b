"""Build libcola.so in-tree for sm_103a (nvcc, one process per translation unit)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libcola.so")
SOURCES = ["kernels_fft.cu", "kernels_pm.cu", "kernels_ic.cu", "host_cosmo.cpp", "cola_api.cpp",
           "pk_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def flags(verbose_ptxas: bool = False) -> list[str]:
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
         "-I", SRC] + ARCH
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _compile(src: str, obj: str, verbose_ptxas: bool) -> tuple[str, int, str]:
    cmd = [nvcc(), "-c", os.path.join(SRC, src), "-o", obj] + flags(verbose_ptxas)
    p = subprocess.run(cmd, capture_output=True, text=True)
    return src, p.returncode, p.stdout + p.stderr


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = True) -> str:
    """Compile every translation unit in parallel and link the shared library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = [os.path.join(SRC, s) for s in SOURCES]
    headers = [os.path.join(SRC, h) for h in os.listdir(SRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "cola.h"))
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in srcs + headers + [__file__])
        if os.path.getmtime(LIB) >= newest:
            return LIB
    objs = [os.path.join(OUT_DIR, s + ".o") for s in SOURCES]
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda a: _compile(*a), [(s, o, verbose_ptxas) for s, o in zip(SOURCES, objs)]))
    failed = [r for r in results if r[1] != 0]
    for src, rc, log in results:
        if log.strip() and (not quiet or rc != 0 or verbose_ptxas):
            sys.stderr.write(f"--- {src} (rc={rc})\n{log}\n")
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(r[0] for r in failed))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + p.stdout + p.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False)
    print(LIB)
