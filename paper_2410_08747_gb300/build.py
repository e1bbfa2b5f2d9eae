"""Builds the CUDA library ``libmcx.so`` in-tree for sm_103a with nvcc.

Every translation unit under ``csrc/`` is compiled in parallel into
``csrc/_build/`` and linked into ``paper_2410_08747_gb300/libmcx.so``.  Tracer
units (the ones that decide counts) are compiled with ``-fmad=false`` and all
host code with ``-ffp-contract=off`` so that their rounding follows the
written operation sequence on both x86-64 and aarch64 hosts.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(CSRC, "_build")
LIB = os.path.join(HERE, "libmcx.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# translation units whose arithmetic decides counts: no FMA contraction
NO_FMA = {"mcx_trace.cu", "mcx_batch.cu", "mcx_static.cu", "mcx_starts.cu", "mcx_mlp.cu"}


def cuda_home() -> str:
    h = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if h:
        return h
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
           if f.endswith((".cu", ".cuh", ".h"))]
    out.append(os.path.join(ROOT, "include", "mcx.h"))
    return out


# device headers handed to the run-time compiler as text (mcx_jit.cu)
EMBED = (("kEmbedInternalH", "mcx_internal.h"), ("kEmbedTracerCuh", "mcx_tracer.cuh"))
EMBED_DELIM = "MCXEMBED"


def write_embed() -> None:
    """csrc/_build/mcx_embed.h: each device header as a raw string literal."""
    out = ["// generated by build.py from the device headers; do not edit", "#pragma once"]
    for name, f in EMBED:
        text = open(os.path.join(CSRC, f)).read()
        if f")({EMBED_DELIM}" in text or f"){EMBED_DELIM}" in text:
            raise RuntimeError(f"{f} contains the raw-string delimiter")
        out.append(f'static const char {name}[] = R"{EMBED_DELIM}({text}){EMBED_DELIM}";')
    path = os.path.join(BUILD, "mcx_embed.h")
    text = "\n".join(out) + "\n"
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as fh:
            fh.write(text)


def _compile(src: str, nvcc: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include"),
           "-I", BUILD, "-c", os.path.join(CSRC, src), "-o", obj]
    if src in NO_FMA:
        cmd.insert(4, "-fmad=false")
    if verbose:
        cmd.append("-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose and r.stderr:
        print(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libmcx.so unless it is newer than every source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in _deps())):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    home = cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc") or "nvcc"
    srcs = sources()
    write_embed()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, verbose), srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    libdir = os.path.join(home, "lib64")
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared", "-lnvrtc",
           "-Xlinker", "-rpath", "-Xlinker", libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
