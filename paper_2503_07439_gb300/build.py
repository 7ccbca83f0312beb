"""Build the CUDA library libme_gb300.so in-tree (nvcc, sm_103a only, no CMake).

Translation units are compiled in parallel, then linked into one shared library next
to this file.  Objects go to ``_build/`` inside the package.  Rebuilds only what is
out of date (source or header newer than the object).
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libme_gb300.so")
FLOPS_TOOL = os.path.join(BUILD, "me_flops")
SOURCES = ["me_core.cu", "me_serve.cu", "me_inst_ee.cu", "me_inst_gg.cu", "me_inst_ggg.cu",
           "me_inst_ggg64.cu", "me_inst_uu.cu", "me_inst_queued.cu", "me_inst_queued_gg.cu", "me_noalloc.cu",
           "me_phase.cu", "me_inst_serve.cu", "me_inst_serve_gg.cu", "me_inst_terms.cu", "me_inst_terms_gg.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def build(verbose: bool = False, extra_flags=()) -> str:
    extra_flags = tuple(extra_flags) + tuple(os.environ.get("ME_NVCC_FLAGS", "").split())
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    newest_header = max(os.path.getmtime(h) for h in _headers())
    procs, objs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), newest_header):
            continue
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, "-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    if procs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
    src = os.path.join(CSRC, "me_flops.cu")
    if not os.path.exists(FLOPS_TOOL) or os.path.getmtime(FLOPS_TOOL) < max(os.path.getmtime(src), newest_header):
        r = subprocess.run([nvcc, "-O1", "-std=c++17", "-diag-suppress", "20014", "-x", "cu", src, "-o", FLOPS_TOOL],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("op-count tool failed to build:\n" + r.stdout + r.stderr)
    return LIB


def block_check_tool() -> str:
    """Build (if out of date) the host program that compares helicity-block and
    single-helicity evaluations (csrc/me_blockcheck.cu), linked against the library."""
    build()
    tool = os.path.join(BUILD, "me_blockcheck")
    src = os.path.join(CSRC, "me_blockcheck.cu")
    newest = max([os.path.getmtime(src), os.path.getmtime(LIB)] + [os.path.getmtime(h) for h in _headers()])
    if not os.path.exists(tool) or os.path.getmtime(tool) < newest:
        r = subprocess.run([_nvcc(), "-O1", "-std=c++17", "-diag-suppress", "20014,20013", "-I", INCLUDE, "-x", "cu", src,
                            "-o", tool, "-L", PKG, "-lme_gb300", "-Xlinker", "-rpath=" + PKG],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("block-check tool failed to build:\n" + r.stdout + r.stderr)
    return tool


def op_counts() -> dict:
    """Algorithmic operation counts per helicity / event (see csrc/me_flops.cu)."""
    import json
    build()  # incremental: rebuilds the tool when its sources changed
    return json.loads(subprocess.run([FLOPS_TOOL], check=True, capture_output=True, text=True).stdout)


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
