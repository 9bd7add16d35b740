"""Builds libsfhad.so (sm_103a) in-tree with nvcc.

The kernel templates are instantiated in several objects (one per precision
mode and dimension) that compile in parallel; the host API, the serving
runtime and the peak benchmarks are separate objects.  Objects are rebuilt
when their source or any header is newer.  Output:
``paper_2306_11665_gb300/libsfhad.so`` (objects under ``_build/``).

``build(debug=True)`` (or ``python -m paper_2306_11665_gb300.build --debug``)
builds the bounds-checked debug library ``libsfhad_debug.so`` from the same
sources with ``-DSFH_DEBUG`` (objects under ``_build_debug/``): every kernel
index into global and shared memory is checked against its buffer, and an
index outside it is reported as SFH_EBOUNDS instead of being used.  The
binding loads it when ``SFH_LIB_VARIANT=debug``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsfhad.so")
OUT_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libsfhad_debug.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-prec-div=true", "-prec-sqrt=true", "-ftz=false", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]

INST = [
    ("fp64_d2", ["-DSFH_INST_FP64", "-DSFH_INST_D=2"]),
    ("fp64_d3", ["-DSFH_INST_FP64", "-DSFH_INST_D=3"]),
    ("fp32k_d2", ["-DSFH_INST_FP32K", "-DSFH_INST_D=2"]),
    ("fp32k_d3", ["-DSFH_INST_FP32K", "-DSFH_INST_D=3"]),
    ("mixed_d2", ["-DSFH_INST_MIXED", "-DSFH_INST_D=2"]),
    ("mixed_d3", ["-DSFH_INST_MIXED", "-DSFH_INST_D=3"]),
    ("vjp_d2", ["-DSFH_INST_VJP", "-DSFH_INST_D=2"]),
    ("vjp_d3", ["-DSFH_INST_VJP", "-DSFH_INST_D=3"]),
]
# Chandrashekar's flux in units of their own (entry points suffixed _ch)
INST += [(name + "_ch", defs + ["-DSFH_INST_CH"]) for name, defs in list(INST)]
# modal / uncollocated entry points (suffixed _modal)
INST += [(name + "_modal", defs + ["-DSFH_INST_MODAL"]) for name, defs in list(INST)]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsfhad")
    return exe


def _units(out=OUT, defs0=()):
    units = []
    for name, defs in INST:
        units.append((os.path.join(CSRC, "sfh_inst.cu"), os.path.join(out, f"inst_{name}.o"), list(defs0) + defs))
    for src in ("sfh_api.cu", "sfh_serve.cu", "sfh_noalloc.cu", "sfh_entropy.cu", "sfh_fig1.cu", "sfh_surface.cu",
                "sfh_modal.cu"):
        units.append((os.path.join(CSRC, src), os.path.join(out, src.replace(".cu", ".o")), list(defs0)))
    return units


def _stale(src: str, obj: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def _compile(src, obj, defs, extra, verbose):
    cmd = [nvcc()] + ARCH + FLAGS + list(extra) + defs + ["-c", src, "-o", obj + ".tmp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    os.replace(obj + ".tmp", obj)
    return res.stdout + res.stderr if verbose else ""


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile every CUDA unit for sm_103a and link libsfhad.so (debug: the
    bounds-checked libsfhad_debug.so); returns its path."""
    out, lib_path = (OUT_DEBUG, LIB_DEBUG) if debug else (OUT, LIB)
    os.makedirs(out, exist_ok=True)
    units = _units(out, ["-DSFH_DEBUG"] if debug else [])
    todo = [u for u in units if force or _stale(u[0], u[1])]
    # the serving unit (every tile body of both Euler fluxes in one kernel)
    # is the longest compile: started first, it does not finish last
    todo.sort(key=lambda u: 0 if os.path.basename(u[0]) == "sfh_serve.cu" else 1)
    jobs = jobs or max(1, min(len(todo) or 1, os.cpu_count() or 1))
    logs = []
    if todo:
        with cf.ThreadPoolExecutor(jobs) as ex:
            futs = [ex.submit(_compile, s, o, d, extra, verbose) for s, o, d in todo]
            for f in futs:
                logs.append(f.result())
    objs = [u[1] for u in units]
    if todo or not os.path.exists(lib_path) or any(os.path.getmtime(o) > os.path.getmtime(lib_path) for o in objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, lib_path)
    if verbose:
        sys.stdout.write("".join(logs))
    return lib_path


if __name__ == "__main__":
    v = "-v" in sys.argv
    f = "-f" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=f or bool(extra), verbose=v or bool(extra), extra=extra, debug="--debug" in sys.argv))
