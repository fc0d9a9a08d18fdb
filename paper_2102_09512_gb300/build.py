"""Builds the CUDA library ``_build/libelbm.so`` in-tree with nvcc for sm_103a.

The kernel source is compiled once per (lattice, store) combination, in
parallel, and linked with the C-ABI translation unit.  No torch headers are used.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libelbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-diag-suppress", "177",
         "-I", CSRC, "-I", INCLUDE]
STORES = [("f64", 0), ("f32", 1), ("f16", 2), ("bf16", 3)]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libelbm")
    return exe


def _sources_digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            with open(os.path.join(d, name), "rb") as fh:
                h.update(name.encode())
                h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(force: bool = False, verbose: bool = False, extra_flags=(), out_dir: str = BUILD) -> str:
    """Compile (if sources changed) and return the path of libelbm.so (in out_dir)."""
    os.makedirs(out_dir, exist_ok=True)
    lib_path = os.path.join(out_dir, "libelbm.so")
    stamp = os.path.join(out_dir, "digest.txt")
    digest = _sources_digest() + " ".join(extra_flags)
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read() == digest:
                return lib_path
    exe = nvcc()
    jobs = []
    for D in (2, 3):
        for name, st in STORES:
            obj = os.path.join(out_dir, f"elbm_d{D}_{name}.o")
            cmd = [exe, *ARCH, *FLAGS, *extra_flags, f"-DELBM_D={D}", f"-DELBM_ST={st}",
                   f"-DELBM_OPS_NAME=d{D}_{name}", "-c", os.path.join(CSRC, "elbm_kernels.cu"), "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((obj, cmd))
    for name in ("elbm_api", "elbm_noalloc", "elbm_ensemble"):
        obj = os.path.join(out_dir, f"{name}.o")
        jobs.append((obj, [exe, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, f"{name}.cu"), "-o", obj]))
    workers = min(len(jobs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        outs = list(ex.map(lambda j: _run(j[1]), jobs))
    if verbose:
        for (obj, _), out in zip(jobs, outs):
            sys.stdout.write(f"--- {os.path.basename(obj)}\n{out}")
    tmp = lib_path + f".tmp{os.getpid()}"
    _run([exe, *ARCH, "-shared", "-o", tmp, *[j[0] for j in jobs], "-lcudart"])
    os.replace(tmp, lib_path)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
