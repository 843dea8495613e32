"""Builds libseb.so in-tree for sm_103a with nvcc (no cmake, no torch extension).

Each translation unit under ``csrc/`` is compiled in parallel, then linked into
``paper_2503_02412_gb300/libseb.so`` (the CUDA runtime is linked statically, so the library
only needs the CUDA driver at run time).  ``python -m paper_2503_02412_gb300.build`` runs it.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "libseb.so")
# Bounds-checked build (-DSEB_DEBUG): every index check of the kernels is compiled in; a failed
# check raises a bit of the device error word instead of touching memory.  Same entry points.
OUT_DEBUG = os.path.join(PKG, "libseb_debug.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return sorted(hs)


def _flags(extra=()):
    defs = [f"-D{d}" for d in os.environ.get("SEB_DEFINES", "").split() if d]
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                   "--expt-relaxed-constexpr", *defs, *extra]


def _compile(src, extra, build_dir=BUILD):
    os.makedirs(build_dir, exist_ok=True)
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [NVCC, *_flags(extra), "-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "cu")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stamp(extra):
    h = hashlib.sha256()
    for f in _sources() + _headers():
        with open(f, "rb") as fh:
            h.update(f.encode() + fh.read())
    h.update(" ".join(_flags(extra)).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile every CUDA/C++ source of the package and link libseb.so (libseb_debug.so with
    debug=True: the bounds-checked build); returns its path."""
    out = OUT_DEBUG if debug else OUT
    extra = tuple(extra) + (("-DSEB_DEBUG",) if debug else ())
    build_dir = BUILD + ("_debug" if debug else "")
    stamp_file = out + ".stamp"
    stamp = _stamp(extra)
    if not force and os.path.exists(out) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read() == stamp:
                return out
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, build_dir), _sources()))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log.strip():
                print(log, file=sys.stderr)
    tmp = out + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
