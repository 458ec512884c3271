"""In-tree build of libgpflbm.so for sm_103a with nvcc.

Each translation unit under csrc/ compiles in parallel to an object file in
_build/, then nvcc links the shared library (CUDA runtime linked
statically, so the library only needs the driver).  Objects are rebuilt when
their source or any header is newer.
"""
import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgpflbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC,
         "--expt-relaxed-constexpr"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return exe


def _headers_mtime():
    hs = (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
          glob.glob(os.path.join(INCLUDE, "*.h")))
    return max(os.path.getmtime(h) for h in hs)


def _units():
    """(source, object name, defines): every csrc/*.cu once, and each kernel
    instance file a second time with the extended-model kernels."""
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        name = os.path.basename(src)[:-3]
        units.append((src, name, []))
        if name.startswith("inst_"):
            units.append((src, name + "_ext", ["-DGPFLBM_EXT=1"]))
    return units


def _compile(src, name, extra):
    obj = os.path.join(BUILD, name + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _headers_mtime()):
        return obj, None
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return obj, "%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj, None


def build(verbose=False, jobs=None, extra=()):
    """Compile every csrc/*.cu and link _build/libgpflbm.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    units = _units()
    # the long 3D instance files first, so that they do not finish last
    units.sort(key=lambda u: (not u[1].startswith("inst_d3"), u[1]))
    jobs = jobs or min(len(units), max(2, os.cpu_count() or 2))
    with concurrent.futures.ThreadPoolExecutor(jobs) as pool:
        results = list(pool.map(lambda u: _compile(u[0], u[1], u[2] + list(extra)), units))
    errors = [e for _, e in results if e]
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    objs = [o for o, _ in results]
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(LIB + ".tmp", LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
