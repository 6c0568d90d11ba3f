"""Compiles the CUDA sources of the package into an in-tree shared library.

``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` for every
``csrc/*.cu`` translation unit (in parallel), then one ``nvcc -shared`` link
into ``_build/libtb.so``.  Rebuilds only when a source or header is newer than
the library.  The tile shape of the scene kernels (threads per block, elements
per thread) and whether the main tile pass runs as persistent blocks come from
``tuned_shape.json``, written by ``autotune.py``.
"""
import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libtb.so")
SHAPE_FILE = os.path.join(PKG, "tuned_shape.json")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            exe = cand
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtb.so")
    return exe


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    deps = (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])
    if os.path.exists(SHAPE_FILE):
        deps.append(SHAPE_FILE)
    return deps


def tuned_shape():
    """(threads per block, elements per thread) of the scene kernels."""
    import json
    if os.path.exists(SHAPE_FILE):
        with open(SHAPE_FILE) as f:
            d = json.load(f)
        return int(d["threads_per_block"]), int(d["elements_per_thread"])
    return 256, 16


def tuned_persistent():
    """Whether the main tile pass runs as persistent blocks."""
    import json
    if os.path.exists(SHAPE_FILE):
        with open(SHAPE_FILE) as f:
            return bool(json.load(f).get("persistent", False))
    return False


def tuned_matcher():
    """In-tile matcher of the matching-only pass: 0 = the chunk walk (default),
    1 = the binary search over a tree of depths (Fig. "core")."""
    import json
    if os.path.exists(SHAPE_FILE):
        with open(SHAPE_FILE) as f:
            return int(json.load(f).get("matcher", 0))
    return 0


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force=False, verbose=False, shape=None, out_dir=None, persistent=None, debug=False,
          matcher=None):
    """Build the library if needed; returns its path.  shape = (threads per
    block, elements per thread) and persistent override the tuned values and
    out_dir the output folder (the autotuner builds its candidates that
    way); debug=True compiles the kernels' index checks in (TB_DEBUG; give it
    an out_dir of its own); matcher selects the in-tile matcher of the
    matching-only pass (tuned_matcher())."""
    out_dir = OUT_DIR if out_dir is None else out_dir
    lib_path = os.path.join(out_dir, "libtb.so")
    if not force and up_to_date(lib_path):
        return lib_path
    os.makedirs(out_dir, exist_ok=True)
    exe = nvcc()
    nt, kpt = tuned_shape() if shape is None else shape
    persist = tuned_persistent() if persistent is None else bool(persistent)
    match_kind = tuned_matcher() if matcher is None else int(matcher)
    common = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I" + INCLUDE, "-I" + CSRC, "-DTB_NT=%d" % nt, "-DTB_KPT=%d" % kpt,
                     "-DTB_PERSIST=%d" % int(persist), "-DTB_DEBUG=%d" % int(bool(debug)),
              "-DTB_MATCHER=%d" % match_kind]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [exe] + common + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + ".%d.tmp" % os.getpid()
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
