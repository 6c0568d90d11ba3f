"""A monoid of the caller's own through include/tb_monoid.cuh: 2x2 uint32
matrices under the product, compiled from tests/user_monoid_scan.cu.  The
CPU test compiles it (the header must build for sm_103a); the GPU test runs
DOWN and UP scans and compares them with products taken along parent links
on the host, exactly (wrapping 32-bit arithmetic)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "user_monoid_scan.cu")


def _nvcc(args):
    from paper_2205_11659_gb300 import _build
    cmd = [_build.nvcc()] + _build.ARCH + ["-O2", "-std=c++17", "-I" + os.path.join(ROOT, "include")]
    r = subprocess.run(cmd + args, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return r


def test_header_compiles(tmp_path):
    _nvcc(["-c", SRC, "-o", str(tmp_path / "user.o")])


_SIZED = r"""
#include <cstdint>
#include "tb_monoid.cuh"
struct Sized {
  struct V { ELEM e[COUNT]; };
  __device__ static V identity() { V v; for (int i = 0; i < COUNT; ++i) v.e[i] = 0; return v; }
  __device__ static V combine(const V& a, const V& b) {
    V v; for (int i = 0; i < COUNT; ++i) v.e[i] = a.e[i] + b.e[i]; return v;
  }
  __device__ static V load(const void* p, int64_t i) { return static_cast<const V*>(p)[i]; }
  __device__ static void store(void* p, int64_t i, const V& v) { static_cast<V*>(p)[i] = v; }
};
int run(const uint8_t* k, int64_t n, int64_t J, const void* in, void* out, void* ws, size_t nb,
        int32_t* st) {
  return tb::tree_scan<Sized>(TB_DOWN, k, n, J, in, out, ws, nb, st, nullptr);
}
"""


@pytest.mark.parametrize("elem,count,error", [
    ("unsigned", 3, None),                        # 12 bytes: whole words, under the limit
    ("unsigned", 13, "at most 48 bytes"),         # 52 bytes: over the workspace slot
    ("unsigned char", 6, "whole 32-bit words"),   # 6 bytes: not whole words
])
def test_value_size_rules(tmp_path, elem, count, error):
    """The header accepts values of whole 32-bit words up to 48 bytes and
    rejects others at compile time with a message saying why."""
    from paper_2205_11659_gb300 import _build
    src = tmp_path / "sized.cu"
    src.write_text(_SIZED)
    cmd = [_build.nvcc()] + _build.ARCH + ["-O1", "-std=c++17", "-I" + os.path.join(ROOT, "include"),
                                          "-DELEM=" + elem, "-DCOUNT=%d" % count, "-c", str(src),
                                          "-o", str(tmp_path / "sized.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if error is None:
        assert r.returncode == 0, r.stderr
    else:
        assert r.returncode != 0 and error in r.stderr, r.stderr


def test_no_process_wide_launch_state(tmp_path):
    """The launch sequence keeps once-per-kernel flags (shared-memory limit
    raised) in function-local statics.  They must stay private to each
    shared object: as GNU unique symbols ('u' in nm) they would be shared
    with the library and with any other copy, and a copy loaded second
    would launch without raising its own kernels' limit."""
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    from paper_2205_11659_gb300 import _build
    lib = tmp_path / "libuser.so"
    _nvcc(["-shared", "-Xcompiler", "-fPIC", SRC, "-o", str(lib)])
    for path in (str(lib), _build.build()):
        out = subprocess.run([nm, "-D", "--defined-only", path], capture_output=True, text=True).stdout
        unique = [ln for ln in out.splitlines() if len(ln.split()) >= 3 and ln.split()[1] == "u"]
        assert not unique, unique[:3]


def _mul(x, y):
    m = 0xFFFFFFFF
    return ((x[0] * y[0] + x[1] * y[2]) & m, (x[0] * y[1] + x[1] * y[3]) & m,
            (x[2] * y[0] + x[3] * y[2]) & m, (x[2] * y[1] + x[3] * y[3]) & m)


def _reference(kind, vals):
    """DOWN and UP by explicit parent links (stack walk over the stream)."""
    parent, children, stack, r = [], [], [], 0
    for k in kind:
        if k in (1, 2):
            parent.append(stack[-1] if stack else -1)
            children.append([])
            if stack:
                children[stack[-1]].append(r)
            stack.append(r)
            r += 1
        elif k == 3:
            stack.pop()
    J = r
    v = [tuple(int(x) for x in vals[j]) for j in range(J)]
    down = [None] * J
    for j in range(J):
        down[j] = v[j] if parent[j] < 0 else _mul(down[parent[j]], v[j])
    up = [None] * J
    for j in range(J - 1, -1, -1):
        acc = v[j]
        for c in children[j]:
            acc = _mul(acc, up[c])
        up[j] = acc
    return np.array(down, np.uint32), np.array(up, np.uint32)


@pytest.mark.gpu
def test_user_monoid_scans(tmp_path):
    import torch
    from paper_2205_11659_gb300 import binding, inputs
    lib_path = tmp_path / "libuser.so"
    _nvcc(["-shared", "-Xcompiler", "-fPIC", SRC, "-o", str(lib_path)])
    lib = ctypes.CDLL(str(lib_path))
    lib.user_ws_size.argtypes = [ctypes.c_int64]
    lib.user_ws_size.restype = ctypes.c_size_t
    lib.user_scan.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                              ctypes.c_void_p, ctypes.c_void_p]
    lib.user_scan.restype = ctypes.c_int
    rng = np.random.default_rng(5)
    cases = [inputs.skeleton_kinds(6000, 80), inputs.random_walk_scene(30_000, 81)[0],
             inputs.chain_scene(3000, 82)[0]]
    for kind in cases:
        J = int(np.count_nonzero((kind == 1) | (kind == 2)))
        vals = rng.integers(0, 2**32, (J, 4), dtype=np.uint64).astype(np.uint32)
        want_down, want_up = _reference(kind, vals)
        kd = torch.from_numpy(kind).cuda()
        vd = torch.from_numpy(vals.view(np.int32)).cuda()
        nb = lib.user_ws_size(kind.size)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        for d, want in ((binding.TB_DOWN, want_down), (binding.TB_UP, want_up)):
            out = torch.empty_like(vd)
            rc = lib.user_scan(d, kd.data_ptr(), kind.size, J, vd.data_ptr(), out.data_ptr(),
                               ws.data_ptr(), nb, status.data_ptr(), None)
            assert rc == binding.TB_OK
            torch.cuda.synchronize()
            assert int(status.item()) == binding.TB_OK
            assert np.array_equal(out.cpu().numpy().view(np.uint32), want)
