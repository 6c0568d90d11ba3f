"""Sequential CPU oracle (test infrastructure only).

This package is test infrastructure, not the product: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path and
never imports it.  The arithmetic lives in ``tb_oracle.c`` (plain C, compiled
here with gcc); this module only builds it and marshals numpy arrays.

Every routine restates a definition of Levien, "Fast GPU bounding boxes on
tree-structured scenes" (arXiv 2205.11659):

* :func:`bic`            Sec. 3 -- bicyclic semigroup reduction.
* :func:`stack_slice`    Sec. 4 -- stack monoid ``Stk(enum(s))``.
* :func:`match_parens`   Sec. 2, Fig. 1 -- the strong matching problem.
* :func:`bboxes`         Sec. 1 and Sec. 6 -- clip intersection down the tree,
  blend union up the tree.
* :func:`open_positions` Sec. 1.1 -- stream compaction of the opens.
* :func:`clip_out`       Sec. 9 -- the running clip intersection per element.
* :func:`tree_scan_i32`, :func:`tree_scan_box`, :func:`affine_forward`,
  :func:`affine_up` -- Sec. 1 / Sec. 13, any monoid over the tree.
* :func:`affine_backward` -- adjoint of the root-path transform product.
* :func:`rigid_scan` -- the same folds over rigid transforms (quaternion and
  translation).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

OK = 0
UNBALANCED = 2
BAD_KIND = 3
DOWN = 0
UP = 1
ISECT = 0
UNION = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile tb_oracle.c into a shared library next to it (gcc -O2)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, p = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.orc_bic.argtypes = [p, i64, p, p]
            lib.orc_stack_slice.argtypes = [p, i64, p, p]
            lib.orc_stack_slice.restype = i64
            lib.orc_match_parens.argtypes = [p, i64, p, p]
            lib.orc_bboxes.argtypes = [p, p, i64, p, p, p]
            lib.orc_bboxes_batched.argtypes = [p, p, p, i64, p, p, p]
            lib.orc_open_positions.argtypes = [p, i64, p, i64, p]
            lib.orc_clip_out.argtypes = [p, p, i64, p]
            lib.orc_tree_scan_i32.argtypes = [i32, p, i64, p, p]
            lib.orc_tree_scan_box.argtypes = [i32, i32, p, i64, p, p]
            lib.orc_affine_forward.argtypes = [p, i64, p, p]
            lib.orc_rigid_scan.argtypes = [ctypes.c_int, p, i64, p, p]
            lib.orc_tree_structure.argtypes = [p, i64, p, p, p]
            lib.orc_affine_up.argtypes = [p, i64, p, p]
            lib.orc_affine_loss.argtypes = [p, i64, p, p, i64, p]
            lib.orc_affine_backward.argtypes = [p, i64, p, p, p, i64]
            for f in (lib.orc_bic, lib.orc_match_parens, lib.orc_bboxes,
                      lib.orc_bboxes_batched, lib.orc_open_positions, lib.orc_clip_out,
                      lib.orc_tree_scan_i32,
                      lib.orc_tree_scan_box, lib.orc_affine_forward,
                      lib.orc_affine_up, lib.orc_affine_loss,
                      lib.orc_affine_backward, lib.orc_rigid_scan, lib.orc_tree_structure):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _kinds(kind):
    return np.ascontiguousarray(kind, dtype=np.uint8)


def bic(kind):
    """Bic(s) of the whole stream as (a, b) -- Sec. 3."""
    k = _kinds(kind)
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    st = _load().orc_bic(_ptr(k), k.size, ctypes.byref(a), ctypes.byref(b))
    if st:
        raise ValueError("bad kind")
    return a.value, b.value


def stack_slice(kind):
    """Stk(enum(s)) as (a, list of unmatched open indices, bottom first)."""
    k = _kinds(kind)
    out = np.empty(max(k.size, 1), np.int64)
    a = ctypes.c_int64()
    m = _load().orc_stack_slice(_ptr(k), k.size, ctypes.byref(a), _ptr(out))
    return a.value, out[:m].copy()


def match_parens(kind):
    """(status, parent, match) of Fig. 1's strong matching problem."""
    k = _kinds(kind)
    parent = np.empty(k.size, np.int32)
    match = np.empty(k.size, np.int32)
    st = _load().orc_match_parens(_ptr(k), k.size, _ptr(parent), _ptr(match))
    return st, parent, match


def bboxes(kind, box):
    """(status, parent, match, box_out) -- Sec. 1 / Sec. 6 definitions."""
    k = _kinds(kind)
    b = np.ascontiguousarray(box, dtype=np.float32).reshape(-1, 4)
    assert b.shape[0] == k.size
    parent = np.empty(k.size, np.int32)
    match = np.empty(k.size, np.int32)
    out = np.empty((k.size, 4), np.float32)
    st = _load().orc_bboxes(_ptr(k), _ptr(b), k.size, _ptr(parent), _ptr(match),
                            _ptr(out))
    return st, parent, match, out


def bboxes_batched(kind, box, offsets):
    """Per-scene bboxes with scene-local parent/match indices."""
    k = _kinds(kind)
    b = np.ascontiguousarray(box, dtype=np.float32).reshape(-1, 4)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    parent = np.empty(k.size, np.int32)
    match = np.empty(k.size, np.int32)
    out = np.empty((k.size, 4), np.float32)
    st = _load().orc_bboxes_batched(_ptr(k), _ptr(b), _ptr(off), off.size - 1,
                                    _ptr(parent), _ptr(match), _ptr(out))
    return st, parent, match, out


def open_positions(kind, cap=None):
    """(status, pos, count): indices of the opens in stream order -- Sec. 1.1.
    Only the first ``cap`` (default: all) are returned."""
    k = _kinds(kind)
    c = ctypes.c_int64()
    cap = k.size if cap is None else int(cap)
    pos = np.empty(max(cap, 0), np.int32)
    st = _load().orc_open_positions(_ptr(k), k.size, _ptr(pos), cap, ctypes.byref(c))
    return st, pos[:min(cap, c.value)].copy(), c.value


def clip_out(kind, box):
    """(status, clip): per element the intersection of its box with every clip
    ancestor's box (Sec. 9); blends pass the clip in force on, a close gets
    its open's value."""
    k = _kinds(kind)
    b = np.ascontiguousarray(box, dtype=np.float32).reshape(-1, 4)
    out = np.zeros((k.size, 4), np.float32)
    st = _load().orc_clip_out(_ptr(k), _ptr(b), k.size, _ptr(out))
    return st, out


def _num_opens(k):
    return int(np.count_nonzero((k == 1) | (k == 2)))


def tree_scan_i32(direction, kind, values):
    """ADD over int32 values given per open in pre-order."""
    k = _kinds(kind)
    v = np.ascontiguousarray(values, dtype=np.int32)
    out = np.zeros(_num_opens(k), np.int32)
    st = _load().orc_tree_scan_i32(direction, _ptr(k), k.size, _ptr(v), _ptr(out))
    return st, out


def tree_scan_box(monoid, direction, kind, values):
    """Box intersection (monoid 0) or union (monoid 1) over the tree."""
    k = _kinds(kind)
    v = np.ascontiguousarray(values, dtype=np.float32).reshape(-1, 4)
    out = np.zeros((_num_opens(k), 4), np.float32)
    st = _load().orc_tree_scan_box(monoid, direction, _ptr(k), k.size, _ptr(v),
                                   _ptr(out))
    return st, out


def affine_forward(kind, local):
    """world_r = world_parent * L_r (fp64), local of shape (J, 3, 4)."""
    k = _kinds(kind)
    L = np.ascontiguousarray(local, dtype=np.float64).reshape(-1, 12)
    world = np.zeros_like(L)
    st = _load().orc_affine_forward(_ptr(k), k.size, _ptr(L), _ptr(world))
    return st, world.reshape(-1, 3, 4)


def affine_up(kind, values):
    """Stream-order product of each joint's subtree transforms (fp64)."""
    k = _kinds(kind)
    v = np.ascontiguousarray(values, dtype=np.float64).reshape(-1, 12)
    out = np.zeros_like(v)
    st = _load().orc_affine_up(_ptr(k), k.size, _ptr(v), _ptr(out))
    return st, out.reshape(-1, 3, 4)


def rigid_scan(direction, kind, values):
    """Rigid transforms (qx, qy, qz, qw, tx, ty, tz, unused) per joint, fp64:
    DOWN (0) root-path products, UP (1) stream-order subtree products."""
    k = _kinds(kind)
    v = np.ascontiguousarray(values, dtype=np.float64).reshape(-1, 8)
    out = np.zeros_like(v)
    st = _load().orc_rigid_scan(int(direction), _ptr(k), k.size, _ptr(v), _ptr(out))
    return st, out


def tree_structure(kind):
    """(status, depth, parent, left_sibling) per joint (the r-th open): int32."""
    k = _kinds(kind)
    J = _num_opens(k)
    d = np.zeros(J, np.int32)
    p_ = np.zeros(J, np.int32)
    l = np.zeros(J, np.int32)
    st = _load().orc_tree_structure(_ptr(k), k.size, _ptr(d), _ptr(p_), _ptr(l))
    return st, d, p_, l


def affine_loss(kind, local, W):
    """sum_r <W_r, world_r> in fp64."""
    k = _kinds(kind)
    L = np.ascontiguousarray(local, dtype=np.float64).reshape(-1, 12)
    Wm = np.ascontiguousarray(W, dtype=np.float64).reshape(-1, 12)
    out = ctypes.c_double()
    st = _load().orc_affine_loss(_ptr(k), k.size, _ptr(L), _ptr(Wm), L.shape[0],
                                 ctypes.byref(out))
    return st, out.value


def affine_backward(kind, local, grad_world):
    """d loss / d local for loss = sum <grad_world_r, world_r> (fp64)."""
    k = _kinds(kind)
    L = np.ascontiguousarray(local, dtype=np.float64).reshape(-1, 12)
    G = np.ascontiguousarray(grad_world, dtype=np.float64).reshape(-1, 12)
    out = np.zeros_like(L)
    st = _load().orc_affine_backward(_ptr(k), k.size, _ptr(L), _ptr(G), _ptr(out),
                                     L.shape[0])
    return st, out.reshape(-1, 3, 4)
