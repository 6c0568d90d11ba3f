"""Python binding of the C ABI declared in ``include/tb.h``.

Argument marshalling only: torch tensors supply device memory and the
current CUDA stream, every step of the computation runs in the CUDA kernels
of ``_build/libtb.so``.  There is no CPU implementation behind these calls:
if the library is not built, or a tensor is not on a CUDA device, they raise.

The ``tb_*`` functions mirror the C entry points one to one.  ``match_parens``,
``bboxes``, ``bboxes_batched``, ``tree_scan`` and ``affine_backward`` are
conveniences that allocate outputs and workspace with torch, check the device
status word and raise on errors.  ``TreeTransform`` is the autograd function
of the affine root-path product (forward: DOWN scan, backward: the
hand-written adjoint).
"""
import ctypes
import os
import threading

import torch

from . import _build

TB_OK = 0
TB_ERR_INVALID_ARG = 1
TB_ERR_UNBALANCED = 2
TB_ERR_BAD_KIND = 3
TB_ERR_WORKSPACE = 4
TB_ERR_TIMEOUT = 5
TB_ERR_CUDA = 6
TB_ERR_BOUNDS = 7
STATUS_NAMES = {0: "TB_OK", 1: "TB_ERR_INVALID_ARG", 2: "TB_ERR_UNBALANCED",
                3: "TB_ERR_BAD_KIND", 4: "TB_ERR_WORKSPACE", 5: "TB_ERR_TIMEOUT",
                6: "TB_ERR_CUDA", 7: "TB_ERR_BOUNDS"}

TB_OP_MATCH_PARENS = 0
TB_OP_BBOXES = 1
TB_OP_BBOXES_BATCHED = 2
TB_OP_TREE_SCAN = 3
TB_OP_TREE_BACKWARD = 4
TB_OP_OPEN_POSITIONS = 5

TB_MONOID_BBOX_ISECT = 0
TB_MONOID_BBOX_UNION = 1
TB_MONOID_ADD_I32 = 2
TB_MONOID_AFFINE3X4_F32 = 3
TB_MONOID_RIGID_F32 = 4
TB_DOWN = 0
TB_UP = 1

LEAF, OPEN_CLIP, OPEN_BLEND, CLOSE = 0, 1, 2, 3


class TBError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s: %s" % (where, STATUS_NAMES.get(code, str(code))))
        self.code = code


_lock = threading.Lock()
_lib = None


def library_path():
    return _build.LIB


def lib():
    """The loaded libtb.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError("libtb.so is not built (%s); run "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
            L = ctypes.CDLL(path)
            p, i64, sz, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t, ctypes.c_int
            L.tb_workspace_size.argtypes = [i32, i64, i64]
            L.tb_workspace_size.restype = sz
            L.tb_match_parens.argtypes = [p, i64, p, p, p, sz, p, p]
            L.tb_bboxes.argtypes = [p, p, i64, p, p, p, p, sz, p, p]
            L.tb_bboxes_batched.argtypes = [p, p, p, i64, i64, p, p, p, p, sz, p, p]
            L.tb_set_phase_events.argtypes = [p, i32]
            L.tb_bboxes_static_ws.argtypes = [p, p, i64, p, p, p, p, p]
            L.tb_tree_scan.argtypes = [i32, i32, p, i64, i64, p, p, p, sz, p, p]
            L.tb_debug_withhold_tile.argtypes = [i32]
            L.tb_debug_withhold_tile.restype = i32
            L.tb_tree_scan_affine_backward.argtypes = [p, i64, i64, p, p, p, p, sz, p, p]
            L.tb_tree_scan_affine_backward_reuse.argtypes = [p, i64, i64, p, p, p, p, sz, p, p]
            L.tb_open_positions.argtypes = [p, i64, p, i64, p, p, sz, p, p]
            L.tb_bboxes_clip.argtypes = [p, p, p, i64, i64, p, p, p, p, p, sz, p, p]
            L.tb_tree_structure.argtypes = [p, i64, i64, p, p, p, p, sz, p, p]
            for f in (L.tb_match_parens, L.tb_bboxes, L.tb_bboxes_batched, L.tb_set_phase_events,
                      L.tb_bboxes_static_ws, L.tb_tree_scan, L.tb_tree_scan_affine_backward,
                      L.tb_tree_scan_affine_backward_reuse, L.tb_open_positions,
                      L.tb_bboxes_clip, L.tb_tree_structure):
                f.restype = i32
            L.tb_version.argtypes = []
            L.tb_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _check(code, where):
    if code != TB_OK:
        raise TBError(code, where)


# --------------------------------------------------------- raw entry points
def tb_version():
    return lib().tb_version().decode()


def tb_workspace_size(op, n, num_scenes=0):
    return int(lib().tb_workspace_size(int(op), int(n), int(num_scenes)))


def tb_match_parens(kind, n, parent, match, ws, ws_bytes, d_status, stream=None):
    return lib().tb_match_parens(_ptr(kind), int(n), _ptr(parent), _ptr(match), _ptr(ws),
                                 int(ws_bytes), _ptr(d_status), _stream(stream))


def tb_bboxes(kind, box, n, parent, match, box_out, ws, ws_bytes, d_status, stream=None):
    return lib().tb_bboxes(_ptr(kind), _ptr(box), int(n), _ptr(parent), _ptr(match),
                           _ptr(box_out), _ptr(ws), int(ws_bytes), _ptr(d_status),
                           _stream(stream))


def tb_open_positions(kind, n, pos, max_opens, d_count, ws, ws_bytes, d_status, stream=None):
    return lib().tb_open_positions(_ptr(kind), int(n), _ptr(pos), int(max_opens), _ptr(d_count),
                                   _ptr(ws), int(ws_bytes), _ptr(d_status), _stream(stream))


def tb_bboxes_batched(kind, box, offsets, num_scenes, n_total, parent, match, box_out, ws,
                      ws_bytes, d_status, stream=None):
    return lib().tb_bboxes_batched(_ptr(kind), _ptr(box), _ptr(offsets), int(num_scenes),
                                   int(n_total), _ptr(parent), _ptr(match), _ptr(box_out),
                                   _ptr(ws), int(ws_bytes), _ptr(d_status), _stream(stream))


def tb_bboxes_clip(kind, box, offsets, num_scenes, n, parent, match, box_out, clip_out, ws,
                   ws_bytes, d_status, stream=None):
    return lib().tb_bboxes_clip(_ptr(kind), _ptr(box), _ptr(offsets), int(num_scenes), int(n),
                                _ptr(parent), _ptr(match), _ptr(box_out), _ptr(clip_out),
                                _ptr(ws), int(ws_bytes), _ptr(d_status), _stream(stream))


def tb_bboxes_static_ws(kind, box, n, parent, match, box_out, d_status, stream=None):
    """tb_bboxes with the library's own fixed scratch: no workspace argument,
    nothing allocated (n <= TB_STATIC_WS_MAX_N)."""
    return lib().tb_bboxes_static_ws(_ptr(kind), _ptr(box), int(n), _ptr(parent), _ptr(match),
                                     _ptr(box_out), _ptr(d_status), _stream(stream))


TB_STATIC_WS_MAX_N = 1 << 17


def tb_tree_scan(monoid, direction, kind, n, num_joints, values, out, ws, ws_bytes, d_status,
                 stream=None):
    return lib().tb_tree_scan(int(monoid), int(direction), _ptr(kind), int(n), int(num_joints),
                              _ptr(values), _ptr(out), _ptr(ws), int(ws_bytes), _ptr(d_status),
                              _stream(stream))


def tb_tree_scan_affine_backward(kind, n, num_joints, local, grad_world, grad_local, ws,
                                 ws_bytes, d_status, stream=None):
    return lib().tb_tree_scan_affine_backward(_ptr(kind), int(n), int(num_joints), _ptr(local),
                                              _ptr(grad_world), _ptr(grad_local), _ptr(ws),
                                              int(ws_bytes), _ptr(d_status), _stream(stream))


def tb_tree_scan_affine_backward_reuse(kind, n, num_joints, local, grad_world, grad_local, ws,
                                       ws_bytes, d_status, stream=None):
    return lib().tb_tree_scan_affine_backward_reuse(
        _ptr(kind), int(n), int(num_joints), _ptr(local), _ptr(grad_world), _ptr(grad_local),
        _ptr(ws), int(ws_bytes), _ptr(d_status), _stream(stream))


def tb_tree_structure(kind, n, num_joints, depth_out, parent_out, left_sibling_out, ws, ws_bytes,
                      d_status, stream=None):
    return lib().tb_tree_structure(_ptr(kind), int(n), int(num_joints), _ptr(depth_out),
                                   _ptr(parent_out), _ptr(left_sibling_out), _ptr(ws), int(ws_bytes),
                                   _ptr(d_status), _stream(stream))


def tb_debug_withhold_tile(tile):
    """Test hook: element tile `tile` of the depth pass of the following tree
    scans on this thread never publishes its look-back word (-1 turns it
    off)."""
    return lib().tb_debug_withhold_tile(int(tile))


def tb_set_phase_events(events):
    """events: 1 to 16 torch.cuda.Event objects (recorded in launch order), or
    None to disable."""
    if events is None:
        return lib().tb_set_phase_events(None, 0)
    arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
    return lib().tb_set_phase_events(arr, len(events))


# ------------------------------------------------------------ conveniences
class Workspace:
    """Grow-only device scratch buffer (one per device), plus a status word."""

    def __init__(self, device):
        self.device = torch.device(device)
        self.buf = torch.empty(0, dtype=torch.uint8, device=self.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.device)

    def get(self, nbytes):
        if self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf

    def reserve(self, op, n, num_scenes=0):
        """Grow now, so that later calls of up to n elements allocate nothing
        (needed before capturing calls into a CUDA graph)."""
        self.get(tb_workspace_size(op, n, num_scenes))


_ws = {}


def workspace(device):
    d = torch.device(device)
    key = (d.type, d.index if d.index is not None else torch.cuda.current_device())
    if key not in _ws:
        _ws[key] = Workspace(torch.device("cuda", key[1]))
    return _ws[key]


def _on_device(t, dtype, name, device):
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if t.device.type != "cuda":
        t = t.to(device, non_blocking=True)
    return t.contiguous()


def check_status(ws, where):
    code = int(ws.status.item())
    _check(code, where)


def match_parens(kind, check=True):
    """(parent, match) int32 tensors for a uint8 kind tensor."""
    dev = kind.device if kind.is_cuda else torch.device("cuda", torch.cuda.current_device())
    k = _on_device(kind, torch.uint8, "kind", dev)
    n = k.numel()
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    match = torch.empty(n, dtype=torch.int32, device=dev)
    ws = workspace(dev)
    nb = tb_workspace_size(TB_OP_MATCH_PARENS, n)
    _check(tb_match_parens(k, n, parent, match, ws.get(nb), nb, ws.status), "tb_match_parens")
    if check:
        check_status(ws, "tb_match_parens")
    if not kind.is_cuda:
        return parent.cpu(), match.cpu()
    return parent, match


def open_positions(kind, max_opens=None, check=True):
    """Stream indices of the opens, in stream order (int32 tensor), and their
    count.  max_opens (default n: room for any byte stream) sizes the output.
    With check the call synchronises, raises on a data error and trims the
    result to the count (the count is then an int); otherwise it returns the
    untrimmed buffer and the device count."""
    dev = kind.device if kind.is_cuda else torch.device("cuda", torch.cuda.current_device())
    k = _on_device(kind, torch.uint8, "kind", dev)
    n = k.numel()
    cap = n if max_opens is None else int(max_opens)
    pos = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int32, device=dev)
    ws = workspace(dev)
    nb = tb_workspace_size(TB_OP_OPEN_POSITIONS, n)
    _check(tb_open_positions(k, n, pos, cap, count, ws.get(nb), nb, ws.status), "tb_open_positions")
    if not check:
        return pos, count
    check_status(ws, "tb_open_positions")
    c = int(count.item())
    pos = pos[:min(c, cap)]
    return (pos.cpu() if not kind.is_cuda else pos), c


def bboxes(kind, box, want_indices=True, check=True, out=None):
    """(parent, match, box_out) for a scene; box is float32 (n, 4).

    Device tensors in, device tensors out.  Host tensors are copied to the
    current device and the results copied back (pinned host memory makes the
    copies asynchronous)."""
    host = not kind.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device()) if host else kind.device
    k = _on_device(kind, torch.uint8, "kind", dev)
    b = _on_device(box, torch.float32, "box", dev).reshape(-1, 4)
    n = k.numel()
    if b.shape[0] != n:
        raise ValueError("box must have shape (n, 4)")
    if out is None:
        parent = torch.empty(n, dtype=torch.int32, device=dev) if want_indices else None
        match = torch.empty(n, dtype=torch.int32, device=dev) if want_indices else None
        box_out = torch.empty(n, 4, dtype=torch.float32, device=dev)
    else:
        parent, match, box_out = out
    ws = workspace(dev)
    nb = tb_workspace_size(TB_OP_BBOXES, n)
    _check(tb_bboxes(k, b, n, parent, match, box_out, ws.get(nb), nb, ws.status), "tb_bboxes")
    if check:
        check_status(ws, "tb_bboxes")
    if host:
        return tuple(None if t is None else t.cpu() for t in (parent, match, box_out))
    return parent, match, box_out


def bboxes_clip(kind, box, offsets=None, want_indices=True, check=True):
    """(parent, match, box_out, clip_out): bboxes (offsets None) or
    bboxes_batched, plus per element the running clip intersection (Sec. 9)."""
    host = not kind.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device()) if host else kind.device
    k = _on_device(kind, torch.uint8, "kind", dev)
    b = _on_device(box, torch.float32, "box", dev).reshape(-1, 4)
    off = None if offsets is None else _on_device(offsets, torch.int64, "offsets", dev)
    n = k.numel()
    if b.shape[0] != n:
        raise ValueError("box must have shape (n, 4)")
    S = 0 if off is None else off.numel() - 1
    parent = torch.empty(n, dtype=torch.int32, device=dev) if want_indices else None
    match = torch.empty(n, dtype=torch.int32, device=dev) if want_indices else None
    box_out = torch.empty(n, 4, dtype=torch.float32, device=dev)
    clip_out = torch.empty(n, 4, dtype=torch.float32, device=dev)
    ws = workspace(dev)
    nb = tb_workspace_size(TB_OP_BBOXES, n)
    _check(tb_bboxes_clip(k, b, off, S, n, parent, match, box_out, clip_out, ws.get(nb), nb,
                          ws.status), "tb_bboxes_clip")
    if check:
        check_status(ws, "tb_bboxes_clip")
    res = (parent, match, box_out, clip_out)
    if host:
        return tuple(None if t is None else t.cpu() for t in res)
    return res


def bboxes_batched(kind, box, offsets, want_indices=True, check=True):
    """Per-scene (parent, match, box_out) for scenes laid end to end;
    offsets is int64 of length num_scenes + 1; indices are scene-local."""
    host = not kind.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device()) if host else kind.device
    k = _on_device(kind, torch.uint8, "kind", dev)
    b = _on_device(box, torch.float32, "box", dev).reshape(-1, 4)
    off = _on_device(offsets, torch.int64, "offsets", dev)
    n = k.numel()
    S = off.numel() - 1
    parent = torch.empty(n, dtype=torch.int32, device=dev) if want_indices else None
    match = torch.empty(n, dtype=torch.int32, device=dev) if want_indices else None
    box_out = torch.empty(n, 4, dtype=torch.float32, device=dev)
    ws = workspace(dev)
    nb = tb_workspace_size(TB_OP_BBOXES_BATCHED, n, S)
    _check(tb_bboxes_batched(k, b, off, S, n, parent, match, box_out, ws.get(nb), nb, ws.status),
           "tb_bboxes_batched")
    if check:
        check_status(ws, "tb_bboxes_batched")
    if host:
        return tuple(None if t is None else t.cpu() for t in (parent, match, box_out))
    return parent, match, box_out


def _host_call(fn_name, host_inputs, out_h, extra):
    """Pinned host inputs in, pinned host outputs filled: the H2D copies, the
    C-ABI call and the D2H copies are enqueued on the current stream, which is
    then synchronised and the status word checked."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    d_in = [t.to(dev, non_blocking=True) for t in host_inputs]
    parent_h, match_h, box_h = out_h
    n = d_in[0].numel()
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    match = torch.empty(n, dtype=torch.int32, device=dev)
    box_out = torch.empty(n, 4, dtype=torch.float32, device=dev)
    ws = workspace(dev)
    if fn_name == "tb_bboxes":
        nb = tb_workspace_size(TB_OP_BBOXES, n)
        rc = tb_bboxes(d_in[0], d_in[1], n, parent, match, box_out, ws.get(nb), nb, ws.status, stream)
    else:
        S = d_in[2].numel() - 1
        nb = tb_workspace_size(TB_OP_BBOXES_BATCHED, n, S)
        rc = tb_bboxes_batched(d_in[0], d_in[1], d_in[2], S, n, parent, match, box_out,
                               ws.get(nb), nb, ws.status, stream)
    _check(rc, fn_name)
    parent_h.copy_(parent, non_blocking=True)
    match_h.copy_(match, non_blocking=True)
    box_h.copy_(box_out, non_blocking=True)
    stream.synchronize()
    check_status(ws, fn_name)
    return out_h


def bboxes_host(kind, box, out):
    """bboxes() for pinned host tensors: fills out = (parent, match, box_out),
    pinned host tensors of shapes (n,), (n,), (n, 4)."""
    return _host_call("tb_bboxes", [kind, box.reshape(-1, 4)], out, None)


def bboxes_batched_host(kind, box, offsets, out):
    """bboxes_batched() for pinned host tensors, filling ``out``."""
    return _host_call("tb_bboxes_batched", [kind, box.reshape(-1, 4), offsets], out, None)


# ------------------------------------------------------------- tree scans
_VALUE_SHAPE = {TB_MONOID_BBOX_ISECT: ((4,), torch.float32),
                TB_MONOID_BBOX_UNION: ((4,), torch.float32),
                TB_MONOID_ADD_I32: ((), torch.int32),
                TB_MONOID_AFFINE3X4_F32: ((3, 4), torch.float32),
                TB_MONOID_RIGID_F32: ((8,), torch.float32)}


def tree_scan(monoid, direction, kind, values, check=True):
    """tb_tree_scan on device tensors: values holds one monoid value per open
    of ``kind`` in stream order ((J, 4) float32 boxes, (J,) int32,
    (J, 3, 4) float32 affine transforms or (J, 8) float32 rigid transforms);
    returns a tensor of the same shape."""
    shape, dtype = _VALUE_SHAPE[monoid]
    dev = kind.device
    if not kind.is_cuda or not values.is_cuda:
        raise ValueError("tree_scan takes CUDA tensors")
    k = _on_device(kind, torch.uint8, "kind", dev)
    v = _on_device(values, dtype, "values", dev)
    J = v.shape[0] if v.dim() > 0 else 0
    if tuple(v.shape[1:]) != shape:
        raise ValueError("values must have shape (J,) + %s" % (shape,))
    n = k.numel()
    out = torch.empty_like(v)
    ws = workspace(dev)
    nb = tb_workspace_size(TB_OP_TREE_SCAN, n)
    _check(tb_tree_scan(monoid, direction, k, n, J, v, out, ws.get(nb), nb, ws.status),
           "tb_tree_scan")
    if check:
        check_status(ws, "tb_tree_scan")
    return out


def tree_structure(kind, check=True):
    """tb_tree_structure on a device kind tensor: (depth, parent,
    left_sibling), three (J,) int32 tensors over the J opens of ``kind``."""
    if not kind.is_cuda:
        raise ValueError("tree_structure takes a CUDA tensor")
    dev = kind.device
    k = _on_device(kind, torch.uint8, "kind", dev)
    n = k.numel()
    J = int(((k == OPEN_CLIP) | (k == OPEN_BLEND)).sum().item())
    outs = [torch.empty(J, dtype=torch.int32, device=dev) for _ in range(3)]
    ws = workspace(dev)
    nb = tb_workspace_size(TB_OP_TREE_SCAN, n)
    _check(tb_tree_structure(k, n, J, outs[0], outs[1], outs[2], ws.get(nb), nb, ws.status),
           "tb_tree_structure")
    if check:
        check_status(ws, "tb_tree_structure")
    return tuple(outs)


def affine_backward(kind, local, grad_world, check=True):
    """grad_local of sum_r <grad_world_r, world_r> for world = DOWN affine
    scan of ``local`` ((J, 3, 4) float32 device tensors)."""
    dev = kind.device
    if not kind.is_cuda or not local.is_cuda or not grad_world.is_cuda:
        raise ValueError("affine_backward takes CUDA tensors")
    k = _on_device(kind, torch.uint8, "kind", dev)
    L = _on_device(local, torch.float32, "local", dev)
    G = _on_device(grad_world, torch.float32, "grad_world", dev)
    if L.shape != G.shape or tuple(L.shape[1:]) != (3, 4):
        raise ValueError("local and grad_world must both have shape (J, 3, 4)")
    n, J = k.numel(), L.shape[0]
    out = torch.empty_like(L)
    ws = workspace(dev)
    nb = tb_workspace_size(TB_OP_TREE_BACKWARD, n)
    _check(tb_tree_scan_affine_backward(k, n, J, L, G, out, ws.get(nb), nb, ws.status),
           "tb_tree_scan_affine_backward")
    if check:
        check_status(ws, "tb_tree_scan_affine_backward")
    return out


class TreeTransform(torch.autograd.Function):
    """world = TreeTransform.apply(kind, local[, check[, keep_structure]]).

    local: (J, 3, 4) float32 local transforms, one per open of ``kind`` in
    stream order; world[r] = world[parent(r)] * local[r].  The backward pass
    recomputes world inside the library and runs the hand-written adjoint.
    By default nothing but kind and local is saved.  With
    keep_structure=True the forward runs in a workspace of its own that the
    node keeps until its backward, which then reads the joint structure from
    it (tb_tree_scan_affine_backward_reuse) instead of computing it again;
    the price is that workspace (tb_workspace_size(TB_OP_TREE_BACKWARD, n)
    bytes) per node.  With check=False no call reads the device status word,
    so forward and backward can be captured in a CUDA graph (reserve the
    shared workspace first)."""

    @staticmethod
    def forward(ctx, kind, local, check=True, keep_structure=False):
        ctx.check = check
        ctx.keep = bool(keep_structure)
        if not ctx.keep:
            ctx.save_for_backward(kind, local)
            return tree_scan(TB_MONOID_AFFINE3X4_F32, TB_DOWN, kind, local.detach(), check=check)
        dev = kind.device
        k = _on_device(kind, torch.uint8, "kind", dev)
        L = _on_device(local.detach(), torch.float32, "local", dev)
        if tuple(L.shape[1:]) != (3, 4):
            raise ValueError("local must have shape (J, 3, 4)")
        n, J = k.numel(), L.shape[0]
        nb = tb_workspace_size(TB_OP_TREE_BACKWARD, n)
        buf = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        world = torch.empty_like(L)
        _check(tb_tree_scan(TB_MONOID_AFFINE3X4_F32, TB_DOWN, k, n, J, L, world, buf, nb, status),
               "tb_tree_scan")
        if check:
            _check(int(status.item()), "tb_tree_scan")
        ctx.buf, ctx.nb, ctx.status = buf, nb, status
        ctx.save_for_backward(k, L)
        return world

    @staticmethod
    def backward(ctx, grad_world):
        kind, local = ctx.saved_tensors
        if not ctx.keep:
            g = affine_backward(kind, local, grad_world.contiguous(), check=ctx.check)
            return None, g, None, None
        G = _on_device(grad_world.contiguous(), torch.float32, "grad_world", kind.device)
        g = torch.empty_like(local)
        _check(tb_tree_scan_affine_backward_reuse(kind, kind.numel(), local.shape[0], local, G, g,
                                                  ctx.buf, ctx.nb, ctx.status),
               "tb_tree_scan_affine_backward_reuse")
        if ctx.check:
            _check(int(ctx.status.item()), "tb_tree_scan_affine_backward_reuse")
        ctx.buf = None
        return None, g, None, None


# ----------------------------------------------------- host pipelines
class HostPipeline:
    """tb_bboxes (or, with boxes=False, tb_match_parens) over a sequence of
    scenes held in pinned host memory, with the copies overlapped: while the
    pass runs on scene i, scene i+1 is copied in and the results of scene
    i-1 are copied out (three CUDA streams, two sets of device buffers, one
    workspace).

    run(kinds, boxes, outs): kinds[i] uint8 (n_i,), boxes[i] float32
    (n_i, 4) (None for a matching-only pipeline), outs[i] = (parent, match,
    box_out) pinned host tensors of shapes (n_i,), (n_i,), (n_i, 4), or
    (parent, match) for a matching-only pipeline.  An entry may repeat a
    tensor: the copies of consecutive scenes are ordered on their own stream.
    Returns after the last result is in host memory and raises TBError if any
    scene's status word is not TB_OK."""

    def __init__(self, n_max, device=None, boxes=True):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        dev = self.device
        self.n_max = int(n_max)
        self.boxes = bool(boxes)
        self.sets = []
        for _ in range(2):
            S = {
                "kind": torch.empty(self.n_max, dtype=torch.uint8, device=dev),
                "parent": torch.empty(self.n_max, dtype=torch.int32, device=dev),
                "match": torch.empty(self.n_max, dtype=torch.int32, device=dev),
                "status": torch.zeros(1, dtype=torch.int32, device=dev),
                "ev_in": torch.cuda.Event(), "ev_comp": torch.cuda.Event(),
                "ev_out": torch.cuda.Event(), "used": False,
            }
            if self.boxes:
                S["box"] = torch.empty(self.n_max, 4, dtype=torch.float32, device=dev)
                S["box_out"] = torch.empty(self.n_max, 4, dtype=torch.float32, device=dev)
            self.sets.append(S)
        self.op = TB_OP_BBOXES if self.boxes else TB_OP_MATCH_PARENS
        self.ws_bytes = tb_workspace_size(self.op, max(self.n_max, 1))
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        self.s_in = torch.cuda.Stream(dev)
        self.s_comp = torch.cuda.Stream(dev)
        self.s_out = torch.cuda.Stream(dev)

    def run(self, kinds, boxes, outs):
        if boxes is None:
            if self.boxes:
                raise ValueError("this pipeline computes boxes: pass the boxes of every scene")
            boxes = [None] * len(kinds)
        elif not self.boxes:
            raise ValueError("a matching-only pipeline takes boxes=None")
        if not (len(kinds) == len(boxes) == len(outs)):
            raise ValueError("kinds, boxes and outs must have the same length")
        name = "tb_bboxes" if self.boxes else "tb_match_parens"
        statuses = torch.zeros(len(kinds), dtype=torch.int32).pin_memory()
        for i, (k_h, b_h, o_h) in enumerate(zip(kinds, boxes, outs)):
            n = k_h.numel()
            if n > self.n_max:
                raise ValueError("scene %d has %d elements, more than n_max" % (i, n))
            S = self.sets[i % 2]
            with torch.cuda.stream(self.s_in):
                if S["used"]:
                    self.s_in.wait_event(S["ev_comp"])  # inputs no longer read
                S["kind"][:n].copy_(k_h, non_blocking=True)
                if self.boxes:
                    S["box"][:n].copy_(b_h.reshape(-1, 4), non_blocking=True)
                S["ev_in"].record(self.s_in)
            self.s_comp.wait_event(S["ev_in"])
            if S["used"]:
                self.s_comp.wait_event(S["ev_out"])  # outputs already copied out
            if self.boxes:
                rc = tb_bboxes(S["kind"], S["box"], n, S["parent"], S["match"], S["box_out"],
                               self.ws, self.ws_bytes, S["status"], self.s_comp)
            else:
                rc = tb_match_parens(S["kind"], n, S["parent"], S["match"], self.ws, self.ws_bytes,
                                     S["status"], self.s_comp)
            _check(rc, name)
            S["ev_comp"].record(self.s_comp)
            with torch.cuda.stream(self.s_out):
                self.s_out.wait_event(S["ev_comp"])
                o_h[0].copy_(S["parent"][:n], non_blocking=True)
                o_h[1].copy_(S["match"][:n], non_blocking=True)
                if self.boxes:
                    o_h[2].copy_(S["box_out"][:n], non_blocking=True)
                statuses[i:i + 1].copy_(S["status"], non_blocking=True)
                S["ev_out"].record(self.s_out)
            S["used"] = True
        self.s_out.synchronize()
        self.s_comp.synchronize()
        self.s_in.synchronize()
        for i in range(len(kinds)):
            _check(int(statuses[i]), "%s (scene %d)" % (name, i))
        return outs


class TreePipeline:
    """The affine tree scan and its adjoint over a sequence of skeleton jobs
    held in pinned host memory, with the copies overlapped: while job i runs
    (tb_tree_scan, then tb_tree_scan_affine_backward_reuse on the same
    workspace), job i+1 is copied in and the results of job i-1 are copied
    out (three CUDA streams, two sets of device buffers, one workspace).

    run(kinds, locals_, grad_worlds, outs): kinds[i] uint8 (n_i,),
    locals_[i] and grad_worlds[i] float32 (J_i, 3, 4), outs[i] = (world,
    grad_local) pinned host tensors of shape (J_i, 3, 4).  An entry may
    repeat a tensor: the copies of consecutive jobs are ordered on their own
    stream.  Returns after the last result is in host memory and raises
    TBError if any job's status word is not TB_OK."""

    def __init__(self, n_max, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        dev = self.device
        self.n_max = int(n_max)
        j_max = max(self.n_max // 2, 1)
        self.sets = []
        for _ in range(2):
            self.sets.append({
                "kind": torch.empty(max(self.n_max, 1), dtype=torch.uint8, device=dev),
                "local": torch.empty(j_max, 3, 4, dtype=torch.float32, device=dev),
                "grad_world": torch.empty(j_max, 3, 4, dtype=torch.float32, device=dev),
                "world": torch.empty(j_max, 3, 4, dtype=torch.float32, device=dev),
                "grad_local": torch.empty(j_max, 3, 4, dtype=torch.float32, device=dev),
                "status": torch.zeros(2, dtype=torch.int32, device=dev),  # forward, backward
                "ev_in": torch.cuda.Event(), "ev_comp": torch.cuda.Event(),
                "ev_out": torch.cuda.Event(), "used": False,
            })
        self.ws_bytes = tb_workspace_size(TB_OP_TREE_BACKWARD, max(self.n_max, 1))
        self.ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        self.s_in = torch.cuda.Stream(dev)
        self.s_comp = torch.cuda.Stream(dev)
        self.s_out = torch.cuda.Stream(dev)

    def run(self, kinds, locals_, grad_worlds, outs):
        if not (len(kinds) == len(locals_) == len(grad_worlds) == len(outs)):
            raise ValueError("kinds, locals_, grad_worlds and outs must have the same length")
        statuses = torch.zeros(len(kinds), 2, dtype=torch.int32).pin_memory()
        for i, (k_h, l_h, g_h, o_h) in enumerate(zip(kinds, locals_, grad_worlds, outs)):
            n, J = k_h.numel(), l_h.shape[0]
            if n > self.n_max:
                raise ValueError("job %d has %d elements, more than n_max" % (i, n))
            if tuple(l_h.shape) != (J, 3, 4) or tuple(g_h.shape) != (J, 3, 4):
                raise ValueError("job %d: local and grad_world must have shape (J, 3, 4)" % i)
            S = self.sets[i % 2]
            with torch.cuda.stream(self.s_in):
                if S["used"]:
                    self.s_in.wait_event(S["ev_comp"])  # inputs no longer read
                S["kind"][:n].copy_(k_h, non_blocking=True)
                S["local"][:J].copy_(l_h, non_blocking=True)
                S["grad_world"][:J].copy_(g_h, non_blocking=True)
                S["ev_in"].record(self.s_in)
            self.s_comp.wait_event(S["ev_in"])
            if S["used"]:
                self.s_comp.wait_event(S["ev_out"])  # outputs already copied out
            _check(tb_tree_scan(TB_MONOID_AFFINE3X4_F32, TB_DOWN, S["kind"], n, J, S["local"],
                                S["world"], self.ws, self.ws_bytes, S["status"][0:1], self.s_comp),
                   "tb_tree_scan")
            _check(tb_tree_scan_affine_backward_reuse(S["kind"], n, J, S["local"], S["grad_world"],
                                                      S["grad_local"], self.ws, self.ws_bytes,
                                                      S["status"][1:2], self.s_comp),
                   "tb_tree_scan_affine_backward_reuse")
            S["ev_comp"].record(self.s_comp)
            with torch.cuda.stream(self.s_out):
                self.s_out.wait_event(S["ev_comp"])
                o_h[0].copy_(S["world"][:J], non_blocking=True)
                o_h[1].copy_(S["grad_local"][:J], non_blocking=True)
                statuses[i].copy_(S["status"], non_blocking=True)
                S["ev_out"].record(self.s_out)
            S["used"] = True
        self.s_out.synchronize()
        self.s_comp.synchronize()
        self.s_in.synchronize()
        for i in range(len(kinds)):
            _check(int(statuses[i, 0]), "tree job %d (forward)" % i)
            _check(int(statuses[i, 1]), "tree job %d (backward)" % i)
        return outs
