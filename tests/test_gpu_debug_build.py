"""The debug build (TB_DEBUG: every data-dependent index is checked before
use, a failed check reports TB_ERR_BOUNDS and skips the access) on the
workloads' shapes: no check may fire on valid input, and the results must
equal the oracle's as in the normal build.  The build goes to its own folder
and is swapped in for these tests only."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2205_11659_gb300 import _build, binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def debug_build():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    lib_path = _build.build(debug=True, out_dir=os.path.join(_build.OUT_DIR, "debug"))
    saved = _build.LIB
    binding._lib = None
    _build.LIB = lib_path
    yield lib_path
    binding._lib = None
    _build.LIB = saved


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same_bits(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def _scenes():
    yield "rw ragged", inputs.random_walk_scene(4096 * 9 + 1234, 60)
    yield "rw 2^22", inputs.random_walk_scene(1 << 22, 61)
    yield "chain", inputs.chain_scene(1 << 16, 62)
    yield "flat", inputs.flat_scene(1 << 18, 63)


@pytest.mark.parametrize("name", [n for n, _ in _scenes()])
def test_scene_passes(debug_build, name):
    kind, box = dict(_scenes())[name]
    st, op, om, ob = oracle.bboxes(kind, box)
    assert st == oracle.OK
    p, m, o = binding.bboxes(_dev(kind), _dev(box))  # raises on TB_ERR_BOUNDS
    assert np.array_equal(p.cpu().numpy(), op)
    assert np.array_equal(m.cpu().numpy(), om)
    assert same_bits(o.cpu().numpy(), ob)
    pm, mm = binding.match_parens(_dev(kind))
    assert np.array_equal(pm.cpu().numpy(), op) and np.array_equal(mm.cpu().numpy(), om)


def test_batched(debug_build):
    kind, box, off = inputs.batched_scenes(200, 64, 4.0, 14.0)
    st, op, om, ob = oracle.bboxes_batched(kind, box, off)
    assert st == oracle.OK
    p, m, o = binding.bboxes_batched(_dev(kind), _dev(box), _dev(off))
    assert np.array_equal(p.cpu().numpy(), op) and np.array_equal(m.cpu().numpy(), om)
    assert same_bits(o.cpu().numpy(), ob)


def test_unbalanced_still_reported_as_such(debug_build):
    kind, box = inputs.random_walk_scene(4096 * 6 + 5, 65)
    kind = kind.copy()
    kind[np.nonzero(kind == 3)[0][0]] = 0
    with pytest.raises(binding.TBError) as ei:
        binding.bboxes(_dev(kind), _dev(box))
    assert ei.value.code == binding.TB_ERR_UNBALANCED


def test_tree_scans(debug_build):
    k, L, W = inputs.skeleton(300_000, 66)
    J = L.shape[0]
    v = (np.arange(J, dtype=np.int64) % 11 - 5).astype(np.int32)
    kd = _dev(k)
    for d in (oracle.DOWN, oracle.UP):
        st, ref = oracle.tree_scan_i32(d, k, v)
        out = binding.tree_scan(binding.TB_MONOID_ADD_I32,
                                binding.TB_DOWN if d == oracle.DOWN else binding.TB_UP, kd, _dev(v))
        assert np.array_equal(out.cpu().numpy(), ref)
    local = _dev(L).requires_grad_(True)
    world = binding.TreeTransform.apply(kd, local, True, True)
    (world * _dev(W)).sum().backward()
    st, wref = oracle.affine_forward(k, L.astype(np.float64))
    st, gref = oracle.affine_backward(k, L.astype(np.float64), W.astype(np.float64))

    def rel(x, ref):
        d = np.abs(x.astype(np.float64) - ref).reshape(ref.shape[0], -1).max(1)
        return float((d / np.maximum(np.abs(ref).reshape(ref.shape[0], -1).max(1), 1e-30)).max())
    assert rel(world.detach().cpu().numpy(), wref) < 1e-4
    assert rel(local.grad.cpu().numpy(), gref) < 1e-4
