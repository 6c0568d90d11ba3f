"""GPU parity of tb_bboxes_clip: the per-element running clip intersection of
the stack snapshot (Sec. 9), bit for bit against oracle.clip_out, with the
other outputs equal to tb_bboxes'.  Leaves and clip opens get their box meet
the clip in force, blends the clip in force, closes their open's value; the
raw intersection is written (zero-area and negative-area results included)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_11659_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

TILE = 4096


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2205_11659_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


def _check(kind, box, offsets=None):
    k = torch.from_numpy(np.ascontiguousarray(kind)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(box)).cuda()
    off = None if offsets is None else torch.from_numpy(np.asarray(offsets, np.int64)).cuda()
    p, m, o, c = binding.bboxes_clip(k, b, off)
    torch.cuda.synchronize()
    p, m, o, c = (t.cpu().numpy() for t in (p, m, o, c))
    if offsets is None:
        st, oc = oracle.clip_out(kind, box)
        assert st == oracle.OK
        st, op, om, ob = oracle.bboxes(kind, box)
    else:
        parts = [oracle.clip_out(kind[a:e], box[a:e])[1] for a, e in zip(offsets[:-1], offsets[1:])]
        oc = np.concatenate(parts) if parts else np.zeros((0, 4), np.float32)
        st, op, om, ob = oracle.bboxes_batched(kind, box, offsets)
    assert st == oracle.OK
    bad = np.nonzero(np.any(_bits(c) != _bits(oc), axis=1))[0]
    assert bad.size == 0, ("clip_out", bad[:8], kind[bad[:8]], c[bad[:2]], oc[bad[:2]])
    assert np.array_equal(p, op) and np.array_equal(m, om)
    assert np.array_equal(_bits(o), _bits(ob))


def test_hand_scene():
    k = np.array([1, 0, 2, 0, 1, 0, 3, 3, 3, 0], np.uint8)
    box = np.zeros((10, 4), np.float32)
    for i, b in {0: [0, 0, 100, 100], 1: [10, 10, 50, 50], 3: [80, 80, 150, 150],
                 4: [200, 200, 300, 300], 5: [210, 210, 220, 220], 9: [5, 5, 6, 6]}.items():
        box[i] = b
    _check(k, box)
    _, c = oracle.clip_out(k, box)
    assert np.array_equal(c[5], np.array([210, 210, 100, 100], np.float32))  # raw, not canonical


@pytest.mark.parametrize("n", [1, 17, 4095, 4097, 3 * TILE + 5, 300_001, 1 << 22])
def test_random_walk(n):
    _check(*inputs.random_walk_scene(n, 300 + n))


def test_wide_scene():
    k = inputs.random_walk_kinds(4 * TILE + 9, 79)
    _check(k, inputs.scene_boxes(k, 80, center_hi=1e6, leaf_wh=(1.0, 4.0), clip_wh=(1e5, 3e6)))


def test_zero_area_grid():
    k = inputs.random_walk_kinds(5 * TILE + 123, 77)
    _check(k, inputs.grid_boxes(k, 78))


@pytest.mark.parametrize("depth", [2049, 1 << 23])
def test_chain(depth):
    _check(*inputs.chain_scene(depth, depth))


def test_flat_and_degenerate():
    _check(*inputs.flat_scene(1 << 20, 4))
    rng = np.random.default_rng(1)
    for k in (np.zeros(10_000, np.uint8), np.array([1, 3] * 5000, np.uint8),
              np.concatenate([np.full(9000, 2, np.uint8), np.full(9000, 3, np.uint8)])):
        _check(k, inputs.scene_boxes(k, int(rng.integers(1 << 30))))


def test_batched():
    k, b, off = inputs.batched_scenes(64, 9, log2_lo=6, log2_hi=14)
    _check(k, b, off)


def test_argument_errors():
    k = torch.zeros(8, dtype=torch.uint8, device="cuda")
    b = torch.zeros(8, 4, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    nb = binding.tb_workspace_size(binding.TB_OP_BBOXES, 8)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    assert binding.tb_bboxes_clip(k, b, None, 0, 8, None, None, b, None, ws, nb, st) \
        == binding.TB_ERR_INVALID_ARG
    flat = torch.zeros(40, dtype=torch.float32, device="cuda")
    misaligned = flat[1:33]  # 4 bytes past a 16-byte boundary
    assert binding.tb_bboxes_clip(k, b, None, 0, 8, None, None, b, misaligned, ws, nb, st) \
        == binding.TB_ERR_INVALID_ARG
