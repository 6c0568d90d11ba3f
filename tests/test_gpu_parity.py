"""GPU parity of the C ABI against the CPU oracle.

Matching and bounding boxes are exact results (integer indices; fp32 min/max
is exact), so every comparison here is bit for bit on every element,
including at the full workload sizes the benchmark uses.
"""
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
    return torch.device("cuda", 0)


def run_bboxes(kind, box, want_indices=True):
    k = torch.from_numpy(np.ascontiguousarray(kind)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(box)).cuda()
    p, m, o = binding.bboxes(k, b, want_indices=want_indices)
    torch.cuda.synchronize()
    return (None if p is None else p.cpu().numpy(), None if m is None else m.cpu().numpy(),
            o.cpu().numpy())


def same_bits(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def assert_bboxes_equal(kind, box):
    st, op, om, ob = oracle.bboxes(kind, box)
    assert st == oracle.OK
    p, m, o = run_bboxes(kind, box)
    bad_p = np.nonzero(p != op)[0]
    bad_m = np.nonzero(m != om)[0]
    assert bad_p.size == 0, ("parent", bad_p[:8], p[bad_p[:8]], op[bad_p[:8]])
    assert bad_m.size == 0, ("match", bad_m[:8], m[bad_m[:8]], om[bad_m[:8]])
    bad_b = np.nonzero(np.any(o.view(np.uint32) != ob.view(np.uint32), axis=1))[0]
    assert bad_b.size == 0, ("box_out", bad_b[:8], kind[bad_b[:8]])


def test_hand_scene():
    k = np.array([1, 0, 2, 0, 1, 0, 3, 3, 3, 0], np.uint8)
    box = np.zeros((10, 4), np.float32)
    for i, b in {0: [0, 0, 100, 100], 1: [10, 10, 50, 50], 3: [80, 80, 150, 150],
                 4: [200, 200, 300, 300], 5: [210, 210, 220, 220], 9: [5, 5, 6, 6]}.items():
        box[i] = b
    assert_bboxes_equal(k, box)


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 255, 4095, 4096, 4097, 3 * TILE + 5,
                               50_000, 300_001, 1 << 20])
def test_random_walk_sizes(n):
    k, b = inputs.random_walk_scene(n, n)
    assert_bboxes_equal(k, b)


@pytest.mark.parametrize("seed", range(6))
def test_random_walk_seeds(seed):
    k, b = inputs.random_walk_scene(200_000 + 977 * seed, 1000 + seed)
    assert_bboxes_equal(k, b)


@pytest.mark.parametrize("n", [1, 4097, 123_457, 1 << 20])
def test_match_only(n):
    k, _ = inputs.random_walk_scene(n, 7 + n)
    st, op, om = oracle.match_parens(k)
    p, m = binding.match_parens(torch.from_numpy(k).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(p.cpu().numpy(), op) and np.array_equal(m.cpu().numpy(), om)


@pytest.mark.parametrize("depth", [1, 2047, 2048, 2049, 1 << 14])
def test_chain(depth):
    k, b = inputs.chain_scene(depth, depth)
    assert_bboxes_equal(k, b)


def test_flat():
    k, b = inputs.flat_scene(1 << 20, 3)
    assert_bboxes_equal(k, b)


def test_degenerate_shapes():
    rng = np.random.default_rng(0)
    cases = [
        np.zeros(10_000, np.uint8),                                   # all leaves
        np.array([1, 3] * 5000, np.uint8),                            # empty nodes
        np.concatenate([np.full(9000, 2, np.uint8), np.full(9000, 3, np.uint8)]),  # blend chain
        np.concatenate([np.ones(5000, np.uint8), np.zeros(3, np.uint8), np.full(5000, 3, np.uint8)]),
    ]
    # staircase: each tile leaves one open unmatched, then all close at once
    cases.append(np.concatenate([np.array([1] + [1, 0, 3] * 1365, np.uint8) for _ in range(20)]
                                + [np.full(20, 3, np.uint8)]))
    for k in cases:
        b = inputs.scene_boxes(k, int(rng.integers(1 << 30)))
        assert_bboxes_equal(k, b)


def test_indices_optional_and_host_path():
    k, b = inputs.random_walk_scene(70_000, 5)
    st, op, om, ob = oracle.bboxes(k, b)
    p, m, o = run_bboxes(k, b, want_indices=False)
    assert p is None and m is None and same_bits(o, ob)
    # host tensors in, host tensors out
    p, m, o = binding.bboxes(torch.from_numpy(k).pin_memory(), torch.from_numpy(b).pin_memory())
    assert np.array_equal(p.numpy(), op) and np.array_equal(m.numpy(), om)
    assert same_bits(o.numpy(), ob)


def test_deterministic_repeat():
    k, b = inputs.random_walk_scene(500_000, 11)
    r1 = run_bboxes(k, b)
    r2 = run_bboxes(k, b)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])
    assert same_bits(r1[2], r2[2])


def test_batched_small_and_empty_scenes():
    k, b, off = inputs.batched_scenes(64, 5, 0.0, 13.0)
    off = np.sort(np.concatenate([off, off[3:6], off[[0, 0, -1]]]))
    st, op, om, ob = oracle.bboxes_batched(k, b, off)
    assert st == oracle.OK
    p, m, o = binding.bboxes_batched(torch.from_numpy(k).cuda(), torch.from_numpy(b).cuda(),
                                     torch.from_numpy(off).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(p.cpu().numpy(), op) and np.array_equal(m.cpu().numpy(), om)
    assert same_bits(o.cpu().numpy(), ob)


def status_of(kind, box, offsets=None):
    k = torch.from_numpy(kind).cuda()
    b = torch.from_numpy(box).cuda()
    try:
        if offsets is None:
            binding.bboxes(k, b)
        else:
            binding.bboxes_batched(k, b, torch.from_numpy(offsets).cuda())
    except binding.TBError as e:
        return e.code
    return binding.TB_OK


def test_error_statuses():
    k, b = inputs.random_walk_scene(40_000, 2)
    bad = k.copy()
    bad[20_000] = 9
    assert status_of(bad, b) == binding.TB_ERR_BAD_KIND
    extra_open = k.copy()
    extra_open[np.nonzero(k == 0)[0][500]] = 1
    assert status_of(extra_open, b) == binding.TB_ERR_UNBALANCED
    lead_close = np.concatenate([np.array([3], np.uint8), k[:-1]])
    assert status_of(lead_close, b) == binding.TB_ERR_UNBALANCED
    # globally balanced, but scene 0 leaves an open that scene 1 closes
    kk = np.array([1, 0, 0, 3, 1, 0, 3, 0], np.uint8)
    off = np.array([0, 6, 8], np.int64)
    assert status_of(kk, inputs.scene_boxes(kk, 0), off) == binding.TB_ERR_UNBALANCED
    # more unmatched opens than a balanced stream can have: the slice slots
    # (sized for balanced streams) run out, which is reported, not overrun
    for kk in (np.ones(40_001, np.uint8), np.full(40_001, 2, np.uint8),
               np.concatenate([np.ones(30_000, np.uint8), np.full(10_000, 3, np.uint8)])):
        assert status_of(kk, inputs.scene_boxes(kk, 3)) == binding.TB_ERR_UNBALANCED
        try:
            binding.match_parens(torch.from_numpy(kk).cuda())
        except binding.TBError as e:
            assert e.code == binding.TB_ERR_UNBALANCED
        else:
            raise AssertionError("unbalanced stream accepted by the matching pass")
    assert status_of(np.full(40_001, 3, np.uint8), np.zeros((40_001, 4), np.float32)) \
        == binding.TB_ERR_UNBALANCED
    # a clean call after errors still works
    assert_bboxes_equal(k, b)


def test_workspace_and_alignment_errors():
    k = torch.zeros(100, dtype=torch.uint8, device="cuda")
    b = torch.zeros(100, 4, dtype=torch.float32, device="cuda")
    out = torch.empty(100, 4, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    need = binding.tb_workspace_size(binding.TB_OP_BBOXES, 100)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    assert binding.tb_bboxes(k, b, 100, None, None, out, ws, need - 1, st) == binding.TB_ERR_WORKSPACE
    kk = torch.zeros(120, dtype=torch.uint8, device="cuda")
    assert binding.tb_bboxes(kk[3:], b, 100, None, None, out, ws, need, st) == binding.TB_ERR_INVALID_ARG
    assert binding.tb_bboxes(k, b, 0, None, None, out, ws, need, st) == binding.TB_OK
    torch.cuda.synchronize()


# ---- full workload sizes, in the launch configuration the benchmark times

def test_full_random_walk_2_26():
    k, b = inputs.random_walk_scene(1 << 26, 0)
    assert_bboxes_equal(k, b)


def test_full_chain_2_24():
    k, b = inputs.chain_scene(1 << 23, 0)
    assert_bboxes_equal(k, b)


def test_full_flat_2_24():
    k, b = inputs.flat_scene(1 << 24, 0)
    assert_bboxes_equal(k, b)


def test_full_batched_4096_scenes():
    k, b, off = inputs.batched_scenes(4096, 0)
    st, op, om, ob = oracle.bboxes_batched(k, b, off)
    assert st == oracle.OK
    p, m, o = binding.bboxes_batched(torch.from_numpy(k).cuda(), torch.from_numpy(b).cuda(),
                                     torch.from_numpy(off).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(p.cpu().numpy(), op) and np.array_equal(m.cpu().numpy(), om)
    assert same_bits(o.cpu().numpy(), ob)


def test_host_pipeline_matches_oracle():
    """Scenes streamed from pinned host memory with overlapped copies give
    the oracle's results, including a repeated scene and a size change."""
    scenes = [inputs.random_walk_scene(n, 900 + n) for n in (70_001, 4096, 300_000, 70_001)]
    pipe = binding.HostPipeline(300_000)
    kinds = [torch.from_numpy(k).pin_memory() for k, _ in scenes]
    boxes = [torch.from_numpy(b).pin_memory() for _, b in scenes]
    outs = [(torch.empty(k.size, dtype=torch.int32).pin_memory(),
             torch.empty(k.size, dtype=torch.int32).pin_memory(),
             torch.empty(k.size, 4, dtype=torch.float32).pin_memory()) for k, _ in scenes]
    for _ in range(2):
        pipe.run(kinds, boxes, outs)
        for (k, b), (p, m, o) in zip(scenes, outs):
            st, op, om, ob = oracle.bboxes(k, b)
            assert st == oracle.OK
            assert np.array_equal(p.numpy(), op) and np.array_equal(m.numpy(), om)
            assert same_bits(o.numpy(), ob)


def test_host_pipeline_matching_only():
    """The matching-only pipeline gives the oracle's parent and match, and
    reports an unbalanced scene of the sequence."""
    scenes = [inputs.random_walk_scene(n, 950 + n)[0] for n in (50_001, 200_000, 4097)]
    pipe = binding.HostPipeline(200_000, boxes=False)
    kinds = [torch.from_numpy(k).pin_memory() for k in scenes]
    outs = [(torch.empty(k.size, dtype=torch.int32).pin_memory(),
             torch.empty(k.size, dtype=torch.int32).pin_memory()) for k in scenes]
    pipe.run(kinds, None, outs)
    for k, (p, m) in zip(scenes, outs):
        st, op, om = oracle.match_parens(k)
        assert st == oracle.OK
        assert np.array_equal(p.numpy(), op) and np.array_equal(m.numpy(), om)
    bad = scenes[1].copy()
    bad[np.nonzero(bad == 3)[0][0]] = 0  # one close fewer
    kinds[1] = torch.from_numpy(bad).pin_memory()
    with pytest.raises(binding.TBError):
        pipe.run(kinds, None, outs)
    with pytest.raises(ValueError):
        pipe.run(kinds, kinds, outs)


def test_withhold_hook_leaves_scene_passes_alone():
    """The scene passes have no cross-block wait (the tile depths come from
    a one-block scan): the look-back test hook does not affect them."""
    k, b = inputs.random_walk_scene(64 * TILE, 77)
    kd, bd = torch.from_numpy(k).cuda(), torch.from_numpy(b).cuda()
    assert binding.tb_debug_withhold_tile(5) == binding.TB_OK
    try:
        p, m, o = binding.bboxes(kd, bd)
    finally:
        assert binding.tb_debug_withhold_tile(-1) == binding.TB_OK
    st, op, om, ob = oracle.bboxes(k, b)
    assert np.array_equal(p.cpu().numpy(), op) and np.array_equal(m.cpu().numpy(), om)
    assert same_bits(o.cpu().numpy(), ob)


# A clip node A=(0,0,16,16) holding a clip node B=(16,0,32,16) whose raw
# intersection with A has zero width, two leaves under B (one live box, one of
# zero width), then under A a leaf touching A's right edge and a live leaf.
# Every leaf under B and the touching leaf are empty (x0 >= x1 is empty), so
# node B is empty and node A is the live leaf's box (2,2,6,6).
_ZERO_KINDS = np.array([1, 1, 0, 0, 3, 0, 0, 3], np.uint8)
_ZERO_BOXES = np.array([[0, 0, 16, 16], [16, 0, 32, 16], [4, 4, 20, 12], [8, 8, 8, 12],
                        [0, 0, 0, 0], [16, 2, 24, 10], [2, 2, 6, 6], [0, 0, 0, 0]], np.float32)


def _zero_area_scene():
    """Grid-box random walks with the pattern above placed across a tile
    boundary (elements 4094..4101), inside a chunk and across a chunk
    boundary."""
    starts = [TILE - 2, 2 * TILE + 16 * 7 + 5, 3 * TILE + 16 * 9 - 1]
    ks, bs, pos = [], [], 0
    for i, s in enumerate(starts + [None]):
        length = 3000 if s is None else s - pos
        k = inputs.random_walk_kinds(length, 40 + i)
        ks.append(k)
        bs.append(inputs.grid_boxes(k, 50 + i))
        pos += length
        if s is not None:
            ks.append(_ZERO_KINDS)
            bs.append(_ZERO_BOXES)
            pos += _ZERO_KINDS.size
    return np.concatenate(ks), np.concatenate(bs)


def _touching_leaves(kind, box):
    """Leaves whose raw clipped box has zero width or height exactly."""
    st, raw = oracle.clip_out(kind, box)
    assert st == oracle.OK
    leaf = kind == 0
    zero = (raw[:, 0] == raw[:, 2]) | (raw[:, 1] == raw[:, 3])
    return int(np.count_nonzero(leaf & zero))


@pytest.mark.parametrize("n", [0, 3 * TILE + 5, 50_000])
def test_zero_area_rule(n):
    """Empty is x0 >= x1 or y0 >= y1 (touching edges and zero-width leaves are
    empty), applied to leaves before any union; bit for bit vs the oracle."""
    if n == 0:
        k, b = _zero_area_scene()
        st, _, _, ob = oracle.bboxes(k, b)
        empty = np.array([np.inf, np.inf, -np.inf, -np.inf], np.float32)
        for s in (TILE - 2, 2 * TILE + 16 * 7 + 5, 3 * TILE + 16 * 9 - 1):
            assert all(same_bits(ob[s + j], empty) for j in (1, 2, 3, 4, 5))
            assert same_bits(ob[s], np.array([2, 2, 6, 6], np.float32))
    else:
        k = inputs.random_walk_kinds(n, 60 + n)
        b = inputs.grid_boxes(k, 61 + n)
    assert _touching_leaves(k, b) > 0   # the case separates >= from >
    assert_bboxes_equal(k, b)


@pytest.mark.parametrize("n", [3 * TILE + 5, 200_003, 1 << 22])
def test_wide_scene_unions(n):
    """Small leaves spread over a wide area under clips that cover it all: a
    node's union depends on every descendant (random-walk scenes on the 4096
    square saturate to nearly the whole square), so a union that drops or
    adds a part shows."""
    k = inputs.random_walk_kinds(n, 900 + n)
    b = inputs.scene_boxes(k, 901 + n, center_hi=1e6, leaf_wh=(1.0, 4.0), clip_wh=(1.5e6, 3e6))
    assert_bboxes_equal(k, b)


def test_graph_capture_replays_the_pass():
    """The whole pass (its cooperative launch included) captured in a CUDA
    graph and replayed gives the plain call's outputs, on new inputs too."""
    k1, b1 = inputs.random_walk_scene(5 * TILE + 3, 41)
    k2, b2 = inputs.random_walk_scene(5 * TILE + 3, 42)
    kd = torch.from_numpy(k1).cuda()
    bd = torch.from_numpy(b1).cuda()
    n = k1.size
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    match = torch.empty(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, 4, dtype=torch.float32, device="cuda")
    nb = binding.tb_workspace_size(binding.TB_OP_BBOXES, n)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        assert binding.tb_bboxes(kd, bd, n, parent, match, out, ws, nb, st, s) == binding.TB_OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rc = binding.tb_bboxes(kd, bd, n, parent, match, out, ws, nb, st, None)
    assert rc == binding.TB_OK
    for k, b in ((k1, b1), (k2, b2)):
        kd.copy_(torch.from_numpy(k))
        bd.copy_(torch.from_numpy(b))
        g.replay()
        torch.cuda.synchronize()
        assert int(st.item()) == binding.TB_OK
        s_, op, om, ob = oracle.bboxes(k, b)
        assert np.array_equal(parent.cpu().numpy(), op) and np.array_equal(match.cpu().numpy(), om)
        assert same_bits(out.cpu().numpy(), ob)
