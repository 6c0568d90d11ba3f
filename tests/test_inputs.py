"""The seeded input generators produce the workloads as their recipe states
them: exact lengths, balanced streams, the stated kind frequencies, depth
limits and box size ranges, and determinism per seed."""
import numpy as np
import pytest

from paper_2205_11659_gb300 import inputs


def depth_profile(k):
    step = np.where((k == 1) | (k == 2), 1, np.where(k == 3, -1, 0))
    return np.cumsum(step)


def assert_balanced(k):
    d = depth_profile(k)
    assert d.size == 0 or (d.min() >= 0 and d[-1] == 0)


def box_wh(box):
    return box[:, 2] - box[:, 0], box[:, 3] - box[:, 1]


def test_random_walk_scene():
    n = 1 << 20
    k, box = inputs.random_walk_scene(n, 3)
    assert k.dtype == np.uint8 and k.size == n and box.shape == (n, 4) and box.dtype == np.float32
    assert_balanced(k)
    frac = np.bincount(k, minlength=4) / n
    assert abs(frac[1] + frac[2] - 0.2) < 0.01       # opens
    assert abs(frac[1] - frac[2]) < 0.01              # clip / blend 50/50
    assert abs(frac[3] - 0.2) < 0.01                  # closes (depth rarely 0)
    leaf, clip = k == 0, k == 1
    w, h = box_wh(box)
    assert w[leaf].min() >= 1 - 1e-3 and w[leaf].max() <= 256 + 1e-3
    assert h[clip].min() >= 64 - 1e-2 and h[clip].max() <= 2048 + 1e-2
    cx = (box[leaf | clip, 0] + box[leaf | clip, 2]) / 2
    assert cx.min() >= -1e-3 and cx.max() < 4096 + 1e-3
    assert not box[(k == 2) | (k == 3)].any()          # blend and close slots are zero
    # depth grows like sqrt(n)
    assert 100 < depth_profile(k).max() < 20 * np.sqrt(n)


def test_seeds():
    a = inputs.random_walk_scene(10_000, 5)
    b = inputs.random_walk_scene(10_000, 5)
    c = inputs.random_walk_scene(10_000, 6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


@pytest.mark.parametrize("n", [1, 2, 3, 17, 4096 * 3 + 5])
def test_random_walk_exact_small_lengths(n):
    k, _ = inputs.random_walk_scene(n, n)
    assert k.size == n
    assert_balanced(k)


def test_chain_scene():
    k, box = inputs.chain_scene(1000, 1)
    assert k.size == 2001
    assert (k[:1000] == 1).all() and k[1000] == 0 and (k[1001:] == 3).all()
    cx = (box[:1001, 0] + box[:1001, 2]) / 2
    assert np.allclose(cx, 2048.0)


def test_flat_scene():
    n = 300_001
    k, _ = inputs.flat_scene(n, 2)
    assert k.size == n
    assert_balanced(k)
    assert depth_profile(k).max() <= 4
    assert 0.85 < np.mean(k == 0) < 0.95


def test_batched_scenes():
    k, box, off = inputs.batched_scenes(64, 7)
    assert off[0] == 0 and off[-1] == k.size == box.shape[0] and np.all(np.diff(off) > 0)
    sizes = np.diff(off)
    assert sizes.min() >= 256 and sizes.max() <= 1 << 18
    for s in range(64):
        assert_balanced(k[off[s]:off[s + 1]])


@pytest.mark.parametrize("J", [1, 2, 64, 5000])
def test_skeleton(J):
    k, L, W = inputs.skeleton(J, 11)
    assert k.size == 2 * J
    assert np.count_nonzero(k == 1) == J and np.count_nonzero(k == 3) == J
    d = depth_profile(k)
    assert d.min() >= 0 and d[-1] == 0 and d.max() <= 64
    assert (d[:-1] > 0).all()                        # one tree: the root closes last
    assert L.shape == (J, 3, 4) and W.shape == (J, 3, 4)
    R = L[:, :, :3].astype(np.float64)
    assert np.allclose(R @ R.transpose(0, 2, 1), np.eye(3), atol=1e-5)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-5)


def test_batched_skeletons():
    k, L, W, eoff, joff = inputs.batched_skeletons(16, 3)
    assert eoff[-1] == k.size and joff[-1] == L.shape[0] == W.shape[0]
    assert np.array_equal(np.diff(eoff), 2 * np.diff(joff))
    j = np.diff(joff)
    assert j.min() >= 1024 and j.max() <= 1 << 16
    for s in range(16):
        assert_balanced(k[eoff[s]:eoff[s + 1]])
