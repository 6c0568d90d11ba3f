"""Seeded synthetic inputs: flattened scene trees and skeleton transforms.

This module only draws random inputs; it holds none of the method's
arithmetic (no matching, no clipping, no unions, no transform products), so
the CUDA path and the CPU oracle can both be fed from it.  Every generator
takes an integer seed and uses numpy's PCG64.

Element kinds: 0 = LEAF, 1 = OPEN_CLIP, 2 = OPEN_BLEND, 3 = CLOSE.  Boxes are
float32 (x0, y0, x1, y1); blend and close slots hold zeros.

Workloads (the paper's inputs are random push/pop sequences, Sec. 11):

* :func:`random_walk_scene` -- OPEN w.p. 0.2 (clip/blend 50/50), CLOSE w.p.
  0.2 when the depth is positive, else LEAF; closes are forced at the end so
  the stream has exactly ``n`` elements and ends at depth 0.
* :func:`chain_scene` -- ``d`` nested clip opens, one leaf, ``d`` closes.
* :func:`flat_scene` -- depth at most 4, about 90% leaves.
* :func:`batched_scenes` -- many random-walk scenes with log-uniform sizes.
* :func:`skeleton` / :func:`batched_skeletons` -- OPEN/CLOSE joint trees with
  depth at most 64 and random 3x4 affine local transforms.
"""
import math

import numpy as np

LEAF, OPEN_CLIP, OPEN_BLEND, CLOSE = 0, 1, 2, 3

_CHUNK = 1 << 22


def _rng(seed, *stream):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), *stream])))


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def random_walk_kinds(n, seed, p_open=0.2, p_close=0.2):
    """Kinds of a random-walk scene of exactly ``n`` elements ending at depth 0."""
    n = int(n)
    rng = _rng(seed, 1)
    kinds = np.empty(n, np.uint8)
    u_all = np.empty(n, np.float64)
    depth_before = np.empty(n, np.int64)
    carry_x, carry_m = 0, 0          # running walk value and running minimum
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        u = rng.random(e - s)
        v = rng.random(e - s)
        u_all[s:e] = u
        want_open = u < p_open
        want_close = (u >= p_open) & (u < p_open + p_close)
        step = want_open.astype(np.int64) - want_close.astype(np.int64)
        x = carry_x + np.cumsum(step)
        m = np.minimum(carry_m, np.minimum.accumulate(np.minimum(x, 0)))
        d_after = x - m               # walk reflected at depth 0
        d_before = np.empty_like(d_after)
        d_before[0] = carry_x - carry_m
        d_before[1:] = d_after[:-1]
        depth_before[s:e] = d_before
        k = np.zeros(e - s, np.uint8)
        k[want_open] = np.where(v[want_open] < 0.5, OPEN_CLIP, OPEN_BLEND)
        k[want_close & (d_before > 0)] = CLOSE
        kinds[s:e] = k
        carry_x, carry_m = int(x[-1]), int(m[-1])
    # exact-length rule: from the first position whose depth reaches the
    # remaining length minus one, opens are forbidden and closes are forced
    # once depth equals the remaining length.
    remaining = n - np.arange(n, dtype=np.int64)
    hit = np.nonzero(depth_before >= remaining - 1)[0]
    if hit.size:
        p0 = int(hit[0])
        d = int(depth_before[p0])
        tail_v = rng.random(n - p0)
        for p in range(p0, n):
            r = n - p
            u = u_all[p]
            if d >= r:
                kinds[p] = CLOSE
                d -= 1
            elif u < p_open:
                if d < r - 1:
                    kinds[p] = OPEN_CLIP if tail_v[p - p0] < 0.5 else OPEN_BLEND
                    d += 1
                else:
                    kinds[p] = LEAF
            elif u < p_open + p_close and d > 0:
                kinds[p] = CLOSE
                d -= 1
            else:
                kinds[p] = LEAF
    return kinds


def scene_boxes(kinds, seed, center_lo=0.0, center_hi=4096.0, leaf_wh=(1.0, 256.0),
                clip_wh=(64.0, 2048.0), center=None):
    """float32 boxes: centres U[lo,hi)^2, log-uniform w/h; zeros for blend/close."""
    n = kinds.size
    rng = _rng(seed, 2)
    out = np.zeros((n, 4), np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        k = kinds[s:e]
        m = e - s
        if center is None:
            cx = rng.uniform(center_lo, center_hi, m)
            cy = rng.uniform(center_lo, center_hi, m)
        else:
            cx = np.full(m, float(center[0]))
            cy = np.full(m, float(center[1]))
        lw = _log_uniform(rng, leaf_wh[0], leaf_wh[1], m)
        lh = _log_uniform(rng, leaf_wh[0], leaf_wh[1], m)
        cw = _log_uniform(rng, clip_wh[0], clip_wh[1], m)
        ch = _log_uniform(rng, clip_wh[0], clip_wh[1], m)
        is_leaf = k == LEAF
        is_clip = k == OPEN_CLIP
        w = np.where(is_leaf, lw, cw)
        h = np.where(is_leaf, lh, ch)
        blk = np.stack([cx - w / 2, cy - h / 2, cx + w / 2, cy + h / 2], axis=1)
        keep = (is_leaf | is_clip)[:, None]
        out[s:e] = np.where(keep, blk, 0.0).astype(np.float32)
    return out


def grid_boxes(kinds, seed, cells=6, cell=8.0):
    """float32 boxes on a coarse integer grid, for edge cases of the empty-box
    rule: corners at multiples of ``cell`` in [0, cells * cell], so leaves of
    zero width or height and clip edges that exactly touch a leaf's edge are
    common; zeros for blend and close slots."""
    rng = _rng(seed, 5)
    n = kinds.size
    a = rng.integers(0, cells + 1, (n, 2)) * cell
    w = rng.integers(0, 3, (n, 2)) * cell          # widths/heights 0, cell, 2 cell
    blk = np.concatenate([a, a + w], axis=1)
    keep = ((kinds == LEAF) | (kinds == OPEN_CLIP))[:, None]
    return np.where(keep, blk, 0.0).astype(np.float32)


def random_walk_scene(n, seed):
    """(kinds, boxes) of the random-walk workload."""
    k = random_walk_kinds(n, seed)
    return k, scene_boxes(k, seed)


def chain_scene(depth, seed):
    """A single chain: ``depth`` nested clip opens, one leaf at the bottom,
    ``depth`` closes (``2*depth + 1`` elements).

    Clip boxes and the leaf are centred at (2048, 2048) so the running
    intersection stays non-empty all the way down."""
    h = int(depth)
    assert h >= 1
    k = np.empty(2 * h + 1, np.uint8)
    k[:h] = OPEN_CLIP
    k[h] = LEAF
    k[h + 1:] = CLOSE
    return k, scene_boxes(k, seed, center=(2048.0, 2048.0))


def _clamped_walk_depths(steps, lo, hi, block=4096):
    """depth_before for depth_after = clip(depth_before + step, lo, hi), start lo.

    Each step is the map x -> clip(x + s, lo, hi) on the small state set
    lo..hi; maps are composed per block (vectorised over blocks), chained
    across blocks, then expanded per position."""
    n = steps.size
    nb = (n + block - 1) // block
    pad = np.zeros(nb * block, np.int64)
    pad[:n] = steps
    st = pad.reshape(nb, block)
    states = np.arange(lo, hi + 1, dtype=np.int64)
    table = np.tile(states, (nb, 1))
    for j in range(block):
        table = np.clip(table + st[:, j:j + 1], lo, hi)
    start = np.empty(nb, np.int64)
    d = lo
    for b in range(nb):
        start[b] = d
        d = int(table[b, d - lo])
    out = np.empty((nb, block), np.int64)
    cur = start.copy()
    for j in range(block):
        out[:, j] = cur
        cur = np.clip(cur + st[:, j], lo, hi)
    return out.reshape(-1)[:n]


def flat_scene(n, seed, max_depth=4, p=0.05):
    """OPEN w.p. p while depth < max_depth, CLOSE w.p. p while depth > 0, else
    LEAF; closes forced at the end."""
    n = int(n)
    rng = _rng(seed, 3)
    u = rng.random(n)
    v = rng.random(n)
    # reserve the last max_depth slots for forced closes
    body = n - max_depth
    step = np.zeros(body, np.int64)
    step[u[:body] < p] = 1
    step[(u[:body] >= p) & (u[:body] < 2 * p)] = -1
    d_before = _clamped_walk_depths(step, 0, max_depth)
    d_after = np.clip(d_before + step, 0, max_depth)
    k = np.zeros(n, np.uint8)
    opened = d_after > d_before
    closed = d_after < d_before
    k[:body][opened] = np.where(v[:body][opened] < 0.5, OPEN_CLIP, OPEN_BLEND)
    k[:body][closed] = CLOSE
    final = int(d_after[-1]) if body > 0 else 0
    k[body:body + final] = CLOSE
    k[body + final:] = LEAF
    return k, scene_boxes(k, seed)


def batched_scenes(num_scenes, seed, log2_lo=8.0, log2_hi=18.0):
    """Concatenated random-walk scenes with sizes round(2^U[log2_lo, log2_hi]).

    Returns (kinds, boxes, offsets) with offsets of length num_scenes+1."""
    rng = _rng(seed, 4)
    sizes = np.rint(2.0 ** rng.uniform(log2_lo, log2_hi, num_scenes)).astype(np.int64)
    offsets = np.zeros(num_scenes + 1, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    kinds = np.empty(total, np.uint8)
    boxes = np.empty((total, 4), np.float32)
    for s in range(num_scenes):
        b, e = int(offsets[s]), int(offsets[s + 1])
        sub = (int(seed) << 20) + s + 1
        kinds[b:e] = random_walk_kinds(e - b, sub)
        boxes[b:e] = scene_boxes(kinds[b:e], sub)
    return kinds, boxes, offsets


def skeleton_kinds(num_joints, seed, max_depth=64):
    """OPEN/CLOSE stream of one joint tree with ``num_joints`` opens.

    Start with an open; at depth 1 always open (one root); at max_depth
    always close; otherwise open or close with probability 1/2; after the
    last open, close everything."""
    J = int(num_joints)
    rng = _rng(seed, 5)
    if J == 1:
        return np.array([OPEN_CLIP, CLOSE], np.uint8)
    steps_needed = 2 * J + 2 * max_depth + 64
    u = rng.random(steps_needed)
    # state = depth before the step, 1..max_depth after the first open
    nb_block = 1024
    n = steps_needed
    nb = (n + nb_block - 1) // nb_block
    pad = np.ones(nb * nb_block)
    pad[:n] = u
    uu = pad.reshape(nb, nb_block)
    states = np.arange(1, max_depth + 1, dtype=np.int64)

    def step(d, draw):
        up = draw < 0.5
        nd = np.where(up, d + 1, d - 1)
        nd = np.where(d == 1, 2, nd)
        nd = np.where(d == max_depth, max_depth - 1, nd)
        return nd

    table = np.tile(states, (nb, 1))
    for j in range(nb_block):
        table = step(table, uu[:, j:j + 1])
    start = np.empty(nb, np.int64)
    d = 1
    for b in range(nb):
        start[b] = d
        d = int(table[b, d - 1])
    before = np.empty((nb, nb_block), np.int64)
    cur = start.copy()
    for j in range(nb_block):
        before[:, j] = cur
        cur = step(cur, uu[:, j])
    before = before.reshape(-1)[:n]
    after = step(before, u)
    is_open = after > before
    # the first element is the root open; opens after it are counted until J
    cum = np.cumsum(is_open)
    last = int(np.searchsorted(cum, J - 1))  # index of the (J-1)-th extra open
    body_open = is_open[:last + 1]
    depth_end = int(after[last])
    k = np.empty(1 + (last + 1) + depth_end, np.uint8)
    k[0] = OPEN_CLIP
    k[1:last + 2] = np.where(body_open, OPEN_CLIP, CLOSE)
    k[last + 2:] = CLOSE
    return k


def affine_locals(num_joints, seed, angle_sigma=0.3):
    """(J, 3, 4) float32 local transforms: rotation by N(0, angle_sigma) about
    a uniform random axis (Rodrigues, fp64), translation N(0, 1)^3."""
    rng = _rng(seed, 6)
    J = int(num_joints)
    axis = rng.normal(size=(J, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = rng.normal(0.0, angle_sigma, J)
    c, s = np.cos(ang), np.sin(ang)
    x, y, z = axis[:, 0], axis[:, 1], axis[:, 2]
    C = 1.0 - c
    R = np.empty((J, 3, 3))
    R[:, 0, 0] = c + x * x * C
    R[:, 0, 1] = x * y * C - z * s
    R[:, 0, 2] = x * z * C + y * s
    R[:, 1, 0] = y * x * C + z * s
    R[:, 1, 1] = c + y * y * C
    R[:, 1, 2] = y * z * C - x * s
    R[:, 2, 0] = z * x * C - y * s
    R[:, 2, 1] = z * y * C + x * s
    R[:, 2, 2] = c + z * z * C
    t = rng.normal(size=(J, 3))
    out = np.concatenate([R, t[:, :, None]], axis=2)
    return out.astype(np.float32)


def rigid_locals(num_joints, seed, angle_sigma=0.3):
    """(J, 8) float32 rigid transforms (qx, qy, qz, qw, tx, ty, tz, 0): a
    rotation by N(0, angle_sigma) about a uniform random axis as a unit
    quaternion (fp64, then rounded), translation N(0, 1)^3."""
    rng = _rng(seed, 8)
    J = int(num_joints)
    axis = rng.normal(size=(J, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    half = 0.5 * rng.normal(0.0, angle_sigma, J)
    out = np.zeros((J, 8))
    out[:, :3] = axis * np.sin(half)[:, None]
    out[:, 3] = np.cos(half)
    out[:, 4:7] = rng.normal(size=(J, 3))
    return out.astype(np.float32)


def grad_weights(num_joints, seed):
    """W_r ~ N(0,1)^{3x4}: the loss is sum_r <W_r, world_r>."""
    rng = _rng(seed, 7)
    return rng.normal(size=(int(num_joints), 3, 4)).astype(np.float32)


def skeleton(num_joints, seed, max_depth=64):
    """(kinds, local, W) for one skeleton of ``num_joints`` joints."""
    k = skeleton_kinds(num_joints, seed, max_depth)
    return k, affine_locals(num_joints, seed), grad_weights(num_joints, seed)


def batched_skeletons(num, seed, log2_lo=10.0, log2_hi=16.0, max_depth=64):
    """Concatenated skeletons with joint counts round(2^U[log2_lo, log2_hi]).

    Returns (kinds, local, W, elem_offsets, joint_offsets)."""
    rng = _rng(seed, 8)
    joints = np.rint(2.0 ** rng.uniform(log2_lo, log2_hi, num)).astype(np.int64)
    ks = []
    for s in range(num):
        ks.append(skeleton_kinds(int(joints[s]), (int(seed) << 20) + s + 1, max_depth))
    eoff = np.zeros(num + 1, np.int64)
    np.cumsum([k.size for k in ks], out=eoff[1:])
    joff = np.zeros(num + 1, np.int64)
    np.cumsum(joints, out=joff[1:])
    kinds = np.concatenate(ks)
    J = int(joff[-1])
    return kinds, affine_locals(J, seed), grad_weights(J, seed), eoff, joff
