"""Pins for the CPU oracle against things other than itself.

* values printed in the paper (Sec. 3 and Sec. 7.1 worked examples),
* brute force on tiny inputs through an independent characterisation:
  the Bic-slice definition of the match (Sec. 3: parenmatch(s)[j] is the
  largest i with Bic(s[i..j]).b = 1), explicit ancestor enumeration for the
  clip (Sec. 6.1 definition) and explicit descendant ranges for the union
  (Sec. 6.2: descendants are the contiguous slice from open to close),
* invariants that hold at any size,
* closed forms for the transform monoid and finite differences for its
  adjoint.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2205_11659_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")
CH = {"(": 1, ")": 3, "L": 0, "C": 1, "B": 2, "X": 3}
EMPTY = np.array([np.inf, np.inf, -np.inf, -np.inf], np.float32)


def gold():
    with open(GOLD) as f:
        return json.load(f)


def kinds_of(s):
    return np.array([CH[c] for c in s], np.uint8)


# --- independent brute force --------------------------------------------

def bic_elem(k):
    if k in (1, 2):
        return (0, 1)
    if k == 3:
        return (1, 0)
    return (0, 0)


def bic_cat(x, y):
    m = min(x[1], y[0])
    return (x[0] + y[0] - m, x[1] + y[1] - m)


def brute_parent(kind):
    """Sec. 3: parenmatch(s)[j] = max i with Bic(s[i..j]).b == 1 (else -1)."""
    n = len(kind)
    par = np.full(n, -1, np.int64)
    for j in range(n):
        acc = (0, 0)
        for i in range(j - 1, -1, -1):
            acc = bic_cat(bic_elem(int(kind[i])), acc)
            if acc[1] == 1:
                par[j] = i
                break
    return par


def brute_match(kind):
    """Depth counting: an open's close is the first later element after which
    the depth returns to the open's depth-before."""
    k = np.asarray(kind)
    step = np.where((k == 1) | (k == 2), 1, np.where(k == 3, -1, 0))
    after = np.cumsum(step)
    before = after - step
    m = np.full(len(k), -1, np.int64)
    for o in np.nonzero(step == 1)[0]:
        rest = np.nonzero(after[o:] == before[o])[0]
        c = o + int(rest[0])
        m[o] = c
        m[c] = o
    return m


def balanced(kind):
    k = np.asarray(kind)
    step = np.where((k == 1) | (k == 2), 1, np.where(k == 3, -1, 0))
    d = np.cumsum(step)
    return d.size == 0 or (d.min() >= 0 and d[-1] == 0)


def isect(a, b):
    return np.concatenate([np.maximum(a[:2], b[:2]), np.minimum(a[2:], b[2:])])


def unite(a, b):
    return np.concatenate([np.minimum(a[:2], b[:2]), np.maximum(a[2:], b[2:])])


def canon(b):
    return EMPTY.copy() if (b[0] >= b[2] or b[1] >= b[3]) else b


def brute_bboxes(kind, box):
    par = brute_parent(kind)
    mat = brute_match(kind)
    n = len(kind)
    out = np.zeros((n, 4), np.float32)
    leaf_out = {}
    for i in range(n):
        if kind[i] == 0:
            acc = box[i].copy()
            a = par[i]
            while a >= 0:                      # explicit ancestor enumeration
                if kind[a] == 1:
                    acc = isect(acc, box[a])
                a = par[a]
            leaf_out[i] = canon(acc)
            out[i] = leaf_out[i]
    for o in range(n):
        if kind[o] in (1, 2):
            u = EMPTY.copy()
            for j in range(o + 1, mat[o]):      # contiguous descendant slice
                if kind[j] == 0:
                    u = unite(u, leaf_out[j])
            out[o] = u
            out[mat[o]] = u
    return par, mat, out


def same_bits(a, b):
    a = np.ascontiguousarray(a, np.float32)
    b = np.ascontiguousarray(b, np.float32)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


# --- printed values -------------------------------------------------------

def test_bic_printed_value():
    g = gold()["bic_example"]
    assert oracle.bic(kinds_of(g["string"])) == tuple(g["bic"])
    acc = (0, 0)
    for k in kinds_of(g["string"]):
        acc = bic_cat(acc, bic_elem(int(k)))
    assert acc == tuple(g["bic"])


def test_reverse_scan_and_slice_printed_values():
    g = gold()["reverse_scan_example"]
    k = kinds_of(g["string"])
    scan = [oracle.bic(k[i:]) for i in range(len(k))]
    assert scan == [tuple(x) for x in g["reverse_bic_scan"]]
    a, lst = oracle.stack_slice(k)
    assert a == g["unmatched_closes"]
    assert list(lst) == g["unmatched_opens"]
    # slot of each unmatched open from the reverse scan, as Sec. 7.1 states
    total_b = scan[0][1]
    for i in g["unmatched_opens"]:
        assert total_b - scan[i][1] == g["slot_of_open"][str(i)]
        assert list(lst).index(i) == g["slot_of_open"][str(i)]


def test_stack_slice_is_bic_with_indices():
    rng = np.random.default_rng(5)
    for _ in range(200):
        k = rng.choice([0, 1, 2, 3], size=int(rng.integers(0, 40))).astype(np.uint8)
        a, lst = oracle.stack_slice(k)
        assert (a, len(lst)) == oracle.bic(k)
        # every listed open is unmatched in the string: depth never returns
        step = np.where((k == 1) | (k == 2), 1, np.where(k == 3, -1, 0))
        after = np.cumsum(step)
        for o in lst:
            assert k[o] in (1, 2)
            assert after[o:].min() >= after[o]


def test_bic_and_stack_laws():
    """Sec. 3 and Sec. 4 laws on random strings: Bic is a monoid homomorphism
    (Bic(st) = Bic(s) . Bic(t), identity (0, 0)); the stack slice combines
    by dropping the first a(t) unmatched opens from the top of s's slice and
    appending t's (shifted); Bic(s[i..j]).b never grows as i moves right."""
    rng = np.random.default_rng(11)
    assert oracle.bic(np.zeros(0, np.uint8)) == (0, 0)
    for _ in range(300):
        s = rng.choice([0, 1, 2, 3], size=int(rng.integers(0, 30))).astype(np.uint8)
        t = rng.choice([0, 1, 2, 3], size=int(rng.integers(0, 30))).astype(np.uint8)
        st = np.concatenate([s, t])
        assert oracle.bic(st) == bic_cat(oracle.bic(s), oracle.bic(t))
        a_s, ls = oracle.stack_slice(s)
        a_t, lt = oracle.stack_slice(t)
        a_st, lst = oracle.stack_slice(st)
        keep = max(len(ls) - a_t, 0)
        assert a_st == a_s + max(a_t - len(ls), 0)
        assert list(lst) == list(ls[:keep]) + [int(i) + len(s) for i in lt]
        j = len(st)
        bs = [oracle.bic(st[i:j])[1] for i in range(j + 1)]
        assert all(x >= y for x, y in zip(bs, bs[1:]))


# --- matching -------------------------------------------------------------

def test_matching_exhaustive_small():
    count = 0
    for n in range(0, 10):
        for t in itertools.product((0, 1, 3), repeat=n):
            k = np.array(t, np.uint8)
            st, par, mat = oracle.match_parens(k)
            if not balanced(k):
                assert st == oracle.UNBALANCED
                continue
            count += 1
            assert st == oracle.OK
            assert np.array_equal(par, brute_parent(k))
            assert np.array_equal(mat, brute_match(k))
    assert count > 1000


@pytest.mark.parametrize("n,seed", [(64, 0), (257, 1), (1000, 2), (1500, 3)])
def test_matching_random_vs_brute(n, seed):
    k = inputs.random_walk_kinds(n, seed)
    st, par, mat = oracle.match_parens(k)
    assert st == oracle.OK
    assert np.array_equal(par, brute_parent(k))
    assert np.array_equal(mat, brute_match(k))


def test_unbalanced_and_bad_kind():
    assert oracle.match_parens(kinds_of(")("))[0] == oracle.UNBALANCED
    assert oracle.match_parens(kinds_of("(()"))[0] == oracle.UNBALANCED
    assert oracle.match_parens(np.array([0, 4, 0], np.uint8))[0] == oracle.BAD_KIND
    box = np.zeros((3, 4), np.float32)
    assert oracle.bboxes(kinds_of("())"), box)[0] == oracle.UNBALANCED
    assert oracle.bboxes(np.array([1, 7, 3], np.uint8), box)[0] == oracle.BAD_KIND
    assert oracle.match_parens(np.zeros(0, np.uint8))[0] == oracle.OK


def test_matching_invariants_large():
    k = inputs.random_walk_kinds(200_000, 7)
    st, par, mat = oracle.match_parens(k)
    assert st == oracle.OK
    n = k.size
    idx = np.arange(n)
    opens = (k == 1) | (k == 2)
    closes = k == 3
    leaves = k == 0
    step = np.where(opens, 1, np.where(closes, -1, 0))
    after = np.cumsum(step)
    before = after - step
    assert before.min() >= 0 and after[-1] == 0
    assert np.all(mat[leaves] == -1)
    assert np.all(mat[mat[~leaves]] == idx[~leaves])
    assert np.all(mat[opens] > idx[opens]) and np.all(mat[closes] < idx[closes])
    assert np.all(par < idx)
    has_p = par >= 0
    assert np.all(np.isin(k[par[has_p]], (1, 2)))
    # depth relation: every non-close sits one below its parent's depth-after
    nc = has_p & ~closes
    assert np.all(before[nc] == after[par[nc]])
    assert np.all(before[~has_p & ~closes] == 0)
    assert np.all(par[closes] == mat[closes])
    # proper nesting: for opens o1 < o2 < close(o1), close(o2) < close(o1)
    o = idx[opens]
    c = mat[opens]
    enclosing = par[o]
    ok = enclosing < 0
    ok |= (o < mat[np.maximum(enclosing, 0)]) & (c < mat[np.maximum(enclosing, 0)])
    assert np.all(ok)


# --- bounding boxes ---------------------------------------------------------

def test_hand_scene():
    g = gold()["hand_scene"]
    k = kinds_of(g["kinds"])
    box = np.zeros((k.size, 4), np.float32)
    for i, b in g["boxes"].items():
        box[int(i)] = b
    st, par, mat, out = oracle.bboxes(k, box)
    assert st == oracle.OK
    assert list(par) == g["parent"]
    assert list(mat) == g["match"]
    for i, b in g["box_out"].items():
        want = EMPTY if b == "EMPTY" else np.array(b, np.float32)
        assert same_bits(out[int(i)], want), (i, out[int(i)], want)
    p2, m2, o2 = brute_bboxes(k, box)
    assert np.array_equal(p2, par) and np.array_equal(m2, mat) and same_bits(o2, out)


# --- stream compaction of the opens (Sec. 1.1) -----------------------------

def test_open_positions_hand_scene():
    """The opens of the hand-worked scene are its C and B elements; they are
    also exactly the elements whose printed match lies after them."""
    g = gold()["hand_scene"]
    k = kinds_of(g["kinds"])
    st, pos, count = oracle.open_positions(k)
    assert st == oracle.OK and count == 3
    assert list(pos) == [0, 2, 4]
    assert list(pos) == [i for i, m in enumerate(g["match"]) if m > i]


def test_open_positions_closed_form_without_leaves():
    """Without leaves, an open at i with depth d before it has (i + d) / 2
    opens before it (opens - closes = d, opens + closes = i), so it is entry
    (i + d) / 2.  Every balanced string of length <= 12."""
    for n in range(0, 13, 2):
        for bits in itertools.product((1, 3), repeat=n):
            d, ok = 0, True
            for b in bits:
                d += 1 if b == 1 else -1
                ok &= d >= 0
            if not ok or d != 0:
                continue
            k = np.array(bits, np.uint8)
            st, pos, count = oracle.open_positions(k)
            assert st == oracle.OK and count == n // 2
            d = 0
            for i, b in enumerate(bits):
                if b == 1:
                    assert pos[(i + d) // 2] == i
                    d += 1
                else:
                    d -= 1


@pytest.mark.parametrize("seed", [0, 1])
def test_open_positions_index_the_joints(seed):
    """Entry r is joint r of the tree scans: the stream depth just after
    that element equals joint r's depth from an ADD DOWN scan of ones."""
    k, _ = inputs.random_walk_scene(20_000, 90 + seed)
    st, pos, count = oracle.open_positions(k)
    assert st == oracle.OK
    st, dep = oracle.tree_scan_i32(oracle.DOWN, k, np.ones(count, np.int32))
    assert st == oracle.OK
    stream_depth = np.cumsum(np.where((k == 1) | (k == 2), 1, np.where(k == 3, -1, 0)))
    assert np.array_equal(stream_depth[pos], dep)
    assert np.all(np.diff(pos) > 0)


def test_open_positions_cap_and_bad_kind():
    k, _ = inputs.random_walk_scene(5000, 95)
    st, full, count = oracle.open_positions(k)
    st2, part, count2 = oracle.open_positions(k, cap=17)
    assert st2 == oracle.OK and count2 == count and np.array_equal(part, full[:17])
    st3, _, _ = oracle.open_positions(np.array([1, 4, 3], np.uint8))
    assert st3 == oracle.BAD_KIND


# --- the running clip per element (Sec. 9 stack snapshot) -------------------

UNIVERSE = np.array([-np.inf, -np.inf, np.inf, np.inf], np.float32)


def brute_clip_out(kind, box):
    """Own box (universe for a blend) intersected with the box of every clip
    ancestor, found by following brute-force parent links; a close takes its
    open's value (brute-force match)."""
    par = brute_parent(kind)
    mat = brute_match(kind)
    out = np.zeros((len(kind), 4), np.float32)
    for i in range(len(kind)):
        j = mat[i] if kind[i] == 3 else i
        acc = UNIVERSE.copy() if kind[j] == 2 else box[j].copy()
        a = par[j]
        while a >= 0:
            if kind[a] == 1:
                acc = isect(acc, box[a])
            a = par[a]
        out[i] = acc
    return out


def test_clip_out_hand_scene():
    """Hand-derived from the scene's definition: the blend passes the outer
    clip on, node 4's clip is its box cut by node 0's, leaf 5's chain
    intersection is (210,210,100,100) (empty, written raw), closes repeat
    their opens."""
    g = gold()["hand_scene"]
    k = kinds_of(g["kinds"])
    box = np.zeros((k.size, 4), np.float32)
    for i, b in g["boxes"].items():
        box[int(i)] = b
    st, c = oracle.clip_out(k, box)
    assert st == oracle.OK
    want = [(0, 0, 100, 100), (10, 10, 50, 50), (0, 0, 100, 100), (80, 80, 100, 100),
            (200, 200, 100, 100), (210, 210, 100, 100), (200, 200, 100, 100),
            (0, 0, 100, 100), (0, 0, 100, 100), (5, 5, 6, 6)]
    assert same_bits(c, np.array(want, np.float32))


@pytest.mark.parametrize("maker,n,seed", [("rw", 300, 0), ("rw", 1200, 1), ("flat", 800, 2),
                                          ("chain", 150, 3)])
def test_clip_out_vs_brute(maker, n, seed):
    if maker == "rw":
        k, box = inputs.random_walk_scene(n, seed)
    elif maker == "flat":
        k, box = inputs.flat_scene(n, seed)
    else:
        k, box = inputs.chain_scene(n, seed)
    st, c = oracle.clip_out(k, box)
    assert st == oracle.OK
    assert same_bits(c, brute_clip_out(k, box))


def test_clip_out_agrees_with_leaf_boxes():
    """A leaf's clip value, made canonical, is its output box of the
    bounding-box pass; at the root the clip is the element's own box."""
    k, box = inputs.random_walk_scene(50_000, 7)
    st, c = oracle.clip_out(k, box)
    st2, par, _, out = oracle.bboxes(k, box)
    assert st == st2 == oracle.OK
    leaves = np.nonzero(k == 0)[0]
    canon_c = c[leaves].copy()
    empty = (canon_c[:, 0] >= canon_c[:, 2]) | (canon_c[:, 1] >= canon_c[:, 3])
    canon_c[empty] = EMPTY
    assert same_bits(canon_c, out[leaves])
    roots = np.nonzero((par == -1) & ((k == 0) | (k == 1)))[0]
    assert same_bits(c[roots], box[roots])
    st3, _ = oracle.clip_out(np.array([1, 0], np.uint8), np.zeros((2, 4), np.float32))
    assert st3 == oracle.UNBALANCED


def test_zero_area_is_empty():
    # a leaf of zero width is empty; a unit-width one is kept
    k = np.array([0, 0, 1, 0, 3], np.uint8)
    box = np.array([[10, 10, 10, 20], [10, 10, 11, 20], [0, 0, 100, 100],
                    [50, 5, 50, 6], [0, 0, 0, 0]], np.float32)
    st, _, _, out = oracle.bboxes(k, box)
    assert st == oracle.OK
    assert same_bits(out[0], EMPTY)
    assert same_bits(out[1], box[1])
    assert same_bits(out[3], EMPTY)
    assert same_bits(out[2], EMPTY) and same_bits(out[4], EMPTY)
    # touching clip edge: the intersection has zero width, so it is empty
    k = np.array([1, 0, 3], np.uint8)
    box = np.array([[0, 0, 10, 10], [10, 0, 20, 10], [0, 0, 0, 0]], np.float32)
    _, _, _, out = oracle.bboxes(k, box)
    assert same_bits(out[1], EMPTY)


def test_bboxes_exhaustive_shapes():
    rng = np.random.default_rng(11)
    tried = 0
    for n in range(1, 9):
        for t in itertools.product((0, 1, 2, 3), repeat=n):
            k = np.array(t, np.uint8)
            if not balanced(k):
                continue
            if n > 6 and rng.random() > 0.2:
                continue
            c = rng.uniform(0, 64, (n, 2))
            wh = rng.uniform(1, 48, (n, 2))
            box = np.concatenate([c - wh / 2, c + wh / 2], 1).astype(np.float32)
            box[(k == 2) | (k == 3)] = 0
            st, par, mat, out = oracle.bboxes(k, box)
            assert st == oracle.OK
            p2, m2, o2 = brute_bboxes(k, box)
            assert np.array_equal(par, p2) and np.array_equal(mat, m2)
            assert same_bits(out, o2)
            tried += 1
    assert tried > 500


@pytest.mark.parametrize("maker,n,seed", [
    (inputs.random_walk_scene, 600, 0),
    (inputs.random_walk_scene, 1200, 3),
    (inputs.chain_scene, 150, 1),
    (inputs.flat_scene, 800, 2),
])
def test_bboxes_random_vs_brute(maker, n, seed):
    k, box = maker(n, seed)
    st, par, mat, out = oracle.bboxes(k, box)
    assert st == oracle.OK
    p2, m2, o2 = brute_bboxes(k, box)
    assert np.array_equal(par, p2) and np.array_equal(mat, m2)
    assert same_bits(out, o2)


def test_bbox_invariants_large():
    k, box = inputs.random_walk_scene(100_000, 9)
    st, par, mat, out = oracle.bboxes(k, box)
    assert st == oracle.OK
    n = k.size
    leaves = np.nonzero(k == 0)[0]
    # a non-empty leaf output lies inside its own box and every ancestor clip
    lo = out[leaves]
    nonempty = lo[:, 0] < lo[:, 2]
    L = leaves[nonempty]
    assert np.all(out[L, :2] >= box[L, :2]) and np.all(out[L, 2:] <= box[L, 2:])
    a = par[L].copy()
    while np.any(a >= 0):
        live = a >= 0
        ai = a[live]
        clip = k[ai] == 1
        li, ci = L[live][clip], ai[clip]
        assert np.all(out[li, :2] >= box[ci, :2]) and np.all(out[li, 2:] <= box[ci, 2:])
        a[live] = par[ai]
    # a node box is the union of its children's boxes (leaf children: their
    # clipped box; node children: their node box)
    acc = np.tile(EMPTY, (n, 1))
    child = np.nonzero((par >= 0) & (k != 3))[0]
    p = par[child]
    np.minimum.at(acc[:, 0], p, out[child, 0])
    np.minimum.at(acc[:, 1], p, out[child, 1])
    np.maximum.at(acc[:, 2], p, out[child, 2])
    np.maximum.at(acc[:, 3], p, out[child, 3])
    opens = np.nonzero((k == 1) | (k == 2))[0]
    assert same_bits(acc[opens], out[opens])
    assert same_bits(out[mat[opens]], out[opens])


def test_batched_oracle_is_per_scene():
    k, box, off = inputs.batched_scenes(12, 3, 4.0, 9.0)
    st, par, mat, out = oracle.bboxes_batched(k, box, off)
    assert st == oracle.OK
    for s in range(len(off) - 1):
        b, e = off[s], off[s + 1]
        st2, p2, m2, o2 = oracle.bboxes(k[b:e], box[b:e])
        assert st2 == oracle.OK
        assert np.array_equal(par[b:e], p2) and np.array_equal(mat[b:e], m2)
        assert same_bits(out[b:e], o2)


# --- tree scans over other monoids -----------------------------------------

def _opens_ranges(k):
    mat = brute_match(k)
    par = brute_parent(k)
    opens = np.nonzero((k == 1) | (k == 2))[0]
    rank = {int(o): r for r, o in enumerate(opens)}
    return opens, mat, par, rank


def test_tree_scan_i32_depth_and_size():
    k = inputs.random_walk_kinds(700, 4)
    opens, mat, par, rank = _opens_ranges(k)
    ones = np.ones(opens.size, np.int32)
    st, down = oracle.tree_scan_i32(oracle.DOWN, k, ones)
    assert st == oracle.OK
    step = np.where((k == 1) | (k == 2), 1, np.where(k == 3, -1, 0))
    after = np.cumsum(step)
    assert np.array_equal(down, after[opens])          # depth of each open
    st, up = oracle.tree_scan_i32(oracle.UP, k, ones)
    size = [int(np.count_nonzero(((k == 1) | (k == 2))[o:mat[o] + 1])) for o in opens]
    assert list(up) == size                             # opens in the subtree
    vals = np.random.default_rng(1).integers(-50, 50, opens.size).astype(np.int32)
    _, down = oracle.tree_scan_i32(oracle.DOWN, k, vals)
    _, up = oracle.tree_scan_i32(oracle.UP, k, vals)
    for o in opens:
        s, a = 0, int(o)
        while a >= 0:
            s += int(vals[rank[a]])
            a = int(par[a])
        assert down[rank[int(o)]] == s
        sub = [rank[int(j)] for j in opens if o <= j < mat[o]]
        assert up[rank[int(o)]] == int(vals[sub].sum())


def test_tree_scan_box_monoids():
    k = inputs.random_walk_kinds(400, 6)
    opens, mat, par, rank = _opens_ranges(k)
    rng = np.random.default_rng(2)
    c = rng.uniform(0, 100, (opens.size, 2))
    wh = rng.uniform(10, 200, (opens.size, 2))
    vals = np.concatenate([c - wh / 2, c + wh / 2], 1).astype(np.float32)
    _, down = oracle.tree_scan_box(oracle.ISECT, oracle.DOWN, k, vals)
    _, up = oracle.tree_scan_box(oracle.UNION, oracle.UP, k, vals)
    for o in opens:
        acc = vals[rank[int(o)]].copy()
        a = int(par[o])
        while a >= 0:
            acc = isect(acc, vals[rank[a]])
            a = int(par[a])
        assert same_bits(down[rank[int(o)]], acc)
        u = EMPTY.copy()
        for j in opens:
            if o <= j < mat[o]:
                u = unite(u, vals[rank[int(j)]])
        assert same_bits(up[rank[int(o)]], u)


# --- affine transform monoid -------------------------------------------------

def _hom(m):
    h = np.eye(4)
    h[:3, :] = m
    return h


def test_affine_forward_vs_ancestor_products():
    k, L, _ = inputs.skeleton(150, 3, max_depth=12)
    st, world = oracle.affine_forward(k, L)
    assert st == oracle.OK
    opens, mat, par, rank = _opens_ranges(k)
    for o in opens:
        chain = []
        a = int(o)
        while a >= 0:
            chain.append(rank[a])
            a = int(par[a])
        w = np.eye(4)
        for r in reversed(chain):               # root first: ancestor on the left
            w = w @ _hom(L[r].astype(np.float64))
        assert np.allclose(world[rank[int(o)]], w[:3], rtol=1e-12, atol=1e-12)


def test_affine_integer_translations_exact():
    k = inputs.skeleton_kinds(300, 8, max_depth=20)
    J = int(np.count_nonzero(k == 1))
    rng = np.random.default_rng(0)
    L = np.zeros((J, 3, 4))
    L[:, :, :3] = np.eye(3)
    L[:, :, 3] = rng.integers(-1000, 1000, (J, 3))
    st, world = oracle.affine_forward(k, L)
    opens, mat, par, rank = _opens_ranges(k)
    for o in opens:
        t = np.zeros(3)
        a = int(o)
        while a >= 0:
            t += L[rank[a], :, 3]
            a = int(par[a])
        assert np.array_equal(world[rank[int(o)], :, 3], t)
        assert np.array_equal(world[rank[int(o)], :, :3], np.eye(3))
    _, up = oracle.affine_up(k, L)
    for o in opens:
        sub = [rank[int(j)] for j in opens if o <= j < mat[o]]
        assert np.array_equal(up[rank[int(o)], :, 3], L[sub, :, 3].sum(0))


def test_affine_fixed_axis_angles_add():
    k = inputs.skeleton_kinds(200, 9, max_depth=30)
    J = int(np.count_nonzero(k == 1))
    th = np.random.default_rng(4).normal(0, 0.3, J)
    L = np.zeros((J, 3, 4))
    L[:, 0, 0] = np.cos(th)
    L[:, 0, 1] = -np.sin(th)
    L[:, 1, 0] = np.sin(th)
    L[:, 1, 1] = np.cos(th)
    L[:, 2, 2] = 1.0
    _, world = oracle.affine_forward(k, L)
    opens, mat, par, rank = _opens_ranges(k)
    for o in opens:
        s, a = 0.0, int(o)
        while a >= 0:
            s += th[rank[a]]
            a = int(par[a])
        w = world[rank[int(o)]]
        assert abs(w[0, 0] - np.cos(s)) < 1e-12 and abs(w[1, 0] - np.sin(s)) < 1e-12


def test_affine_backward_vs_finite_differences():
    k, L, W = inputs.skeleton(64, 1, max_depth=64)
    L = L.astype(np.float64)
    W = W.astype(np.float64)
    st, g = oracle.affine_backward(k, L, W)
    assert st == oracle.OK
    h = 1e-6
    fd = np.zeros_like(L)
    for idx in np.ndindex(*L.shape):
        Lp = L.copy()
        Lp[idx] += h
        Lm = L.copy()
        Lm[idx] -= h
        fd[idx] = (oracle.affine_loss(k, Lp, W)[1] - oracle.affine_loss(k, Lm, W)[1]) / (2 * h)
    err = np.abs(fd - g).max() / np.abs(g).max()
    assert err < 1e-7, err


def test_affine_up_stream_order_with_rotations():
    """UP folds a joint's own value first, then its descendants' in stream
    order (Sec. 6.2's contiguous slice; the order matters for a monoid that
    does not commute, Sec. 13).  With random rotations the 4x4 products do
    not commute, so a swapped composition fails here."""
    for seed, (k, L) in enumerate([inputs.skeleton(120, 5, max_depth=10)[:2],
                                   inputs.skeleton(90, 6, max_depth=40)[:2]]):
        L = L.astype(np.float64)
        st, up = oracle.affine_up(k, L)
        assert st == oracle.OK
        opens, mat, par, rank = _opens_ranges(k)
        swapped_differs = False
        for o in opens:
            sub = [rank[int(j)] for j in opens if o <= j < mat[o]]  # stream order, o first
            acc = np.eye(4)
            rev = np.eye(4)
            for r in sub:
                acc = acc @ _hom(L[r])
                rev = _hom(L[r]) @ rev
            assert np.allclose(up[rank[int(o)]], acc[:3], rtol=1e-12, atol=1e-12)
            if len(sub) > 1 and not np.allclose(acc[:3], rev[:3], rtol=1e-6, atol=1e-6):
                swapped_differs = True
        assert swapped_differs  # the pin separates the two orders on these inputs


def _quat_matrix(q):
    """Rotation matrix of unit quaternion (x, y, z, w): the textbook closed form."""
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _rigid_as_affine(v):
    out = np.zeros((v.shape[0], 3, 4))
    for r in range(v.shape[0]):
        out[r, :, :3] = _quat_matrix(v[r, :4])
        out[r, :, 3] = v[r, 4:7]
    return out


@pytest.mark.parametrize("direction", [0, 1])
def test_rigid_scan_matches_affine_forms(direction):
    """Rigid transforms compose like their 3x4 matrices (rotation matrix of
    the quaternion, translation): both scan directions agree with the affine
    oracle functions on the matrix forms (a different arithmetic path)."""
    for k in (inputs.skeleton_kinds(300, 21, max_depth=25), inputs.random_walk_kinds(2000, 22)):
        J = int(np.count_nonzero((k == 1) | (k == 2)))
        v = inputs.rigid_locals(J, 23).astype(np.float64)
        v[:, :4] /= np.linalg.norm(v[:, :4], axis=1, keepdims=True)
        st, out = oracle.rigid_scan(direction, k, v)
        assert st == oracle.OK
        aff = _rigid_as_affine(v)
        st, ref = (oracle.affine_forward(k, aff) if direction == 0 else oracle.affine_up(k, aff))
        assert st == oracle.OK
        assert np.allclose(_rigid_as_affine(out), ref, rtol=1e-11, atol=1e-11)
        assert np.allclose(np.linalg.norm(out[:, :4], axis=1), 1.0, atol=1e-12)


def test_rigid_scan_hamilton_rules_and_translation_sums():
    # a chain of three joints with quaternions i, j, k: root-path products
    # i, ij = k, ijk = -1 (Hamilton's rules)
    k = np.array([1, 1, 1, 3, 3, 3], np.uint8)
    v = np.zeros((3, 8))
    v[0, 0] = v[1, 1] = v[2, 2] = 1.0
    st, out = oracle.rigid_scan(0, k, v)
    assert st == oracle.OK
    assert np.allclose(out[:, :4], [[1, 0, 0, 0], [0, 0, 1, 0], [0, 0, 0, -1]])
    # identity rotations: translations add along the root path (DOWN) and
    # over the subtree (UP)
    k = inputs.skeleton_kinds(200, 24, max_depth=20)
    J = int(np.count_nonzero(k == 1))
    v = np.zeros((J, 8))
    v[:, 3] = 1.0
    v[:, 4:7] = np.random.default_rng(5).integers(-50, 50, (J, 3))
    opens, mat, par, rank = _opens_ranges(k)
    _, down = oracle.rigid_scan(0, k, v)
    _, up = oracle.rigid_scan(1, k, v)
    for o in opens:
        t, a = np.zeros(3), int(o)
        while a >= 0:
            t += v[rank[a], 4:7]
            a = int(par[a])
        assert np.array_equal(down[rank[int(o)], 4:7], t)
        sub = [rank[int(j)] for j in opens if o <= j < mat[o]]
        assert np.array_equal(up[rank[int(o)], 4:7], v[sub, 4:7].sum(0))


def _structure_brute(k):
    """Depth, parent and left sibling of every joint by brute force: the
    depth counts the opens before it minus the closes before it, plus one;
    the parent is the last earlier joint one level up (everything between a
    parent and its child is inside the parent); the left sibling is the last
    earlier joint with the same parent."""
    opens = [i for i in range(k.size) if k[i] in (1, 2)]
    delta = np.where((k == 1) | (k == 2), 1, np.where(k == 3, -1, 0))
    depth = [int(delta[:o].sum()) + 1 for o in opens]
    parent = []
    for r, d in enumerate(depth):
        p = -1
        for q in range(r - 1, -1, -1):
            if depth[q] == d - 1:
                p = q
                break
            if depth[q] < d - 1:
                break
        parent.append(p)
    left = []
    for r in range(len(opens)):
        q = -1
        for j in range(r - 1, -1, -1):
            if parent[j] == parent[r] and depth[j] == depth[r]:
                q = j
                break
        left.append(q)
    return np.array(depth), np.array(parent), np.array(left)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tree_structure_brute_force(seed):
    for k in (inputs.skeleton_kinds(150, seed, max_depth=6), inputs.random_walk_kinds(400, seed),
              np.concatenate([inputs.skeleton_kinds(40, seed + 10), inputs.skeleton_kinds(30, seed + 20)])):
        st, d, p, l = oracle.tree_structure(k)
        assert st == oracle.OK
        bd, bp, bl = _structure_brute(k)
        assert np.array_equal(d, bd) and np.array_equal(p, bp) and np.array_equal(l, bl)
        # the depth is also the ADD root-path fold of ones
        _, d2 = oracle.tree_scan_i32(0, k, np.ones(d.size, np.int32))
        assert np.array_equal(d, d2)


def test_tree_structure_closed_forms():
    m = 9
    # a chain: depth r + 1, parent r - 1, no siblings
    st, d, p, l = oracle.tree_structure(np.array([1] * m + [3] * m, np.uint8))
    assert st == oracle.OK
    assert np.array_equal(d, np.arange(1, m + 1)) and np.array_equal(p, np.arange(-1, m - 1))
    assert np.array_equal(l, np.full(m, -1))
    # m roots one after another: each root's left sibling is the one before
    st, d, p, l = oracle.tree_structure(np.array([2, 0, 3] * m, np.uint8))
    assert np.array_equal(d, np.ones(m)) and np.array_equal(p, np.full(m, -1))
    assert np.array_equal(l, np.arange(-1, m - 1))
    # a star: one root with m children
    st, d, p, l = oracle.tree_structure(np.array([1] + [2, 3] * m + [3], np.uint8))
    assert np.array_equal(p, np.array([-1] + [0] * m))
    assert np.array_equal(l, np.array([-1, -1] + list(range(1, m))))
    # errors
    assert oracle.tree_structure(np.array([1, 3, 3], np.uint8))[0] == oracle.UNBALANCED
    assert oracle.tree_structure(np.array([1, 5, 3], np.uint8))[0] == oracle.BAD_KIND
