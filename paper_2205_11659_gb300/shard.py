"""Single-scene sharding over R ranks: the exchange-and-resolve protocol.

One scene (a flattened tree of kinds and boxes) is split into R contiguous
ranges, one per rank.  Matching and the box passes only need, at each range
start, the part of the stack that the range reaches below its start, and
for the unions of pairs that cross ranges, each range's partial unions.  The
protocol therefore has two exchange steps, each an all-gather of per-range
summaries whose size is bounded by the range's unmatched elements (Sec. 3:
a range's bicyclic element (a, b) counts them):

1. ``summarize`` (per rank): Bic(range) = (a, b); the stream indices of the
   a unmatched closes and of the b unmatched opens (the range's stack slice,
   Sec. 7.1) with the running intersection of the slice's clip boxes
   (Sec. 9), relative to whatever clip is in force below the slice.
   All-gather.
2. ``resolve_contexts`` (every rank, the same fold): the ranges' slices are
   stacked in order (Sec. 4's stack monoid at range granularity): range r
   pops a_r entries and pushes its slice, whose absolute clips are its
   relative ones meet the clip of the entry below it.  The result is, for
   each range, the top a_r + 1 entries of the stack at its start (index and
   clip; -1 and the universe below the root), and every pair whose open and
   close lie in different ranges.
3. ``local_pass`` (per rank) with that context: parents, matches, leaf boxes
   and the unions of pairs inside the range, plus the partial unions of the
   cross pairs: for each unmatched open the union of the range's leaves
   after it, for each unmatched close the union before it, and the union of
   all the range's leaves.  All-gather.
4. ``finish_cross_pairs`` (every rank, for its own elements): the union of a
   cross pair is (open's range after the open) + (whole ranges between) +
   (close's range before the close), written at both ends (Sec. 6.2: the
   descendants are a contiguous slice); the open's match is its close.

The per-range steps (1 and 3) are passed in as callables: on a GPU they are
the tile kernels run over the range with the context injected at its start.
This module holds only the exchange and the host-side fold over the
summaries, whose size is the number of unmatched elements, not the range
length.
"""
from dataclasses import dataclass, field

import numpy as np

UNIVERSE = np.array([-np.inf, -np.inf, np.inf, np.inf], np.float32)
EMPTY = np.array([np.inf, np.inf, -np.inf, -np.inf], np.float32)

OK, UNBALANCED = 0, 2


def isect(a, b):
    """Intersection of boxes (x0, y0, x1, y1), row-wise (Sec. 6.1)."""
    return np.concatenate([np.maximum(a[..., :2], b[..., :2]), np.minimum(a[..., 2:], b[..., 2:])],
                          axis=-1).astype(np.float32)


def unite(a, b):
    """Union of boxes, row-wise (Sec. 6.2)."""
    return np.concatenate([np.minimum(a[..., :2], b[..., :2]), np.maximum(a[..., 2:], b[..., 2:])],
                          axis=-1).astype(np.float32)


@dataclass
class RangeSummary:
    """Step 1's result for one range."""
    close_pos: np.ndarray   # int64[a]: unmatched closes, stream order
    open_pos: np.ndarray    # int64[b]: unmatched opens, stream order (bottom of the slice first)
    rel_clip: np.ndarray    # float32[b, 4]: running clip intersection along the slice
    status: int = OK


@dataclass
class Context:
    """The top a + 1 entries of the stack at a range start, top first."""
    idx: np.ndarray         # int64[a + 1]; -1 below the root
    clip: np.ndarray        # float32[a + 1, 4]; the universe below the root


@dataclass
class CrossPairs:
    """Pairs whose open and close lie in different ranges."""
    open_rank: list = field(default_factory=list)
    open_slot: list = field(default_factory=list)    # k: the open is open_pos[k] of its range
    close_rank: list = field(default_factory=list)
    close_slot: list = field(default_factory=list)   # m: the close is close_pos[m] of its range


@dataclass
class RangePartials:
    """Step 3's partial unions for one range."""
    usuf: np.ndarray        # float32[b, 4]: union of the range's leaves after each unmatched open
    upre: np.ndarray        # float32[a, 4]: union of the range's leaves before each unmatched close
    total: np.ndarray       # float32[4]: union of all the range's leaves


def resolve_contexts(summaries):
    """Step 2: (status, contexts, cross pairs) from all ranges' summaries."""
    stack_idx, stack_clip, stack_rank, stack_slot = [], [], [], []
    contexts, pairs, status = [], CrossPairs(), OK
    for r, s in enumerate(summaries):
        if s.status != OK and status == OK:
            status = s.status
        a = len(s.close_pos)
        idx = np.full(a + 1, -1, np.int64)
        clip = np.tile(UNIVERSE, (a + 1, 1))
        top = len(stack_idx)
        for m in range(min(a + 1, top)):
            idx[m] = stack_idx[top - 1 - m]
            clip[m] = stack_clip[top - 1 - m]
        contexts.append(Context(idx, clip))
        for m in range(a):
            if not stack_idx:
                status = UNBALANCED if status == OK else status
                break
            stack_idx.pop()
            stack_clip.pop()
            pairs.open_rank.append(stack_rank.pop())
            pairs.open_slot.append(stack_slot.pop())
            pairs.close_rank.append(r)
            pairs.close_slot.append(m)
        below = stack_clip[-1] if stack_clip else UNIVERSE
        for k in range(len(s.open_pos)):
            stack_idx.append(int(s.open_pos[k]))
            stack_clip.append(isect(below, s.rel_clip[k]))
            stack_rank.append(r)
            stack_slot.append(k)
    if stack_idx and status == OK:
        status = UNBALANCED
    return status, contexts, pairs


def finish_cross_pairs(rank, summaries, partials, pairs, match, box_out, start):
    """Step 4 for the elements of `rank` (arrays indexed from `start`)."""
    totals = [p.total for p in partials]
    for ro, ko, rc, mc in zip(pairs.open_rank, pairs.open_slot, pairs.close_rank,
                              pairs.close_slot):
        if ro != rank and rc != rank:
            continue
        u = unite(partials[ro].usuf[ko], partials[rc].upre[mc])
        for q in range(ro + 1, rc):
            u = unite(u, totals[q])
        o = int(summaries[ro].open_pos[ko])
        c = int(summaries[rc].close_pos[mc])
        if ro == rank:
            match[o - start] = c
            box_out[o - start] = u
        if rc == rank:
            box_out[c - start] = u


def run_rank(rank, world, kind, box, start, summarize, local_pass, all_gather):
    """The whole protocol on one rank.

    kind, box: this rank's range (numpy), starting at stream index `start`.
    summarize(kind, box, start) -> RangeSummary; local_pass(kind, box, start,
    context) -> (parent, match, box_out, RangePartials); all_gather(obj) ->
    list of every rank's obj (e.g. torch.distributed.all_gather_object).
    Returns (status, parent, match, box_out) for the range, indices global."""
    summaries = all_gather(summarize(kind, box, start))
    status, contexts, pairs = resolve_contexts(summaries)
    if status != OK:
        return status, None, None, None
    parent, match, box_out, part = local_pass(kind, box, start, contexts[rank])
    partials = all_gather(part)
    finish_cross_pairs(rank, summaries, partials, pairs, match, box_out, start)
    return OK, parent, match, box_out


def torch_all_gather(group=None):
    """all_gather over torch.distributed (gloo or NCCL) for step objects."""
    import torch.distributed as dist

    def gather(obj):
        out = [None] * dist.get_world_size(group)
        dist.all_gather_object(out, obj, group=group)
        return out
    return gather
