"""CPU restatement of the two per-range steps of the sharding protocol
(paper_2205_11659_gb300/shard.py), standing in for the tile kernels run over
one range: a sequential stack walk over the range (Fig. 1), with the clip
intersection flowing down (Sec. 6.1) and the union flowing up (Sec. 6.2).
Test infrastructure: it shares nothing with the oracle, which checks the
assembled result."""
import numpy as np

from paper_2205_11659_gb300 import shard

LEAF, CLIP, BLEND, CLOSE = 0, 1, 2, 3


def _canon(b):
    return shard.EMPTY.copy() if (b[0] >= b[2] or b[1] >= b[3]) else b


def summarize(kind, box, start):
    """Bic(range) with the unmatched closes and the slice of unmatched opens,
    each open's clip relative to the clip in force below the slice."""
    stack, closes, status = [], [], shard.OK
    for i, k in enumerate(kind):
        if k > 3:
            status = 3
        elif k in (CLIP, BLEND):
            stack.append(i)
        elif k == CLOSE:
            if stack:
                stack.pop()
            else:
                closes.append(start + i)
    rel = np.tile(shard.UNIVERSE, (len(stack), 1))
    acc = shard.UNIVERSE
    for k_, i in enumerate(stack):
        if kind[i] == CLIP:
            acc = shard.isect(acc, box[i])
        rel[k_] = acc
    return shard.RangeSummary(np.array(closes, np.int64), np.array([start + i for i in stack], np.int64),
                              rel, status)


def local_pass(kind, box, start, ctx):
    """Parents, matches and boxes of the range given the stack entries below
    its start, and the partial unions of the pairs that cross its ends."""
    n = len(kind)
    parent = np.full(n, -1, np.int32)
    match = np.full(n, -1, np.int32)
    out = np.tile(shard.EMPTY, (n, 1))
    stack = []          # in-range opens: [stream index, clip, union so far]
    m = 0               # context entries popped so far
    total = shard.EMPTY.copy()
    upre = []
    for i in range(n):
        e, k = start + i, kind[i]
        if stack:
            top_idx, top_clip = stack[-1][0], stack[-1][1]
        else:
            top_idx, top_clip = int(ctx.idx[m]), ctx.clip[m]
        parent[i] = top_idx
        if k == LEAF:
            b = _canon(shard.isect(box[i], top_clip))
            out[i] = b
            total = shard.unite(total, b)
            if stack:
                stack[-1][2] = shard.unite(stack[-1][2], b)
        elif k in (CLIP, BLEND):
            clip = shard.isect(box[i], top_clip) if k == CLIP else top_clip
            stack.append([e, clip, shard.EMPTY.copy()])
        else:
            if stack:
                o, _, u = stack.pop()
                match[i], match[o - start] = o, e
                out[i] = u
                out[o - start] = u
                if stack:
                    stack[-1][2] = shard.unite(stack[-1][2], u)
            else:
                match[i] = top_idx
                upre.append(total.copy())
                m += 1
    usuf = np.tile(shard.EMPTY, (len(stack), 1))
    run = shard.EMPTY.copy()
    for k_ in range(len(stack) - 1, -1, -1):
        run = shard.unite(run, stack[k_][2])
        usuf[k_] = run
    upre = np.array(upre, np.float32).reshape(-1, 4)
    return parent, match, out, shard.RangePartials(usuf, upre, total)
