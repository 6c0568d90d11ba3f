"""Single-scene sharding over R ranks (gloo, CPU processes): each rank holds a
contiguous range of one scene, the ranks exchange their range summaries and
then their partial unions (two all-gathers), and every rank resolves its own
elements.  The per-range steps are the CPU restatement in shard_cpu.py; the
assembled parent, match and box outputs must equal the oracle's bit for bit
on the whole scene, whatever the split (deep nesting across ranks, ranges
of one element, empty ranges)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene(name):
    import sys
    sys.path.insert(0, ROOT)
    from paper_2205_11659_gb300 import inputs
    if name == "walk":
        return inputs.random_walk_scene(40_000, 11)
    if name == "chain":
        return inputs.chain_scene(3000, 12)
    if name == "wide":            # small leaves over a wide area: unions do not saturate
        k = inputs.random_walk_kinds(30_000, 15)
        return k, inputs.scene_boxes(k, 16, center_hi=1e6, leaf_wh=(1.0, 4.0),
                                     clip_wh=(1.5e6, 3e6))
    if name == "grid":
        k = inputs.random_walk_kinds(9000, 13)
        return k, inputs.grid_boxes(k, 14)
    if name == "unbalanced":
        k = np.array([1, 0, 1, 0, 3, 0, 0, 1, 3], np.uint8)
        return k, np.zeros((k.size, 4), np.float32)
    raise ValueError(name)


def _cuts(n, world, name):
    if name == "chain":           # splits inside the nesting, one range of a single element
        return [0, 1000, 1001, 4500, n][:world] + [n]
    rng = np.random.default_rng(world)
    inner = sorted(rng.choice(np.arange(1, n), world - 1, replace=False).tolist())
    if world == 4:
        inner[1] = inner[0]        # an empty range
    return [0] + inner + [n]


def _rank_main(rank, world, port, name, q):
    import sys
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import shard_cpu
    from paper_2205_11659_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        kind, box = _scene(name)
        cuts = _cuts(kind.size, world, name)
        s, e = cuts[rank], cuts[rank + 1]
        st, p, m, o = shard.run_rank(rank, world, kind[s:e], box[s:e], s, shard_cpu.summarize,
                                     shard_cpu.local_pass, shard.torch_all_gather())
        q.put((rank, st, p, m, o))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,name", [(2, "walk"), (4, "walk"), (2, "chain"), (4, "chain"),
                                        (4, "grid"), (4, "wide"), (2, "unbalanced")])
def test_sharded_scene_equals_oracle(world, name):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = mp.start_processes(_rank_main, args=(world, _free_port(), name, q), nprocs=world,
                               start_method="spawn", join=False)
    got = sorted([q.get(timeout=300) for _ in range(world)], key=lambda t: t[0])
    procs.join()
    kind, box = _scene(name)
    st, op, om, ob = oracle.bboxes(kind, box)
    if name == "unbalanced":
        assert st == oracle.UNBALANCED and all(g[1] == 2 for g in got)
        return
    assert st == oracle.OK and all(g[1] == 0 for g in got)
    p = np.concatenate([g[2] for g in got])
    m = np.concatenate([g[3] for g in got])
    o = np.concatenate([g[4] for g in got])
    assert np.array_equal(p, op)
    assert np.array_equal(m, om)
    assert np.array_equal(o.view(np.uint32), ob.view(np.uint32))
