"""GPU parity of tb_open_positions (stream compaction of the opens, Sec.
1.1) against the oracle, bit for bit: small streams that span several
4096-element tiles with a ragged tail, the degenerate shapes, the full
benchmark sizes, short output buffers and bad kind bytes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_11659_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)


def _compare(k, cap=None):
    st, want, count = oracle.open_positions(k, cap)
    assert st == oracle.OK
    pos, c = binding.open_positions(torch.from_numpy(k).cuda(), max_opens=cap)
    assert c == count
    assert np.array_equal(pos.cpu().numpy(), want)


def _streams():
    rng = np.random.default_rng(11)
    yield "rw ragged", inputs.random_walk_scene(4096 * 9 + 1234, 60)[0]
    yield "rw one tile minus one", inputs.random_walk_scene(4095, 61)[0]
    yield "rw 2^20", inputs.random_walk_scene(1 << 20, 62)[0]
    yield "skeleton", inputs.skeleton_kinds(70_001, 63)
    yield "chain", inputs.chain_scene(1 << 15, 64)[0]
    yield "flat", inputs.flat_scene(300_001, 65)[0]
    yield "single leaf", np.zeros(1, np.uint8)
    yield "one node", np.array([2, 3], np.uint8)
    yield "all leaves", np.zeros(50_000, np.uint8)
    yield "random bytes 0..3", rng.integers(0, 4, 123_457).astype(np.uint8)
    yield "all opens", rng.integers(1, 3, 40_000).astype(np.uint8)


STREAMS = dict(_streams())


@pytest.mark.parametrize("name", list(STREAMS))
def test_parity(name):
    _compare(STREAMS[name])


def test_empty_stream():
    pos, c = binding.open_positions(torch.empty(0, dtype=torch.uint8, device="cuda"))
    assert c == 0 and pos.numel() == 0


@pytest.mark.parametrize("cap", [0, 1, 4095, 4097, 9_000])
def test_short_output_buffer(cap):
    """Only the first cap entries are written (the guard words after them
    keep their values) and the count still covers every open."""
    k = inputs.random_walk_scene(100_003, 70)[0]
    st, want, count = oracle.open_positions(k)
    kd = torch.from_numpy(k).cuda()
    guard = 64
    pos = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    ws = binding.workspace(kd.device)
    nb = binding.tb_workspace_size(binding.TB_OP_OPEN_POSITIONS, k.size)
    rc = binding.tb_open_positions(kd, k.size, pos if cap > 0 else None, cap, cnt, ws.get(nb), nb,
                                   ws.status)
    assert rc == binding.TB_OK
    torch.cuda.synchronize()
    assert int(ws.status.item()) == binding.TB_OK
    assert int(cnt.item()) == count
    got = pos.cpu().numpy()
    assert np.array_equal(got[:min(cap, count)], want[:cap])
    assert np.all(got[min(cap, count):] == -7)


def test_bad_kind_reported():
    k = inputs.random_walk_scene(50_000, 71)[0].copy()
    k[40_000] = 7
    with pytest.raises(binding.TBError) as ei:
        binding.open_positions(torch.from_numpy(k).cuda())
    assert ei.value.code == binding.TB_ERR_BAD_KIND


def test_positions_index_the_tree_scan_joints():
    """Entry r is joint r of tb_tree_scan: the stream depth just after it
    is joint r's depth from the GPU ADD DOWN scan of ones."""
    k = inputs.skeleton_kinds(200_000, 72)
    kd = torch.from_numpy(k).cuda()
    pos, c = binding.open_positions(kd)
    dep = binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_DOWN, kd,
                            torch.ones(c, dtype=torch.int32, device="cuda"))
    stream_depth = np.cumsum(np.where((k == 1) | (k == 2), 1, np.where(k == 3, -1, 0)))
    assert np.array_equal(stream_depth[pos.cpu().numpy()], dep.cpu().numpy())


# ---- full workload sizes
def test_full_random_walk_2_26():
    _compare(inputs.random_walk_scene(1 << 26, 0)[0])


def test_full_chain_2_24():
    _compare(inputs.chain_scene(1 << 23, 1)[0])


def test_full_flat_2_24():
    _compare(inputs.flat_scene(1 << 24, 2)[0])
