"""GPU parity of the main pass in the launch mode the tuned build does not
use: persistent blocks drawing tiles from a ticket counter, or one block per
tile.  The other build goes to its own folder and is swapped in for these
tests only; its outputs must equal the oracle's bit for bit."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2205_11659_gb300 import _build, binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def other_mode():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    persist = not _build.tuned_persistent()
    nt, kpt = _build.tuned_shape()
    lib_path = _build.build(shape=(nt, kpt), persistent=persist,
                            out_dir=os.path.join(_build.OUT_DIR, "mode_%d_%d_%d" % (nt, kpt, persist)))
    saved = _build.LIB
    binding._lib = None
    _build.LIB = lib_path
    yield persist
    binding._lib = None
    _build.LIB = saved


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same_bits(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("n,seed", [(1, 0), (4096 * 3 + 777, 1), (1 << 20, 2), ((1 << 22) + 5, 3)])
def test_bboxes_and_matching(other_mode, n, seed):
    kind, box = inputs.random_walk_scene(n, seed)
    st, op, om, ob = oracle.bboxes(kind, box)
    assert st == oracle.OK
    p, m, o = binding.bboxes(_dev(kind), _dev(box))
    assert np.array_equal(p.cpu().numpy(), op)
    assert np.array_equal(m.cpu().numpy(), om)
    assert same_bits(o.cpu().numpy(), ob)
    pm, mm = binding.match_parens(_dev(kind))
    assert np.array_equal(pm.cpu().numpy(), op)
    assert np.array_equal(mm.cpu().numpy(), om)


def test_batched(other_mode):
    kind, box, off = inputs.batched_scenes(300, 5, 4.0, 14.0)
    st, op, om, ob = oracle.bboxes_batched(kind, box, off)
    assert st == oracle.OK
    p, m, o = binding.bboxes_batched(_dev(kind), _dev(box), _dev(off))
    assert np.array_equal(p.cpu().numpy(), op)
    assert np.array_equal(m.cpu().numpy(), om)
    assert same_bits(o.cpu().numpy(), ob)


def test_unbalanced_reported(other_mode):
    kind, box = inputs.random_walk_scene(4096 * 5 + 3, 6)
    kind = kind.copy()
    kind[np.nonzero(kind == 3)[0][-1]] = 0  # one close fewer: ends above depth 0
    with pytest.raises(binding.TBError):
        binding.bboxes(_dev(kind), _dev(box))
