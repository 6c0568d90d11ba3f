"""The allocation-free entry point tb_bboxes_static_ws.

Some callers cannot allocate device memory while they run (a renderer's
per-frame path with a fixed memory budget, a plug-in whose host owns all
device memory); this entry point takes no workspace and uses the library's
own fixed scratch array instead.  Here it is called through the C ABI and
checked, bit for bit (the tolerance of every other box test), against the
ordinary workspace form tb_bboxes on the same inputs, and directly against the
CPU oracle, for two calls in a row: the second call runs on the scratch the
first one left behind.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_11659_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2205_11659_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def _run(fn, kind, box):
    n = kind.numel()
    parent = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    match = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    box_out = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    if fn == "static":
        rc = binding.tb_bboxes_static_ws(kind, box, n, parent, match, box_out, status)
    else:
        nb = binding.tb_workspace_size(binding.TB_OP_BBOXES, n)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
        rc = binding.tb_bboxes(kind, box, n, parent, match, box_out, ws, nb, status)
    assert rc == binding.TB_OK
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_OK
    return parent.cpu().numpy(), match.cpu().numpy(), box_out.cpu().numpy()


def test_static_scratch_matches_workspace_form_twice():
    scenes = [inputs.random_walk_scene(binding.TB_STATIC_WS_MAX_N, 1),  # at the limit, 32 tiles
              inputs.random_walk_scene(9_999, 2)]                     # ragged tail
    for kind_np, box_np in scenes:  # two calls in a row
        kind = torch.from_numpy(kind_np).cuda()
        box = torch.from_numpy(box_np).cuda()
        p1, m1, b1 = _run("static", kind, box)
        p2, m2, b2 = _run("workspace", kind, box)
        assert np.array_equal(p1, p2)
        assert np.array_equal(m1, m2)
        assert np.array_equal(b1.view(np.uint32), b2.view(np.uint32))
        st, op, om, ob = oracle.bboxes(kind_np, box_np)
        assert st == oracle.OK
        assert np.array_equal(p1, op) and np.array_equal(m1, om)
        assert np.array_equal(b1.view(np.uint32), ob.view(np.uint32))


def test_static_scratch_rejects_sizes_beyond_its_limit():
    k = torch.zeros(8, dtype=torch.uint8, device="cuda")
    b = torch.zeros(8, 4, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = binding.tb_bboxes_static_ws(k, b, binding.TB_STATIC_WS_MAX_N + 1, None, None, b, st)
    assert rc == binding.TB_ERR_WORKSPACE
    rc = binding.tb_bboxes_static_ws(k, b, -1, None, None, b, st)
    assert rc == binding.TB_ERR_INVALID_ARG
