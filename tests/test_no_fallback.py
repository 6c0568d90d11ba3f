"""The product path has no CPU fallback: without the built library, or
without a CUDA device, the binding raises instead of computing anything."""
import numpy as np
import pytest
import torch

from paper_2205_11659_gb300 import _build, binding, inputs


def test_missing_library_raises(tmp_path, monkeypatch):
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent" / "libtb.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        binding.lib()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
@pytest.mark.parametrize("call", ["match_parens", "bboxes", "open_positions", "tree_scan"])
def test_no_gpu_raises(call):
    k, box = inputs.random_walk_scene(1000, 1)
    kind = torch.from_numpy(k)
    with pytest.raises((RuntimeError, ValueError)):
        if call == "match_parens":
            binding.match_parens(kind)
        elif call == "bboxes":
            binding.bboxes(kind, torch.from_numpy(box))
        elif call == "open_positions":
            binding.open_positions(kind)
        else:
            J = int(np.count_nonzero((k == 1) | (k == 2)))
            binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_DOWN, kind,
                              torch.zeros(J, dtype=torch.int32))
