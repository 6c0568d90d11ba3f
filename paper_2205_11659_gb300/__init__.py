"""GB300 (sm_103a) implementation of the data-parallel core of Levien,
"Fast GPU bounding boxes on tree-structured scenes" (arXiv 2205.11659).

``binding`` wraps the C ABI of ``include/tb.h`` (CUDA kernels in ``csrc/``,
built into ``_build/libtb.so`` by ``_build.build()``); ``inputs`` draws the
seeded synthetic scenes and skeletons.
"""
from .binding import (  # noqa: F401
    HostPipeline, TBError, TreePipeline, TreeTransform, affine_backward, bboxes, bboxes_batched,
    bboxes_clip, tb_bboxes_clip,
    match_parens, open_positions, tb_bboxes, tb_bboxes_batched, tb_match_parens, tb_open_positions,
    tb_set_phase_events, tb_tree_scan,
    tb_tree_scan_affine_backward, tb_tree_scan_affine_backward_reuse, tb_tree_structure, tb_version,
    tb_workspace_size, tree_scan, tree_structure,
)
