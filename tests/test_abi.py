"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every entry point declared in include/tb.h; workspace sizing;
argument errors are reported before any work is enqueued."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tb_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_11659_gb300 import _build, binding
    _build.build()
    return binding.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("tb_workspace_size", "tb_match_parens", "tb_bboxes", "tb_bboxes_batched",
              "tb_tree_scan", "tb_tree_scan_affine_backward",
              "tb_tree_scan_affine_backward_reuse", "tb_set_phase_events",
              "tb_debug_withhold_tile", "tb_version", "tb_open_positions"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_2205_11659_gb300 import binding
    assert "sm_103a" in binding.tb_version()


def test_workspace_size(lib):
    from paper_2205_11659_gb300 import binding as b
    assert b.tb_workspace_size(b.TB_OP_BBOXES, 0) == 0
    s1 = b.tb_workspace_size(b.TB_OP_BBOXES, 1)
    s2 = b.tb_workspace_size(b.TB_OP_BBOXES, 1 << 20)
    m2 = b.tb_workspace_size(b.TB_OP_MATCH_PARENS, 1 << 20)
    assert 0 < s1 < s2 and 0 < m2 < s2
    assert b.tb_workspace_size(b.TB_OP_BBOXES_BATCHED, 1 << 20, 7) == s2
    # workspace grows linearly in n
    assert b.tb_workspace_size(b.TB_OP_BBOXES, 1 << 22) < 4.5 * s2
    # slots for the unmatched elements a balanced stream can have (n / 2 per
    # side), not for every element of every tile: below the 41 bytes per
    # element of the pass's own inputs and outputs
    big = 1 << 26
    assert b.tb_workspace_size(b.TB_OP_BBOXES, big) < 33 * big
    assert b.tb_workspace_size(b.TB_OP_MATCH_PARENS, big) < 9 * big
    t2 = b.tb_workspace_size(b.TB_OP_TREE_SCAN, 1 << 20)
    g2 = b.tb_workspace_size(b.TB_OP_TREE_BACKWARD, 1 << 20)
    assert m2 < t2 < g2
    # the adjoint adds two transforms per joint (at most n / 2 joints)
    assert g2 - t2 >= 2 * 48 * (1 << 19)
    assert b.tb_workspace_size(b.TB_OP_TREE_SCAN, 0) == 0
    assert b.tb_workspace_size(99, 1 << 20) == 0
    # tile counts and tile offsets: two int32 per tile of 16384 elements
    o1 = b.tb_workspace_size(b.TB_OP_OPEN_POSITIONS, 1)
    o2 = b.tb_workspace_size(b.TB_OP_OPEN_POSITIONS, 1 << 26)
    assert 0 < o1 <= 512 and 2 * 4 * (1 << 12) <= o2 <= 2 * 4 * (1 << 12) + 512
    assert b.tb_workspace_size(b.TB_OP_OPEN_POSITIONS, 0) == 0


def test_argument_errors_before_any_launch(lib):
    # These are rejected by host checks before any CUDA call is made.
    from paper_2205_11659_gb300 import binding as b
    p = ctypes.c_void_p
    fake = 1 << 20          # never dereferenced: the checks fail first
    assert lib.tb_bboxes(p(fake), p(fake), -1, None, None, p(fake), p(fake), 1 << 30, p(fake), None) \
        == b.TB_ERR_INVALID_ARG
    assert lib.tb_bboxes(None, p(fake), 10, None, None, p(fake), p(fake), 1 << 30, p(fake), None) \
        == b.TB_ERR_INVALID_ARG
    assert lib.tb_bboxes(p(fake + 1), p(fake), 10, None, None, p(fake), p(fake), 1 << 30, p(fake),
                         None) == b.TB_ERR_INVALID_ARG
    assert lib.tb_bboxes(p(fake), p(fake), 10, None, None, p(fake), p(fake), 16, p(fake), None) \
        == b.TB_ERR_WORKSPACE
    assert lib.tb_match_parens(p(fake), 10, None, p(fake), p(fake), 1 << 30, p(fake), None) \
        == b.TB_ERR_INVALID_ARG
    assert lib.tb_bboxes_batched(p(fake), p(fake), None, 1, 10, None, None, p(fake), p(fake),
                                 1 << 30, p(fake), None) == b.TB_ERR_INVALID_ARG
    assert lib.tb_bboxes(p(fake), p(fake), 1 << 31, None, None, p(fake), p(fake), 1 << 40, p(fake),
                         None) == b.TB_ERR_INVALID_ARG
    assert lib.tb_set_phase_events(None, 0) == b.TB_OK
    assert lib.tb_debug_withhold_tile(-2) == b.TB_ERR_INVALID_ARG
    assert lib.tb_debug_withhold_tile(-1) == b.TB_OK


def test_open_positions_argument_errors(lib):
    from paper_2205_11659_gb300 import binding as b
    p = ctypes.c_void_p
    fake, big = 1 << 20, 1 << 40

    def call(kind=fake, n=10, pos=fake, cap=5, count=fake + 64, ws=fake, nb=big, status=fake + 128):
        return lib.tb_open_positions(p(kind) if kind else None, n, p(pos) if pos else None, cap,
                                     p(count) if count else None, p(ws) if ws else None, nb,
                                     p(status) if status else None, None)

    assert call(n=-1) == b.TB_ERR_INVALID_ARG
    assert call(n=1 << 31) == b.TB_ERR_INVALID_ARG
    assert call(cap=-1) == b.TB_ERR_INVALID_ARG
    assert call(kind=0) == b.TB_ERR_INVALID_ARG
    assert call(kind=fake + 1) == b.TB_ERR_INVALID_ARG
    assert call(pos=0) == b.TB_ERR_INVALID_ARG          # room for 5 but no buffer
    assert call(pos=fake + 2) == b.TB_ERR_INVALID_ARG
    assert call(count=0) == b.TB_ERR_INVALID_ARG
    assert call(status=0) == b.TB_ERR_INVALID_ARG
    assert call(ws=0) == b.TB_ERR_INVALID_ARG
    assert call(nb=8) == b.TB_ERR_WORKSPACE


def test_tree_scan_argument_errors(lib):
    from paper_2205_11659_gb300 import binding as b
    p = ctypes.c_void_p
    fake, big = 1 << 20, 1 << 40
    out = fake + (1 << 12)

    def scan(monoid=b.TB_MONOID_ADD_I32, d=b.TB_DOWN, kind=fake, n=10, J=5, vin=fake, vout=out,
             ws=fake, nb=big):
        return lib.tb_tree_scan(monoid, d, p(kind), n, J, p(vin), p(vout), p(ws), nb, p(fake), None)

    assert scan(monoid=5) == b.TB_ERR_INVALID_ARG
    assert scan(monoid=-1) == b.TB_ERR_INVALID_ARG
    assert scan(d=2) == b.TB_ERR_INVALID_ARG
    assert scan(J=6) == b.TB_ERR_INVALID_ARG          # more joints than n / 2
    assert scan(J=-1) == b.TB_ERR_INVALID_ARG
    assert scan(n=-1, J=0) == b.TB_ERR_INVALID_ARG
    assert scan(vout=fake) == b.TB_ERR_INVALID_ARG    # in and out alias
    assert scan(vin=fake + 4) == b.TB_ERR_INVALID_ARG  # misaligned values
    assert scan(kind=fake + 1) == b.TB_ERR_INVALID_ARG
    assert scan(nb=16) == b.TB_ERR_WORKSPACE
    assert lib.tb_tree_scan(0, 0, p(fake), 10, 5, p(fake), p(out), p(fake), big, None, None) \
        == b.TB_ERR_INVALID_ARG                         # no status word

    def bwd(J=5, local=fake, g=fake + 4096, gl=fake + 8192, nb=big):
        return lib.tb_tree_scan_affine_backward(p(fake), 10, J, p(local), p(g), p(gl), p(fake), nb,
                                                p(fake), None)

    assert bwd(J=6) == b.TB_ERR_INVALID_ARG
    assert bwd(gl=fake) == b.TB_ERR_INVALID_ARG
    assert bwd(local=fake + 8) == b.TB_ERR_INVALID_ARG
    assert bwd(nb=1 << 10) == b.TB_ERR_WORKSPACE

    def structure(J=5, n=10, kind=fake, d=fake, par=fake + 4096, left=fake + 8192, nb=big, st=fake):
        return lib.tb_tree_structure(p(kind), n, J, p(d), p(par), p(left), p(fake), nb, p(st), None)

    assert structure(J=6) == b.TB_ERR_INVALID_ARG
    assert structure(n=-1, J=0) == b.TB_ERR_INVALID_ARG
    assert structure(kind=fake + 1) == b.TB_ERR_INVALID_ARG
    assert structure(left=fake + 2) == b.TB_ERR_INVALID_ARG  # misaligned output
    assert structure(nb=16) == b.TB_ERR_WORKSPACE
    assert structure(st=0) == b.TB_ERR_INVALID_ARG           # no status word

    def bwd_reuse(J=5, local=fake, g=fake + 4096, gl=fake + 8192, nb=big):
        return lib.tb_tree_scan_affine_backward_reuse(p(fake), 10, J, p(local), p(g), p(gl),
                                                      p(fake), nb, p(fake), None)

    assert bwd_reuse(J=6) == b.TB_ERR_INVALID_ARG
    assert bwd_reuse(gl=fake) == b.TB_ERR_INVALID_ARG
    assert bwd_reuse(g=fake + 4) == b.TB_ERR_INVALID_ARG
    assert bwd_reuse(nb=1 << 10) == b.TB_ERR_WORKSPACE


def test_phase_event_count_limits(lib):
    from paper_2205_11659_gb300 import binding as b
    arr = (ctypes.c_void_p * 17)(*([1 << 20] * 17))
    assert lib.tb_set_phase_events(arr, 17) == b.TB_ERR_INVALID_ARG
    assert lib.tb_set_phase_events(arr, 0) == b.TB_ERR_INVALID_ARG
    assert lib.tb_set_phase_events(None, 0) == b.TB_OK


def test_tuned_shape_is_a_candidate():
    from paper_2205_11659_gb300 import _build, autotune
    assert _build.tuned_shape() + (_build.tuned_persistent(), _build.tuned_matcher()) \
        in autotune.CANDIDATES
    assert (256, 16, False, 0) in autotune.CANDIDATES and (128, 16, False, 1) in autotune.CANDIDATES


def test_static_scratch_argument_errors(lib):
    # tb_bboxes_static_ws: host checks come before any CUDA call.
    from paper_2205_11659_gb300 import binding as b
    p = ctypes.c_void_p
    fake = 1 << 20
    assert lib.tb_bboxes_static_ws(p(fake), p(fake), -1, None, None, p(fake), p(fake), None) \
        == b.TB_ERR_INVALID_ARG
    assert lib.tb_bboxes_static_ws(p(fake), p(fake), b.TB_STATIC_WS_MAX_N + 1, None, None, p(fake),
                                   p(fake), None) == b.TB_ERR_WORKSPACE


def _host_sources():
    d = os.path.join(ROOT, "paper_2205_11659_gb300", "csrc")
    out = {}
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            src = open(os.path.join(d, f)).read()
            out[f] = re.sub(r"//[^\n]*", "", src)
    return out


def test_launch_state_is_per_device():
    """A kernel attribute (the raised shared-memory limit) and the SM count
    belong to one device.  Launch code keeps them per device ordinal in
    atomic masks and arrays (tb_device_once.h), never in a process-wide
    flag, and takes the SM count from the device, not from a literal."""
    srcs = _host_sources()
    for f, src in srcs.items():
        assert not re.search(r"\bstatic\s+bool\b", src), f
        assert not re.search(r"\bstatic\s+int\s+\w+\s*\[", src), f  # plain per-process caches
        assert not re.search(r"\b152\b", src), f
    # every raised shared-memory limit goes through the per-device helper
    raw = [f for f, src in srcs.items()
           if "cudaFuncAttributeMaxDynamicSharedMemorySize" in src and f != "tb_device_once.h"]
    assert not raw, raw
    assert "smem_limit_once" in srcs["tb_api.cu"] and "smem_limit_once" in srcs["tb_tree_launch.cuh"]
