"""GPU parity of the tree scans (tb_tree_scan, tb_tree_scan_affine_backward
and the TreeTransform autograd function) against the CPU oracle.

int32 and box monoids are exact (wrapping adds, fp32 min/max), so they are
compared bit for bit.  The affine transforms are fp32 on the GPU and fp64 in
the oracle; they are compared per joint with the relative error
    max_i |gpu_i - ref_i| / max_i |ref_i|   over the 12 entries of joint r,
which must stay below 1e-4 (skeletons of depth <= 64, and the deeper chain
cases here).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2205_11659_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4
JT = 1024  # joints per tile of the tree kernels


@pytest.fixture(scope="module", autouse=True)
def device():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2205_11659_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def n_opens(k):
    return int(np.count_nonzero((k == 1) | (k == 2)))


def gpu_scan(monoid, d, k, v):
    out = binding.tree_scan(monoid, d, torch.from_numpy(k).cuda(),
                            torch.from_numpy(np.ascontiguousarray(v)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def rel_err(x, ref):
    J = ref.shape[0]
    if J == 0:
        return 0.0
    d = np.abs(x.astype(np.float64) - ref).reshape(J, -1).max(1)
    s = np.abs(ref).reshape(J, -1).max(1)
    return float((d / np.maximum(s, 1e-30)).max())


def boxes_for(J, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, 4096, (J, 2))
    wh = np.exp(rng.uniform(0, np.log(3000), (J, 2)))
    return np.concatenate([c - wh / 2, c + wh / 2], 1).astype(np.float32)


def streams():
    yield "skel1", inputs.skeleton_kinds(1, 1)
    yield "skel700", inputs.skeleton_kinds(700, 2)
    yield "skel1024", inputs.skeleton_kinds(JT, 3)
    yield "skel1025", inputs.skeleton_kinds(JT + 1, 4)
    yield "skel5000", inputs.skeleton_kinds(5000, 5)
    yield "skel60000", inputs.skeleton_kinds(60_000, 6)
    yield "skel9000_d8", inputs.skeleton_kinds(9000, 7, max_depth=8)
    yield "rw50000", inputs.random_walk_scene(50_000, 8)[0]
    yield "chain9000", inputs.chain_scene(9000, 9)[0]
    yield "flat30000", inputs.flat_scene(30_000, 10)[0]
    yield "forest", np.concatenate([inputs.skeleton_kinds(j, 20 + j) for j in (1030, 1, 2047, 300)])


STREAMS = dict(streams())


@pytest.mark.parametrize("name", list(STREAMS))
@pytest.mark.parametrize("d", [binding.TB_DOWN, binding.TB_UP])
def test_add_i32(name, d):
    k = STREAMS[name]
    v = np.random.default_rng(1).integers(-1000, 1000, n_opens(k)).astype(np.int32)
    st, ref = oracle.tree_scan_i32(d, k, v)
    assert st == oracle.OK
    out = gpu_scan(binding.TB_MONOID_ADD_I32, d, k, v)
    bad = np.nonzero(out != ref)[0]
    assert bad.size == 0, (bad[:8], out[bad[:8]], ref[bad[:8]])


@pytest.mark.parametrize("name", list(STREAMS))
@pytest.mark.parametrize("monoid", [binding.TB_MONOID_BBOX_ISECT, binding.TB_MONOID_BBOX_UNION])
@pytest.mark.parametrize("d", [binding.TB_DOWN, binding.TB_UP])
def test_boxes(name, monoid, d):
    k = STREAMS[name]
    bx = boxes_for(n_opens(k), 2)
    st, ref = oracle.tree_scan_box(monoid, d, k, bx)
    assert st == oracle.OK
    out = gpu_scan(monoid, d, k, bx)
    bad = np.nonzero(np.any(out.view(np.uint32) != ref.view(np.uint32), axis=1))[0]
    assert bad.size == 0, (bad[:8], out[bad[:8]], ref[bad[:8]])


@pytest.mark.parametrize("name", list(STREAMS))
@pytest.mark.parametrize("d", [binding.TB_DOWN, binding.TB_UP])
def test_affine(name, d):
    k = STREAMS[name]
    L = inputs.affine_locals(n_opens(k), 3)
    if d == binding.TB_DOWN:
        st, ref = oracle.affine_forward(k, L.astype(np.float64))
    else:
        st, ref = oracle.affine_up(k, L.astype(np.float64))
    assert st == oracle.OK
    out = gpu_scan(binding.TB_MONOID_AFFINE3X4_F32, d, k, L)
    assert rel_err(out, ref) < REL_TOL


@pytest.mark.parametrize("name", list(STREAMS))
@pytest.mark.parametrize("d", [binding.TB_DOWN, binding.TB_UP])
def test_rigid(name, d):
    """Rigid transforms (unit quaternion + translation, Sec. 1 / Sec. 13: any
    monoid) in fp32 against the fp64 oracle, per joint as for the affine
    transforms; the quaternion parts also against the unit norm."""
    k = STREAMS[name]
    J = n_opens(k)
    v = inputs.rigid_locals(J, 41)
    st, ref = oracle.rigid_scan(d, k, v.astype(np.float64))
    assert st == oracle.OK
    got = gpu_scan(binding.TB_MONOID_RIGID_F32, d, k, v)
    assert got.shape == (J, 8)
    assert rel_err(got[:, :4], ref[:, :4]) < REL_TOL, name
    assert rel_err(got[:, 4:7], ref[:, 4:7]) < REL_TOL, name
    if J:
        assert np.abs(np.linalg.norm(got[:, :4].astype(np.float64), axis=1) - 1.0).max() < 1e-4


@pytest.mark.parametrize("name", list(STREAMS))
def test_tree_structure(name):
    """Joint depth, parent and left-sibling vectors, bit for bit."""
    k = STREAMS[name]
    d, p, l = binding.tree_structure(torch.from_numpy(k).cuda())
    torch.cuda.synchronize()
    st, od, op, ol = oracle.tree_structure(k)
    assert st == oracle.OK
    assert np.array_equal(d.cpu().numpy(), od)
    assert np.array_equal(p.cpu().numpy(), op)
    assert np.array_equal(l.cpu().numpy(), ol)


def test_tree_structure_large_and_errors():
    k = inputs.skeleton_kinds(1 << 20, 31)
    d, p, l = binding.tree_structure(torch.from_numpy(k).cuda())
    torch.cuda.synchronize()
    st, od, op, ol = oracle.tree_structure(k)
    assert np.array_equal(d.cpu().numpy(), od) and np.array_equal(p.cpu().numpy(), op)
    assert np.array_equal(l.cpu().numpy(), ol)
    with pytest.raises(binding.TBError):
        binding.tree_structure(torch.tensor([1, 3, 3], dtype=torch.uint8, device="cuda"))


def test_rigid_large_skeleton():
    k = inputs.skeleton_kinds(1 << 20, 42)
    J = n_opens(k)
    v = inputs.rigid_locals(J, 43)
    for d in (binding.TB_DOWN, binding.TB_UP):
        st, ref = oracle.rigid_scan(d, k, v.astype(np.float64))
        got = gpu_scan(binding.TB_MONOID_RIGID_F32, d, k, v)
        assert rel_err(got[:, :4], ref[:, :4]) < REL_TOL
        assert rel_err(got[:, 4:7], ref[:, 4:7]) < REL_TOL


@pytest.mark.parametrize("name", list(STREAMS))
def test_affine_backward(name):
    k = STREAMS[name]
    J = n_opens(k)
    L = inputs.affine_locals(J, 4)
    W = inputs.grad_weights(J, 4)
    st, ref = oracle.affine_backward(k, L.astype(np.float64), W.astype(np.float64))
    assert st == oracle.OK
    g = binding.affine_backward(torch.from_numpy(k).cuda(), torch.from_numpy(L).cuda(),
                                torch.from_numpy(W).cuda())
    torch.cuda.synchronize()
    assert rel_err(g.cpu().numpy(), ref) < REL_TOL


def test_skeleton_2p20_forward_backward():
    """One skeleton of 2^20 joints, depth <= 64: forward and adjoint against
    the fp64 oracle on every joint."""
    k, L, W = inputs.skeleton(1 << 20, 11)
    st, world_ref = oracle.affine_forward(k, L.astype(np.float64))
    assert st == oracle.OK
    st, grad_ref = oracle.affine_backward(k, L.astype(np.float64), W.astype(np.float64))
    assert st == oracle.OK
    kd, Ld, Wd = (torch.from_numpy(a).cuda() for a in (k, L, W))
    world = binding.tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, kd, Ld)
    grad = binding.affine_backward(kd, Ld, Wd)
    torch.cuda.synchronize()
    e_fwd = rel_err(world.cpu().numpy(), world_ref)
    e_bwd = rel_err(grad.cpu().numpy(), grad_ref)
    assert e_fwd < REL_TOL, e_fwd
    assert e_bwd < REL_TOL, e_bwd


@pytest.mark.parametrize("J", [1 << 21, 2_400_000])
def test_many_joint_tiles(J):
    """2048 and 2344 joint tiles: the pointer jumping over tiles keeps its
    buffers in shared memory (2048 tiles) or in the workspace (2344), and
    the tile-level trees have several thousand leaves."""
    k, L, W = inputs.skeleton(J, 31)
    v = (np.arange(J, dtype=np.int64) * 2654435761 % 1000 - 500).astype(np.int32)
    kd = torch.from_numpy(k).cuda()
    for d in (oracle.DOWN, oracle.UP):
        st, ref = oracle.tree_scan_i32(d, k, v)
        assert st == oracle.OK
        out = binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_DOWN if d == oracle.DOWN
                                else binding.TB_UP, kd, torch.from_numpy(v).cuda())
        assert np.array_equal(out.cpu().numpy(), ref)
    Ld, Wd = torch.from_numpy(L).cuda(), torch.from_numpy(W).cuda()
    world = binding.tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, kd, Ld)
    grad = binding.affine_backward(kd, Ld, Wd)
    st, world_ref = oracle.affine_forward(k, L.astype(np.float64))
    assert st == oracle.OK
    assert rel_err(world.cpu().numpy(), world_ref) < REL_TOL
    st, grad_ref = oracle.affine_backward(k, L.astype(np.float64), W.astype(np.float64))
    assert st == oracle.OK
    assert rel_err(grad.cpu().numpy(), grad_ref) < REL_TOL


def test_backward_vs_fp64_finite_differences():
    """64-joint skeleton: the GPU adjoint against central differences of the
    fp64 oracle loss."""
    k, L, W = inputs.skeleton(64, 12)
    L64, W64 = L.astype(np.float64), W.astype(np.float64)
    h = 1e-6
    fd = np.zeros_like(L64)
    for idx in np.ndindex(*L64.shape):
        Lp = L64.copy()
        Lp[idx] += h
        Lm = L64.copy()
        Lm[idx] -= h
        fp = oracle.affine_loss(k, Lp, W64)[1]
        fm = oracle.affine_loss(k, Lm, W64)[1]
        fd[idx] = (fp - fm) / (2 * h)
    g = binding.affine_backward(torch.from_numpy(k).cuda(), torch.from_numpy(L).cuda(),
                                torch.from_numpy(W).cuda())
    torch.cuda.synchronize()
    assert rel_err(g.cpu().numpy(), fd) < REL_TOL


def test_tree_transform_autograd():
    k, L, W = inputs.skeleton(20_000, 13)
    kd = torch.from_numpy(k).cuda()
    local = torch.from_numpy(L).cuda().requires_grad_(True)
    Wd = torch.from_numpy(W).cuda()
    world = binding.TreeTransform.apply(kd, local)
    loss = (world * Wd).sum()
    loss.backward()
    torch.cuda.synchronize()
    st, ref = oracle.affine_backward(k, L.astype(np.float64), W.astype(np.float64))
    assert rel_err(local.grad.cpu().numpy(), ref) < REL_TOL
    st, wref = oracle.affine_forward(k, L.astype(np.float64))
    assert rel_err(world.detach().cpu().numpy(), wref) < REL_TOL


def test_batched_skeletons_match_separate_calls_and_graph():
    """Skeletons laid end to end form a forest: one call over the batch
    equals the per-skeleton calls (bit for bit for int32, within tolerance
    for fp32 transforms, whose rounding depends on the tile split).  The
    forward + backward through TreeTransform is then captured in one CUDA
    graph and replayed."""
    k, L, W, eoff, joff = inputs.batched_skeletons(24, 14, 6.0, 12.0)
    J = L.shape[0]
    kd, Ld, Wd = (torch.from_numpy(a).cuda() for a in (k, L, W))
    v = np.arange(J, dtype=np.int32) % 7 - 3
    vd = torch.from_numpy(v).cuda()
    whole_i = binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_UP, kd, vd)
    whole_w = binding.tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, kd, Ld)
    whole_g = binding.affine_backward(kd, Ld, Wd)
    torch.cuda.synchronize()
    for s in range(len(eoff) - 1):
        ks = kd[eoff[s]:eoff[s + 1]].clone()  # a fresh, aligned buffer
        js = slice(int(joff[s]), int(joff[s + 1]))
        part_i = binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_UP, ks, vd[js].clone())
        assert torch.equal(part_i, whole_i[js])
        part_w = binding.tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, ks,
                                   Ld[js].clone())
        ref = part_w.double().cpu().numpy()
        assert rel_err(whole_w[js].cpu().numpy(), ref) < REL_TOL
        part_g = binding.affine_backward(ks, Ld[js].clone(), Wd[js].clone())
        assert rel_err(whole_g[js].cpu().numpy(), part_g.double().cpu().numpy()) < REL_TOL

    # One graph for forward + backward, no status reads inside.
    ws = binding.workspace(kd.device)
    ws.reserve(binding.TB_OP_TREE_BACKWARD, k.size)
    local = Ld.clone().requires_grad_(True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):  # warm-up outside the graph
            local.grad = None
            (binding.TreeTransform.apply(kd, local, False) * Wd).sum().backward()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    local.grad = None
    with torch.cuda.graph(g):
        world = binding.TreeTransform.apply(kd, local, False)
        (world * Wd).sum().backward()
    g.replay()
    torch.cuda.synchronize()
    assert int(ws.status.item()) == binding.TB_OK
    assert torch.equal(world.detach(), whole_w)
    assert torch.equal(local.grad, whole_g)


def test_all_leaves_and_empty():
    k = np.zeros(5000, np.uint8)
    out = gpu_scan(binding.TB_MONOID_ADD_I32, binding.TB_DOWN, k, np.zeros(0, np.int32))
    assert out.shape == (0,)
    e = binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_UP,
                          torch.zeros(0, dtype=torch.uint8, device="cuda"),
                          torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert e.numel() == 0


def test_errors_reported_in_status():
    k = inputs.skeleton_kinds(3000, 15)
    J = n_opens(k)
    kd = torch.from_numpy(k).cuda()
    # wrong joint count
    with pytest.raises(binding.TBError) as ei:
        binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_DOWN, kd,
                          torch.zeros(J - 1, dtype=torch.int32, device="cuda"))
    assert ei.value.code == binding.TB_ERR_INVALID_ARG
    # unbalanced: the last close becomes a leaf
    k_unb = k.copy()
    k_unb[-1] = 0
    ku = torch.from_numpy(k_unb).cuda()
    with pytest.raises(binding.TBError) as ei:
        binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_UP, ku,
                          torch.zeros(J, dtype=torch.int32, device="cuda"))
    assert ei.value.code == binding.TB_ERR_UNBALANCED
    # a bad kind byte
    kb = k.copy()
    kb[100] = 9
    with pytest.raises(binding.TBError) as ei:
        binding.affine_backward(torch.from_numpy(kb).cuda(),
                                torch.zeros(J, 3, 4, device="cuda"),
                                torch.zeros(J, 3, 4, device="cuda"))
    assert ei.value.code == binding.TB_ERR_BAD_KIND
    # the context is still usable afterwards
    v = torch.ones(J, dtype=torch.int32, device="cuda")
    out = binding.tree_scan(binding.TB_MONOID_ADD_I32, binding.TB_UP, kd, v)
    st, ref = oracle.tree_scan_i32(oracle.UP, k, np.ones(J, np.int32))
    assert np.array_equal(out.cpu().numpy(), ref)


def test_lookback_timeout_reported_and_recovered():
    """An element tile of the depth pass that never publishes makes the
    bounded look-back waits of the tiles after it give up: the call reports
    TB_ERR_TIMEOUT (after about a second), and the next call on the same
    context is correct."""
    import time
    k, L, _ = inputs.skeleton(1 << 16, 21)  # 2^17 elements: 32 element tiles
    kd, Ld = torch.from_numpy(k).cuda(), torch.from_numpy(L).cuda()
    assert binding.tb_debug_withhold_tile(5) == binding.TB_OK
    try:
        t0 = time.perf_counter()
        with pytest.raises(binding.TBError) as ei:
            binding.tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, kd, Ld)
        assert ei.value.code == binding.TB_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 30.0
    finally:
        assert binding.tb_debug_withhold_tile(-1) == binding.TB_OK
    world = binding.tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, kd, Ld)
    st, ref = oracle.affine_forward(k, L.astype(np.float64))
    assert st == oracle.OK
    assert rel_err(world.cpu().numpy(), ref) < REL_TOL
    assert binding.tb_debug_withhold_tile(-2) == binding.TB_ERR_INVALID_ARG


def _forward_into(ws, status, kd, Ld, world):
    nb = ws.numel()
    rc = binding.tb_tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, kd, kd.numel(),
                              Ld.shape[0], Ld, world, ws, nb, status)
    assert rc == binding.TB_OK


def _reuse_into(ws, status, kd, Ld, Wd, grad):
    rc = binding.tb_tree_scan_affine_backward_reuse(kd, kd.numel(), Ld.shape[0], Ld, Wd, grad, ws,
                                                    ws.numel(), status)
    assert rc == binding.TB_OK


def test_backward_reuse_matches_full_backward():
    """The backward that reads the joint structure a forward left in its
    workspace gives the full backward's gradients bit for bit."""
    k, L, W = inputs.skeleton(200_000, 41)
    kd, Ld, Wd = (torch.from_numpy(a).cuda() for a in (k, L, W))
    n = k.size
    ws = torch.empty(binding.tb_workspace_size(binding.TB_OP_TREE_BACKWARD, n), dtype=torch.uint8,
                     device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    world = torch.empty_like(Ld)
    grad = torch.empty_like(Ld)
    _forward_into(ws, status, kd, Ld, world)
    _reuse_into(ws, status, kd, Ld, Wd, grad)
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_OK
    full = binding.affine_backward(kd, Ld, Wd)
    assert torch.equal(grad.view(torch.int32), full.view(torch.int32))
    st, ref = oracle.affine_backward(k, L.astype(np.float64), W.astype(np.float64))
    assert rel_err(grad.cpu().numpy(), ref) < REL_TOL
    # a second backward on the same workspace (the structure is still there)
    grad2 = torch.empty_like(Ld)
    _reuse_into(ws, status, kd, Ld, Wd, grad2)
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_OK
    assert torch.equal(grad2.view(torch.int32), full.view(torch.int32))


def test_backward_reuse_rejects_a_missing_structure():
    """After a forward over another joint count, or a failed forward, the
    reusing backward reports TB_ERR_INVALID_ARG; a fresh forward makes it
    work again."""
    k, L, W = inputs.skeleton(30_000, 42)
    k2, L2, _ = inputs.skeleton(29_000, 43)
    n = max(k.size, k2.size)
    ws = torch.empty(binding.tb_workspace_size(binding.TB_OP_TREE_BACKWARD, n), dtype=torch.uint8,
                     device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    kd, Ld, Wd = (torch.from_numpy(a).cuda() for a in (k, L, W))
    kd2, Ld2 = torch.from_numpy(k2).cuda(), torch.from_numpy(L2).cuda()
    grad = torch.empty_like(Ld)
    _forward_into(ws, status, kd2, Ld2, torch.empty_like(Ld2))
    _reuse_into(ws, status, kd, Ld, Wd, grad)
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_ERR_INVALID_ARG
    kb = k.copy()
    kb[10] = 9  # a bad kind: the forward fails and leaves no structure
    _forward_into(ws, status, torch.from_numpy(kb).cuda(), Ld, torch.empty_like(Ld))
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_ERR_BAD_KIND
    _reuse_into(ws, status, kd, Ld, Wd, grad)
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_ERR_INVALID_ARG
    _forward_into(ws, status, kd, Ld, torch.empty_like(Ld))
    _reuse_into(ws, status, kd, Ld, Wd, grad)
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_OK
    assert torch.equal(grad.view(torch.int32), binding.affine_backward(kd, Ld, Wd).view(torch.int32))


def test_tree_transform_keep_structure():
    """TreeTransform with keep_structure=True gives the same world and
    gradients as the default."""
    k, L, W = inputs.skeleton(50_000, 44)
    kd, Wd = torch.from_numpy(k).cuda(), torch.from_numpy(W).cuda()
    outs = []
    for keep in (False, True):
        local = torch.from_numpy(L).cuda().requires_grad_(True)
        world = binding.TreeTransform.apply(kd, local, True, keep)
        (world * Wd).sum().backward()
        torch.cuda.synchronize()
        outs.append((world.detach(), local.grad))
    assert torch.equal(outs[0][0].view(torch.int32), outs[1][0].view(torch.int32))
    assert torch.equal(outs[0][1].view(torch.int32), outs[1][1].view(torch.int32))


def test_tree_pipeline_matches_separate_calls():
    """Skeleton jobs streamed from pinned host memory with overlapped copies
    give the device calls' world and gradients (a repeated job and a size
    change included); a bad job raises with its forward status."""
    jobs = [inputs.skeleton(j, 70 + j) for j in (40_000, 3_000, 40_000, 25_000)]
    pipe = binding.TreePipeline(max(k.size for k, _, _ in jobs))
    kinds = [torch.from_numpy(k).pin_memory() for k, _, _ in jobs]
    locs = [torch.from_numpy(L).pin_memory() for _, L, _ in jobs]
    gws = [torch.from_numpy(W).pin_memory() for _, _, W in jobs]
    outs = [(torch.empty(L.shape, dtype=torch.float32).pin_memory(),
             torch.empty(L.shape, dtype=torch.float32).pin_memory()) for _, L, _ in jobs]
    pipe.run(kinds, locs, gws, outs)
    for (k, L, W), (world_h, grad_h) in zip(jobs, outs):
        kd, Ld, Wd = (torch.from_numpy(a).cuda() for a in (k, L, W))
        world = binding.tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, kd, Ld)
        grad = binding.affine_backward(kd, Ld, Wd)
        assert torch.equal(world_h.view(torch.int32), world.cpu().view(torch.int32))
        assert torch.equal(grad_h.view(torch.int32), grad.cpu().view(torch.int32))
    bad = jobs[1][0].copy()
    bad[7] = 9
    kinds[1] = torch.from_numpy(bad).pin_memory()
    with pytest.raises(binding.TBError) as ei:
        pipe.run(kinds, locs, gws, outs)
    assert ei.value.code == binding.TB_ERR_BAD_KIND

