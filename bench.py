"""Benchmark of the bounding-box + parentheses-matching pass and of the
differentiable transform tree scan on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rw26|match26|chain24|flat24|batched|rw24|rw16|skel20|skel20s|skelbatch]

Scene workloads: one step = one full pass (tile summaries and tile scan,
tile-level resolve, main tile pass, cross-tile unions) over one synthetic
scene already resident in HBM.  Skeleton workloads: one step = the affine
DOWN scan (forward) plus its adjoint (backward) over the joint stream.
Prints one JSON line (rank 0).  With N > 1 (torchrun), each rank runs its own
replica of the workload on its own GPU (independent scenes, no collective on
the data path) and the value is the whole-job throughput.

``--impl reference`` times the sequential CPU oracle on the same workload on
the host cores instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gelem/s bbox+paren pass & fwd+bwd tree scan; % HBM roofline; batched vs plain"
BYTES_PER_ELEM = 41  # kind 1 + box 16 read; parent 4 + match 4 + box_out 16 written
MATCH_BYTES_PER_ELEM = 9  # kind 1 read; parent 4 + match 4 written

WORKLOADS = {
    "rw26": "bbox+paren pass, one random-walk scene (OPEN 0.2 clip/blend 50/50, CLOSE 0.2), N=2^26",
    "chain24": "bbox+paren pass, one chain scene: 2^23 nested clip opens, a leaf, 2^23 closes",
    "flat24": "bbox+paren pass, one flat scene of depth <= 4 (~90% leaves), N=2^24",
    "batched": "bbox+paren pass, 4096 random-walk scenes with N_s = round(2^U[8,18]), one batched call",
    "rw16": "bbox+paren pass, one random-walk scene, N=2^16 (launch-latency size)",
    "rw24": "bbox+paren pass, one random-walk scene, N=2^24 (profiling size)",
    "match26": "parentheses matching only (parent and match indices), one random-walk scene, N=2^26",
    "opens26": "stream compaction of the opens (clip and blend nodes) of one random-walk scene, "
               "N=2^26",
    "skel20": "affine tree scan forward + adjoint, one skeleton of J=2^20 joints (N=2J), depth <= 64",
    "skel20s": "affine tree scan forward + adjoint, one skeleton of J=2^18 joints (profiling size)",
    "skelbatch": "affine tree scan forward + adjoint through TreeTransform, 256 skeletons with "
                 "J_s = round(2^U[10,16]), one CUDA graph per step",
}
TREE_WORKLOADS = ("skel20", "skel20s", "skelbatch")
FWD_BYTES_PER_JOINT = 98   # 2 kinds + 48 local read, 48 world written
BWD_BYTES_PER_JOINT = 146  # 2 kinds + 48 local + 48 grad_world read, 48 grad_local written

# DRAM bytes per launch of the main tile pass measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the hash of the
# kernel sources they were taken on; a changed kernel reports null.
NCU_TRAFFIC = {
    # 641.5 MB per launch measured on the 2^24 random walk (2048-element
    # tiles, profiles/k3_tile_bbox_rw24.md); the 2^26 entry scales it by the
    # element count (traffic tracks the 41 B/elem).
    "33758ae913d869fc": {"rw24": 641.5e6, "rw26": 641.5e6 * 4},
}
# The same for one tb_open_positions call (its three launches summed), keyed
# by the hash of the compaction sources: the kinds read twice, and the part
# of the positions that already left L2 when the scatter ended.
OPEN_NCU_TRAFFIC = {"3df41487eb6d93e2": {"opens26": 139.3e6}}


def make_workload(name, seed=0):
    from paper_2205_11659_gb300 import inputs
    if name in ("rw26", "match26", "opens26"):
        k, b = inputs.random_walk_scene(1 << 26, seed)
        return k, b, None
    if name == "rw24":
        k, b = inputs.random_walk_scene(1 << 24, seed)
        return k, b, None
    if name == "rw16":
        k, b = inputs.random_walk_scene(1 << 16, seed)
        return k, b, None
    if name == "chain24":
        k, b = inputs.chain_scene(1 << 23, seed)
        return k, b, None
    if name == "flat24":
        k, b = inputs.flat_scene(1 << 24, seed)
        return k, b, None
    if name == "batched":
        return inputs.batched_scenes(4096, seed)
    if name == "skel20":
        k, L, W = inputs.skeleton(1 << 20, seed)
        return k, L, W, None, None
    if name == "skel20s":
        k, L, W = inputs.skeleton(1 << 18, seed)
        return k, L, W, None, None
    if name == "skelbatch":
        return inputs.batched_skeletons(256, seed)
    raise ValueError(name)


SCENE_SOURCES = ("tb_api.cu", "tb_core.cuh", "tb_prims.cuh", "tb_scene_kernels.cuh")
OPEN_SOURCES = ("tb_open_api.cu", "tb_core.cuh", "tb_prims.cuh", "tb_open_kernels.cuh")
TREE_SOURCES = ("tb_core.cuh", "tb_prims.cuh", "tb_tree_api.cu", "tb_tree_kernels.cuh")


def kernel_hash(sources=SCENE_SOURCES):
    """Hash of the CUDA sources a workload's kernels are built from (and of
    the tuned build parameters), naming the kernels a traffic figure was
    measured on."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2205_11659_gb300", "csrc")
    for f in sources:
        h.update(open(os.path.join(csrc, f), "rb").read())
    from paper_2205_11659_gb300 import _build
    nt, kpt = _build.tuned_shape()
    if (nt, kpt) != (256, 16):
        h.update(b"shape %d %d" % (nt, kpt))
    if _build.tuned_persistent():
        h.update(b"persistent")
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def job_time_ms(ms_local, world, device):
    """Whole-job duration of a timed region: the maximum over the ranks."""
    if world <= 1:
        return ms_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


L2_BYTES = 130e6  # GB300 L2 (129 MB), rounded up


class L2Flush:
    """Evicts L2 between timed steps when a workload's inputs fit in it: a
    256 MB write (twice the L2) issued before each step, outside the step's
    timed event pair.  Inactive (no buffer, no writes) when the inputs are
    larger than L2."""

    def __init__(self, torch, dev, input_bytes):
        self.active = input_bytes <= L2_BYTES
        self.buf = torch.empty(64 << 20, dtype=torch.float32, device=dev) if self.active else None

    def __call__(self):
        if self.active:
            self.buf.fill_(1.0)

    def describe(self, input_bytes):
        return l2_description(input_bytes)


def l2_description(input_bytes):
    """How the timed steps of a workload with these input bytes treat L2."""
    if input_bytes <= L2_BYTES:
        return ("inputs (%.1f MB) fit in L2: 256 MB written before each timed step, outside "
                "its events" % (input_bytes / 1e6))
    return "inputs (%.2f GB) larger than L2, no flush" % (input_bytes / 1e9)


def parallelism(world):
    return "replicas" if world > 1 else "single"


def scene_config(workload, n, scenes, input_bytes, world):
    """config of a scene workload's line (both arms print the same)."""
    return {"workload": WORKLOADS[workload], "n": int(n), "seed": 0, "scenes": int(scenes),
            "l2": l2_description(input_bytes), "parallelism": parallelism(world)}


def opens_config(workload, n, opens, input_bytes, world):
    return {"workload": WORKLOADS[workload], "n": int(n), "opens": int(opens), "seed": 0,
            "l2": l2_description(input_bytes), "parallelism": parallelism(world)}


def tree_config(workload, n, joints, batched, input_bytes, world):
    return {"workload": WORKLOADS[workload], "n": int(n), "joints": int(joints), "seed": 0,
            "step": "one CUDA graph of TreeTransform forward + backward (keep_structure=True)"
                    if batched else "one CUDA graph of tb_tree_scan (affine DOWN) + "
                                    "tb_tree_scan_affine_backward_reuse",
            "l2": l2_description(input_bytes), "parallelism": parallelism(world)}


def timed_each(torch, stream, call, K, flush):
    """Mean ms of K calls, each between its own pair of events on `stream`,
    with flush() before each call (outside the pair)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    for a, b in ev:
        flush()
        a.record(stream)
        call()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / K


def job_rate(units_per_rank, world, ms_step):
    """Whole-job throughput in G units/s: every rank processes its own copy
    of the workload (replicas, weak scaling)."""
    return world * units_per_rank / (ms_step * 1e-3) / 1e9


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def time_oracle(kind, box, offsets, match_only=False, budget_s=12.0, min_runs=1, max_runs=50):
    import oracle
    oracle.build()
    runs, t0 = 0, time.perf_counter()
    while True:
        if match_only:
            st = oracle.match_parens(kind)[0]
        elif offsets is None:
            st = oracle.bboxes(kind, box)[0]
        else:
            st = oracle.bboxes_batched(kind, box, offsets)[0]
        assert st == oracle.OK
        runs += 1
        el = time.perf_counter() - t0
        if (runs >= min_runs and el >= budget_s) or runs >= max_runs:
            return kind.size * runs / el / 1e9, runs, el


def time_oracle_opens(kind, budget_s=12.0, max_runs=50):
    import oracle
    oracle.build()
    runs, t0 = 0, time.perf_counter()
    while True:
        assert oracle.open_positions(kind)[0] == oracle.OK
        runs += 1
        el = time.perf_counter() - t0
        if el >= budget_s or runs >= max_runs:
            return kind.size * runs / el / 1e9, runs, el


def run_opens(args, torch, world, rank, dev):
    """tb_open_positions over the 2^26 random walk: device-timed calls with
    the kinds resident in HBM (L2 flushed before each), the same call as a
    CUDA graph, and end to end from pinned host memory."""
    from paper_2205_11659_gb300 import binding
    kind, _, _ = make_workload(args.workload, seed=0)
    n = int(kind.size)
    k_d = torch.from_numpy(kind).to(dev)
    cap = n // 2 + 1
    pos = torch.empty(cap, dtype=torch.int32, device=dev)
    count = torch.empty(1, dtype=torch.int32, device=dev)
    nb = binding.tb_workspace_size(binding.TB_OP_OPEN_POSITIONS, n)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        rc = binding.tb_open_positions(k_d, n, pos, cap, count, ws, nb, status, stream)
        if rc != binding.TB_OK:
            raise binding.TBError(rc, "bench step")

    flush = L2Flush(torch, dev, kind.nbytes)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_OK
    J = int(count.item())
    K = args.steps
    phase = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    for evs in phase:
        for e in evs:
            e.record(stream)
    steps_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(K)]
    clocks = ClockSampler(dev.index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(K):
        flush()
        steps_ev[i][0].record(stream)
        binding.tb_set_phase_events(phase[i])
        step()
        steps_ev[i][1].record(stream)
    binding.tb_set_phase_events(None)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_step = job_time_ms(sum(a.elapsed_time(b) for a, b in steps_ev), world, dev) / K
    assert int(status.item()) == binding.TB_OK and int(count.item()) == J
    names = ["count", "offsets", "scatter"]
    phases = {nm: statistics.mean(phase[i][j].elapsed_time(phase[i][j + 1]) for i in range(K))
              for j, nm in enumerate(names)}
    value = job_rate(n, world, ms_step)

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rcg = binding.tb_open_positions(k_d, n, pos, cap, count, ws, nb, status, None)
    assert rcg == binding.TB_OK
    g.replay()
    torch.cuda.synchronize()
    graph_ms = timed_each(torch, stream, g.replay, K, flush)
    del g

    # end to end: kinds from pinned host memory, the call, then the count and
    # the positions back (the count decides how many positions to copy)
    kind_h = torch.from_numpy(kind).pin_memory()
    pos_h = torch.empty(cap, dtype=torch.int32).pin_memory()
    count_h = torch.empty(1, dtype=torch.int32).pin_memory()

    def e2e_step():
        k_d.copy_(kind_h, non_blocking=True)
        step()
        count_h.copy_(count, non_blocking=True)
        torch.cuda.synchronize()
        c = int(count_h[0])
        pos_h[:c].copy_(pos[:c], non_blocking=True)
        torch.cuda.synchronize()
    e2e_step()
    e2e_steps = max(3, K)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    peak, peak_src = measured_peaks()
    alg = n + 4 * J  # kinds read once, one int32 per open written
    achieved = alg / (ms_step * 1e-3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, runs, el = time_oracle_opens(kind)
        cpu = {"value": round(v, 4), "unit": "Gelem/s", "cores": 1, "kind": "oracle",
               "sample": "the full workload (%d elements) x %d runs, %.1f s, single thread"
                         % (n, runs, el)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gelem/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": opens_config(args.workload, n, J, kind.nbytes, world),
            "roofline": {"bound": "hbm",
                         "kernel": "tb_open_positions (count, offsets, scatter launches)",
                         "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": OPEN_NCU_TRAFFIC.get(kernel_hash(OPEN_SOURCES), {}).get(
                             args.workload),
                         "algorithmic_bytes_per_launch": int(alg)},
            "phases_ms": {k: round(v, 4) for k, v in phases.items()},
            "graph": {"ms_per_step": round(graph_ms, 4),
                      "value": round(world * n / (graph_ms * 1e-3) / 1e9, 3), "unit": "Gelem/s",
                      "note": "the same call replayed as one CUDA graph"},
            "cpu_baseline": cpu,
            "e2e": {"value": round(world * n / e2e_s / 1e9, 3), "unit": "Gelem/s",
                    "h2d_bytes_per_step": int(kind.nbytes), "d2h_bytes_per_step": int(4 + 4 * J),
                    "how": "copy in, the call, count and positions copied back, one scene at a "
                           "time"},
            "gpu_launches": 3 * K,
            "clocks": clk,
            "kernel_hash": kernel_hash(OPEN_SOURCES),
        }
        print(json.dumps(line), flush=True)
    return 0


def time_oracle_tree(kind, L, W, budget_s=12.0, max_runs=50):
    import oracle
    oracle.build()
    L64, W64 = L.astype(np.float64), W.astype(np.float64)
    runs, t0 = 0, time.perf_counter()
    while True:
        assert oracle.affine_forward(kind, L64)[0] == oracle.OK
        assert oracle.affine_backward(kind, L64, W64)[0] == oracle.OK
        runs += 1
        el = time.perf_counter() - t0
        if el >= budget_s or runs >= max_runs:
            return kind.size * runs / el / 1e9, runs, el


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    if args.workload in TREE_WORKLOADS:
        return run_reference_tree(args, world)
    kind, box, offsets = make_workload(args.workload)
    import oracle
    oracle.build()

    def once():
        if args.workload == "match26":
            return oracle.match_parens(kind)[0]
        if args.workload == "opens26":
            return oracle.open_positions(kind)[0]
        if offsets is None:
            return oracle.bboxes(kind, box)[0]
        return oracle.bboxes_batched(kind, box, offsets)[0]
    for _ in range(args.warmup):
        assert once() == oracle.OK
    t0 = time.perf_counter()
    for _ in range(args.steps):
        assert once() == oracle.OK
    el = time.perf_counter() - t0
    value = kind.size * args.steps / el / 1e9
    sample = "full workload (%d elements) per step, single thread" % kind.size
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Gelem/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "u8" if args.workload == "opens26" else "f32", "data": "synthetic",
            "config": (opens_config(args.workload, kind.size, int(np.count_nonzero((kind == 1) | (kind == 2))),
                                    kind.nbytes, world) if args.workload == "opens26" else
                       scene_config(args.workload, kind.size,
                                    1 if offsets is None else offsets.size - 1,
                                    kind.nbytes + (0 if args.workload == "match26" else box.nbytes),
                                    world)),
            "cpu_baseline": {"value": round(value, 4), "unit": "Gelem/s", "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "Gelem/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_tree(args, world):
    kind, L, W = make_workload(args.workload)[:3]
    import oracle
    oracle.build()
    L64, W64 = L.astype(np.float64), W.astype(np.float64)

    def once():
        assert oracle.affine_forward(kind, L64)[0] == oracle.OK
        assert oracle.affine_backward(kind, L64, W64)[0] == oracle.OK
    for _ in range(args.warmup):
        once()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        once()
    el = time.perf_counter() - t0
    value = kind.size * args.steps / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Gelem/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": tree_config(args.workload, kind.size, L.shape[0],
                                  args.workload == "skelbatch", kind.nbytes + L.nbytes + W.nbytes,
                                  world),
            "cpu_baseline": {"value": round(value, 4), "unit": "Gelem/s", "cores": 1,
                             "kind": "oracle",
                             "sample": "full workload (%d elements) forward + backward per step, "
                                       "single thread, fp64" % kind.size},
            "e2e": {"value": round(value, 4), "unit": "Gelem/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_tree(args, torch, world, rank, dev):
    """Skeleton workloads: forward (affine DOWN scan) + adjoint per step.
    Returns rank 0's line (None on the other ranks); args.light skips the
    end-to-end leg and the CPU baseline."""
    from paper_2205_11659_gb300 import binding
    light = getattr(args, "light", False)
    kind, L, W, eoff, joff = make_workload(args.workload, seed=0)
    n, J = int(kind.size), int(L.shape[0])
    k_d = torch.from_numpy(kind).to(dev)
    L_d = torch.from_numpy(L).to(dev)
    W_d = torch.from_numpy(W).to(dev)
    world_d = torch.empty_like(L_d)
    grad_d = torch.empty_like(L_d)
    nb = binding.tb_workspace_size(binding.TB_OP_TREE_BACKWARD, n)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    batched = eoff is not None

    def fwd():
        rc = binding.tb_tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, k_d, n, J, L_d,
                                  world_d, ws, nb, status, stream)
        if rc != binding.TB_OK:
            raise binding.TBError(rc, "forward")

    def bwd():
        rc = binding.tb_tree_scan_affine_backward(k_d, n, J, L_d, W_d, grad_d, ws, nb, status,
                                                  stream)
        if rc != binding.TB_OK:
            raise binding.TBError(rc, "backward")

    def bwd_reuse(st):
        # the backward that reads the joint structure the forward left in ws
        return binding.tb_tree_scan_affine_backward_reuse(k_d, n, J, L_d, W_d, grad_d, ws, nb,
                                                          status, st)

    graph = None
    if not batched:
        # the forward and the structure-reusing backward, captured once in a
        # CUDA graph
        fwd()
        assert bwd_reuse(stream) == binding.TB_OK
        torch.cuda.synchronize()
        assert int(status.item()) == binding.TB_OK
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            rc1 = binding.tb_tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, k_d, n, J,
                                       L_d, world_d, ws, nb, status, None)
            rc2 = bwd_reuse(None)
        assert rc1 == binding.TB_OK and rc2 == binding.TB_OK
    if batched:
        # forward + backward through the autograd function, one graph
        bws = binding.workspace(dev)
        bws.reserve(binding.TB_OP_TREE_BACKWARD, n)
        local = L_d.clone().requires_grad_(True)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(2):
                local.grad = None
                (binding.TreeTransform.apply(k_d, local, False, True) * W_d).sum().backward()
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        local.grad = None
        with torch.cuda.graph(graph):
            (binding.TreeTransform.apply(k_d, local, False, True) * W_d).sum().backward()

    in_bytes = kind.nbytes + L.nbytes + W.nbytes
    flush = L2Flush(torch, dev, in_bytes)
    for _ in range(max(args.warmup, 3)):
        fwd()
        bwd()
        if graph is not None:
            graph.replay()
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_OK, int(status.item())
    if graph is not None:
        assert int(binding.workspace(dev).status.item()) == binding.TB_OK

    K = args.steps
    nf, nbk = 7, 9
    ev_f = [[torch.cuda.Event(enable_timing=True) for _ in range(nf)] for _ in range(K)]
    ev_b = [[torch.cuda.Event(enable_timing=True) for _ in range(nbk)] for _ in range(K)]
    for evs in ev_f + ev_b:
        for e in evs:
            e.record(stream)
    steps_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(K)]
    clocks = ClockSampler(dev.index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(K):
        flush()
        steps_ev[i][0].record(stream)
        if graph is not None:
            graph.replay()
        else:
            binding.tb_set_phase_events(ev_f[i])
            fwd()
            binding.tb_set_phase_events(ev_b[i])
            bwd()
        steps_ev[i][1].record(stream)
    binding.tb_set_phase_events(None)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = job_time_ms(sum(a.elapsed_time(b) for a, b in steps_ev), world, dev)
    ms_step = ms_total / K
    value = job_rate(n, world, ms_step)

    # per-kernel times of the plain calls (event pairs in launch order)
    fnames = ["depth", "minmax", "min_tree", "jstruct_chain", "down_tiles", "down_tile"]
    bnames = fnames[:5] + ["adjoint_tile", "up_tiles", "up_cross"]
    if graph is not None:
        for i in range(K):
            flush()
            binding.tb_set_phase_events(ev_f[i])
            fwd()
            binding.tb_set_phase_events(ev_b[i])
            bwd()
        binding.tb_set_phase_events(None)
        torch.cuda.synchronize()

    def spans(evs, names):
        return {nm: statistics.mean(evs[i][j].elapsed_time(evs[i][j + 1]) for i in range(K))
                for j, nm in enumerate(names)}
    fph = spans(ev_f, fnames)
    bph = spans(ev_b, bnames)
    fwd_calls_ms = statistics.mean(ev_f[i][0].elapsed_time(ev_f[i][nf - 1]) for i in range(K))
    bwd_calls_ms = statistics.mean(ev_b[i][0].elapsed_time(ev_b[i][nbk - 1]) for i in range(K))

    # forward and backward each captured alone and replayed: their launches
    # without host gaps (the roofline fractions use these)
    def graph_ms(call):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            call(None)
        g.replay()
        torch.cuda.synchronize()
        return timed_each(torch, stream, g.replay, K, flush)
    fwd_ms = graph_ms(lambda st: binding.tb_tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN,
                                                      k_d, n, J, L_d, world_d, ws, nb, status, st))
    bwd_ms = graph_ms(lambda st: binding.tb_tree_scan_affine_backward(k_d, n, J, L_d, W_d, grad_d, ws,
                                                                      nb, status, st))
    # the structure-reusing backward alone (ws holds the structure of the
    # same stream from the calls above)
    bwd_reuse_ms = graph_ms(bwd_reuse)
    assert int(status.item()) == binding.TB_OK

    per_scene = None
    if batched:
        # the same skeletons as 256 separate plain forward + backward calls
        S = len(eoff) - 1
        parts = []
        for sidx in range(S):
            e0, e1, j0, j1 = int(eoff[sidx]), int(eoff[sidx + 1]), int(joff[sidx]), int(joff[sidx + 1])
            parts.append((k_d[e0:e1].clone(), L_d[j0:j1].clone(), W_d[j0:j1].clone(),
                          torch.empty_like(L_d[j0:j1]), torch.empty_like(L_d[j0:j1])))

        def per_scene_step():
            for kk, ll, wg, wo, go in parts:
                ns, js = kk.numel(), ll.shape[0]
                binding.tb_tree_scan(binding.TB_MONOID_AFFINE3X4_F32, binding.TB_DOWN, kk, ns, js, ll,
                                     wo, ws, nb, status, stream)
                binding.tb_tree_scan_affine_backward_reuse(kk, ns, js, ll, wg, go, ws, nb, status,
                                                           stream)
        per_scene_step()
        torch.cuda.synchronize()
        reps = max(2, min(K, 5))
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(reps):
            per_scene_step()
        p1.record(stream)
        torch.cuda.synchronize()
        ps_ms = p0.elapsed_time(p1) / reps
        assert int(status.item()) == binding.TB_OK
        per_scene = {"value": round(n / (ps_ms * 1e-3) / 1e9, 3), "unit": "Gelem/s",
                     "ms_per_step": round(ps_ms, 4), "launches": "%d x (forward + structure-reusing backward) plain calls" % S,
                     "batched_over_per_scene": round(ps_ms / ms_step, 2)}

    # end to end through the public API with pinned host buffers: K jobs
    # streamed through TreePipeline (copies of consecutive jobs overlap the
    # forward + backward; the pipeline's fill and drain are timed)
    e2e_steps, e2e_s = 0, float("nan")
    if not light:
        kind_h = torch.from_numpy(kind).pin_memory()
        L_h = torch.from_numpy(L).pin_memory()
        W_h = torch.from_numpy(W).pin_memory()
        out_h = (torch.empty_like(L_h).pin_memory(), torch.empty_like(L_h).pin_memory())
        e2e_steps = max(3, K)
        tpipe = binding.TreePipeline(n, dev)
        tpipe.run([kind_h], [L_h], [W_h], [out_h])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tpipe.run([kind_h] * e2e_steps, [L_h] * e2e_steps, [W_h] * e2e_steps, [out_h] * e2e_steps)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        del tpipe

    peak, peak_src = measured_peaks()
    bwd_alg = BWD_BYTES_PER_JOINT * J
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not light:
        v, runs, el = time_oracle_tree(kind, L, W)
        cpu = {"value": round(v, 4), "unit": "Gelem/s", "cores": 1, "kind": "oracle",
               "sample": "the full workload (%d elements) forward + backward x %d runs, %.1f s, "
                         "single thread, fp64" % (n, runs, el)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gelem/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": tree_config(args.workload, n, J, batched, in_bytes, world),
            "gjoint_per_s": round(world * J / (ms_step * 1e-3) / 1e9, 3),
            "roofline": {"bound": "hbm",
                         "kernel": "tb_tree_scan_affine_backward_reuse (all its launches; the joint "
                                   "structure the step's forward left in the workspace)",
                         "achieved": round(bwd_alg / (bwd_reuse_ms * 1e-3) / 1e9, 1), "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s",
                         "frac": round(bwd_alg / (bwd_reuse_ms * 1e-3) / 1e9 / peak, 4),
                         "traffic": None, "algorithmic_bytes_per_launch": bwd_alg},
            "forward_roofline_frac": round(FWD_BYTES_PER_JOINT * J / (fwd_ms * 1e-3) / 1e9 / peak, 4),
            "standalone_backward_roofline_frac": round(bwd_alg / (bwd_ms * 1e-3) / 1e9 / peak, 4),
            "forward_ms": round(fwd_ms, 4), "backward_reuse_ms": round(bwd_reuse_ms, 4),
            "standalone_backward_ms": round(bwd_ms, 4),
            "step_roofline_frac": round((FWD_BYTES_PER_JOINT + BWD_BYTES_PER_JOINT) * world * J /
                                        (ms_step * 1e-3) / 1e9 / peak, 4),
            "forward_backward_plain_calls_ms": [round(fwd_calls_ms, 4), round(bwd_calls_ms, 4)],
            "backward_gjoint_per_s": round(J / (bwd_reuse_ms * 1e-3) / 1e9, 3),
            "phases_ms": {"forward": {k: round(v, 4) for k, v in fph.items()},
                          "backward": {k: round(v, 4) for k, v in bph.items()}},
            "per_scene": per_scene,
            "cpu_baseline": cpu,
            "e2e": None if light else {
                "value": round(world * n / e2e_s / 1e9, 3), "unit": "Gelem/s",
                "h2d_bytes_per_step": int(kind.nbytes + L.nbytes + W.nbytes),
                "d2h_bytes_per_step": int(2 * L.nbytes), "jobs": e2e_steps,
                "how": "TreePipeline: copies of consecutive jobs overlap the forward + "
                       "structure-reusing backward; fill and drain timed"},
            "gpu_launches": (6 + 5) * K,
            "clocks": clk,
            "kernel_hash": kernel_hash(TREE_SOURCES),
        }
        return line
    return None


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2205_11659_gb300 import _build
    _build.build()
    if args.workload == "opens26":
        rc = run_opens(args, torch, world, rank, dev)
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return rc
    line = (run_tree if args.workload in TREE_WORKLOADS else measure_scene)(
        args, torch, world, rank, dev)
    if line is not None and args.workload == "rw26" and world == 1 and not args.no_sub:
        line["sub"] = sub_records(args, torch, world, rank, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


SUB_WORKLOADS = ("chain24", "flat24", "batched", "skel20", "skelbatch")


def sub_records(args, torch, world, rank, dev):
    """The other configurations of the benchmark, each measured the same way
    as its own line (device-timed steps with inputs resident in HBM, L2
    flushed when they would fit in it, clocks sampled) with fewer steps and
    without the end-to-end leg and CPU baseline; summarised per workload."""
    out = {}
    for wl in SUB_WORKLOADS:
        sub = argparse.Namespace(**vars(args))
        sub.workload, sub.steps, sub.warmup, sub.light = wl, 10, 3, True
        sub.no_cpu_baseline = True
        t0 = time.perf_counter()
        ln = (run_tree if wl in TREE_WORKLOADS else measure_scene)(sub, torch, world, rank, dev)
        torch.cuda.empty_cache()
        if ln is None:
            continue
        rec = {"workload": WORKLOADS[wl], "n": ln["config"]["n"], "steps": 10,
               "ms_per_step": ln["ms_per_step"], "value": ln["value"], "unit": ln["unit"],
               "roofline": {k: ln["roofline"][k] for k in ("kernel", "achieved", "frac")},
               "step_roofline_frac": ln["step_roofline_frac"], "l2": ln["config"]["l2"],
               "clocks": ln["clocks"], "wall_s": round(time.perf_counter() - t0, 1)}
        if wl in TREE_WORKLOADS:
            rec.update({"joints": ln["config"]["joints"], "gjoint_per_s": ln["gjoint_per_s"],
                        "forward_ms": ln["forward_ms"], "backward_reuse_ms": ln["backward_reuse_ms"],
                        "forward_roofline_frac": ln["forward_roofline_frac"],
                        "backward_roofline_frac": ln["roofline"]["frac"],
                        "standalone_backward_roofline_frac": ln["standalone_backward_roofline_frac"]})
        else:
            rec.update({"phases_ms": ln["phases_ms"], "graph_value": ln["graph"]["value"]})
        if ln.get("per_scene"):
            rec["per_scene"] = ln["per_scene"]
        out[wl] = rec
    return out


def measure_scene(args, torch, world, rank, dev):
    """Scene workloads: one full bounding-box (or matching) pass per step.
    Returns rank 0's line (None on the other ranks); args.light skips the
    end-to-end leg and the CPU baseline."""
    from paper_2205_11659_gb300 import binding
    light = getattr(args, "light", False)
    kind, box, offsets = make_workload(args.workload, seed=0)
    n = int(kind.size)
    k_d = torch.from_numpy(kind).to(dev)
    b_d = torch.from_numpy(box).to(dev)
    off_d = torch.from_numpy(offsets).to(dev) if offsets is not None else None
    S = 0 if offsets is None else int(offsets.size - 1)
    parent = torch.empty(n, dtype=torch.int32, device=dev)
    match = torch.empty(n, dtype=torch.int32, device=dev)
    box_out = torch.empty(n, 4, dtype=torch.float32, device=dev)
    match_only = args.workload == "match26"
    bytes_per_elem = MATCH_BYTES_PER_ELEM if match_only else BYTES_PER_ELEM
    op = binding.TB_OP_MATCH_PARENS if match_only else (
        binding.TB_OP_BBOXES if offsets is None else binding.TB_OP_BBOXES_BATCHED)
    nb = binding.tb_workspace_size(op, n, S)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def call(st):
        if match_only:
            return binding.tb_match_parens(k_d, n, parent, match, ws, nb, status, st)
        if offsets is None:
            return binding.tb_bboxes(k_d, b_d, n, parent, match, box_out, ws, nb, status, st)
        return binding.tb_bboxes_batched(k_d, b_d, off_d, S, n, parent, match, box_out, ws, nb,
                                         status, st)

    def step():
        rc = call(stream)
        if rc != binding.TB_OK:
            raise binding.TBError(rc, "bench step")

    in_bytes = kind.nbytes + (0 if match_only else box.nbytes)
    flush = L2Flush(torch, dev, in_bytes)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_OK, int(status.item())

    # ---- device-timed region: inputs resident in HBM (L2 flushed before
    # each step when they would fit in it)
    K = args.steps
    phase = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    for evs in phase:           # create the event handles
        for e in evs:
            e.record(stream)
    steps_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(K)]
    clocks = ClockSampler(dev.index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(K):
        flush()
        steps_ev[i][0].record(stream)
        binding.tb_set_phase_events(phase[i])
        step()
        steps_ev[i][1].record(stream)
    binding.tb_set_phase_events(None)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = job_time_ms(sum(a.elapsed_time(b) for a, b in steps_ev), world, dev)
    ms_step = ms_total / K
    assert int(status.item()) == binding.TB_OK
    names = ["k1_tile_summary", "k2_tile_resolve", "k3_tile", "k4_cross_tile_unions"]
    phases = {nm: statistics.mean(phase[i][j].elapsed_time(phase[i][j + 1]) for i in range(K))
              for j, nm in enumerate(names)}
    value = job_rate(n, world, ms_step)

    # ---- the same step captured once in a CUDA graph and replayed (what a
    # caller repeating the pass would do; at small sizes launch latency
    # dominates the plain calls)
    gstep = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gstep):
        rcg = call(None)
    assert rcg == binding.TB_OK
    gstep.replay()
    torch.cuda.synchronize()
    assert int(status.item()) == binding.TB_OK
    graph_step_ms = timed_each(torch, stream, gstep.replay, K, flush)
    del gstep

    # ---- batched: the same scenes as separate plain calls, same outputs
    per_scene = None
    if offsets is not None:
        parent2 = torch.empty_like(parent)
        match2 = torch.empty_like(match)
        box2 = torch.empty_like(box_out)
        calls = []
        for sidx in range(S):
            e0, e1 = int(offsets[sidx]), int(offsets[sidx + 1])
            if e1 > e0:
                # kind needs 16-byte alignment: a copy per scene; the other
                # buffers are 16-byte aligned views
                calls.append((k_d[e0:e1].clone(), b_d[e0:e1], e1 - e0, parent2[e0:e1],
                              match2[e0:e1], box2[e0:e1]))
        nb1 = binding.tb_workspace_size(binding.TB_OP_BBOXES, max(c[2] for c in calls))

        def per_scene_step():
            for kk, bb, ns, pp, mm, oo in calls:
                rc = binding.tb_bboxes(kk, bb, ns, pp, mm, oo, ws, nb1, status, stream)
                if rc != binding.TB_OK:
                    raise binding.TBError(rc, "per-scene step")
        per_scene_step()
        torch.cuda.synchronize()
        assert int(status.item()) == binding.TB_OK
        same = (torch.equal(parent, parent2) and torch.equal(match, match2) and
                torch.equal(box_out.view(torch.int32), box2.view(torch.int32)))
        reps = max(2, min(K, 5))
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(reps):
            per_scene_step()
        p1.record(stream)
        torch.cuda.synchronize()
        ps_ms = p0.elapsed_time(p1) / reps
        # the batched call captured once in a CUDA graph and replayed
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            rc = binding.tb_bboxes_batched(k_d, b_d, off_d, S, n, parent2, match2, box2, ws, nb,
                                           status, None)
        assert rc == binding.TB_OK
        g.replay()
        torch.cuda.synchronize()
        assert int(status.item()) == binding.TB_OK
        same_graph = (torch.equal(parent, parent2) and torch.equal(match, match2) and
                      torch.equal(box_out.view(torch.int32), box2.view(torch.int32)))
        p0.record(stream)
        for _ in range(reps):
            g.replay()
        p1.record(stream)
        torch.cuda.synchronize()
        graph_ms = p0.elapsed_time(p1) / reps
        per_scene = {"value": round(n / (ps_ms * 1e-3) / 1e9, 3), "unit": "Gelem/s",
                     "ms_per_step": round(ps_ms, 4),
                     "launches": "%d plain tb_bboxes calls on one stream" % len(calls),
                     "outputs_identical": bool(same),
                     "batched_over_per_scene": round(ps_ms / ms_step, 2),
                     "graph_ms_per_step": round(graph_ms, 4),
                     "graph_outputs_identical": bool(same_graph)}
        del parent2, match2, box2, calls, g

    # ---- end to end through the public API with host buffers
    e2e = None
    if not light:
        e2e = scene_e2e(torch, binding, dev, kind, box, offsets, match_only, n, K, world)

    peak, peak_src = measured_peaks()
    k3_ms = phases["k3_tile"]
    achieved = bytes_per_elem * n / (k3_ms * 1e-3) / 1e9
    traffic = NCU_TRAFFIC.get(kernel_hash(), {}).get(args.workload)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not light:
        v, runs, el = time_oracle(kind, box, offsets, match_only)
        cpu = {"value": round(v, 4), "unit": "Gelem/s", "cores": 1, "kind": "oracle",
               "sample": "the full workload (%d elements) x %d runs, %.1f s, single thread"
                         % (n, runs, el)}

    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": round(value, 3), "unit": "Gelem/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": scene_config(args.workload, n, S if S else 1, in_bytes, world),
        "roofline": {"bound": "hbm", "kernel": "k3_tile", "achieved": round(achieved, 1),
                     "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "algorithmic_bytes_per_launch": bytes_per_elem * n},
        "step_roofline_frac": round(bytes_per_elem * n / (ms_step * 1e-3) / 1e9 / peak, 4),
        "phases_ms": {k: round(v, 4) for k, v in phases.items()},
        "graph": {"ms_per_step": round(graph_step_ms, 4),
                  "value": round(world * n / (graph_step_ms * 1e-3) / 1e9, 3),
                  "unit": "Gelem/s", "note": "the same step replayed as one CUDA graph"},
        "per_scene": per_scene,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": (6 if match_only else 8) * K,
        "clocks": clk,
        "kernel_hash": kernel_hash(),
    }


def scene_e2e(torch, binding, dev, kind, box, offsets, match_only, n, K, world):
    """The scene metric end to end through the public API: inputs copied from
    pinned host memory and outputs copied back inside the timed region."""
    kind_h = torch.from_numpy(kind).pin_memory()
    box_h = torch.from_numpy(box).pin_memory()
    off_h = torch.from_numpy(offsets) if offsets is not None else None
    outs_h = (torch.empty(n, dtype=torch.int32).pin_memory(),
              torch.empty(n, dtype=torch.int32).pin_memory(),
              torch.empty(n, 4, dtype=torch.float32).pin_memory())

    if offsets is None:
        # K scenes streamed from pinned host memory: copies in, the pass and
        # copies out of consecutive scenes overlap (HostPipeline); the
        # pipeline's fill and drain are inside the timed region
        e2e_steps = max(3, K)
        pipe = binding.HostPipeline(n, dev, boxes=not match_only)
        outs_p = outs_h[:2] if match_only else outs_h
        boxes_p = None if match_only else [box_h] * e2e_steps
        pipe.run([kind_h], None if match_only else [box_h], [outs_p])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pipe.run([kind_h] * e2e_steps, boxes_p, [outs_p] * e2e_steps)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        del pipe
    else:
        e2e_steps = max(3, min(K, 6))

        def e2e_step():
            binding.bboxes_batched_host(kind_h, box_h, off_h, outs_h)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = kind.nbytes + (0 if match_only else box.nbytes) + (offsets.nbytes if offsets is not None else 0)
    d2h = 4 * n + 4 * n + (0 if match_only else 16 * n)
    return {"value": round(world * n / e2e_s / 1e9, 3), "unit": "Gelem/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "scenes": e2e_steps,
            "how": ("HostPipeline: copies of consecutive scenes overlap the pass; fill and "
                    "drain timed" if offsets is None else
                    "bboxes_batched_host: copies in, the batched pass, copies out")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rw26", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="rw26 only: skip the sub-records of the other configurations")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
