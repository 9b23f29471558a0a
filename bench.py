#!/usr/bin/env python3
"""Benchmark of the polyhedral spatial-join hot path on GB300.

Headline workload (one "step"): the chunked streaming within-tau join of
2,000,000 nuclei-like blobs (R, icosphere subdivision 1/2/3 with SH radial
noise, streamed in 64 chunks of 31,250) against 20,000 vessel-like tubes
(S, 2k-50k facets, 3 LoDs) in a cube of side 5,000, tau = 1.0, with every
tuned feature on: single precision with the FP64 re-decide, unit pruning,
the autotuned LoD schedule, the learned start LoD (fitted on a seed-1
chunk) and per-chunk graph replay.

* ``value``: the chunk arrays resident in device memory when the timed
  region starts (read in place by the set-building kernels); candidate
  object pairs resolved exactly per second.
* ``e2e``: the same join with the chunk arrays in pinned host memory, copied
  to the device inside the timed region through the C ABI (no packing),
  results copied back.
* sub-records under ``configs``: the resident workloads blobs20k,
  knn50k and tubes2k, each tuned against the plain FP64 path on the same
  inputs, so the tuned / plain ratios are measured in the same run.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
       [--workload stream2m|blobs20k|knn50k|tubes2k] [--no-sub]
"""
from __future__ import annotations

import argparse
import copy
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "object-pairs joined/sec & tri-pair tests/sec, tuned vs plain GPU path, exact"
UNIT = "object-pairs/s"
WORKLOADS = {
    "stream2m": ("stream2m: 2,000,000 SH-noised icosphere blobs (LoDs sub 1/2/3 = 80/320/1280 facets) streamed "
                 "in 64 chunks of 31,250 against 20,000 tubes (16-segment swept circles, arc length 50-800, "
                 "2k-50k facets, 3 LoDs), cube side 5,000, within tau = 1.0"),
    "blobs20k": ("blobs20k: R, S = 20,000 SH-noised icosphere blobs each (LoDs sub 1/2/3), cube side 400, "
                 "intersection (tau=0) + within tau=1.0 per step"),
    "knn50k": ("knn50k: R, S = 50,000 sub-3 blobs each, 20-cluster Gaussian mixture (sigma 15) in a cube of "
               "side 1,000, k = 3; proposal fitted on the seed-1 run"),
    "tubes2k": "tubes2k: 2,000 tubes (2k-50k facets, 3 LoDs) x 200,000 sub-3 blobs, cube side 2,320, within tau = 2",
    "voxels_tubes2k": ("voxels_tubes2k: voxel-pair filtering (section 3.2, Algorithms 1 and 2) of the tubes2k box "
                       "candidates (2,000 tubes x 200,000 blobs, within tau = 2), voxels of 2 % of the facets"),
}
WORKLOAD = WORKLOADS["stream2m"]
STREAM = dict(n=2_000_000, chunks=64, tubes=20_000, side=5000.0, tau=1.0)
# FP32 floating-point operations of one triangle-pair test of the refine
# kernel (FMA = 2): 27 differences, 2 x 3 x 22 for the vertex-to-face cases,
# 9 x 45 for the edge-to-edge cases.
FLOPS_PER_TEST = 564
# the single-precision refinement kernel the tuned path runs; the traffic
# counters in profiles/ name it
REFINE_KERNEL_ID = "k_refine<float>+staged+masks+dealt+crossq"
RESULT_BYTES_PER_PAIR = 4 + 4 + 8 + 8 + 8 + 1


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stream2m", choices=list(WORKLOADS),
                    help="the headline line's workload (default: stream2m, the largest)")
    ap.add_argument("--stream-chunks", type=int, default=STREAM["chunks"],
                    help="stream2m: chunks of 31,250 blobs streamed (64 = the full 2,000,000)")
    ap.add_argument("--n", type=int, default=0, help="blobs20k: objects per set (0 = 20,000)")
    ap.add_argument("--no-sub", action="store_true", help="skip the per-config sub-records")
    ap.add_argument("--no-plain", action="store_true", help="skip the FP64 plain-path measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sample-pairs", type=int, default=8,
                    help="cpu_baseline: candidate blob-tube pairs of the oracle sample (about 1.5 core-minutes "
                         "each); the reference arm's steps take half as many")
    ap.add_argument("--options", default=None, help="context options as a JSON object")
    return ap.parse_args(argv)


def alu_peak(nsm: int, mhz: float = 2070.0) -> float:
    """FP32 ALU peak in TFLOP/s: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return nsm * 128 * 2 * mhz * 1e6 / 1e12


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- arrays

def _map_arrays(ms, fn, fields=("verts", "vert_off", "faces", "face_off", "hd", "ph")):
    """A shallow copy of a mesh set with fn applied to its arrays (shared
    arrays stay shared)."""
    out = copy.copy(ms)
    cache = {}

    def f(a):
        if a is None:
            return None
        if id(a) not in cache:
            cache[id(a)] = fn(a)
        return cache[id(a)]

    for name in fields:
        setattr(out, name, [f(a) for a in getattr(ms, name)])
    out.anchor = f(ms.anchor)
    return out


def pinned_copy(ms):
    """The mesh set's arrays copied into pinned host memory."""
    import torch
    return _map_arrays(ms, lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy())


def device_copy(ms):
    """verts, faces, hd, ph, anchor as CUDA tensors (offsets stay host arrays)."""
    import torch
    return _map_arrays(ms, lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda(),
                       fields=("verts", "faces", "hd", "ph"))


def h2d_bytes(ms) -> int:
    seen, tot = set(), 0
    for arrs in (ms.verts, ms.vert_off, ms.faces, ms.face_off, ms.hd, ms.ph, [ms.anchor]):
        for a in arrs:
            if a is None or id(a) in seen:
                continue
            seen.add(id(a))
            tot += a.nbytes
    return tot


# ----------------------------------------------------------------- ranks

def dist_init(backend: str | None = None):
    """Process group of a multi-rank run (one replica of the join per rank,
    no data-path collective).  NCCL on GPUs; gloo when asked (CPU tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend or "nccl")
    return world, rank, local


def _reduce(x: float, world: int, op_name: str) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The slowest rank's time: the job finishes when every replica has."""
    return _reduce(x, world, "MAX")


def sum_over_ranks(x: float, world: int) -> float:
    """Units processed by all ranks together."""
    return _reduce(x, world, "SUM")


# ----------------------------------------------------------------- generation
# every input is drawn in spawned processes before the first CUDA call

def _gen(task):
    from synth import configs
    kind = task[0]
    if kind == "chunk":
        _, c, seed, chunks = task
        return configs.stream2m_R_chunk(c, seed=seed, n=STREAM["n"], chunks=chunks, side=STREAM["side"])
    if kind == "tubes":
        _, n, side, seed, set_id, start, count = task
        return configs.tube_set(n, side, seed, set_id, start=start, count=count)
    if kind == "blobs":
        _, n, side, seed, set_id, start, count, gmm = task
        g = configs.gmm_centres(seed, 20, side) if gmm else None
        return configs.blob_set(n, side, seed, set_id, start=start, count=count, gmm=g)
    raise ValueError(kind)


def _parts(kind, n, side, seed, set_id, pieces, gmm=False):
    step = max(1, (n + pieces - 1) // pieces)
    out = []
    for a in range(0, n, step):
        c = min(step, n - a)
        out.append(("tubes", n, side, seed, set_id, a, c) if kind == "tubes" else
                   ("blobs", n, side, seed, set_id, a, c, gmm))
    return out


def generate(args, seed: int):
    """Every input of this run: name -> MeshSet (or list of chunks)."""
    import multiprocessing as mp
    from synth.mesh import concat
    procs = max(1, min(16, os.cpu_count() or 1))
    plan = {}
    if args.impl == "ours":
        w = args.workload
        if w == "stream2m":
            plan["stream_S"] = _parts("tubes", STREAM["tubes"], STREAM["side"], seed, 1, 4 * procs)
            plan["chunks"] = [("chunk", c, seed, STREAM["chunks"]) for c in range(args.stream_chunks)]
            plan["chunk_seed1"] = [("chunk", 0, seed + 1, STREAM["chunks"])]
        subs = [] if args.no_sub else [x for x in ("blobs20k", "knn50k", "tubes2k") if x != w]
        for name in ([w] if w != "stream2m" else []) + subs:
            if name == "voxels_tubes2k":
                name = "tubes2k"
            if name == "blobs20k":
                n = args.n or 20_000
                side = 400.0 * (n / 20_000) ** (1 / 3)
                plan["b20_R"] = _parts("blobs", n, side, seed, 0, procs)
                plan["b20_S"] = _parts("blobs", n, side, seed, 1, procs)
            elif name == "knn50k":
                for s, tag in ((seed, ""), (seed + 1, "1")):
                    plan["knn_R" + tag] = _parts("blobs", 50_000, 1000.0, s, 0, procs, gmm=True)
                    plan["knn_S" + tag] = _parts("blobs", 50_000, 1000.0, s, 1, procs, gmm=True)
            elif name == "tubes2k":
                plan["t2_R"] = _parts("tubes", 2000, 2320.0, seed, 0, 2 * procs)
                plan["t2_S"] = _parts("blobs", 200_000, 2320.0, seed, 1, 2 * procs)
    tasks = [t for v in plan.values() for t in v]
    if not tasks:
        return {}
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_gen, tasks, chunksize=1)
    out, i = {}, 0
    for k, v in plan.items():
        part = res[i:i + len(v)]
        i += len(v)
        out[k] = part if k == "chunks" else (part[0] if len(part) == 1 else concat(part))
    return out


# ----------------------------------------------------------------- oracle sample

def _mindist(lo, hi, blo, bhi):
    gap = np.maximum(0, np.maximum(blo - hi, lo - bhi))
    return np.sqrt((gap ** 2).sum(-1))


def stream_oracle_sample(target_pairs: int, seed: int = 0):
    """Blobs of the streamed R (from its first chunk) with every tube of S
    within tau of their boxes, chosen from the boxes alone (tubes are
    screened by the box their centre and length bound, then generated
    alone): (R sample, S sample, candidate pairs, description)."""
    from synth import configs
    from synth.mesh import subset
    tau = STREAM["tau"]
    per = STREAM["n"] // STREAM["chunks"]
    c, L = configs.tube_params(STREAM["tubes"], STREAM["side"], seed, 1)
    tlo, thi = c - (L[:, None] / 2 + 2.01), c + (L[:, None] / 2 + 2.01)
    rng = np.random.default_rng(seed)
    blobs = configs.blob_set(STREAM["n"], STREAM["side"], seed, 0, start=0, count=min(per, 4096))
    mb = blobs.mbb().astype(np.float64)
    chosen, tubes, pairs = [], {}, 0
    for r in rng.permutation(blobs.n):
        near = np.nonzero(_mindist(mb[r, :3], mb[r, 3:], tlo, thi) <= tau)[0]
        if len(near) == 0:
            continue
        T = configs.tube_list(STREAM["tubes"], STREAM["side"], seed, 1, near)
        tm = T.mbb().astype(np.float64)
        hit = near[_mindist(mb[r, :3], mb[r, 3:], tm[:, :3], tm[:, 3:]) <= tau]
        if len(hit) == 0:
            continue
        chosen.append(int(r))
        for t in hit:
            tubes[int(t)] = True
        pairs += len(hit)
        if pairs >= target_pairs:
            break
    ids = sorted(tubes)
    Rs = subset(blobs, np.array(sorted(chosen)))
    Ss = configs.tube_list(STREAM["tubes"], STREAM["side"], seed, 1, ids)
    desc = (f"{len(chosen)} blobs of the first chunk with all {pairs} candidate tubes (within tau = 1, "
            f"{len(ids)} tubes), full-resolution facet pairs in FP64")
    return Rs, Ss, pairs, desc


def time_oracle(Rs, Ss, tau, steps, warmup):
    import oracle
    soups = (oracle.soup(Rs), oracle.soup(Ss))
    threads = oracle.default_threads()
    for _ in range(warmup):
        oracle.join_within(Rs, Ss, tau, threads=threads, soups=soups)
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.join_within(Rs, Ss, tau, threads=threads, soups=soups)
    return (time.perf_counter() - t0) / steps, threads


# ----------------------------------------------------------------- reference arm

def reference_arm(args):
    """The CPU oracle as it stands, on a bounded sample of the headline
    workload, on the host cores; only rank 0 works."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    Rs, Ss, pairs, sample = stream_oracle_sample(max(1, args.sample_pairs // 2))
    dt, threads = time_oracle(Rs, Ss, STREAM["tau"], max(1, args.steps), args.warmup)
    v = pairs / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU helpers

def _traffic():
    prof = os.path.join(ROOT, "profiles", "refine_fp32_traffic.json")
    try:
        tr = json.load(open(prof))
        # counters of another kernel (or an older build of it) do not apply
        return tr.get("bytes_per_launch") if tr.get("kernel_id") == REFINE_KERNEL_ID else None
    except (OSError, ValueError):
        return None


def roofline(stats_list, nsm, measured32):
    tests = sum(s["tests_fp32"] for s in stats_list)
    kms = sum(s["refine_ms_fp32"] for s in stats_list)
    peak = alu_peak(nsm)
    ach = tests * FLOPS_PER_TEST / (kms / 1000.0) / 1e12 if kms > 0 else 0.0
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": _traffic(),
            "kernel": "k_refine<float> (single-precision refinement, facet-ball culling; full-resolution steps "
                      "include their k_unit_masks pre-pass in the timed window)",
            "peak_kind": f"derived: {nsm} SMs x 128 FP32 lanes x 2 flops x 2.070 GHz",
            "measured_fma_peak": measured32, "frac_of_measured": ach / measured32 if measured32 else None,
            "flops_per_test": FLOPS_PER_TEST, "kernel_ms": kms, "tests": tests,
            "kernel_timing": "CUDA events around each refinement launch on its stream, direct (non-graph) steps"}


def timed(ctx, stream, fn, steps):
    """Run fn() steps times between CUDA events on stream (synchronized on
    both sides); returns (ms, [stats])."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    e0.record(stream)
    for _ in range(steps):
        fn()
        out.append(ctx.stats())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def host_timed(fn, steps):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = [fn() for _ in range(steps)]
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1000.0, out


# ----------------------------------------------------------------- headline: stream2m

def stream_headline(args, data, ctx, pj, stream, world, rank, nsm, measured32):
    import torch
    S = data["stream_S"]
    chunks = data["chunks"]
    n_total = sum(c.n for c in chunks)
    gS = ctx.load_set(S)
    # learned start LoD: fitted on a seed-1 chunk against S
    g1 = ctx.load_set(data["chunk_seed1"])
    rmse = ctx.mlp_fit(g1, gS, pj.WITHIN, tau=STREAM["tau"], max_pairs=200_000, epochs=30, seed=1)
    g1.free()
    dev_chunks = [device_copy(c) for c in chunks]
    gR = ctx.load_set_streamed(n_total, len(chunks), lambda c: dev_chunks[c])
    tau = STREAM["tau"]
    tuned = dict(prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE | pj.USE_MLP | pj.USE_GRAPH)
    direct = dict(prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE | pj.USE_MLP)

    def join(R, mode):
        return ctx.join(R, gS, pj.WITHIN, tau=tau, stream=stream.cuda_stream, **mode)

    for _ in range(max(3, args.warmup)):
        join(gR, tuned)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    # the NVTX range marks the timed steps for a profiler's launch list
    torch.cuda.nvtx.range_push("timed")
    ms, stats = timed(ctx, stream, lambda: join(gR, tuned), args.steps)
    torch.cuda.nvtx.range_pop()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(ms, world)
    pairs = sum(s["candidates"] for s in stats)
    value = sum_over_ranks(pairs, world) / (ms / 1000.0)
    tests = sum(s["tests_fp32"] + s["tests_fp64"] for s in stats)
    launches = int(sum(s["launches"] for s in stats))
    join(gR, direct)   # tunes the direct key first, so the measured pass runs no trials
    _, kst = timed(ctx, stream, lambda: join(gR, direct), 1)
    roof = roofline(kst, nsm, measured32)
    last = stats[-1]
    config = {"workload": WORKLOAD, "objects_R": n_total, "chunks": len(chunks), "objects_S": S.n,
              "precision": "fp32 + fp64 re-decide",
              "flags": "TILE_PRUNE | AUTOTUNE | USE_MLP | USE_GRAPH", "candidate_pairs_per_step": pairs // args.steps,
              "results_per_step": last["results"], "proposal_rmse_log1p": rmse,
              "inputs": "chunk arrays resident in device memory (read in place), S resident; "
                        f"{h2d_bytes(chunks[0]) * len(chunks) / 1e9:.1f} GB of raw chunk arrays, larger than L2",
              "l2": "inputs larger than L2 (129 MB): every step reads all chunks"}
    gR.free()
    gR._cb = gR._keep = None
    dev_chunks.clear()
    torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        pin_chunks = [pinned_copy(c) for c in chunks]
        gRp = ctx.load_set_streamed(n_total, len(pin_chunks), lambda c: pin_chunks[c])
        # warm passes: the first copies from freshly pinned pages run well
        # below the link rate
        for _ in range(3):
            join(gRp, tuned)
        ke = max(1, min(args.steps, 5))
        e2e_stats = []

        e2e_ms = []

        def e2e_step():
            t0 = time.perf_counter()
            res = join(gRp, tuned)
            e2e_ms.append((time.perf_counter() - t0) * 1000.0)
            st = ctx.stats()
            e2e_stats.append(st)
            return st["candidates"], res.n, st["bytes_h2d"], st.get("h2d_gbs", 0.0)

        ems, outs = host_timed(e2e_step, ke)
        ems = max_over_ranks(ems, world)
        e2e = {"value": sum_over_ranks(sum(o[0] for o in outs), world) / (ems / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(sum(o[2] for o in outs) / ke),
               "d2h_bytes_per_step": int(sum(o[1] for o in outs) / ke * RESULT_BYTES_PER_PAIR),
               "ms_per_step": ems / ke, "h2d_gbs_during_join": statistics.median(o[3] for o in outs),
               "host_read_bytes_max_per_step": e2e_stats[-1].get("bytes_host_read_max"),
               "join_call_ms": e2e_ms, "join_ms_total": [x.get("ms_total") for x in e2e_stats],
               "how": "pj_join of the streamed R with every chunk array in pinned host memory (copied by the "
                      "library's copy stream without packing, overlapped with the previous chunk's join; the "
                      "hd / ph of the middle LoD read in place by the kernels for the objects that reach it) + "
                      "result copy, host clock; 3 untimed warm passes",
               "last_step_stats": {k: e2e_stats[-1].get(k) for k in (
                   "bytes_h2d", "bytes_host_read_max", "ms_h2d", "h2d_gbs", "ms_fill", "ms_pack", "ms_wait_loader",
                   "ms_build", "ms_join",
                   "ms_filter", "ms_total", "graph_replays", "graph_captures")}}
        gRp.free()
        gRp._cb = gRp._keep = None
        pin_chunks.clear()
        # the pinned host-to-device copy rate of this machine: 1 GiB, best of 5
        h = torch.empty(1 << 28, dtype=torch.float32).pin_memory()
        dd = torch.empty_like(h, device="cuda")
        best = 0.0
        for _ in range(5):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            dd.copy_(h, non_blocking=True)
            a1.record()
            torch.cuda.synchronize()
            best = max(best, h.numel() * 4 / (a0.elapsed_time(a1) / 1000.0) / 1e9)
        e2e["h2d_peak_gbs"] = best
        del h, dd

    plain = None
    if not args.no_plain:
        from synth.mesh import subset
        part = subset(chunks[0], np.arange(min(4096, chunks[0].n)))
        gP = ctx.load_set(part)
        join(gP, direct)
        pms, pst = host_timed(lambda: (join(gP, dict(prec=pj.FP64, flags=0)), ctx.stats())[1], 1)
        tms, tst = host_timed(lambda: (join(gP, direct), ctx.stats())[1], 3)
        tms /= 3
        plain = {"inputs": f"the first {part.n} blobs of chunk 0 against all of S",
                 "value": pst[0]["candidates"] / (pms / 1000.0), "ms": pms, "dtype": "f64",
                 "tri_tests_per_s": (pst[0]["tests_fp64"] + pst[0]["tests_fp32"]) / (pms / 1000.0),
                 "tuned_same_inputs": {"value": tst[0]["candidates"] / (tms / 1000.0), "ms": tms},
                 "speedup": (tst[0]["candidates"] / tms) / (pst[0]["candidates"] / pms)}
        gP.free()
    gS.free()
    return {"value": value, "ms": ms, "tests": tests, "launches": launches, "roofline": roof, "config": config,
            "e2e": e2e, "plain": plain, "clocks": clk, "last_stats": {k: v for k, v in last.items() if k != "steps"}}


# ----------------------------------------------------------------- resident workloads

def blobs20k_record(args, data, ctx, pj, stream, nsm, measured32, steps):
    R, S = data["b20_R"], data["b20_S"]
    gR, gS = ctx.load_set(R), ctx.load_set(S)
    tuned = dict(prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE | pj.USE_GRAPH)
    direct = dict(prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE)

    def cands(sts):
        return sum(s["candidates"] for s in sts)

    for _ in range(3):
        _two(ctx, gR, gS, pj, stream, tuned)
    sts = []
    ms, _ = timed(ctx, stream, lambda: sts.extend(_two(ctx, gR, gS, pj, stream, tuned)), steps)
    kst = []
    _two(ctx, gR, gS, pj, stream, direct)   # tunes the direct keys first
    timed(ctx, stream, lambda: kst.extend(_two(ctx, gR, gS, pj, stream, direct)), 2)
    rec = {"workload": WORKLOADS["blobs20k"], "value": cands(sts) / (ms / 1000.0), "ms_per_step": ms / steps,
           "tri_tests_per_s": sum(s["tests_fp32"] + s["tests_fp64"] for s in sts) / (ms / 1000.0),
           "flags": "TILE_PRUNE | AUTOTUNE | USE_GRAPH", "roofline": roofline(kst, nsm, measured32)}
    if not args.no_plain:
        pst = []
        pms, _ = timed(ctx, stream, lambda: pst.extend(_two(ctx, gR, gS, pj, stream, dict(prec=pj.FP64, flags=0))),
                       1)
        rec["plain"] = {"value": cands(pst) / (pms / 1000.0), "ms_per_step": pms, "dtype": "f64",
                        "inputs": "the same sets"}
        rec["speedup_vs_plain"] = rec["value"] / rec["plain"]["value"]
    gR.free()
    gS.free()
    return rec


def _two(ctx, gR, gS, pj, stream, mode):
    out = []
    for t in (0.0, 1.0):
        ctx.join(gR, gS, pj.WITHIN, tau=t, stream=stream.cuda_stream, **mode)
        out.append(ctx.stats())
    return out


def knn50k_record(args, data, ctx, pj, stream, nsm, measured32, steps):
    from synth.mesh import subset
    a, b = ctx.load_set(data["knn_R1"]), ctx.load_set(data["knn_S1"])
    rmse = ctx.mlp_fit(a, b, pj.KNN, k=3, max_pairs=200_000, epochs=30, seed=1)
    a.free()
    b.free()
    R, S = data["knn_R"], data["knn_S"]
    gR, gS = ctx.load_set(R), ctx.load_set(S)
    tuned = dict(prec=pj.FP32, flags=pj.TILE_PRUNE | pj.USE_MLP)

    def run(Rset, mode):
        ctx.join(Rset, gS, pj.KNN, k=3, stream=stream.cuda_stream, **mode)

    run(gR, tuned)
    ms, sts = timed(ctx, stream, lambda: run(gR, tuned), steps)
    rec = {"workload": WORKLOADS["knn50k"], "value": sum(s["candidates"] for s in sts) / (ms / 1000.0),
           "ms_per_step": ms / steps,
           "tri_tests_per_s": sum(s["tests_fp32"] + s["tests_fp64"] for s in sts) / (ms / 1000.0),
           "flags": "TILE_PRUNE | USE_MLP", "proposal_rmse_log1p": rmse, "roofline": roofline(sts, nsm, measured32)}
    _, nst = timed(ctx, stream, lambda: run(gR, dict(prec=pj.FP32, flags=pj.TILE_PRUNE)), 1)
    rec["without_proposal"] = {"tests": nst[0]["tests_fp32"] + nst[0]["tests_fp64"],
                               "with_proposal_tests": sts[-1]["tests_fp32"] + sts[-1]["tests_fp64"]}
    if not args.no_plain:
        gP = ctx.load_set(subset(R, np.arange(2000)))
        pms, pst = host_timed(lambda: (run(gP, dict(prec=pj.FP64, flags=0)), ctx.stats())[1], 1)
        run(gP, tuned)
        tms, tst = host_timed(lambda: (run(gP, tuned), ctx.stats())[1], 3)
        tms /= 3
        rec["plain"] = {"inputs": "the first 2,000 objects of R against all of S (the full plain join is minutes "
                                  "of FP64 work)", "value": pst[0]["candidates"] / (pms / 1000.0), "ms": pms,
                        "dtype": "f64", "tuned_same_inputs": {"value": tst[0]["candidates"] / (tms / 1000.0),
                                                              "ms": tms}}
        rec["speedup_vs_plain"] = (tst[0]["candidates"] / tms) / (pst[0]["candidates"] / pms)
        gP.free()
    gR.free()
    gS.free()
    return rec


def tubes2k_record(args, data, ctx, pj, stream, nsm, measured32, steps):
    from synth.mesh import subset
    R, S = data["t2_R"], data["t2_S"]
    gR, gS = ctx.load_set(R), ctx.load_set(S)
    tuned = dict(prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE | pj.USE_GRAPH)
    direct = dict(prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE)

    def run(Rset, mode):
        ctx.join(Rset, gS, pj.WITHIN, tau=2.0, stream=stream.cuda_stream, **mode)

    for _ in range(3):
        run(gR, tuned)
    ms, sts = timed(ctx, stream, lambda: run(gR, tuned), steps)
    run(gR, direct)   # tunes the direct key first
    _, kst = timed(ctx, stream, lambda: run(gR, direct), 1)
    rec = {"workload": WORKLOADS["tubes2k"], "value": sum(s["candidates"] for s in sts) / (ms / 1000.0),
           "ms_per_step": ms / steps,
           "tri_tests_per_s": sum(s["tests_fp32"] + s["tests_fp64"] for s in sts) / (ms / 1000.0),
           "flags": "TILE_PRUNE | AUTOTUNE | USE_GRAPH", "roofline": roofline(kst, nsm, measured32)}
    if not args.no_plain:
        gP = ctx.load_set(subset(R, np.arange(100)))
        pms, pst = host_timed(lambda: (run(gP, dict(prec=pj.FP64, flags=0)), ctx.stats())[1], 1)
        run(gP, direct)
        tms, tst = host_timed(lambda: (run(gP, direct), ctx.stats())[1], 3)
        tms /= 3
        rec["plain"] = {"inputs": "the first 100 tubes of R against all of S (the full plain join is many "
                                  "minutes of FP64 work)", "value": pst[0]["candidates"] / (pms / 1000.0),
                        "ms": pms, "dtype": "f64",
                        "tuned_same_inputs": {"value": tst[0]["candidates"] / (tms / 1000.0), "ms": tms}}
        rec["speedup_vs_plain"] = (tst[0]["candidates"] / tms) / (pst[0]["candidates"] / pms)
        gP.free()
    gR.free()
    gS.free()
    return rec


def _object_boxes(ms):
    """[n, 6] boxes of every object's original-LoD vertices (host)."""
    L = ms.n_lods - 1
    v = ms.verts[L].astype(np.float64)
    vo = np.asarray(ms.vert_off[L], np.int64)
    return np.concatenate([np.minimum.reduceat(v, vo[:-1]), np.maximum.reduceat(v, vo[:-1])], axis=1)


def box_candidates(R, S, tau):
    """Object pairs whose boxes lie within tau, grouped by r, s ascending: a
    sweep along x over S's boxes (bench input for the voxel filter)."""
    a, b = _object_boxes(R), _object_boxes(S)
    order = np.argsort(b[:, 0], kind="stable")
    slo = b[order, 0]
    ext = float((b[:, 3] - b[:, 0]).max()) if len(b) else 0.0
    prs, pss = [], []
    for r in range(len(a)):
        i0 = np.searchsorted(slo, a[r, 0] - tau - ext, side="left")
        i1 = np.searchsorted(slo, a[r, 3] + tau, side="right")
        c = order[i0:i1]
        bb = b[c]
        g = np.maximum(0.0, np.maximum(bb[:, :3] - a[r, 3:], a[r, :3] - bb[:, 3:]))
        c = np.sort(c[(g * g).sum(1) <= tau * tau])
        prs.append(np.full(len(c), r, np.int32))
        pss.append(c.astype(np.int32))
    return np.concatenate(prs), np.concatenate(pss)


VOXEL_KEYS = ("voxel_pairs_per_s", "inputs", "voxels", "kept", "kept_frac", "decided", "step_ms", "f64",
              "speedup_f32_vs_f64")
VOXEL_BATCH = 1 << 27     # voxel pairs per pj_voxel_filter call (2 GB of bounds, 1 GB of survivors)
# double-precision operations of one voxel pair's bounds in k_vp_bound:
# MINDIST 6 differences, 6 maxima, 3 squares, 2 sums, 1 root; anchor
# distance 3 differences, 3 squares, 2 sums, 1 root
VOXEL_OPS = 27


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) of this machine's GPUs, else the
    fallback figure; and which one it is."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def voxels_tubes2k_record(args, data, ctx, pj, stream, nsm, measured32, steps):
    import torch
    R, S = data["t2_R"], data["t2_S"]
    tau = 2.0
    vctx = pj.Context(torch.cuda.current_device(), {"voxels": 1})
    t0 = time.perf_counter()
    gR, gS = vctx.load_set(R), vctx.load_set(S)
    load_s = time.perf_counter() - t0
    kr = np.diff(vctx.voxel_offsets(gR))
    ks = np.diff(vctx.voxel_offsets(gS))
    pr, ps = box_candidates(R, S, tau)
    sz = kr[pr].astype(np.int64) * ks[ps]
    cum = np.cumsum(sz)
    n = int(np.searchsorted(cum, VOXEL_BATCH, side="right"))   # pairs of the first batch
    n = max(1, min(n, len(pr)))
    cap = int(cum[n - 1])
    # algorithmic bytes of one k_vp_bound launch: the bounds written (2 x 8 B
    # per voxel pair), each pair's voxel records read once (box 24 B + anchor
    # 12 B per voxel), ids, offsets, object-pair bounds and status (65 B)
    bound_bytes = 16 * cap + 36 * int(kr[pr[:n]].sum() + ks[ps[:n]].sum()) + 65 * n
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dpr, dps = dev(pr[:n]), dev(ps[:n])
    out = {"op_lb": torch.empty(n, dtype=torch.float64, device="cuda"),
           "op_ub": torch.empty(n, dtype=torch.float64, device="cuda"),
           "status": torch.empty(n, dtype=torch.uint8, device="cuda"),
           "vp_off": torch.empty(n + 1, dtype=torch.int64, device="cuda"),
           "vp_lb": torch.empty(cap, dtype=torch.float64, device="cuda"),
           "vp_ub": torch.empty(cap, dtype=torch.float64, device="cuda"),
           "kept_off": torch.empty(n + 1, dtype=torch.int64, device="cuda"),
           "kept": torch.empty(2 * cap, dtype=torch.int32, device="cuda")}
    ptr = {k: v.data_ptr() for k, v in out.items()}

    def measure(prec):
        run = lambda: vctx.voxel_filter(gR, gS, dpr.data_ptr(), dps.data_ptr(), n, tau, ptr, cap, prec=prec,
                                        stream=stream.cuda_stream)
        for _ in range(3):
            kept = run()
        ms, sts = timed(vctx, stream, run, steps)
        status = out["status"].cpu().numpy()
        return {"ms": ms, "kept": kept, "bound_ms": sum(x["ms_bound"] for x in sts) / len(sts),
                "step_ms": {k: sts[-1][k] for k in ("ms_sizes", "ms_bound", "ms_count", "ms_scan", "ms_compact")},
                "decided": {"results": int((status == 1).sum()), "pruned": int((status == 2).sum()),
                            "undecided": int((status == 0).sum())}}

    f32 = measure(pj.FP32)
    f64 = measure(pj.FP64)
    peak, kind = hbm_peak()
    gbs = bound_bytes / (f32["bound_ms"] / 1000.0) / 1e9
    peak64 = vctx.fma_peak(True) / 1000.0
    ach64 = cap * VOXEL_OPS / (f64["bound_ms"] / 1000.0) / 1e12
    rec = {"workload": WORKLOADS["voxels_tubes2k"], "value": n * steps / (f32["ms"] / 1000.0),
           "ms_per_step": f32["ms"] / steps, "dtype": "f32",
           "voxel_pairs_per_s": cap * steps / (f32["ms"] / 1000.0), "tri_tests_per_s": None,
           "flags": "pj_voxel_filter, PJ_PREC_FP32_REDECIDE (outward-rounded bounds), tau = 2",
           "inputs": f"the first {n:,} of {len(pr):,} box candidates (r ascending), {cap:,} voxel pairs "
                     f"(one call's batch of at most {VOXEL_BATCH:,}); outputs larger than L2",
           "voxels": {"R": int(kr.sum()), "S": int(ks.sum()), "load_s_with_voxels": load_s},
           "kept": f32["kept"], "kept_frac": f32["kept"] / cap, "decided": f32["decided"], "step_ms": f32["step_ms"],
           "f64": {"value": n * steps / (f64["ms"] / 1000.0), "ms_per_step": f64["ms"] / steps,
                   "voxel_pairs_per_s": cap * steps / (f64["ms"] / 1000.0), "kept": f64["kept"],
                   "decided": f64["decided"], "step_ms": f64["step_ms"],
                   "roofline": {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                                "frac": ach64 / peak64, "kernel": "k_vp_bound<double>",
                                "peak_kind": "measured FP64 FMA throughput (pj_fma_peak, FMA = 2 flops)",
                                "ops_per_voxel_pair": VOXEL_OPS, "kernel_ms": f64["bound_ms"]}},
           "speedup_f32_vs_f64": f64["ms"] / f32["ms"],
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "traffic": None, "kernel": "k_vp_bound<float> (Algorithm 1, outward-rounded single precision)",
                        "peak_kind": f"{kind} HBM copy bandwidth", "bytes_per_launch": bound_bytes,
                        "kernel_ms": f32["bound_ms"],
                        "kernel_timing": "CUDA events around the launch inside pj_voxel_filter"}}
    gR.free()
    gS.free()
    vctx.close()
    return rec


SUB_RECORDS = {"blobs20k": blobs20k_record, "knn50k": knn50k_record, "tubes2k": tubes2k_record,
               "voxels_tubes2k": voxels_tubes2k_record}


# ----------------------------------------------------------------- our arm

def ours_arm(args):
    world, rank, local = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))
    data = generate(args, seed=rank)        # weak scaling: one independent batch per rank
    cpu_sample = None
    if world == 1 and not args.no_cpu and args.workload == "stream2m":
        cpu_sample = stream_oracle_sample(max(1, args.sample_pairs))
    import torch
    from paper_2604_19982_gb300 import pj
    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    opts = {"refine_variant": 1}
    opts.update(json.loads(args.options) if args.options else {})
    ctx = pj.Context(local, opts)
    stream = torch.cuda.Stream()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    measured32 = ctx.fma_peak(False) / 1000.0

    if args.workload == "stream2m":
        h = stream_headline(args, data, ctx, pj, stream, world, rank, nsm, measured32)
        for k in ("stream_S", "chunks", "chunk_seed1"):
            data.pop(k, None)
        line = {"metric": METRIC, "value": h["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": h["ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": h["config"], "tri_tests_per_s": h["tests"] / (h["ms"] / 1000.0),
                "plain": h["plain"], "speedup_vs_plain": h["plain"]["speedup"] if h["plain"] else None,
                "roofline": h["roofline"], "e2e": h["e2e"], "gpu_launches": h["launches"], "clocks": h["clocks"],
                "last_step_stats": h["last_stats"]}
    else:
        fn = SUB_RECORDS[args.workload]
        clocks = ClockSampler(local)
        clocks.start()
        rec = fn(args, data, ctx, pj, stream, nsm, measured32, args.steps)
        clk = clocks.stop()
        line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": rec["workload"], "flags": rec["flags"]},
                "tri_tests_per_s": rec["tri_tests_per_s"], "plain": rec.get("plain"),
                "speedup_vs_plain": rec.get("speedup_vs_plain"), "roofline": rec["roofline"], "e2e": None,
                "gpu_launches": None, "clocks": clk}
        line["dtype"] = rec.get("dtype", "f32")
        line.update({k: rec[k] for k in VOXEL_KEYS if k in rec})
    ctx.close()
    if not args.no_sub:
        # each workload in a context of its own (workspace, graphs and tuned
        # choices of one workload do not weigh on the next)
        subs = {}
        for name, fn in SUB_RECORDS.items():
            if name == args.workload:
                continue
            c = pj.Context(local, opts)
            subs[name] = fn(args, data, c, pj, stream, nsm, measured32, max(1, min(args.steps, 5)))
            c.close()
        line["configs"] = subs
    if cpu_sample is not None:
        Rs, Ss, pairs, sample = cpu_sample
        dt, threads = time_oracle(Rs, Ss, STREAM["tau"], 1, 0)
        line["cpu_baseline"] = {"value": pairs / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": sample + f", {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
