"""Benchmark: moved-point updates per second of the kinetic Delaunay step.

Headline workload (the largest one that fits one GPU): 16,000,000 integer points on
[0, 2^24)^2, a 32-component Gaussian mixture (sigma 2^18) plus 5 % on an exact lattice
(cocircular quadruples), 256 x 256 equal-area partitions, 1-16 moved points per
partition per step (about 165,000 moves), each move 1-8 units right/left/up/down,
synthetic and seeded.  A step is one call of kdt_step: bucket the moves per partition,
delete + re-insert each moved point, certify the touched triangles.

Printed JSON line (rank 0), for the headline workload:
  value        updates/s with the moves already resident in HBM: CUDA events around
               every kdt_step on a handle without instrumentation (the 1.15 GB store is
               larger than L2, so no flush is needed);
  e2e          the same metric through the C ABI with the moves in pinned host memory
               (host->device copy and the status read inside the timed region);
  roofline     the kinetic kernel's algorithmic bytes per update (from the degrees of
               the moved points in the oracle's triangulations before and after a step)
               x moves per launch / its event-timed duration (a separate instrumented
               pass over the same moves), against the measured HBM copy bandwidth;
  comparators  the GPU full rebuild, quad-tree partitions and the two in-place variants
               on the same steps and GPU;
  workloads    the 1e6-point uniform workload (c2), the 512-instance batch (c4, plain,
               with the learned proposal, one handle per instance, rebuild), and the
               learned proposal on c2 (c5), each with its own value and comparators;
  cpu_baseline the CPU oracle rebuilding one step's point set on every host core.

--workload c2|c3|c4|c5 prints that workload's line alone.  --impl reference times the
oracle alone (the deliberately slow reference).  Under torchrun (N > 1) every rank
advances its own independent instance of the headline workload (replicas; "weak"
scaling) and value = all ranks' updates / max-over-ranks time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "moved-point updates/sec (1 GB300, bit-exact) vs plain GPU update and full rebuild"
WORKLOADS = {
    "c2": ("1e6 uniform points on [0,2^24)^2, 64x64 partitions, 4096 moves/step "
           "(1 per partition, 1-8 units R/L/U/D)"),
    "c3": ("16e6 points: 32-Gaussian mixture (sigma 2^18) + 5 % lattice on [0,2^24)^2, "
           "256x256 partitions, 1-16 moves per partition per step (1-8 units R/L/U/D)"),
    "c4": ("512 instances, sizes log-uniform 1e3-2e5 (seeded), uniform on [0,2^20)^2, "
           "~256 points per partition, 1-4 moves per partition per step (1-8 units)"),
    "c5": ("1e6 uniform points on [0,2^24)^2, 64x64 partitions, 4096 moves/step, "
           "learned locate proposal on"),
}

# Algorithmic bytes of one update, from the degrees k_old and k_new of the moved point
# before and after the move: star triangles read and written (vertices + neighbours,
# 32 B each), the outer neighbours' back-pointers (16 B each) and the coordinates of
# the star's vertices and of p (8 B each).  At the mean planar degree k = 6: 688 B.
def bytes_per_update(k_old, k_new):
    return 32.0 * (k_old + k_new) + 16.0 * (k_old + k_new) + 8.0 * (k_old + k_new + 2)


BYTES_K6 = bytes_per_update(6, 6)

# DRAM bytes (read + write) per moved point of one k_kinetic launch, from ncu's
# dram__bytes_read.sum + dram__bytes_write.sum (profiles/), valid only for the kernel
# sources it was taken on (their SHA-256 prefix) and the workload it was taken on; the
# bench line reports it scaled to the launch's moves, null otherwise.
KINETIC_TRAFFIC = {
    # 16e6-point workload, 3 launches of 165,068 moves: 441.5, 440.9, 438.7 MB (the
    # triangle store as 32-byte records)
    "c3": {"sources": "505f12924c6ce36f", "bytes_per_move": 2668.0},
    # 1e6-point workload, 2 launches of 4,096 moves: 15.64, 15.69 MB, taken with the
    # two halves of a triangle in separate arrays (no capture of the current sources:
    # the traffic is reported as null)
    "c2": {"sources": "0a5e0b49bcda6ab7", "bytes_per_move": 3824.0},
}


def kernel_sources_hash():
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2308_06484_gb300", "csrc", "*.cu*"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kinetic_traffic(workload, moves_per_launch):
    t = KINETIC_TRAFFIC.get(workload)
    if not t or kernel_sources_hash() != t["sources"]:
        return None
    return t["bytes_per_move"] * moves_per_launch


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.25)  # the first sample lands before the timed region
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(local_updates, local_seconds, local_e2e_seconds, group=None):
    """Whole-job numbers: sum of updates over ranks, max of times over ranks."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return local_updates, local_seconds, local_e2e_seconds
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    u = torch.tensor([float(local_updates)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(local_seconds), float(local_e2e_seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(t[0].item()), float(t[1].item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- the oracle leg
#
# Only this leg (and --impl reference) runs the oracle.  One step's rebuild of a large
# point set is split into the tiles of a T x T division of the domain, one oracle call
# per tile, the tiles spread over every host core: the same Bowyer-Watson work as one
# rebuild of the whole set (without the seams), in parallel.

def _tiles(xy, bits, T):
    """Index arrays of the points in each tile of a T x T division of [0, 2^bits)^2."""
    xy = np.asarray(xy, dtype=np.int64)
    t = ((xy[:, 1] * T) >> bits) * T + ((xy[:, 0] * T) >> bits)
    order = np.argsort(t, kind="stable")
    cuts = np.searchsorted(t[order], np.arange(T * T + 1))
    return [order[cuts[i]:cuts[i + 1]] for i in range(T * T)]


def _oracle_tiles(xy, tiles, threads):
    """Oracle rebuild of every tile with >= 3 points on `threads` threads; returns
    (wall seconds, {tile: triangles in global ids})."""
    import oracle
    oracle.lib()
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    out = {}

    def one(i):
        idx = tiles[i]
        if idx.shape[0] < 3:
            return i, None
        try:
            tri = oracle.delaunay(xy[idx])
        except oracle.OracleError:
            return i, None  # a degenerate tile (all collinear): nothing to rebuild
        return i, idx[tri]

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as pool:
        for i, r in pool.map(one, range(len(tiles))):
            out[i] = r
    return time.perf_counter() - t0, out


def _degrees(tri_global, n):
    """Vertex degrees in a triangulation closed by ghost triangles: finite triangles at
    each vertex, plus 2 for a hull vertex (its two ghost triangles)."""
    deg = np.bincount(tri_global.ravel(), minlength=n).astype(np.int64)
    e = np.concatenate([tri_global[:, [0, 1]], tri_global[:, [1, 2]], tri_global[:, [2, 0]]]).astype(np.int64)
    fwd = e[:, 0] * n + e[:, 1]
    rev = e[:, 1] * n + e[:, 0]
    boundary = ~np.isin(fwd, rev)
    hull = np.zeros(n, dtype=bool)
    hull[e[boundary, 0]] = True
    deg[hull] += 2
    return deg


def oracle_leg(xy_before, xy_after, moves, bits, tiles_per_side, threads, model_tiles):
    """The CPU baseline and the bytes-per-update model of one step.

    Baseline: the oracle rebuilds the point set before the step (tiled, every core);
    updates/s = moves of the step / wall time.  Model: for the moves whose old and new
    positions lie in the inner half of one of `model_tiles` tiles (so their stars do not
    reach the tile's border), k_old and k_new are their degrees in the oracle's
    triangulations of that tile before and after the step."""
    n = xy_before.shape[0]
    T = tiles_per_side
    tb = _tiles(xy_before, bits, T)
    wall, tri_b = _oracle_tiles(xy_before, tb, threads)
    ids = moves[:, 0].astype(np.int64)
    side = (1 << bits) // T
    old = xy_before[ids].astype(np.int64)
    new = xy_after[ids].astype(np.int64)
    tile_old = (old[:, 1] // side) * T + old[:, 0] // side
    tile_new = (new[:, 1] // side) * T + new[:, 0] // side
    lo = side // 4

    def inner(p):
        r = p % side
        return (r[:, 0] >= lo) & (r[:, 0] < side - lo) & (r[:, 1] >= lo) & (r[:, 1] < side - lo)

    ok = (tile_old == tile_new) & inner(old) & inner(new)
    # the tiles with the most such moves, rebuilt after the step
    cand = np.bincount(tile_old[ok], minlength=T * T)
    pick = [int(i) for i in np.argsort(-cand, kind="stable")[:model_tiles] if cand[i] > 0 and tri_b.get(int(i)) is not None]
    ta = _tiles(xy_after, bits, T)
    _, tri_a = _oracle_tiles(xy_after, [ta[i] if i in pick else ta[i][:0] for i in range(T * T)], threads)
    ko, kn = [], []
    for i in pick:
        if tri_a.get(i) is None:
            continue
        db = _degrees(tri_b[i], n)
        da = _degrees(tri_a[i], n)
        sel = ids[ok & (tile_old == i)]
        ko.append(db[sel])
        kn.append(da[sel])
    ko = np.concatenate(ko) if ko else np.zeros(0, np.int64)
    kn = np.concatenate(kn) if kn else np.zeros(0, np.int64)
    model = {"bytes_per_update": float(np.mean(bytes_per_update(ko, kn))) if ko.size else BYTES_K6,
             "mean_k_old": float(ko.mean()) if ko.size else None,
             "mean_k_new": float(kn.mean()) if kn.size else None,
             "moves_sampled": int(ko.size),
             "how": ("degrees of the moved points in the oracle's triangulations before and after the step "
                     "(moves inside the inner half of %d of %d tiles)" % (len(pick), T * T))}
    base = {"value": moves.shape[0] / wall, "unit": "updates/s", "cores": threads, "kind": "oracle",
            "sample": ("one oracle rebuild of the %d-point set of a step, as %d tiles (%dx%d division of the "
                       "domain) on %d threads: %.1f s wall" % (n, T * T, T, T, threads, wall))}
    return base, model


# ---------------------------------------------------------------- GPU helpers

def draw_moves(w, nsteps, at):
    """The move lists of nsteps steps, and (positions before, positions after, moves) of
    step `at` (for the oracle leg)."""
    mv = []
    around = None
    for i in range(nsteps):
        before = w.positions if i == at else None
        mv.append(w.next_moves())
        if i == at:
            around = (before, w.positions, mv[-1])
    return mv, around


def _events(k):
    import torch
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]


def timed_steps(tri, moves, warmup, flush=None, stepper=None):
    """Event-timed steps: warm-up on moves[:warmup], then one (start, end) event pair
    around every later step (flush written between steps when given, outside the
    events).  Returns the per-step milliseconds."""
    import torch
    step = stepper or tri.step
    for i in range(warmup):
        step(moves[i])
    tri.reset_stats()
    ev = _events(len(moves) - warmup)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(ev):
        a.record()
        step(moves[warmup + k])
        b.record()
        if flush is not None:
            flush.zero_()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def kernel_pass(make_tri, xy0, moves, warmup, flush=None, stepper=None):
    """The same steps on an instrumented handle (timing = 1): mean event-timed duration
    of the kinetic kernel, and the handle's counters."""
    tri = make_tri(timing=1)
    tri.build(xy0)
    timed_steps(tri, moves, warmup, flush, stepper=(lambda m: stepper(tri, m)) if stepper else None)
    st = tri.stats()
    tri.close()
    return st["kinetic_kernel_ms"] / max(1, st["kinetic_kernel_timed"]), st


def roofline(bpu, moves_per_launch, kernel_ms, traffic):
    peak, kind = measured_peaks()
    achieved = bpu * moves_per_launch / (kernel_ms / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_kinetic", "kernel_ms": kernel_ms, "bytes_per_update": bpu,
            "moves_per_launch": moves_per_launch, "peak_kind": kind + " (hbm_gbs, copy bandwidth)"}


def base_line(value, steps, warmup, sec, workload, extra_cfg):
    cfg = {"workload": WORKLOADS[workload]}
    cfg.update(extra_cfg)
    return {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": 1000.0 * sec / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+int128 exact (fp32 filter)",
            "data": "synthetic", "config": cfg}


# ---------------------------------------------------------------- c3 (headline)

def run_c3(args, rank=0, ws=1, local=0, comparators=True):
    """The 16e6-point mixture + lattice workload at full size."""
    import torch
    from paper_2308_06484_gb300 import kdt, workloads as W
    dev = torch.device("cuda", local)
    w = W.c3(seed=3 + 1000 * rank)
    xy0_h = w.positions
    xy0 = torch.from_numpy(xy0_h).to(dev)
    nsteps = args.warmup + args.steps
    mv_h, around = draw_moves(w, nsteps, args.warmup)
    xy_end = w.positions
    moves = [torch.from_numpy(m).to(dev) for m in mv_h]
    pinned = [torch.from_numpy(m).pin_memory() for m in mv_h]
    mk = lambda **kw: kdt.Triangulation(kdt.default_config(grid=256, domain_bits=24, **kw), device=local)

    # value: moves resident in HBM, uninstrumented handle
    tri = mk()
    tri.build(xy0)
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    ms = timed_steps(tri, moves, args.warmup)
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    st = tri.stats()
    sec = sum(ms) / 1000.0
    launches = st["kernel_launches"]
    # the certificate of the final state, and its positions
    verify_bad = tri.verify()
    points_ok = bool(np.array_equal(tri.export_points(), xy_end))
    rebuild_ms = None
    if comparators:
        a, b = _events(1)[0]
        a.record()
        tri.rebuild()
        b.record()
        torch.cuda.synchronize()
        rebuild_ms = a.elapsed_time(b)
    tri.close()

    # e2e: moves in pinned host memory through the C ABI
    tri2 = mk()
    tri2.build(xy0)
    e2e_ms = timed_steps(tri2, pinned, args.warmup)
    tri2.close()
    e2e_sec = sum(e2e_ms) / 1000.0

    updates, seconds, e2e_seconds = aggregate(st["moves"], sec, e2e_sec)
    if rank != 0:
        return None

    # kernel time: a separate instrumented pass over the same moves
    kin_ms, stk = kernel_pass(mk, xy0, moves, args.warmup)
    m_avg = st["moves"] / args.steps
    line = base_line(updates / seconds, args.steps, args.warmup, seconds, "c3",
                     {"n": int(w.n), "grid": 256, "moves_per_step": m_avg,
                      "l2": "store (1.15 GB) larger than L2: no flush",
                      "parallelism": "replicas" if ws > 1 else "single"})
    line["n_gpus"] = ws
    line["e2e"] = {"value": updates / e2e_seconds, "unit": "updates/s",
                   "h2d_bytes_per_step": int(12 * m_avg), "d2h_bytes_per_step": 4 * 20}
    line["gpu_launches"] = int(launches)
    line["fallbacks"] = int(st["fallbacks"])
    line["clocks"] = clk
    line["verify_violations"] = int(verify_bad)
    line["final_positions_match"] = points_ok
    line["kinetic_counters"] = {k: int(stk[k]) for k in ("staged_to_global", "retries", "deferred", "big_moves",
                                                         "drain_moves", "tail_moves")}
    line["_kernel_ms"] = kin_ms
    line["_m_avg"] = m_avg
    line["_oracle_step"] = around
    if comparators:
        def same_steps(**kw):
            tq = mk(**kw) if "quadtree" not in kw else kdt.Triangulation(
                kdt.default_config(domain_bits=24, quadtree=kw["quadtree"], points_per_partition=256), device=local)
            tq.build(xy0)
            qms = timed_steps(tq, moves, args.warmup)
            stq = tq.stats()
            out = {"value": stq["moves"] / (sum(qms) / 1000.0), "unit": "updates/s",
                   "ms_per_step": sum(qms) / len(qms), "fallbacks": int(stq["fallbacks"]),
                   "moved_in_place": (stq["moves"] - stq["deletes"]) / max(1, stq["moves"]),
                   "cells": tq.num_cells()}
            if kw.get("rebuild_displacement"):
                out["far_rebuilds"] = int(stq["far_rebuilds"])
                out["steps"] = int(stq["steps"])
            tq.close()
            return out

        line["comparators"] = {
            "gpu_kinetic_plain": {"value": line["value"], "unit": "updates/s"},
            "gpu_full_rebuild": {"value": m_avg / (rebuild_ms / 1000.0), "unit": "updates/s",
                                 "ms_per_rebuild": rebuild_ms},
            "gpu_kinetic_quadtree_partitions": same_steps(quadtree=1),
            "gpu_kinetic_quadtree_redivided_every_step": same_steps(quadtree=2),
            "gpu_kinetic_index_order": same_steps(partition_order=1),
            "gpu_kinetic_planned_order": same_steps(plan=1),
            "gpu_kinetic_seven_blocks_per_sm": same_steps(kinetic_blocks_per_sm=7),
            "gpu_kinetic_displacement_rule_f1": same_steps(rebuild_displacement=1.0),
            "gpu_kinetic_variant_in_place": same_steps(variant=1),
            "gpu_kinetic_variant_move_flip": same_steps(variant=2),
        }
    return line


# ---------------------------------------------------------------- c2

def run_c2(args, comparators=True):
    """The 1e6-point uniform workload; --check compares the final state with the oracle
    (in a host thread while the GPU runs)."""
    import torch
    from paper_2308_06484_gb300 import kdt, workloads as W
    dev = torch.device("cuda", 0)
    steps = max(args.steps, args.c2_steps)
    w = W.c2(n=args.n, grid=args.grid)
    xy0_h = w.positions
    xy0 = torch.from_numpy(xy0_h).to(dev)
    nsteps = args.warmup + steps
    mv_h, around = draw_moves(w, nsteps, args.warmup)
    xy_end = w.positions
    pool = ThreadPoolExecutor(1)
    fut = None
    if args.check:
        import oracle
        oracle.lib()
        fut = pool.submit(oracle.delaunay, xy_end)
    moves = [torch.from_numpy(m).to(dev) for m in mv_h]
    pinned = [torch.from_numpy(m).pin_memory() for m in mv_h]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    mk = lambda **kw: kdt.Triangulation(kdt.default_config(grid=args.grid, domain_bits=24, **kw))
    tri = mk()
    tri.build(xy0)
    clocks = ClockSampler(0)
    clocks.start()
    ms = timed_steps(tri, moves, args.warmup, flush)
    clk = clocks.stop()
    st = tri.stats()
    sec = sum(ms) / 1000.0
    verify_bad = tri.verify()
    final = tri.export_triangles() if fut is not None else None
    # rebuild comparator on the final positions
    evr = _events(args.rebuild_steps)
    for a, b in evr:
        a.record()
        tri.rebuild()
        b.record()
        flush.zero_()
    torch.cuda.synchronize()
    rebuild_ms = statistics.median(a.elapsed_time(b) for a, b in evr)
    # d-calculation on the final state (one warm-up call allocates its scratch)
    dcalc = {}
    for N in (1, 4):
        tri.d_values(N)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            info = tri.d_values(N)
        dcalc["N%d" % N] = {"ms": 1000.0 * (time.perf_counter() - t0) / 5, "min_dist": math.sqrt(info["min2"]),
                            "spread": info["spread"]}
    tri.close()
    tri2 = mk()
    tri2.build(xy0)
    e2e_ms = timed_steps(tri2, pinned, args.warmup, flush)
    tri2.close()
    kin_ms, _ = kernel_pass(mk, xy0, moves, args.warmup, flush)
    m = st["moves"] / steps
    line = base_line(st["moves"] / sec, steps, args.warmup, sec, "c2",
                     {"n": args.n, "grid": args.grid, "moves_per_step": m,
                      "l2": "flushed between timed steps (256 MB write)"})
    line["e2e"] = {"value": st["moves"] / (sum(e2e_ms) / 1000.0), "unit": "updates/s",
                   "h2d_bytes_per_step": int(12 * m), "d2h_bytes_per_step": 4 * 20}
    line["gpu_launches"] = int(st["kernel_launches"])
    line["fallbacks"] = int(st["fallbacks"])
    line["clocks"] = clk
    line["verify_violations"] = int(verify_bad)
    line["d_calculation"] = dcalc
    line["_kernel_ms"] = kin_ms
    line["_m_avg"] = m
    comp = {"gpu_kinetic_plain": {"value": line["value"], "unit": "updates/s"},
            "gpu_full_rebuild": {"value": m / (rebuild_ms / 1000.0), "unit": "updates/s",
                                 "ms_per_rebuild": rebuild_ms}}
    if comparators:
        for kw, name in (({"variant": 1}, "gpu_kinetic_variant_in_place"),
                         ({"variant": 2}, "gpu_kinetic_variant_move_flip"),
                         ({"rebuild_displacement": 1.0}, "gpu_kinetic_displacement_rule_f1")):
            t3 = mk(**kw)
            t3.build(xy0)
            vms = timed_steps(t3, moves, args.warmup, flush)
            st3 = t3.stats()
            comp[name] = {"value": st3["moves"] / (sum(vms) / 1000.0), "unit": "updates/s",
                          "moved_in_place": (st3["moves"] - st3["deletes"]) / max(1, st3["moves"]),
                          "fallbacks": int(st3["fallbacks"])}
            if "rebuild_displacement" in kw:
                comp[name]["far_rebuilds"] = int(st3["far_rebuilds"])
                comp[name]["steps"] = int(st3["steps"])
            t3.close()
    line["comparators"] = comp
    if fut is not None:
        line["final_state_matches_oracle"] = bool(np.array_equal(final, fut.result()))
    pool.shutdown()
    line["_oracle_step"] = around
    return line


# ---------------------------------------------------------------- c5 (learned proposal)

MLP_FLOPS_PER_ROW = 2 * 7424 * 3 + 2 * 18 * 64 + 2 * 64 * 64  # forward, backward to inputs of layers 2-3, grads


def _tc_grad_flops_per_tile():
    """BF16 tensor-core FLOPs k_mlp_grad_tc issues per 128-row tile: the row products
    (three parts each: layers 1-3 forward, dOut W3, dZ2 W2, N and K as issued) and the
    weight-gradient products over the 128 rows (G_a 128 x 112, three products; G_b
    128 x 32, two)."""
    row = lambda n, k: 3 * 2 * 128 * n * k
    return (row(64, 32) + row(64, 64) + row(32, 64) + row(64, 32) + row(64, 64)
            + 3 * 2 * 128 * 112 * 128 + 2 * 2 * 128 * 32 * 128)


def bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("bf16_tflops", 1900.0)), "measured"
    return 1900.0, "fallback"


def train_proposal(args):
    """Train the proposal on traces of its training workloads; returns (trainer,
    holder handle, info)."""
    import torch
    from paper_2308_06484_gb300 import kdt, proposal
    t0 = time.time()
    x, y = proposal.collect_traces(proposal.default_training_sources(c3_n=args.c5_c3_n, c3_grid=args.c5_c3_grid,
                                                                     c2_steps=args.c5_train_steps,
                                                                     c3_steps=args.c5_c3_steps),
                                   cap=args.c5_trace_cap)
    gen_s = time.time() - t0
    holder = kdt.Triangulation(kdt.default_config())
    tn = proposal.Trainer(holder, seed=0, lr=args.c5_lr, tensor_cores=bool(args.c5_train_tc))
    torch.cuda.synchronize()
    t1 = time.time()
    loss = tn.fit(x, y, epochs=args.c5_epochs, batch=args.c5_batch, seed=0)
    train_s = time.time() - t1
    rows_big = min(x.shape[0], 1 << 18)
    grad_ms = {}
    for tc in (False, True):  # the gradient on the CUDA cores and on the tensor cores
        for _ in range(3):
            holder.mlp_loss_grad(tn.params, x[:rows_big], y[:rows_big], tn.grad, tn.loss, tensor_cores=tc)
        a, b = _events(1)[0]
        a.record()
        reps = 10
        for _ in range(reps):
            holder.mlp_loss_grad(tn.params, x[:rows_big], y[:rows_big], tn.grad, tn.loss, tensor_cores=tc)
        b.record()
        torch.cuda.synchronize()
        grad_ms[tc] = a.elapsed_time(b) / reps
    acc, mae = tn.evaluate(x, y)
    info = {"rows": int(x.shape[0]), "epochs": args.c5_epochs, "batch": args.c5_batch, "lr": args.c5_lr,
            "on_tensor_cores": bool(args.c5_train_tc), "train_top1": acc, "train_log2_cavity_mae": mae,
            "train_loss": loss, "trace_s": gen_s, "train_s": train_s, "grad_ms": grad_ms[False],
            "grad_tc_ms": grad_ms[True], "grad_rows": rows_big, "tensor_timeouts": int(holder.stats()["tensor_timeouts"])}
    return tn, holder, info


def run_c5(args, tn, holder, tinfo):
    """c2's workload (its own seed) with the proposal off and on: in-step hit rate,
    offline top-1 on the evaluation rows, updates/s, the gain."""
    import torch
    from paper_2308_06484_gb300 import kdt, proposal, workloads as W
    dev = torch.device("cuda", 0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    steps = max(args.steps, args.c2_steps)
    nsteps = args.warmup + steps
    w = W.c2()
    xy0 = torch.from_numpy(w.positions).to(dev)
    moves = [torch.from_numpy(w.next_moves()).to(dev) for _ in range(nsteps)]
    res = {}
    plans = {"off": 0, "in_move": 0, "on": 6, "cuda_cores": 2}
    for mode in ("off", "in_move", "on", "cuda_cores"):
        # on: the network evaluated for all moves by the step planner on the tensor
        # cores (plan = 2 | 4); cuda_cores: by the planner, one thread per move
        # (plan = 2); in_move: evaluated inside each move
        tri = kdt.Triangulation(kdt.default_config(grid=64, domain_bits=24, plan=plans[mode]))
        tri.build(xy0)
        if mode != "off":
            tri.set_proposal(tn.params)
        tr = proposal.Trace(4096 * nsteps)
        tr.attach(tri)
        ms = timed_steps(tri, moves, args.warmup, flush)
        st = tri.stats()
        tr.detach(tri)
        res[mode] = {"ms": ms, "st": st, "trace": tr.view(), "verify": tri.verify()}
        tri.close()
    ex, ey = res["off"]["trace"]
    eval_acc, eval_mae = tn.evaluate(ex, ey)
    counts = torch.bincount(ey[:, 0].long(), minlength=17).float()
    majority = float((counts.max() / counts.sum()).item()) if ey.shape[0] else 0.0
    on_s, off_s = sum(res["on"]["ms"]) / 1000.0, sum(res["off"]["ms"]) / 1000.0
    ston = res["on"]["st"]
    v_on, v_off = ston["moves"] / on_s, res["off"]["st"]["moves"] / off_s
    stin = res["in_move"]["st"]
    v_in = stin["moves"] / (sum(res["in_move"]["ms"]) / 1000.0)
    stcc = res["cuda_cores"]["st"]
    v_cc = stcc["moves"] / (sum(res["cuda_cores"]["ms"]) / 1000.0)
    peak_fp32 = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = MLP_FLOPS_PER_ROW * tinfo["grad_rows"] / (tinfo["grad_ms"] / 1000.0) / 1e12
    line = base_line(v_on, steps, args.warmup, on_s, "c5",
                     {"moves_per_step": ston["moves"] / steps, "l2": "flushed between timed steps (256 MB write)",
                      "train": tinfo})
    line["dtype"] = "int64+int128 exact (fp32 filter); proposal net bf16 weights, fp32 accumulate"
    line["proposal"] = {"in_step_hit_rate": ston["proposal_hits"] / max(1, ston["proposal_moves"]),
                        "in_step_proposals_per_step": ston["proposal_moves"] / steps,
                        "eval_top1": eval_acc, "eval_majority_class": majority, "eval_log2_cavity_mae": eval_mae,
                        "eval_rows": int(ex.shape[0]), "gain": v_on / v_off - 1.0,
                        "in_move_evaluation": {"value": v_in, "gain": v_in / v_off - 1.0,
                                               "hit_rate": stin["proposal_hits"] / max(1, stin["proposal_moves"])},
                        "tensor_timeouts": int(ston["tensor_timeouts"]),
                        "planner_on_cuda_cores": {"value": v_cc, "gain": v_cc / v_off - 1.0,
                                                  "hit_rate": stcc["proposal_hits"] / max(1, stcc["proposal_moves"]),
                                                  "ms_per_step": sum(res["cuda_cores"]["ms"]) / steps}}
    line["training_kernel"] = {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                               "frac": achieved / peak_fp32, "kernel": "k_mlp_grad", "kernel_ms": tinfo["grad_ms"],
                               "rows": tinfo["grad_rows"],
                               "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    # the tensor-core form: BF16 tensor FLOPs as issued (splits and padding included)
    # against the measured dense BF16 peak, and the network's own FLOPs per second
    tiles = (tinfo["grad_rows"] + 127) // 128
    tc_tflops = _tc_grad_flops_per_tile() * tiles / (tinfo["grad_tc_ms"] / 1000.0) / 1e12
    pk, pk_kind = bf16_peak()
    line["training_kernel_tensor_cores"] = {
        "bound": "tensor", "achieved": tc_tflops, "peak": pk, "unit": "TFLOP/s", "frac": tc_tflops / pk,
        "kernel": "k_mlp_grad_tc", "kernel_ms": tinfo["grad_tc_ms"], "rows": tinfo["grad_rows"],
        "peak_kind": pk_kind + " dense BF16 (burst)", "bf16_flops_per_tile": _tc_grad_flops_per_tile(),
        "network_tflops": MLP_FLOPS_PER_ROW * tinfo["grad_rows"] / (tinfo["grad_tc_ms"] / 1000.0) / 1e12,
        "speedup_vs_cuda_cores": tinfo["grad_ms"] / tinfo["grad_tc_ms"]}
    line["comparators"] = {"gpu_kinetic_plain": {"value": v_off, "unit": "updates/s",
                                                 "ms_per_step": 1000.0 * off_s / steps}}
    line["gpu_launches"] = int(ston["kernel_launches"])
    line["fallbacks"] = int(ston["fallbacks"])
    line["verify_violations"] = sum(int(r["verify"]) for r in res.values())
    return line


# ---------------------------------------------------------------- c4 (batched)

def run_c4(args, tn=None):
    """Every instance advanced by one kdt_step_batch per step (one graph launch), plain
    and with the learned proposal; against the same instances stepped one handle at a
    time and a rebuild of every instance."""
    import torch
    from paper_2308_06484_gb300 import kdt, workloads as W
    dev = torch.device("cuda", 0)
    ws = W.c4()
    warmup = max(args.warmup, 9 + 3) if args.autotune else args.warmup  # the autotuner times 9 steps
    nsteps = warmup + args.steps
    steps = []
    for _ in range(nsteps):
        mv = [w.next_moves() for w in ws]
        offs = np.zeros(len(mv) + 1, dtype=np.int64)
        offs[1:] = np.cumsum([m.shape[0] for m in mv])
        steps.append((torch.from_numpy(np.ascontiguousarray(np.concatenate(mv))).to(dev), offs, mv))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    start = [w.positions for w in W.c4()]
    check = None
    if args.check:
        import oracle
        sample = list(range(0, len(ws), max(1, len(ws) // 16))) + [len(ws) - 1]
        pool = ThreadPoolExecutor(min(8, host_cores()))
        futs = {i: pool.submit(oracle.delaunay, ws[i].positions) for i in sample}
    stepper = lambda t, s: t.step_batch(s[0], s[1])

    def batched(proposal=False, timing=0, plan=0):
        tri = kdt.Triangulation(kdt.default_config(domain_bits=20, timing=timing, autotune=args.autotune, plan=plan))
        tri.build_batch(start)
        if proposal:
            tri.set_proposal(tn.params)
        ms = timed_steps(tri, steps, warmup, flush, stepper=lambda s: stepper(tri, s))
        return tri, ms

    tri, ms = batched()
    st = tri.stats()
    sec = sum(ms) / 1000.0
    verify_bad = tri.verify()
    if args.check:
        check = all(np.array_equal(tri.export_triangles_inst(i), futs[i].result()) for i in futs)
        pool.shutdown()
    a, b = _events(1)[0]
    a.record()
    tri.rebuild()
    b.record()
    torch.cuda.synchronize()
    rebuild_ms = a.elapsed_time(b)
    tri.close()
    tk, _ = batched(timing=1)
    stk = tk.stats()
    kin_ms = stk["kinetic_kernel_ms"] / max(1, stk["kinetic_kernel_timed"])
    tk.close()
    m_avg = st["moves"] / args.steps
    line = base_line(st["moves"] / sec, args.steps, warmup, sec, "c4",
                     {"instances": len(ws), "points": int(sum(w.n for w in ws)), "moves_per_step": m_avg,
                      "l2": "flushed between timed steps (256 MB write)", "autotune": args.autotune,
                      "tuned_points_per_partition": st["tuned_points_per_partition"],
                      "tuned_warps_per_partition": st["tuned_warps_per_partition"]})
    comp = {"gpu_kinetic_batched_plain": {"value": line["value"], "unit": "updates/s"},
            "gpu_full_rebuild_all_instances": {"value": m_avg / (rebuild_ms / 1000.0), "unit": "updates/s",
                                               "ms_per_rebuild": rebuild_ms}}
    tq, qms = batched(plan=1)
    stq = tq.stats()
    comp["gpu_kinetic_batched_planned_order"] = {"value": stq["moves"] / (sum(qms) / 1000.0), "unit": "updates/s",
                                                 "ms_per_step": sum(qms) / len(qms), "verify_violations": tq.verify()}
    tq.close()
    if tn is not None:
        # the network evaluated for all moves at once, on the CUDA cores and on the
        # tensor cores
        for key, plan in (("gpu_kinetic_batched_learned", 2), ("gpu_kinetic_batched_learned_tensor_cores", 6)):
            tp, pms = batched(proposal=True, plan=plan)
            stp = tp.stats()
            comp[key] = {
                "value": stp["moves"] / (sum(pms) / 1000.0), "unit": "updates/s", "ms_per_step": sum(pms) / len(pms),
                "hit_rate": stp["proposal_hits"] / max(1, stp["proposal_moves"]),
                "proposals_per_step": stp["proposal_moves"] / args.steps, "verify_violations": tp.verify(),
                "tensor_timeouts": int(stp["tensor_timeouts"])}
            comp[key]["gain_vs_batched_plain"] = comp[key]["value"] / line["value"] - 1.0
            tp.close()
    if args.c4_plain_steps > 0:
        hs = []
        for x in start:
            t1 = kdt.Triangulation(kdt.default_config(domain_bits=20))
            t1.build(x)
            hs.append(t1)
        for i in range(warmup):
            for t1, m1 in zip(hs, steps[i][2]):
                t1.step(m1)
        evp = []
        torch.cuda.synchronize()
        for k in range(args.c4_plain_steps):
            _, _, mv = steps[warmup + k]
            dm = [torch.from_numpy(m1).to(dev) for m1 in mv]
            flush.zero_()
            a, b = _events(1)[0]
            a.record()
            for t1, m1 in zip(hs, dm):
                t1.step(m1)
            b.record()
            evp.append((a, b, sum(m1.shape[0] for m1 in mv)))
        torch.cuda.synchronize()
        plain_ms = sum(a.elapsed_time(b) for a, b, _ in evp) / len(evp)
        plain_moves = sum(c for _, _, c in evp) / len(evp)
        for t1 in hs:
            t1.close()
        comp["gpu_kinetic_one_handle_per_instance"] = {"value": plain_moves / (plain_ms / 1000.0),
                                                       "unit": "updates/s", "ms_per_step": plain_ms}
    line["comparators"] = comp
    line["gpu_launches"] = int(st["kernel_launches"])
    line["fallbacks"] = int(st["fallbacks"])
    line["verify_violations"] = int(verify_bad)
    line["_kernel_ms"] = kin_ms
    line["_m_avg"] = m_avg
    if check is not None:
        line["sampled_instances_match_oracle"] = check
    return line


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    """--impl reference: the oracle as it stands, on the host cores, for the workload
    of the headline (each step = one rebuild of the step's point set, tiled over every
    core for the 16e6-point set); steps stop after the requested count or when the time
    budget is spent (at least one), so the run ends within a few minutes."""
    ws, rank, _ = dist_info()
    if ws > 1 and rank != 0:
        return
    from paper_2308_06484_gb300 import workloads as W
    threads = max(1, min(host_cores(), args.ref_threads)) if args.ref_threads > 0 else host_cores()
    if args.workload in ("c2", "c5"):
        w, T, key = W.c2(n=args.n, grid=args.grid), 1, "c2"
    else:
        w, T, key = W.c3(n=args.ref_n or 16_000_000), args.ref_tiles, "c3"
    w.next_moves()
    times, moves = [], 0
    t_start = time.perf_counter()
    for s in range(args.steps):
        mv = w.next_moves()
        xy = w.positions
        if T == 1:
            # independent steps in parallel: one rebuild of the whole set per thread
            snaps = [xy]
            for _ in range(threads - 1):
                w.next_moves()
                snaps.append(w.positions)
            import oracle
            oracle.lib()
            t0 = time.perf_counter()
            with ThreadPoolExecutor(threads) as pool:
                list(pool.map(oracle.delaunay, snaps))
            dt = time.perf_counter() - t0
            times.append(dt)
            moves += mv.shape[0] * len(snaps)
        else:
            dt, _ = _oracle_tiles(xy, _tiles(xy, 24, T), threads)
            times.append(dt)
            moves += mv.shape[0]
        if time.perf_counter() - t_start > args.ref_budget_s:
            break
    tot = sum(times)
    value = moves / tot
    steps_done = len(times) if T > 1 else len(times) * threads
    sample = ("%d oracle rebuilds of the %d-point set (one per time step), %d in parallel per round, %.1f s timed"
              % (steps_done, w.n, threads, tot)) if T == 1 else \
        ("%d time steps, each one oracle rebuild of the %d-point set as %d tiles (%dx%d division of the domain) "
         "on %d threads, %.1f s timed" % (steps_done, w.n, T * T, T, T, threads, tot))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s",
        "n_gpus": 1, "steps": steps_done, "warmup": 1, "ms_per_step": 1000.0 * tot / max(1, len(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64+int128 exact", "data": "synthetic",
        "config": {"workload": WORKLOADS[key], "n": int(w.n), "requested_steps": args.steps,
                   "time_budget_s": args.ref_budget_s},
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- main

def finish(line, workload, args, oracle_ok):
    """Add the roofline (with the oracle's bytes model when the oracle leg runs) and
    the CPU baseline; drop the private keys."""
    model = None
    step = line.pop("_oracle_step", None)
    line.pop("_oracle_args", None)
    if oracle_ok and step is not None:
        before, after, mv = step
        T, mt = (args.ref_tiles, 8) if workload == "c3" else (2, 4)
        base, model = oracle_leg(before, after, mv, 24, T, host_cores(), mt)
        if workload == "c3":
            line["cpu_baseline"] = base
        else:
            line["oracle_bytes_model"] = model
    bpu = model["bytes_per_update"] if model else BYTES_K6
    kin_ms, m_avg = line.pop("_kernel_ms", None), line.pop("_m_avg", None)
    if kin_ms:
        line["roofline"] = roofline(bpu, m_avg, kin_ms, kinetic_traffic(workload, m_avg))
        line["roofline"]["bytes_model"] = model if model else "mean planar degree k = 6 (oracle leg not run)"
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="all", choices=["all", "c2", "c3", "c4", "c5"],
                    help="all: the 16e6-point headline with c2, c4, c5 nested; else that workload alone")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--c2-steps", type=int, default=200, help="timed steps of the 1e6-point workload (at least)")
    ap.add_argument("--rebuild-steps", type=int, default=3)
    ap.add_argument("--ref-threads", type=int, default=0, help="reference arm threads (0 = every host core)")
    ap.add_argument("--ref-tiles", type=int, default=8, help="tiles per side of the 16e6-point oracle rebuild")
    ap.add_argument("--ref-n", type=int, default=0, help="reference arm points (0 = the workload's)")
    ap.add_argument("--ref-budget-s", type=float, default=90.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--check", type=int, default=1, help="compare final states with the oracle (outside timing)")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--c4-plain-steps", type=int, default=2)
    ap.add_argument("--c5-train-steps", type=int, default=100)
    ap.add_argument("--c5-c3-n", type=int, default=2_000_000)
    ap.add_argument("--c5-c3-grid", type=int, default=90)
    ap.add_argument("--c5-c3-steps", type=int, default=4)
    ap.add_argument("--c5-trace-cap", type=int, default=1_000_000)
    ap.add_argument("--c5-epochs", type=int, default=4)
    ap.add_argument("--c5-batch", type=int, default=8192)
    ap.add_argument("--c5-lr", type=float, default=2e-3)
    ap.add_argument("--c5-train-tc", type=int, default=1, help="train the proposal with the tensor-core gradient")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    oracle_ok = not args.no_cpu_baseline and ws == 1
    comps = not args.no_comparators
    t0 = time.time()
    if args.workload in ("all", "c3"):
        line = run_c3(args, rank, ws, local, comparators=comps and ws == 1)
        if rank == 0:
            line = finish(line, "c3", args, oracle_ok)
            if args.workload == "all" and ws == 1:
                nested = {}
                nested["c2"] = finish(run_c2(args, comps), "c2", args, oracle_ok)
                tn, holder, tinfo = train_proposal(args)
                nested["c5"] = finish(run_c5(args, tn, holder, tinfo), "c5", args, False)
                nested["c4"] = finish(run_c4(args, tn), "c4", args, False)
                holder.close()
                line["workloads"] = nested
    elif args.workload == "c2":
        line = finish(run_c2(args, comps), "c2", args, oracle_ok)
    elif args.workload == "c5":
        tn, holder, tinfo = train_proposal(args)
        line = finish(run_c5(args, tn, holder, tinfo), "c5", args, False)
        holder.close()
    else:
        tn, holder, tinfo = (None, None, None) if args.no_comparators else train_proposal(args)
        line = finish(run_c4(args, tn), "c4", args, False)
        if holder:
            holder.close()
    if rank == 0:
        line["bench_wall_s"] = time.time() - t0
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
