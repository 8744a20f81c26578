"""Benchmark: moved-point updates per second of the kinetic Delaunay step.

Workload (the configuration the headline metric is quoted on): 1,000,000 distinct
integer points uniform on [0, 2^24)^2, 64 x 64 equal-area partitions, one moved point
per partition per step (4,096 moves), each move 1-8 units right/left/up/down,
synthetic and seeded.  A step is one call of kdt_step: bucket the moves per
partition, delete + re-insert each moved point, certify the touched triangles.

Printed JSON line (rank 0):
  value      updates/s with the moves already resident in HBM (CUDA events around
             every step, L2 flushed between steps: the 72 MB store fits in L2);
  e2e        the same metric through the C ABI with the moves in pinned host memory
             (host->device copy and the status read inside the timed region);
  roofline   the kinetic kernel's algorithmic bytes (688 B per update) / its
             event-timed duration, against the measured HBM copy bandwidth;
  comparators  the GPU full rebuild per step, on the same GB300;
  cpu_baseline the CPU oracle (a Bowyer-Watson rebuild per step) on the host cores.

--impl reference times the oracle alone (the deliberately slow reference).
Under torchrun (N > 1) every rank advances its own independent instance (replicas;
"weak" scaling) and value = all ranks' updates / max-over-ranks time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = 688  # star triangles 32*(k_old+k_new) + back-pointers 16*(k_old+k_new) + coords 8*(k_old+k_new+2), k = 6

# DRAM bytes (read + write) of one k_kinetic launch of the 1e6-point, 4096-move step,
# from `ncu --set full` (profiles/k_kinetic_c2_1e6.md), valid only for the kernel
# sources it was taken on (their SHA-256 prefix); reported as null otherwise.
KINETIC_TRAFFIC = {"sources": "39a3ede9acc55c3d", "bytes": 15688192 + 74240, "moves": 4096}


def kernel_sources_hash():
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2308_06484_gb300", "csrc", "*.cu*"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kinetic_traffic(moves_per_launch):
    if kernel_sources_hash() != KINETIC_TRAFFIC["sources"] or moves_per_launch != KINETIC_TRAFFIC["moves"]:
        return None
    return KINETIC_TRAFFIC["bytes"]
METRIC = "moved-point updates/sec (1 GB300, bit-exact) vs plain GPU update and full rebuild"
WORKLOAD = ("1e6 uniform points on [0,2^24)^2, 64x64 partitions, 4096 moves/step "
            "(1 per partition, 1-8 units R/L/U/D)")


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
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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


def oracle_baseline(snapshots, moves_per_step, threads):
    """Time the oracle (rebuild from scratch) on `threads` step snapshots in parallel."""
    import oracle
    oracle.lib()
    t0 = time.perf_counter()
    out = [None] * len(snapshots)

    def run(i):
        out[i] = oracle.delaunay(snapshots[i]).shape[0]

    ths = [threading.Thread(target=run, args=(i,)) for i in range(len(snapshots))]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    dt = time.perf_counter() - t0
    return len(snapshots) * moves_per_step / dt, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """--impl reference: the oracle as it stands, on the host cores.

    One step of the workload is one oracle rebuild of the 1e6-point set (the DT after
    a time step); `threads` steps run in parallel per round.  Rounds stop after the
    requested count or when the time budget is spent (at least one timed round), so
    the run ends within a few minutes whatever --steps asks for."""
    ws, rank, _ = dist_info()
    if ws > 1 and rank != 0:
        return
    from paper_2308_06484_gb300 import workloads as W
    w = W.c2(n=args.n, grid=args.grid)
    threads = max(1, min(host_cores(), 16, args.ref_threads))
    # warm-up: one single rebuild pages the library and the data in
    mv = w.next_moves()
    oracle_baseline([w.positions], mv.shape[0], 1)
    times, moves = [], 0
    t_start = time.perf_counter()
    for s in range(args.steps):
        snaps = []
        for _ in range(threads):
            mv = w.next_moves()
            snaps.append(w.positions)
        ups, dt = oracle_baseline(snaps, mv.shape[0], threads)
        times.append(dt)
        moves += threads * mv.shape[0]
        if time.perf_counter() - t_start > args.ref_budget_s:
            break
    tot = sum(times)
    value = moves / tot
    steps_done = len(times) * threads
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s",
        "n_gpus": 1, "steps": steps_done, "warmup": 1,
        "ms_per_step": 1000.0 * tot * threads / max(1, steps_done) / threads,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64+int128 exact", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": args.n, "grid": args.grid,
                   "requested_steps": args.steps, "time_budget_s": args.ref_budget_s},
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": threads, "kind": "oracle",
                         "sample": "%d oracle rebuilds of the %d-point set (one per time step), %d in "
                                   "parallel per round, %.1f s timed" % (steps_done, args.n, threads, tot)},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


C4_WORKLOAD = ("512 instances, sizes log-uniform 1e3-2e5 (seeded), uniform on [0,2^20)^2, "
               "~256 points per partition, 1-4 moves per partition per step (1-8 units)")


def run_c4(args):
    """Batched workload: every instance advanced by one kdt_step_batch per step
    (one graph launch), against the same instances stepped one handle at a time and
    against a full rebuild of every instance."""
    import torch
    from paper_2308_06484_gb300 import kdt, workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ws = W.c4()
    # the autotuner times one step of each of its 9 configurations first
    warmup = max(args.warmup, 9 + 3) if args.autotune else args.warmup
    args.warmup = warmup
    nsteps = args.warmup + args.steps
    steps = []
    for _ in range(nsteps):
        mv = [w.next_moves() for w in ws]
        offs = np.zeros(len(mv) + 1, dtype=np.int64)
        offs[1:] = np.cumsum([m.shape[0] for m in mv])
        steps.append((torch.from_numpy(np.ascontiguousarray(np.concatenate(mv))).to(dev), offs, mv))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ws0 = W.c4()  # the same seeded instances from their start positions
    start = [w.positions for w in ws0]
    tri = kdt.Triangulation(kdt.default_config(domain_bits=20, timing=1, autotune=args.autotune))
    tri.build_batch(start)
    for i in range(args.warmup):
        tri.step_batch(steps[i][0], steps[i][1])
    tri.reset_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        d, offs, _ = steps[args.warmup + k]
        ev[k][0].record()
        tri.step_batch(d, offs)
        ev[k][1].record()
        flush.zero_()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    st = tri.stats()
    moves = st["moves"]
    verify_bad = tri.verify()
    check = None
    if args.check:
        import oracle
        # the generators already stand at the final positions (all steps were drawn)
        sample = list(range(0, len(ws), max(1, len(ws) // 32))) + [len(ws) - 1]
        check = all(np.array_equal(tri.export_triangles_inst(i), oracle.delaunay(ws[i].positions))
                    for i in sample)
    # comparator 1: the same instances, one handle each, stepped one after another
    plain_ms = None
    if args.c4_plain_steps > 0:
        hs = []
        for x in start:
            t1 = kdt.Triangulation(kdt.default_config(domain_bits=20))
            t1.build(x)
            hs.append(t1)
        for i in range(args.warmup):
            for t1, m1 in zip(hs, steps[i][2]):
                t1.step(m1)
        evp = []
        torch.cuda.synchronize()
        for k in range(args.c4_plain_steps):
            _, _, mv = steps[args.warmup + k]
            dm = [torch.from_numpy(m1).to(dev) for m1 in mv]
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
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
    # comparator 2: full rebuild of every instance
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    tri.rebuild()
    b.record()
    torch.cuda.synchronize()
    rebuild_ms = a.elapsed_time(b)
    m_avg = moves / args.steps
    peak, peak_kind = measured_peaks()
    kin_ms = st["kinetic_kernel_ms"] / max(1, st["kinetic_kernel_timed"])
    achieved = BYTES_PER_UPDATE * m_avg / (kin_ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": moves / sec, "unit": "updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64+int128 exact (fp32 filter)", "data": "synthetic",
        "config": {"workload": C4_WORKLOAD, "instances": len(ws), "points": int(sum(w.n for w in ws)),
                   "moves_per_step": m_avg, "l2": "flushed between timed steps (256 MB write)",
                   "autotune": args.autotune, "tuned_points_per_partition": st["tuned_points_per_partition"],
                   "tuned_warps_per_partition": st["tuned_warps_per_partition"]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_kinetic", "kernel_ms": kin_ms, "peak_kind": peak_kind},
        "comparators": {
            "gpu_kinetic_one_handle_per_instance": (None if plain_ms is None else
                                                    {"value": plain_moves / (plain_ms / 1000.0), "unit": "updates/s",
                                                     "ms_per_step": plain_ms}),
            "gpu_full_rebuild_all_instances": {"value": m_avg / (rebuild_ms / 1000.0), "unit": "updates/s",
                                               "ms_per_rebuild": rebuild_ms},
        },
        "gpu_launches": int(st["kernel_launches"]), "fallbacks": int(st["fallbacks"]), "clocks": clk,
        "verify_violations": int(verify_bad),
    }
    if check is not None:
        line["sampled_instances_match_oracle"] = check
    print(json.dumps(line), flush=True)
    tri.close()


def _timed_steps(tri, moves, warmup, flush):
    """Per-step CUDA-event times (ms) of tri.step over moves[warmup:], L2 flushed between."""
    import torch
    for i in range(warmup):
        tri.step(moves[i])
    tri.reset_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(len(moves) - warmup)]
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(ev):
        a.record()
        tri.step(moves[warmup + k])
        b.record()
        flush.zero_()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


MLP_FLOPS_PER_ROW = 2 * 7424 * 3 + 2 * 18 * 64 + 2 * 64 * 64  # forward, backward to inputs of layers 2-3, grads


def run_c3(args):
    """The 16e6-point mixture + lattice workload at full size (256x256 partitions, 1-16
    moves per partition): updates/s of kdt_step with the moves in HBM (the 1.15 GB
    store exceeds L2, so no flush is needed), the rebuild comparator, and the GPU
    certificate of the final state."""
    import torch
    from paper_2308_06484_gb300 import kdt, workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = W.c3()
    xy0 = torch.from_numpy(w.positions).to(dev)
    nsteps = args.warmup + args.steps
    moves = [torch.from_numpy(w.next_moves()).to(dev) for _ in range(nsteps)]
    tri = kdt.Triangulation(kdt.default_config(grid=256, domain_bits=24, timing=1))
    tri.build(xy0)
    for i in range(args.warmup):
        tri.step(moves[i])
    tri.reset_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    torch.cuda.synchronize()
    clocks.start()
    for k, (a, b) in enumerate(ev):
        a.record()
        tri.step(moves[args.warmup + k])
        b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    st = tri.stats()
    verify_bad = tri.verify()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    tri.rebuild()
    b.record()
    torch.cuda.synchronize()
    rebuild_ms = a.elapsed_time(b)
    tri.close()

    def same_steps(cfg):
        # the same build and steps with another configuration (a comparator)
        tq = kdt.Triangulation(cfg)
        tq.build(xy0)
        for i in range(args.warmup):
            tq.step(moves[i])
        tq.reset_stats()
        evq = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k, (qa, qb) in enumerate(evq):
            qa.record()
            tq.step(moves[args.warmup + k])
            qb.record()
        torch.cuda.synchronize()
        qsec = sum(qa.elapsed_time(qb) for qa, qb in evq) / 1000.0
        stq = tq.stats()
        out = {"value": stq["moves"] / qsec, "unit": "updates/s", "ms_per_step": 1000.0 * qsec / args.steps,
               "fallbacks": int(stq["fallbacks"]), "moved_in_place": (stq["moves"] - stq["deletes"]) / stq["moves"],
               "cells": tq.num_cells()}
        tq.close()
        return out

    # the paper's quad-tree partitions (threshold 256); the two in-place variants
    quadtree = same_steps(kdt.default_config(domain_bits=24, timing=1, quadtree=1, points_per_partition=256))
    var1 = same_steps(kdt.default_config(grid=256, domain_bits=24, timing=1, variant=1))
    var2 = same_steps(kdt.default_config(grid=256, domain_bits=24, timing=1, variant=2))
    m_avg = st["moves"] / args.steps
    peak, peak_kind = measured_peaks()
    kin_ms = st["kinetic_kernel_ms"] / max(1, st["kinetic_kernel_timed"])
    achieved = BYTES_PER_UPDATE * m_avg / (kin_ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": st["moves"] / sec, "unit": "updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64+int128 exact (fp32 filter)", "data": "synthetic",
        "config": {"workload": "16e6 points: 32-Gaussian mixture (sigma 2^18) + 5 % lattice on [0,2^24)^2, "
                               "256x256 partitions, 1-16 moves per partition per step (1-8 units)",
                   "n": int(w.n), "moves_per_step": m_avg, "l2": "store (1.15 GB) larger than L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_kinetic", "kernel_ms": kin_ms, "peak_kind": peak_kind},
        "comparators": {"gpu_full_rebuild": {"value": m_avg / (rebuild_ms / 1000.0), "unit": "updates/s",
                                             "ms_per_rebuild": rebuild_ms},
                        "gpu_kinetic_quadtree_partitions": quadtree,
                        "gpu_kinetic_variant_in_place": var1, "gpu_kinetic_variant_move_flip": var2},
        "gpu_launches": int(st["kernel_launches"]), "fallbacks": int(st["fallbacks"]), "clocks": clk,
        "verify_violations": int(verify_bad), "staged_to_global": int(st["staged_to_global"]),
        "retries": int(st["retries"]),
    }
    print(json.dumps(line), flush=True)


def run_c5(args):
    """The learned locate proposal: train on traces of c2 and of the c3 distribution
    (training seeds), evaluate on the headline c2 workload (its own seed): offline
    top-1 accuracy, in-step hit rate, and updates/s with the proposal on and off."""
    import time
    import torch
    from paper_2308_06484_gb300 import kdt, proposal, workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    cfg = lambda g, b: kdt.default_config(grid=g, domain_bits=b, timing=1)
    # ---- training rows
    t0 = time.time()
    traces = []
    for (wl, steps, g) in ((W.c2(seed=102), args.c5_train_steps, 64),
                           (W.c3(n=args.c5_c3_n, grid=args.c5_c3_grid, seed=103), args.c5_c3_steps, args.c5_c3_grid)):
        tri = kdt.Triangulation(cfg(g, 24))
        tri.build(torch.from_numpy(wl.positions).to(dev))
        tr = proposal.Trace(args.c5_trace_cap)
        tr.attach(tri)
        for _ in range(steps):
            tri.step(torch.from_numpy(wl.next_moves()).to(dev))
        tr.detach(tri)
        traces.append(tr.view())
        tri.close()
    x = torch.cat([a for a, _ in traces])
    y = torch.cat([b for _, b in traces])
    gen_s = time.time() - t0
    # ---- training (and the gradient kernel's rate on one large batch)
    holder = kdt.Triangulation(kdt.default_config())
    tn = proposal.Trainer(holder, seed=0, lr=args.c5_lr)
    torch.cuda.synchronize()
    t1 = time.time()
    loss = tn.fit(x, y, epochs=args.c5_epochs, batch=args.c5_batch, seed=0)
    train_s = time.time() - t1
    rows_big = min(x.shape[0], 1 << 18)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        holder.mlp_loss_grad(tn.params, x[:rows_big], y[:rows_big], tn.grad, tn.loss)
    a.record()
    reps = 10
    for _ in range(reps):
        holder.mlp_loss_grad(tn.params, x[:rows_big], y[:rows_big], tn.grad, tn.loss)
    b.record()
    torch.cuda.synchronize()
    grad_ms = a.elapsed_time(b) / reps
    train_acc, train_mae = tn.evaluate(x, y)
    # ---- evaluation on the headline workload
    nsteps = args.warmup + args.steps
    w_eval = W.c2()
    moves = [torch.from_numpy(w_eval.next_moves()).to(dev) for _ in range(nsteps)]
    xy0 = torch.from_numpy(W.c2().positions).to(dev)
    res = {}
    for mode in ("off", "on"):
        tri = kdt.Triangulation(cfg(64, 24))
        tri.build(xy0)
        if mode == "on":
            tri.set_proposal(tn.params)
        tr = proposal.Trace(4096 * nsteps)
        tr.attach(tri)
        ms = _timed_steps(tri, moves, args.warmup, flush)
        st = tri.stats()
        tr.detach(tri)
        res[mode] = {"ms": ms, "st": st, "trace": tr.view(), "check": None}
        if args.check:
            import oracle
            res[mode]["check"] = bool(np.array_equal(tri.export_triangles(), oracle.delaunay(w_eval.positions)))
        tri.close()
    ex, ey = res["off"]["trace"]
    eval_acc, eval_mae = tn.evaluate(ex, ey)
    counts = torch.bincount(ey[:, 0].long(), minlength=17).float()
    eval_majority = float((counts.max() / counts.sum()).item()) if ey.shape[0] else 0.0
    m_avg = res["on"]["st"]["moves"] / args.steps
    on_s = sum(res["on"]["ms"]) / 1000.0
    off_s = sum(res["off"]["ms"]) / 1000.0
    ston = res["on"]["st"]
    peak_fp32 = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = MLP_FLOPS_PER_ROW * rows_big / (grad_ms / 1000.0) / 1e12
    line = {
        "metric": METRIC, "value": res["on"]["st"]["moves"] / on_s, "unit": "updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * on_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64+int128 exact (fp32 filter); proposal net bf16 weights, fp32 accumulate",
        "data": "synthetic",
        "config": {"workload": WORKLOAD + ", learned locate proposal on", "moves_per_step": m_avg,
                   "l2": "flushed between timed steps (256 MB write)",
                   "train": {"c2_seed": 102, "c2_steps": args.c5_train_steps, "c3_n": args.c5_c3_n,
                             "c3_grid": args.c5_c3_grid, "c3_seed": 103, "c3_steps": args.c5_c3_steps,
                             "rows": int(x.shape[0]), "epochs": args.c5_epochs, "batch": args.c5_batch,
                             "lr": args.c5_lr}},
        "proposal": {"in_step_hit_rate": ston["proposal_hits"] / max(1, ston["proposal_moves"]),
                     "in_step_proposals": ston["proposal_moves"] / args.steps,
                     "eval_top1": eval_acc, "eval_majority_class": eval_majority,
                     "eval_log2_cavity_mae": eval_mae, "eval_rows": int(ex.shape[0]),
                     "train_top1": train_acc, "train_loss": loss, "trace_s": gen_s, "train_s": train_s,
                     "gain": (res["on"]["st"]["moves"] / on_s) / (res["off"]["st"]["moves"] / off_s) - 1.0},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                     "frac": achieved / peak_fp32, "traffic": None, "kernel": "k_mlp_grad",
                     "kernel_ms": grad_ms, "rows": rows_big,
                     "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
        "comparators": {"gpu_kinetic_plain": {"value": res["off"]["st"]["moves"] / off_s, "unit": "updates/s",
                                              "ms_per_step": 1000.0 * off_s / args.steps}},
        "gpu_launches": int(ston["kernel_launches"]), "fallbacks": int(ston["fallbacks"]),
    }
    if args.check:
        line["final_state_matches_oracle"] = {"on": res["on"]["check"], "off": res["off"]["check"]}
    print(json.dumps(line), flush=True)
    holder.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--rebuild-steps", type=int, default=5)
    ap.add_argument("--cpu-threads", type=int, default=4)
    ap.add_argument("--ref-threads", type=int, default=8)
    ap.add_argument("--ref-budget-s", type=float, default=90.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--check", action="store_true", help="compare the final state with the oracle")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5"],
                    help="c2: the headline single instance; c4: 512 batched instances")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--c4-plain-steps", type=int, default=3)
    ap.add_argument("--c5-train-steps", type=int, default=100)
    ap.add_argument("--c5-c3-n", type=int, default=2_000_000)
    ap.add_argument("--c5-c3-grid", type=int, default=90)
    ap.add_argument("--c5-c3-steps", type=int, default=4)
    ap.add_argument("--c5-trace-cap", type=int, default=1_000_000)
    ap.add_argument("--c5-epochs", type=int, default=4)
    ap.add_argument("--c5-batch", type=int, default=8192)
    ap.add_argument("--c5-lr", type=float, default=2e-3)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c3":
        return run_c3(args)
    if args.workload == "c4":
        return run_c4(args)
    if args.workload == "c5":
        return run_c5(args)

    import torch
    import torch.distributed as dist
    from paper_2308_06484_gb300 import kdt, workloads as W

    ws, rank, local = dist_info()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # workload: every rank its own seeded instance
    w = W.c2(n=args.n, grid=args.grid, seed=2 + 1000 * rank)
    xy0 = w.positions
    nsteps = args.warmup + args.steps
    moves = [w.next_moves() for _ in range(nsteps)]
    m = moves[0].shape[0]
    d_moves = [torch.from_numpy(mv).to(dev) for mv in moves]
    h_moves = [torch.from_numpy(mv).pin_memory() for mv in moves]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    cfg = kdt.default_config(grid=args.grid, domain_bits=24, timing=1)
    tri = kdt.Triangulation(cfg, device=local)
    tri.build(torch.from_numpy(xy0).to(dev))

    # ---- value: device-resident moves
    for i in range(args.warmup):
        tri.step(d_moves[i])
    tri.reset_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        i = args.warmup + k
        ev[k][0].record()
        tri.step(d_moves[i])
        ev[k][1].record()
        flush.zero_()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st = tri.stats()
    local_sec = sum(step_ms) / 1000.0
    local_updates = st["moves"]
    launches = st["kernel_launches"]
    kin_ms = st["kinetic_kernel_ms"] / max(1, st["kinetic_kernel_timed"])
    fallbacks = st["fallbacks"]
    final_xy = w.positions.copy()

    # ---- e2e: host (pinned) moves through the C ABI, on a fresh instance of the same workload
    w2 = W.c2(n=args.n, grid=args.grid, seed=2 + 1000 * rank)
    tri2 = kdt.Triangulation(kdt.default_config(grid=args.grid, domain_bits=24), device=local)
    tri2.build(torch.from_numpy(w2.positions).to(dev))
    for i in range(args.warmup):
        tri2.step(h_moves[i])
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        i = args.warmup + k
        ev2[k][0].record()
        tri2.step(h_moves[i])
        ev2[k][1].record()
        flush.zero_()
    torch.cuda.synchronize()
    e2e_sec = sum(a.elapsed_time(b) for a, b in ev2) / 1000.0
    tri2.close()

    # ---- comparators: the same steps with the in-place variants (kdt_config.variant
    # 1: safe-region test, 2: move and flip)
    variants = {}
    for var in (1, 2):
        w3 = W.c2(n=args.n, grid=args.grid, seed=2 + 1000 * rank)
        tri3 = kdt.Triangulation(kdt.default_config(grid=args.grid, domain_bits=24, variant=var), device=local)
        tri3.build(torch.from_numpy(w3.positions).to(dev))
        for i in range(args.warmup):
            tri3.step(d_moves[i])
        tri3.reset_stats()
        ev3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            i = args.warmup + k
            ev3[k][0].record()
            tri3.step(d_moves[i])
            ev3[k][1].record()
            flush.zero_()
        torch.cuda.synchronize()
        var_sec = sum(a.elapsed_time(b) for a, b in ev3) / 1000.0
        st3 = tri3.stats()
        variants[var] = {"value": local_updates / var_sec, "unit": "updates/s",
                         "moved_in_place": (st3["moves"] - st3["deletes"]) / max(1, st3["moves"]),
                         "fallbacks": int(st3["fallbacks"])}
        tri3.close()

    # ---- comparator: GPU full rebuild of the same point set per step
    tri.reset_stats()
    evr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.rebuild_steps)]
    for k in range(args.rebuild_steps):
        evr[k][0].record()
        tri.rebuild()
        evr[k][1].record()
        flush.zero_()
    torch.cuda.synchronize()
    rebuild_ms = statistics.median(a.elapsed_time(b) for a, b in evr)

    # ---- d-calculation (Section III/IV) on the final state: N-th nearest neighbours of
    # every point, per-partition and global minima (one warm-up call allocates scratch)
    dcalc = {}
    for N in (1, 4):
        tri.d_values(N)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 5
        for _ in range(reps):
            info = tri.d_values(N)
        dcalc["N%d" % N] = {"ms": 1000.0 * (time.perf_counter() - t0) / reps, "min_dist": math.sqrt(info["min2"]),
                            "spread": info["spread"]}

    check = None
    if args.check:
        import oracle
        check = bool(np.array_equal(tri.export_triangles(), oracle.delaunay(final_xy)))

    updates, seconds, e2e_seconds = aggregate(local_updates, local_sec, e2e_sec)
    value = updates / seconds
    e2e_value = updates / e2e_seconds

    if rank == 0:
        peak, peak_kind = measured_peaks()
        achieved = BYTES_PER_UPDATE * m / (kin_ms / 1000.0) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * seconds / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64+int128 exact (fp32 filter)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "grid": args.grid, "moves_per_step": m,
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "e2e": {"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": 12 * m,
                    "d2h_bytes_per_step": 64},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": kinetic_traffic(m),
                         "kernel": "k_kinetic", "kernel_ms": kin_ms, "bytes_per_update": BYTES_PER_UPDATE,
                         "peak_kind": peak_kind},
            "comparators": {
                "gpu_kinetic_plain": {"value": value, "unit": "updates/s"},
                "gpu_full_rebuild": {"value": m / (rebuild_ms / 1000.0), "unit": "updates/s",
                                     "ms_per_rebuild": rebuild_ms},
                "gpu_kinetic_variant_in_place": variants[1],
                "gpu_kinetic_variant_move_flip": variants[2],
            },
            "gpu_launches": int(launches),
            "fallbacks": int(fallbacks),
            "clocks": clk,
            "d_calculation": dcalc,
        }
        if check is not None:
            line["final_state_matches_oracle"] = check
        if not args.no_cpu_baseline and ws == 1:
            threads = max(1, min(host_cores(), args.cpu_threads))
            snaps = []
            wb = W.c2(n=args.n, grid=args.grid, seed=77)
            for _ in range(threads):
                wb.next_moves()
                snaps.append(wb.positions)
            ups, dt = oracle_baseline(snaps, m, threads)
            line["cpu_baseline"] = {"value": ups, "unit": "updates/s", "cores": threads, "kind": "oracle",
                                    "sample": "%d oracle rebuilds of the %d-point set (one per step), "
                                              "in parallel on %d threads, %.1f s wall" % (threads, args.n, threads, dt)}
        print(json.dumps(line), flush=True)
    tri.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
