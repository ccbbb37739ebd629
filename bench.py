"""Benchmark: events/s and hit-triplets/s of the displaced-track Hough on GB300.

A step is one trk_reconstruct call over one synthetic event of the 500-track 10-layer
workload (pack, schedule, triplet fit + vote, peaks, candidates, hit assignment), with
the inputs resident in HBM.  Each timed step is bracketed by CUDA events on the stream the
library runs on, and the L2 is flushed (a 512 MB write) between steps outside the timed
window.  `e2e` runs the same steps through trk_reconstruct_host from pinned host memory
(hits in, candidates and hit ids out).  Under torchrun every rank runs its own replica on
its own GPU (events are independent: no collective on the data path); the barrier and the
max over ranks only frame the timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "barrel10_500trk"
BATCH_WORKLOAD = "barrel10_batch256"
# Algorithmic FP32 work of the vote kernel, counted from its formulas as written: each add,
# subtract, multiply, fused multiply-add, min, max, abs, compare, square root, reciprocal
# square root, reciprocal, division, floor, arcsine and arctangent counts 1; selects, sign
# flips and integer work do not count.
#   every enumerated triplet: the curvature test (4 differences, D, |v|^2, |w|^2, 3 products,
#     1 comparison; the pair's own terms are computed once per pair) = 14;
#   every survivor of it: the transverse fit (differences, compensated determinants,
#     circle, q/pT and d0 with their range tests, perigee) = 65;
#   every triplet with q/pT and d0 in range: the longitudinal fit (first arc 17, two
#     hit-to-hit arcs with the turn choice 2 x 46, least-squares line and range tests 37)
#     = 146;
#   every accepted triplet: phi0 and the five bin indices = 31.
# An arcsine or arctangent counts 1 (each is a polynomial of 8 fused multiply-adds here).
OPS_PER_TRIPLET = 14
OPS_PER_FIT = 65
OPS_PER_EXACT = 146
OPS_PER_VOTE = 31
# The method's own work, independent of how the kernel prunes (the roofline's `achieved`):
# every enumerated triplet needs the determinant, the three squared distances and the
# curvature comparison before it can be rejected (the 14 above) plus the reciprocal and
# the products of the q/pT range test, about 31 operations; every accepted triplet needs
# the whole fit, phi0 and the five bins, 65 + 146 + 31 = 242.
METHOD_OPS_PER_TRIPLET = 31
METHOD_OPS_PER_VOTE = 65 + 146 + 31
# Of those, the operations that go to the special-function (MUFU) pipe (16 per SM per
# clock): square roots and reciprocals (one MUFU operation each):
#   every survivor of the curvature test: the transverse fit's 2 square roots and 4
#     reciprocals = 6;
#   every triplet through the longitudinal fit: 1 reciprocal of |c|, 7 square roots and
#     the slope's reciprocal = 9;
#   every accepted triplet: the arctangent's reciprocal = 1.
MUFU_PER_FIT = 6
MUFU_PER_EXACT = 9
MUFU_PER_VOTE = 1


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-variants", action="store_true",
                   help="skip the batched / plain-on-batch / served measurements")
    p.add_argument("--batch-events", type=int, default=256)
    p.add_argument("--serve-seconds", type=float, default=12.0)
    p.add_argument("--hough2d", default=None, metavar="WORKLOAD",
                   help="only time a per-hit 2-D Hough workload (sht_toy50, curved_ip200, "
                        "sht_jets) and print its line")
    p.add_argument("--with-fit", action="store_true",
                   help="also fit a helix to every candidate inside each timed call")
    p.add_argument("--tuning", default=None, metavar="TI,TJ,LEVEL",
                   help="fixed vote-kernel tile and occupancy level instead of the autotuner "
                        "(profiling runs: every vote launch is then the same kernel)")
    return p.parse_args()


def dist_init(n):
    import torch
    if n <= 1 or "RANK" not in os.environ:
        return 0, 1, int(os.environ.get("LOCAL_RANK", 0))
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), int(os.environ.get("LOCAL_RANK", 0))


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(cfg, batch, seconds, threads=None):
    """The FP64 oracle as it stands, on all host cores (or `threads`), over a bounded sample
    of the workload: the first inner hits of every layer triple, until ~`seconds` of CPU
    work."""
    import oracle
    setup = oracle.OracleSetup.from_workload(cfg)
    threads = threads or oracle.max_threads()
    # grow the number of inner hits per layer triple until the run takes long enough
    n_inner = 8
    while True:
        xyz, lay, keep = _inner_subsample(batch, setup, n_inner)
        t0 = time.perf_counter()
        en = oracle.enumerate_batch(xyz, lay, np.array([0, len(xyz)], np.int64), setup, n_threads=threads)
        dt = time.perf_counter() - t0
        if dt > seconds / 4 or n_inner >= 4096:
            break
        n_inner *= 2
    trip_s = en["n_triplets"] / dt
    return trip_s, threads, ("barrel10_500trk event, every layer triple with its first %d inner-layer "
                             "hits (%d triplets, %.1f s); events/s = triplets/s / triplets per event"
                             % (n_inner, en["n_triplets"], dt))


def _inner_subsample(batch, setup, n_inner):
    """Keep only the first n_inner hits of each layer that is the inner layer of some triple
    (all hits of the other layers): every triple's enumeration shrinks proportionally."""
    inner = {int(t[0]) for t in setup.triples}
    keep = []
    for L in range(setup.n_layers):
        idx = np.nonzero(batch.layer == L)[0]
        keep.extend(idx[:n_inner].tolist() if L in inner else idx.tolist())
    keep = np.array(sorted(keep))
    return batch.xyz[keep], batch.layer[keep], keep


def run_reference(args, cfg, batch, rank, world):
    """The oracle arm: bounded samples of the same workload on the host cores."""
    if rank != 0:
        return
    import oracle
    setup = oracle.OracleSetup.from_workload(cfg)
    threads = oracle.max_threads()
    trip_event = int(batch_triplets(batch, cfg))
    xyz, lay, _ = _inner_subsample(batch, setup, 16)
    offs = np.array([0, len(xyz)], np.int64)
    for _ in range(args.warmup):
        oracle.enumerate_batch(xyz, lay, offs, setup, n_threads=threads)
    t0 = time.perf_counter()
    trip = 0
    for _ in range(args.steps):
        en = oracle.enumerate_batch(xyz, lay, offs, setup, n_threads=threads)
        trip += en["n_triplets"]
    dt = time.perf_counter() - t0
    trip_s = trip / dt
    ev_s = trip_s / trip_event
    sample = "first 16 inner-layer hits of every layer triple of the barrel10_500trk event per step"
    line = {"metric": "events/s", "value": ev_s, "unit": "events/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "events_per_step": 1,
                       "triplets_per_event": trip_event},
            "hit_triplets_per_s": trip_s,
            "cpu_baseline": {"value": ev_s, "unit": "events/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": ev_s, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_triplets(batch, cfg):
    from paper_1305_4855_gb300 import events as ev
    return ev.layer_triplet_count(batch, cfg["geometry"]["triples"]).sum()


def main():
    args = parse()
    from paper_1305_4855_gb300 import events as ev
    cfg = ev.load_workload(args.workload)
    batch = ev.make_batch(cfg, n_events=1)
    rank, world, local = dist_init(args.gpus)
    if args.impl == "reference":
        run_reference(args, cfg, batch, rank, world)
        return
    if args.hough2d:
        import torch
        torch.cuda.set_device(local)
        from paper_1305_4855_gb300 import build
        build.build()
        line = {"metric": "events/s", "workload": args.hough2d, "n_gpus": 1,
                **run_hough2d(args.hough2d, local, reps=max(args.steps, 1))}
        line["value"] = line["events_per_s"]
        print(json.dumps(line), flush=True)
        return

    import torch
    torch.cuda.set_device(local)
    from paper_1305_4855_gb300 import build
    build.build()
    from paper_1305_4855_gb300.trk import Reconstructor

    n_trip = int(batch_triplets(batch, cfg))
    fixed = {}
    if args.tuning:
        ti, tj, lv = (int(x) for x in args.tuning.split(","))
        fixed = {"tile_i": ti, "tile_j": tj, "vote_level": lv}
    rec = Reconstructor(cfg, max_events=1, max_hits=batch.n_hits, device=local,
                        vote_capacity=1 << 28, cand_capacity=1 << 21, assign_capacity=1 << 25,
                        fit_candidates=int(args.with_fit), **fixed)
    stream = torch.cuda.Stream()
    hits = torch.from_numpy(batch.packed()).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    tuning = dict(fixed, source="--tuning") if fixed else rec.autotune(hits, offs, reps=2, stream=stream)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            rc = rec.reconstruct_device(hits, offs, stream=stream)
    stats = rec.stats()
    res = rec.result(rc)
    assert res.rc == 0 and int(res.status[0]) == 0, rec.error()

    # ---- device-resident timing --------------------------------------------------------
    torch.cuda.synchronize()
    barrier(world)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xff)
                starts[i].record(stream)
                rec.reconstruct_device(hits, offs, stream=stream)
                ends[i].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms = max_over_ranks(ms, world)
    value = world * args.steps / (ms / 1000.0)
    clocks = clk.summary()

    # ---- vote kernel alone (roofline), same stream, same call ----------------------------
    vote_ms, stage_ms = vote_kernel_ms(rec, hits, offs, stream, flush, max(3, args.steps // 3))

    # ---- end to end through the host C-ABI path ----------------------------------------
    hp = torch.from_numpy(batch.packed()).pin_memory()
    op = torch.from_numpy(batch.offsets.astype(np.int64)).pin_memory()
    rec.reconstruct_host(hp, op, stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rec.reconstruct_host(hp, op, stream=stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    out = rec.out
    h2d = batch.n_hits * 16 + (batch.n_events + 1) * 8
    d2h = int(out.n_candidates) * 48 + int(out.n_hit_ids) * 4 + 8 * (batch.n_events + 1) + 4 * batch.n_events + 128

    peaks = measured_peaks()
    dev = torch.cuda.get_device_properties(local)
    sm_count = dev.multi_processor_count
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    # FP32 lane-operation peak: 128 FP32 lanes per SM per clock
    alu_peak = sm_count * 128 * sm_mhz * 1e6 / 1e12
    kernel_ops = (OPS_PER_TRIPLET * stats["n_triplets"] + OPS_PER_FIT * stats["n_fit"] +
                  OPS_PER_EXACT * stats["n_exact"] + OPS_PER_VOTE * stats["n_votes"]) / 1e12
    method_ops = (METHOD_OPS_PER_TRIPLET * stats["n_triplets"] +
                  METHOD_OPS_PER_VOTE * stats["n_votes"]) / 1e12
    achieved = method_ops / (vote_ms / 1000.0) if vote_ms else None
    kernel_rate = kernel_ops / (vote_ms / 1000.0) if vote_ms else None
    hbm_peak = peaks.get("hbm_gbs")
    nbins = int(rec.lib.trk_histogram_size(rec.h))
    mufu_peak = sm_count * 16 * sm_mhz * 1e6 / 1e12
    mufu_ops = (MUFU_PER_FIT * stats["n_fit"] + MUFU_PER_EXACT * stats["n_exact"] +
                MUFU_PER_VOTE * stats["n_votes"]) / 1e12
    mufu = mufu_ops / (vote_ms / 1000.0) if vote_ms else None
    line = {
        "metric": "events/s", "value": value, "unit": "events/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "events_per_step": 1, "hits_per_event": batch.n_hits,
                   "triplets_per_event": n_trip, "bins": rec.lib.trk_histogram_size(rec.h),
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": "replicas",
                   "tuning": tuning, "candidate_fit": bool(args.with_fit)},
        "hit_triplets_per_s": value * n_trip,
        "stats": {k: stats[k] for k in ("n_triplets", "n_fit", "n_exact", "n_votes", "n_fp64", "n_candidates",
                                        "n_hit_ids", "n_work_items", "n_plateau", "n_cand_votes")},
        "roofline": {"bound": "alu", "kernel": "k_vote", "achieved": achieved, "peak": alu_peak,
                     "unit": "TFLOP/s", "frac": (achieved / alu_peak) if achieved else None,
                     "traffic": vote_traffic(args.workload, tuning), "vote_kernel_ms": vote_ms,
                     "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (median SM clock under load)"
                                   % (sm_count, sm_mhz),
                     "achieved_basis": "the method's work: %d FP32 ops per enumerated triplet + "
                                       "%d per accepted triplet (vote kernel stats of the call)"
                                       % (METHOD_OPS_PER_TRIPLET, METHOD_OPS_PER_VOTE),
                     "peak_source": "derived (SM count x lanes x sampled clock)",
                     "issue_frac": (kernel_rate / alu_peak) if kernel_rate else None,
                     "issue_basis": "the operations the kernel executes by design: %d per "
                                    "enumerated triplet + %d per curvature survivor + %d per "
                                    "triplet with q/pT and d0 in range + %d per vote"
                                    % (OPS_PER_TRIPLET, OPS_PER_FIT, OPS_PER_EXACT, OPS_PER_VOTE),
                     "mufu": {"achieved": mufu, "peak": mufu_peak, "unit": "T ops/s",
                              "frac": (mufu / mufu_peak) if mufu else None,
                              "basis": "%d special-function ops per curvature survivor + %d "
                                       "per longitudinal fit + %d per vote; %d SMs x 16 per "
                                       "clock" % (MUFU_PER_FIT, MUFU_PER_EXACT, MUFU_PER_VOTE,
                                                  sm_count)}},
        "e2e": {"value": world * args.steps / e2e_s, "unit": "events/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "stage_ms": stage_ms,
        "hbm_rooflines": {
            "peaks": {"kernels": "k_peak_pass1, k_peak_pass2, k_peak_ties (+ bitmap clears)",
                      "bytes": 4 * nbins, "ms": stage_ms.get("peaks"),
                      "achieved_gbs": (4 * nbins / (stage_ms["peaks"] / 1000.0) / 1e9)
                      if stage_ms.get("peaks") else None,
                      "peak_gbs": hbm_peak, "peak_source": "measured (MEASURED_PEAKS.json)",
                      "basis": "one read of the event's dense histogram (4 B per bin)"},
            "assign": {"kernels": "k_assign_scan, k_assign_cvotes, k_cand_hits, scans, k_compact",
                       "bytes": 4 * stats["n_votes"], "ms": stage_ms.get("assign"),
                       "achieved_gbs": (4 * stats["n_votes"] / (stage_ms["assign"] / 1000.0) / 1e9)
                       if stage_ms.get("assign") else None,
                       "peak_gbs": hbm_peak, "peak_source": "measured (MEASURED_PEAKS.json)",
                       "basis": "one read of each vote's bin (4 B per vote)"}},
        "clocks": clocks,
        "gpu_launches": args.steps * (LAUNCHES_PER_CALL + int(args.with_fit)),
    }
    for r in line["hbm_rooflines"].values():
        r["frac"] = (r["achieved_gbs"] / r["peak_gbs"]) if r["achieved_gbs"] and r["peak_gbs"] else None
    rec.close()
    if not args.no_variants:
        line["variants"] = run_variants(args, local)
    if rank == 0 and not args.no_cpu_baseline:
        trip_s, cores, sample = cpu_baseline(cfg, batch, args.cpu_seconds)
        line["cpu_baseline"] = {"value": trip_s / n_trip, "unit": "events/s", "cores": cores,
                                "kind": "oracle", "sample": sample}
        trip_1, _, sample_1 = cpu_baseline(cfg, batch, args.cpu_seconds / 3, threads=1)
        line["cpu_baseline"]["single_thread"] = {"value": trip_1 / n_trip, "unit": "events/s",
                                                 "cores": 1, "sample": sample_1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_variants(args, local):
    """Batched (the 256-event uneven workload in one call when its vote lists fit the free
    device memory, else in the largest memory-sized sub-batches), the same events through
    the plain path one call each, and serving: the plain host path and the continuous-
    batching server driven by the same Poisson arrival stream."""
    import torch
    from paper_1305_4855_gb300 import events as ev
    from paper_1305_4855_gb300.trk import Reconstructor
    cfg = ev.load_workload(BATCH_WORKLOAD)
    batch = ev.make_batch(cfg, n_events=args.batch_events)
    trip_ev = ev.layer_triplet_count(batch, cfg["geometry"]["triples"]).astype(np.int64)
    n_trip = int(trip_ev.sum())
    out = {"candidate_fit": run_fit(args, local),
           "hough2d": {w: run_hough2d(w, local) for w in ("sht_toy50", "curved_ip200", "sht_jets")}}
    per_event_max = int(np.diff(batch.offsets).max())
    packed = torch.from_numpy(batch.packed()).cuda()
    stream = torch.cuda.Stream()
    # --- the same events through the plain path, one call per event (also measures the
    #     acceptance fraction that sizes the batched call's vote list)
    rec = Reconstructor(cfg, max_events=1, max_hits=per_event_max, device=local,
                        vote_capacity=1 << 29, cand_capacity=1 << 21, assign_capacity=1 << 25)
    evs = [(packed[int(batch.offsets[e]):int(batch.offsets[e + 1])].contiguous(),
            torch.tensor([0, int(batch.offsets[e + 1] - batch.offsets[e])], dtype=torch.int64,
                         device="cuda")) for e in range(batch.n_events)]
    rec.autotune(evs[0][0], evs[0][1], reps=1, stream=stream)
    with torch.cuda.stream(stream):
        rec.reconstruct_device(evs[0][0], evs[0][1], stream=stream)
    torch.cuda.synchronize()
    lat, done_t, votes = [], [], 0
    plain_stages = {}

    def add_stages(acc, st):
        for k, v in st.items():
            acc[k] = acc.get(k, 0.0) + v
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for h_, o_ in evs:
            t1 = time.perf_counter()
            rec.reconstruct_device(h_, o_, stream=stream)    # returns after its counts sync
            t2 = time.perf_counter()
            lat.append(t2 - t1)
            done_t.append(t2 - t0)
            votes += rec.stats()["n_votes"]
            add_stages(plain_stages, rec.stage_ms(stream))   # events of the call (no sync left)
    wall = time.perf_counter() - t0
    out["plain_on_batch_events"] = {
        "events_per_s": batch.n_events / wall, "hit_triplets_per_s": n_trip / wall, "ms": 1000 * wall,
        "p50_ms": 1000 * float(np.percentile(lat, 50)), "p99_ms": 1000 * float(np.percentile(lat, 99)),
        "all_at_once": {"p50_ms": 1000 * float(np.percentile(done_t, 50)),
                        "p99_ms": 1000 * float(np.percentile(done_t, 99))},
        "votes": int(votes), "acceptance": votes / n_trip,
        "device_stage_ms": plain_stages}
    rec.close()
    # --- batched: the whole mix in one call if its vote list and histograms fit
    free_b = torch.cuda.mem_get_info()[0]
    nbins = int(np.prod(cfg["binning"]["n"]))
    accept = 1.1 * votes / n_trip                          # 10 % headroom on the measured rate

    def call_bytes(first, last):
        v = accept * trip_ev[first:last].sum()
        e = last - first
        return 8.75 * v + e * (4 * nbins + 8 * ((nbins + 31) // 32)) + (3 << 30)
    sub = batch.n_events
    while sub > 1 and max(call_bytes(s0, min(batch.n_events, s0 + sub))
                          for s0 in range(0, batch.n_events, sub)) > 0.9 * free_b:
        sub //= 2
    vcap = int(max(accept * trip_ev[s0:s0 + sub].sum() for s0 in range(0, batch.n_events, sub)))
    rec = Reconstructor(cfg, max_events=sub, max_hits=int(batch.offsets[-1]), device=local,
                        vote_capacity=vcap, cand_capacity=1 << 25, assign_capacity=1 << 29)
    chunks = []
    for s0 in range(0, batch.n_events, sub):
        s1 = min(batch.n_events, s0 + sub)
        a, b_ = int(batch.offsets[s0]), int(batch.offsets[s1])
        chunks.append((packed[a:b_].contiguous(),
                       torch.from_numpy(batch.offsets[s0:s1 + 1] - a).cuda(), s1 - s0))
    tune_n = min(32, sub)
    a_, b_ = int(batch.offsets[0]), int(batch.offsets[tune_n])
    tuning = rec.autotune(packed[a_:b_].contiguous(),
                          torch.from_numpy(batch.offsets[:tune_n + 1] - a_).cuda(), reps=1,
                          stream=stream)
    with torch.cuda.stream(stream):
        rec.reconstruct_device(chunks[0][0], chunks[0][1], stream=stream)    # graph capture
    torch.cuda.synchronize()
    failed, done_b, batch_stages = 0, [], {}
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for h_, o_, n_ in chunks:
            rc = rec.reconstruct_device(h_, o_, stream=stream)
            failed += int(rc != 0)
            done_b += [time.perf_counter() - t0] * n_
            add_stages(batch_stages, rec.stage_ms(stream))
    wall = time.perf_counter() - t0
    out["batched"] = {"workload": BATCH_WORKLOAD, "events": batch.n_events, "sub_batch": sub,
                      "calls": len(chunks), "events_per_s": batch.n_events / wall,
                      "hit_triplets_per_s": n_trip / wall, "ms": 1000 * wall,
                      "all_at_once": {"p50_ms": 1000 * float(np.percentile(done_b, 50)),
                                      "p99_ms": 1000 * float(np.percentile(done_b, 99))},
                      "calls_with_capacity_errors": failed, "tuning": tuning,
                      "device_stage_ms": batch_stages,
                      "memory": {"free_gb": free_b / 1e9, "vote_capacity": vcap,
                                 "largest_call_gb": max(call_bytes(s0, min(batch.n_events, s0 + sub))
                                                        for s0 in range(0, batch.n_events, sub)) / 1e9,
                                 "whole_mix_gb": call_bytes(0, batch.n_events) / 1e9,
                                 "basis": "8.75 B per vote (bin, code, chunk record) at 1.1 x the "
                                          "measured acceptance, 4 B per bin and 8 B per 32 bins "
                                          "per event, 3 GB of other pools"}}
    rec.close()
    # --- serving, like for like: host events in, results on the host, same arrivals
    out["serving"] = run_serving(args, cfg, batch, local)
    return out


def run_serving(args, cfg, batch, local):
    """Plain host path (one trk_reconstruct_host per event, first come first served, on one
    thread) and the server, each fed the same events at the same Poisson arrival times.
    Latency: arrival to results on the host.  The rate is a stated fraction of the plain
    path's measured capacity; a second run offers every event at once (saturation)."""
    from paper_1305_4855_gb300.trk import Reconstructor, Server
    per_event_max = int(np.diff(batch.offsets).max())
    hosts = [np.ascontiguousarray(batch.packed()[int(batch.offsets[e]):int(batch.offsets[e + 1])])
             for e in range(batch.n_events)]
    import torch
    pinned = [torch.from_numpy(h).pin_memory() for h in hosts]
    offs = [torch.tensor([0, len(h)], dtype=torch.int64).pin_memory() for h in hosts]
    rec = Reconstructor(cfg, max_events=1, max_hits=per_event_max, device=local,
                        vote_capacity=1 << 29, cand_capacity=1 << 21, assign_capacity=1 << 25)
    rec.reconstruct_host(pinned[0], offs[0])
    # plain capacity: every event back to back through the host path
    t0 = time.perf_counter()
    for e in range(len(hosts)):
        rec.reconstruct_host(pinned[e], offs[e])
    cap_plain = len(hosts) / (time.perf_counter() - t0)
    frac = 0.8
    rate = frac * cap_plain
    n = min(len(hosts), max(64, int(rate * args.serve_seconds / 2)))
    rng = np.random.default_rng(5)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))

    def pct(x):
        return {"p50_ms": 1000 * float(np.percentile(x, 50)),
                "p99_ms": 1000 * float(np.percentile(x, 99)),
                "p999_ms": 1000 * float(np.percentile(x, 99.9))}

    def plain_run(arr):
        lat = []
        t0 = time.perf_counter()
        for e in range(n):
            now = time.perf_counter() - t0
            if arr[e] > now:
                time.sleep(arr[e] - now)
            rec.reconstruct_host(pinned[e], offs[e])
            lat.append(time.perf_counter() - t0 - arr[e])
        wall = time.perf_counter() - t0
        return dict(events=n, events_per_s=n / wall, **pct(lat))
    res = {"arrival_rate_hz": rate, "load": "%.1f of the plain path's measured capacity" % frac,
           "plain_capacity_events_per_s": cap_plain, "events": n,
           "plain": plain_run(arrivals), "plain_saturated": plain_run(np.zeros(n))}
    rec.close()

    def served_run(arr, lanes, lane_events):
        srv = Server(cfg, lane_events=lane_events, lane_hits=lane_events * per_event_max,
                     n_lanes=lanes, device=local, vote_capacity=0, cand_capacity=1 << 22,
                     assign_capacity=1 << 26)
        for t in [srv.submit(hosts[i]) for i in range(2 * lanes)]:
            srv.wait(t, 120.0)
        tickets = []
        t0 = time.perf_counter()
        for e in range(n):
            now = time.perf_counter() - t0
            if arr[e] > now:
                time.sleep(arr[e] - now)
            tickets.append(srv.submit(hosts[e]))
        lats, nb = [], []
        for t in tickets:
            info = srv.wait(t, 600.0)
            lats.append(info["latency_s"])
            nb.append(info["batch_events"])
        wall = time.perf_counter() - t0
        srv.close()
        return dict(events=n, events_per_s=n / wall, mean_batch_events=float(np.mean(nb)),
                    lanes=lanes, lane_events=lane_events, **pct(lats))
    res["served"] = served_run(arrivals, 2, 4)
    res["served_saturated"] = served_run(np.zeros(n), 2, 4)
    res["note"] = ("prefix of the 1e6-event stream: %d events of the batch mix; server lanes "
                   "sized from free device memory, graphs captured at creation" % n)
    return res


def run_fit(args, local):
    """The candidate fit on the 500-track event: its stage time inside the call (CUDA
    events around the fit kernel; the stage also holds the final offsets kernel and the
    small count copies), and candidates fitted per second."""
    import torch
    from paper_1305_4855_gb300 import events as ev
    from paper_1305_4855_gb300.trk import Reconstructor
    cfg = ev.load_workload(WORKLOAD)
    batch = ev.make_batch(cfg, n_events=1)
    rec = Reconstructor(cfg, max_events=1, max_hits=batch.n_hits, device=local,
                        vote_capacity=1 << 28, cand_capacity=1 << 21, assign_capacity=1 << 25,
                        fit_candidates=1)
    stream = torch.cuda.Stream()
    hits = torch.from_numpy(batch.packed()).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    fits = []
    for i in range(8):
        with torch.cuda.stream(stream):
            rec.reconstruct_device(hits, offs, stream=stream)
        st = rec.stage_ms(stream)
        if i >= 3:
            fits.append(st["fit"])
    n_cand = rec.stats()["n_candidates"]
    res = rec.result(0)
    rec.close()
    ms = float(np.mean(fits))
    return {"workload": WORKLOAD, "candidates": int(n_cand), "fit_stage_ms": ms,
            "candidates_per_s": n_cand / (ms / 1000.0),
            "status_ok_fraction": float(np.mean(res.tracks["status"] == 0)) if n_cand else None}


def run_hough2d(workload, local, reps=5):
    """A per-hit 2-D Hough workload, all its events in one call (hits resident): events/s of
    the whole call and the vote-and-peak kernel's vote rate (hits x columns per second)."""
    import torch
    from paper_1305_4855_gb300 import events as ev
    from paper_1305_4855_gb300.trk import Hough2D
    cfg = ev.load_workload(workload)
    batch = ev.make_batch(cfg)
    h2 = Hough2D(cfg, max_events=batch.n_events, max_hits=batch.n_hits, device=local,
                 cand_capacity=1 << 22, hit_capacity=1 << 26)
    hits = torch.from_numpy(batch.packed()).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    tot, vp = [], []
    for i in range(reps + 2):
        flush.fill_(i & 0xff)
        torch.cuda.synchronize()
        rc = h2.reconstruct_device(hits, offs)
        assert rc == 0, h2.error()
        ms = h2.last_ms()
        if i >= 2:
            tot.append(ms["total"])
            vp.append(ms["vote_peak"])
    n_cand = int(h2.out.n_candidates)
    n_vtx = int(h2.out.n_vertices)
    h2.close()
    t, v = float(np.mean(tot)), float(np.mean(vp))
    votes = batch.n_hits * cfg["hough2d"]["n_cols"]
    out = {"events": batch.n_events, "hits": batch.n_hits, "candidates": n_cand,
           "call_ms": t, "events_per_s": batch.n_events / (t / 1000.0),
           "vote_peak_ms": v, "hit_columns_per_s": votes / (v / 1000.0),
           "l2": "flushed before each call (512 MB write)"}
    if "vertex" in cfg["hough2d"]:
        out["vertices"] = n_vtx
    return out


# kernels of one trk_reconstruct call for a one-event batch: pack, schedule, vote,
# 2 peak passes + the tie pass, 3 scan kernels x 3 scans, candidate emission, assignment
# (vote stream + candidate votes), hit lists, compaction, finalize
LAUNCHES_PER_CALL = 1 + 1 + 1 + 3 + 9 + 1 + 2 + 1 + 1 + 1

# DRAM traffic of one vote-kernel launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# ncu captures of the bench workload, one record per vote-kernel tuning; a record stands
# only while the vote-kernel sources hash to the recorded digest, and the traffic is
# reported as null for a tuning without a record.
VOTE_TRAFFIC = {"workload": "barrel10_500trk",
                "sources_sha256": "eb2709d8e7a920291cd8b6a360cb81f62862d1a0e5e65b135506fa4f15531037",
                "records": [{"tile_i": 8, "tile_j": 4, "vote_level": 3,
                             "bytes": 0.97245824e9 + 2.792216064e9},
                            {"tile_i": 8, "tile_j": 4, "vote_level": 4,
                             "bytes": 1.099234816e9 + 2.996451328e9}]}
VOTE_SOURCES = ["trk_common.cuh", "trk_vote_kernel.cuh", "trk_vote.cu", "trk_vote_l2.cu",
                "trk_vote_l3.cu", "trk_vote_l4.cu"]


def vote_sources_digest():
    import hashlib
    h = hashlib.sha256()
    for f in VOTE_SOURCES:
        with open(os.path.join(ROOT, "paper_1305_4855_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def vote_traffic(workload, tuning):
    t = VOTE_TRAFFIC
    if workload != t["workload"] or vote_sources_digest() != t["sources_sha256"]:
        return None
    for r in t["records"]:
        if all(tuning.get(k) == r[k] for k in ("tile_i", "tile_j", "vote_level")):
            return r["bytes"]
    return None


def vote_kernel_ms(rec, hits, offs, stream, flush, reps):
    """Average device time of the vote kernel over `reps` calls, from the CUDA events the
    library records around it on the call's stream (L2 flushed before each call)."""
    import torch
    tot = 0.0
    stages = {}
    for i in range(reps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xff)
            rec.reconstruct_device(hits, offs, stream=stream)
        st = rec.stage_ms(stream)
        tot += st["vote"]
        for k, v in st.items():
            stages[k] = stages.get(k, 0.0) + v / reps
    return tot / reps, stages


if __name__ == "__main__":
    main()
