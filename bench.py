#!/usr/bin/env python3
"""Throughput benchmark: macro-particle-turns per second on the 390-bunch fill.

Workload: 390 bunches in buckets 0..389 of an h = 480 SLS-like ring (a
90-bucket ion-cleaning gap), 1e5 macro-particles and 0.5 mA per bunch,
broadband (5 kOhm, 10 GHz, Q = 1) + HOM (1 MOhm, 1.5 GHz, Q = 2e4, short and
long range) wakes, mixed precision (tau FP32, delta FP64, tensor-core wake,
FP64 phasor scan and moments).  A step is one turn of the whole hot path for
every bunch: push kernel (kick, RF, damping + excitation, drift, binning,
moment partials) and post kernel (short-range wake on the tensor cores,
long-range phasor scan, moments).  The state (468 MB) is larger than the
129 MB L2, so no flush is needed between turns.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank tracks its own fill (weak scaling, no data-path
collective); rank 0 prints one JSON line.

Serving: python bench.py --workload serving [--requests R] [--rate HZ]
replays an open-loop Poisson stream of instability-scan requests (sizes
drawn as in mbt_workloads.serving_stream) into the continuous-batching
server and prints one JSON line with the p50/p99 latency (arrival to
result) and the delivered throughput.

L5 scan: python bench.py --workload l5scan tracks the SLS-2 L5 HOM detuning
scan (Sec. 5: the 400 mA uniform and 3/4 fills of the h = 484 ring, 25 HOM
frequencies across one revolution-harmonic period) as one batch and prints
its throughput and the growth-rate table (measured, and Eq. 7 for the
uniform fill).

Resistive-wall current scan: python bench.py --workload rwscan tracks a
single bunch of the 'dc12c' ring in the short-range resistive-wall wake of a
copper pipe of 10 mm radius around the ring (Sec. 3) at 12 currents, one
batch, 50 000 turns, and prints the 'equilibrium' bunch length and energy
spread (averages over the last 5000 turns) per current.

Harmonic-cavity scan: python bench.py --workload hcscan tracks a single 1 mA
bunch of ring R0 with the broadband wake and an active third-harmonic
cavity at fractions 0 ... 1.2 of the flat-potential voltage (one batch) and
prints the equilibrium bunch length per setting.

Transverse plane: python bench.py --workload fill390t tracks the 390-bunch
fill with a horizontal plane (beta 10 m, tune 0.31, chromaticity 1.5,
1 nm) and a transverse HOM (200 kOhm/m, 1.5 GHz, Q 2e4, short and long
range) besides the longitudinal wakes, and prints its throughput and the
push roofline (40 B per macro-particle-turn: tau, delta, x, x').

FP64 tracker: python bench.py --workload three_f64 tracks three bunches of
1e5 macro-particles (broadband + HOM, long and short range) on the FP64 path
and prints its throughput and the FP64 push's time per launch;
--workload fill390_f64 tracks the 390-bunch fill on the FP64 path and on the
mixed path, and prints both throughputs and the FP64 push against the GPU's
measured DFMA throughput.

Cluster-resident tracking: python bench.py --workload resident [--steps K]
tracks one bunch of 1e4 and one of 1e5 macro-particles (broadband wake) and
three bunches of 1e5 with the long-range HOM resident (mbt_track_resident, K
turns in one launch) and through the per-turn kernels, and prints the time
per turn of each.

The default line also carries a bounded serving sample (--serving-requests,
Poisson requests at about the server's capacity: p50/p99 latency) and the
FP64 oracle timed on all host cores (one process per core, each tracking a
contiguous subset of the bunches).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mbt_workloads as W  # noqa: E402

METRIC = "macro-particle-turns/s (390-bunch fill)"
UNIT = "mp-turns/s"
BYTES_PER_MP_TURN = 24          # tau f32 + delta f64, read + written once per turn
FALLBACK_HBM_GBS = 6800.0
PUSH_SOURCES = ["paper_1809_00391_gb300/csrc/k_push.cu", "paper_1809_00391_gb300/csrc/push_core.cuh",
                "paper_1809_00391_gb300/csrc/device_common.cuh", "paper_1809_00391_gb300/csrc/mbt_internal.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "push_stream_fill390_traffic.json")
GRAPH_TURNS = 100      # turns per captured CUDA graph
# batch lanes (mbt_batch_set_lanes) per scan workload: the measured best
LANES = {"l5scan": 4, "rwscan": 3, "hcscan": 2, "serving": 2}
AUTOTUNE_TURNS = 20    # timed turns per push-tile candidate
ROOFLINE_TURNS = 4000  # turns of the event-timed roofline region
SATURATED_TURNS = 200  # turns of the event-timed region in the saturated instability


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--state-file", default="/tmp/mbt_fill390.state", help="state: checkpoint of the fill")
    ap.add_argument("--at-turn", type=int, default=1500, help="state: turn at which the checkpoint is taken")
    ap.add_argument("--transverse", action="store_true", help="state: the 390-bunch fill with a transverse plane")
    ap.add_argument("--serving-requests", type=int, default=40,
                    help="requests of the bounded serving sample in the default line (0 = skip)")
    ap.add_argument("--saturated-turn", type=int, default=1500,
                    help="also time the push from this turn on (saturated instability); 0 = skip")
    ap.add_argument("--lanes", type=int, default=0,
                    help="l5scan, rwscan, hcscan, serving: groups of runs tracked on streams of their own "
                         "(mbt_batch_set_lanes); 0: the workload's default (LANES)")
    ap.add_argument("--tile", type=int, default=0,
                    help="particles per push CTA; 0 = autotune (timed trial turns during warm-up)")
    ap.add_argument("--workload", choices=["fill390", "serving", "l5scan", "rwscan", "hcscan", "fill390t", "three_f64",
                                           "fill390_f64", "state", "resident"],
                    default="fill390")
    ap.add_argument("--requests", type=int, default=200, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: Poisson arrival rate (1/s)")
    ap.add_argument("--max-active", type=int, default=16, help="serving: requests tracked together")
    ap.add_argument("--turns-per-step", type=int, default=200, help="serving: turns between admissions")
    return ap.parse_args()


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest x over the ranks of the process group (x itself alone)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_run(rank: int) -> W.Run:
    """The fill a rank tracks: every rank its own 390-bunch fill (independent
    replicas, weak scaling; no data-path collective)."""
    return W.fill_390(seed=1 + rank, precision=W.PREC_MIXED)


def weak_scaling_value(units_per_rank: int, steps: int, world: int, t_max_ms: float) -> float:
    """Whole-job throughput: all ranks' units x steps over the slowest rank's time."""
    return units_per_rank * steps * world / (t_max_ms * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in PUSH_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(n_particles: int):
    """DRAM bytes per push launch from the committed ncu capture, if it was
    taken on the current kernel source (else None)."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != kernel_source_hash():
        return None
    return float(t["dram_bytes_per_particle"]) * n_particles


# NVML clock-event reason bits reported in the clocks summary
CLOCK_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
                 0x80: "hw_power_brake_slowdown"}


class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml ships with the
    driver): SM clock, its maximum, power and the active clock-event reasons."""

    SM = 1            # NVML_CLOCK_SM

    def __init__(self, local_index: int):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            pr = torch.cuda.get_device_properties(local_index)
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0".encode()
            ok = self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(self.h)) == 0
        except Exception:
            ok = False
        if not ok:
            vis = [x.strip() for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
            idx = int(vis[local_index]) if local_index < len(vis) and vis[local_index].isdigit() else local_index
            if self.lib.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(self.h)) != 0:
                raise RuntimeError("no NVML handle")
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn if fn is not None else self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        v = ctypes.c_uint()
        self.max_mhz = float(v.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, ctypes.byref(v)) == 0 \
            else float("nan")

    def sample(self):
        ct = self.ct
        c, pw, r = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, ct.byref(c)) != 0:
            return None
        self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(pw))
        self.reasons_fn(self.h, ct.byref(r))
        return float(c.value), pw.value / 1000.0, int(r.value)


class ClockSampler:
    """SM clocks and clock-event reasons sampled during the timed region:
    NVML queried from a host thread every ~0.25 ms (so that a region of a few
    milliseconds still gets samples), else nvidia-smi every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_index: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        self.gpu = ids[local_index] if local_index < len(ids) else str(local_index)
        self.local = local_index
        self.proc = None
        self.path = None
        self.nvml = None
        self.rows = []
        self.thread = None
        self.stop = False

    def __enter__(self):
        import threading
        try:
            self.nvml = _Nvml(self.local)
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            first = self.nvml.sample()
            if first is not None:
                self.rows.append(first)

            def loop():
                while not self.stop:
                    x = self.nvml.sample()
                    if x is not None:
                        self.rows.append(x)
                    time.sleep(0.00025)
            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop = True
            self.thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.nvml is not None:
            return self._summary_nvml()
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        sm = np.array([num(r[1]) for r in rows])
        smax = np.array([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(np.nanmax(smax)), "reasons": reasons,
                "samples": len(rows), "source": "nvidia-smi"}

    def _summary_nvml(self):
        rows = list(self.rows)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": self.nvml.max_mhz, "reasons": ["no NVML samples"], "samples": 0,
                    "source": "nvml"}
        sm = np.array([r[0] for r in rows])
        pw = np.array([r[1] for r in rows])
        reasons = sorted({name for r in rows for bit, name in CLOCK_REASONS.items() if r[2] & bit})
        return {"sm_mhz": float(np.median(sm)), "sm_min_mhz": float(sm.min()), "sm_max_mhz": self.nvml.max_mhz,
                "power_w_max": float(pw.max()), "reasons": reasons, "samples": len(rows), "source": "nvml"}


def _oracle_part(args):
    """One worker of the CPU baseline: the oracle (single-threaded) tracking
    bunches [lo, hi) of the fill as a fill of their own."""
    sys.path.insert(0, ROOT)
    import oracle
    run, lo, hi, turns = args
    part = W.Run(run.ring, run.resonators, run.buckets[lo:hi], run.currents_A[lo:hi], run.n_mp[lo:hi],
                 seed=run.seed, turns=turns, precision=run.precision, flags=run.flags, nbins=run.nbins,
                 half_width_sigmas=run.half_width_sigmas)
    s = oracle.OracleSim(part.ring, part.resonators, part.nbins, part.half_width_sigmas, part.buckets,
                         part.currents_A, part.n_mp, part.seed, part.flags)
    s.init_particles()
    t0 = time.perf_counter()
    s.track(turns, record=False)
    dt = time.perf_counter() - t0
    s.close()
    return int(part.n_particles) * turns, dt


def cpu_baseline(run: W.Run, turns: int = 2, workers: int = 0):
    """The FP64 oracle on this host's cores, on a bounded sample: `turns`
    turns of the full fill, its bunches split into one contiguous subset per
    core, each tracked by a single-threaded oracle in a worker process as a
    fill of its own (throughput only: the subsets do not see each other's
    long-range wake).  The pool is started with spawn before any GPU work of
    the worker processes."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    n = workers or (os.cpu_count() or 1)
    n = max(1, min(n, run.nb))
    bounds = [(k * run.nb) // n for k in range(n + 1)]
    jobs = [(run, bounds[k], bounds[k + 1], turns) for k in range(n)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(n) as pool:
        res = pool.map(_oracle_part, jobs)
    wall = time.perf_counter() - t0
    work = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    v = work / busy
    return {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{turns} turns of the full {run.nb}-bunch fill ({run.n_particles} mp), FP64, split into "
                      f"{n} bunch subsets tracked independently by {n} single-threaded oracle processes; "
                      f"slowest worker {busy:.1f} s (wall {wall:.1f} s with process start)",
            "per_core": v / n}


def reference_arm(args, rank, world):
    """The oracle as the reference implementation: each step tracks one turn of
    a bounded sample of the workload (the first 4 bunches of the fill, with
    as many macro-particles per bunch as fit a ~150 s total budget)."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    full = W.fill_390()
    steps, warm = args.steps, args.warmup
    # cost probe: one turn of 4 x 2000 particles
    probe = full.scaled(n_mp_per_bunch=2000, nb=4)
    s = oracle.OracleSim(probe.ring, probe.resonators, probe.nbins, probe.half_width_sigmas, probe.buckets,
                         probe.currents_A, probe.n_mp, probe.seed, probe.flags)
    s.init_particles()
    t0 = time.perf_counter()
    s.track(3, record=False)
    per_mp = (time.perf_counter() - t0) / (3 * probe.n_particles)
    s.close()
    budget = 150.0
    n_per = int(max(2, min(100_000, budget / max(1, steps + warm) / (4 * per_mp))))
    sample = full.scaled(n_mp_per_bunch=n_per, nb=4)
    s = oracle.OracleSim(sample.ring, sample.resonators, sample.nbins, sample.half_width_sigmas, sample.buckets,
                         sample.currents_A, sample.n_mp, sample.seed, sample.flags)
    s.init_particles()
    s.track(warm, record=False)
    t0 = time.perf_counter()
    s.track(steps, record=False)
    dt = time.perf_counter() - t0
    s.close()
    v = sample.n_particles * steps / dt
    desc = f"each step: one turn of the first 4 bunches of the fill with {n_per} mp each (FP64 oracle, 1 core)"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": steps,
            "warmup": warm, "ms_per_step": dt / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": full.name, "sample": desc},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serving_sample(n_requests: int, rate_hz: float, max_active: int = 16, turns_per_step: int = 200,
                   budget: int = 64 << 30, seed: int = 7, lanes: int = 1):
    """Open-loop replay of a Poisson request stream into the continuous-
    batching server: each request is submitted at its arrival time (a host
    thread sleeps until then); latency = result time - submission time on the
    server's clock.  Returns (latencies, queue waits, delivered mp-turns/s,
    stats, span)."""
    import threading
    import paper_1809_00391_gb300 as pkg
    stream = W.serving_stream(n_requests, rate_hz=rate_hz, seed=seed)
    work = np.array([rq.run.turns * rq.run.n_particles for rq in stream], np.float64)
    srv = pkg.Server(hbm_budget_bytes=budget, max_active=max_active, turns_per_step=turns_per_step, lanes=lanes)
    ids = [None] * len(stream)
    t_wall0 = time.perf_counter()

    def feeder():
        for i, rq in enumerate(stream):
            delay = rq.arrival_s - (time.perf_counter() - t_wall0)
            if delay > 0:
                time.sleep(delay)
            ids[i] = srv.submit(rq.run)

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    for rid in ids:
        srv.wait(rid, timeout_s=3600)
    st = [srv.status(rid) for rid in ids]
    lat = np.array([x["t_finish"] - x["t_submit"] for x in st])
    queue = np.array([x["t_start"] - x["t_submit"] for x in st])
    span = max(x["t_finish"] for x in st) - min(x["t_submit"] for x in st)
    stats = srv.stats()
    srv.close()
    return lat, queue, work, stats, span


def serving_bench(args, rank, local):
    """The serving workload: an open-loop Poisson stream of instability-scan
    requests into mbt_server (serving_sample), with p50/p99 latency, queue
    wait and delivered throughput."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    budget = 64 << 30
    with ClockSampler(local) as clk:
        lat, queue, work, stats, span = serving_sample(args.requests, args.rate, args.max_active,
                                                       args.turns_per_step, budget,
                                                       lanes=args.lanes or LANES["serving"])
    clocks = clk.summary()
    thr = work.sum() / span
    line = {"metric": "serving latency p99 (instability-scan requests, open-loop Poisson stream)",
            "value": float(np.percentile(lat, 99)), "unit": "s", "n_gpus": 1, "higher_is_better": False,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "queue_p50_s": float(np.percentile(queue, 50)), "queue_p99_s": float(np.percentile(queue, 99)),
            "throughput": thr, "throughput_unit": UNIT, "span_s": span,
            "busy_s": stats["busy_seconds"], "steps": stats["steps"],
            "capacity_rate_hz": thr / work.mean(),
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Poisson stream, {args.requests} requests at {args.rate} /s (seed 7)",
                       "mean_mp_turns_per_request": float(work.mean()), "offered_mp_turns_per_s":
                       float(work.mean() * args.rate), "max_active": args.max_active,
                       "turns_per_step": args.turns_per_step, "hbm_budget_bytes": budget,
                       "lanes": args.lanes or LANES["serving"],
                       "max_active_seen": stats["max_active_seen"], "max_bytes_seen": stats["max_bytes_seen"]},
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def l5scan_bench(args, rank, local):
    """The L5 detuning scan as one batch: throughput of the tracking (CUDA
    events around the batched turns) and the growth rates per detuning."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    from paper_1809_00391_gb300 import scan as S
    pkg.build()
    ring = W.ring_dc12c()
    f0 = 1.0 / ring["T0_s"]
    det = np.linspace(-600e3, 600e3, 25)
    turns, n_mp = 6000, 5000
    runs = W.l5_scan_runs(det, "uniform", n_mp=n_mp, turns=turns) + \
        W.l5_scan_runs(det, "three_quarter", n_mp=n_mp, turns=turns, seed=211)
    trackers = [pkg.tracker_for_run(r, record_turns=turns) for r in runs]
    stream = torch.cuda.current_stream()
    for t in trackers:
        t.init_particles(stream)
    b = pkg.Batch(trackers)
    b.set_graph(GRAPH_TURNS)
    lanes = args.lanes or LANES["l5scan"]
    b.set_lanes(lanes)   # groups of runs on streams of their own: one group's push beside another's post
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        b.track(turns, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    b.sync()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    mp = sum(r.n_particles for r in runs)
    recs = [t.moments(0, turns) for t in trackers]
    b.close()
    for t in trackers:
        t.close()
    damp = 1.0 / ring["tau_z_s"]
    fit = (1500, 4500)   # mode fits: clear of the start-up and of the nonlinear regime
    table = []
    for i, df in enumerate(det):
        ru, rq = recs[i], recs[len(det) + i]
        eq7 = S.eq7_growth_rates(ring, ring["h"], 0.4 / ring["h"], W.L5_RS_OHM, W.L5_FR_HZ + df, W.L5_Q)
        mu, rate = S.dominant_mode(ru, ring, *fit)

        def factor(rec):
            a = S.rms_amplitude(rec, ring)
            return round(float(np.nanmean(a[turns - 1100:turns - 250]) / np.nanmean(a[250:1100])), 2)

        amp = S.oscillation_amplitudes(rq, ring)
        cap = 0.2 * float(np.mean(rq[:200, :, 1]))
        fml = [S.adaptive_rate(amp[:, m], ring["T0_s"], cap=cap) for m in (0, 181, 362)]
        table.append({"detuning_kHz": round(df / 1e3, 1),
                      "eq7_fastest_mode": int(np.argmax(eq7)),
                      "eq7_max_minus_damping_per_s": round(float(eq7.max() - damp), 1),
                      "uniform_dominant_mode": mu,
                      "uniform_dominant_mode_rate_per_s": None if np.isnan(rate) else round(rate, 1),
                      "uniform_rms_growth_factor": factor(ru),
                      "three_quarter_first_mid_last_per_s": [None if np.isnan(x) else round(x, 1) for x in fml],
                      "three_quarter_rms_growth_factor": factor(rq)})
    line = {"metric": "L5 HOM detuning scan throughput (macro-particle-turns/s)", "value": mp * turns / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": turns, "ms_per_step": ms / turns, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"SLS-2 L5 scan: {len(det)} HOM detunings x (uniform 484 + 3/4 363 bunches), "
                                   f"{n_mp} mp per bunch, 400 mA, {turns} turns, one batch of {len(runs)} runs",
                       "lanes": lanes,
                       "revolution_frequency_Hz": f0, "hom": {"fr_Hz": W.L5_FR_HZ, "Rs_ohm": W.L5_RS_OHM, "Q": W.L5_Q},
                       "radiation_damping_per_s": damp, "fit_turns": list(fit)},
            "growth_rates": table, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def resident_scan(pkg, runs, turns, last):
    """The same scan's runs tracked resident, all members at once
    (mbt_batch_track_resident: one stream per run, forked from and joined into
    the current stream): throughput over `turns` turns from the matched start
    (CUDA events on the current stream) and each run's equilibrium rms length
    over the last `last` turns."""
    import torch
    trackers = [pkg.tracker_for_run(r, record_turns=turns) for r in runs]
    stream = torch.cuda.current_stream()
    for t in trackers:
        t.init_particles(stream)
    b = pkg.Batch(trackers)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.track_resident(turns, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    b.sync()
    ms = ev0.elapsed_time(ev1)
    sig = [round(float(t.moments(turns - last, last)[:, 0, 1].mean()) * 1e12, 4) for t in trackers]
    b.close()
    for t in trackers:
        t.close()
    mp = sum(r.n_particles for r in runs)
    return {"value": mp * turns / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / turns, "turns": turns,
            "mode": "mbt_batch_track_resident: every run's cluster-resident kernel on its own stream, "
                    "concurrently, clusters capped in size so that all runs' clusters are on the GPU at once",
            "sigma_tau_ps": sig}


def rwscan_bench(args, rank, local):
    """Single-bunch current scan in the resistive-wall wake, one batch."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    ring = W.ring_dc12c()
    rw = dict(radius_m=0.01, conductivity_S_per_m=5.8e7, length_m=290.4)
    currents_mA = [0.1, 0.5, 1, 2, 3, 5, 7.5, 10, 15, 20, 30, 40]
    turns, n_mp, hw, last = 50_000, 100_000, 10.0, 5000
    runs = []
    for k, I in enumerate(currents_mA):
        b, c, n = W._fill([0], I * 1e-3, n_mp)
        runs.append(W.Run(ring, [], b, c, n, seed=700 + k, turns=turns, precision=W.PREC_MIXED,
                          half_width_sigmas=hw, resistive_wall=[dict(rw)], name=f"rw {I} mA"))
    trackers = [pkg.tracker_for_run(r, record_turns=turns) for r in runs]
    stream = torch.cuda.current_stream()
    for t in trackers:
        t.init_particles(stream)
    b = pkg.Batch(trackers)
    b.set_graph(GRAPH_TURNS)
    b.set_lanes(args.lanes or LANES["rwscan"])
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        b.track(turns, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    b.sync()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    table = []
    for I, r, t in zip(currents_mA, runs, trackers):
        rec = t.moments(turns - last, last)[:, 0, :]
        table.append({"current_mA": I, "sigma_tau_ps": round(float(rec[:, 1].mean()) * 1e12, 4),
                      "sigma_tau_spread_ps": round(float(rec[:, 1].std()) * 1e12, 4),
                      "sigma_delta_over_sigma_E": round(float(rec[:, 3].mean()) / ring["sigma_delta"], 5),
                      "centroid_ps": round(float(rec[:, 0].mean()) * 1e12, 4),
                      "outside_fraction": round(float(rec[:, 5].mean()) / n_mp, 6)})
    b.close()
    for t in trackers:
        t.close()
    mp = sum(r.n_particles for r in runs)
    line = {"metric": "resistive-wall current scan throughput (macro-particle-turns/s)",
            "value": mp * turns / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": turns, "ms_per_step": ms / turns,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"dc12c single bunch x {len(runs)} currents ({n_mp} mp), copper pipe b = 10 mm "
                                   f"around the ring, {turns} turns, one batch; mesh 256 cells over +-{hw} sigma",
                       "equilibrium": f"averages over the last {last} turns", "sigma_E": ring["sigma_delta"]},
            "scan": table, "clocks": clocks}
    line["resident"] = resident_scan(pkg, runs, turns, last)
    print(json.dumps(line), flush=True)
    return 0


def hcscan_bench(args, rank, local):
    """Bunch lengthening by an active third-harmonic cavity, one batch."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    ring = W.ring_r0()
    n = 3
    u = ring["U0_eV"] / ring["V_rf_V"]
    k_flat = math.sqrt(1 / n ** 2 - u * u / (n * n - 1))
    s_flat = n * n / (n * n - 1) * u
    phih = math.atan2(-s_flat / (n * n * k_flat), -math.sqrt(1 - s_flat * s_flat) / (n * k_flat))
    fractions = [0.0, 0.25, 0.5, 0.75, 0.9, 1.0, 1.1, 1.2]
    turns, n_mp, last = 20_000, 100_000, 4000
    runs = []
    for i, f in enumerate(fractions):
        b, c, nn = W._fill([0], 1e-3, n_mp)
        hcs = [dict(n=n, V_V=f * k_flat * ring["V_rf_V"], phi_rad=phih)] if f > 0 else []
        runs.append(W.Run(ring, [dict(W.BROADBAND)], b, c, nn, seed=900 + i, turns=turns, precision=W.PREC_MIXED,
                          half_width_sigmas=12.0, harmonic_cavities=hcs, name=f"harmonic {f:.2f} x flat"))
    trackers = [pkg.tracker_for_run(r, record_turns=turns) for r in runs]
    stream = torch.cuda.current_stream()
    for t in trackers:
        t.init_particles(stream)
    b = pkg.Batch(trackers)
    b.set_graph(GRAPH_TURNS)
    b.set_lanes(args.lanes or LANES["hcscan"])
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        b.track(turns, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    b.sync()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    table = []
    for f, t in zip(fractions, trackers):
        rec = t.moments(turns - last, last)[:, 0, :]
        table.append({"fraction_of_flat_voltage": f, "V_h_kV": round(f * k_flat * ring["V_rf_V"] / 1e3, 2),
                      "sigma_tau_ps": round(float(rec[:, 1].mean()) * 1e12, 3),
                      "sigma_delta_over_sigma_E": round(float(rec[:, 3].mean()) / ring["sigma_delta"], 4),
                      "centroid_ps": round(float(rec[:, 0].mean()) * 1e12, 3)})
    b.close()
    for t in trackers:
        t.close()
    mp = sum(r.n_particles for r in runs)
    line = {"metric": "harmonic-cavity scan throughput (macro-particle-turns/s)", "value": mp * turns / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": turns, "ms_per_step": ms / turns, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"R0 single bunch 1 mA + broadband wake, third-harmonic cavity at "
                                   f"{len(fractions)} voltages (flat potential: {k_flat * ring['V_rf_V'] / 1e3:.1f} kV,"
                                   f" phase {phih:.4f} rad), {n_mp} mp, {turns} turns, one batch",
                       "equilibrium": f"averages over the last {last} turns"},
            "scan": table, "clocks": clocks}
    line["resident"] = resident_scan(pkg, runs, turns, last)
    print(json.dumps(line), flush=True)
    return 0


def resident_bench(args, rank, local):
    """Time per turn of small fills held in cluster shared memory
    (mbt_track_resident: all K turns in one launch, CUDA events) against the
    same runs through the per-turn kernels (graph replay)."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    K = max(args.steps, 50)
    ring = W.ring_r0()
    cases = []
    for name, buckets, n_mp, res in (("1 bunch x 1e4, BB", [0], 10_000, [dict(W.BROADBAND)]),
                                     ("1 bunch x 1e5, BB", [0], 100_000, [dict(W.BROADBAND)]),
                                     ("3 bunches x 1e5, BB + HOM (long range)", [0, 1, 2], 100_000,
                                      [dict(W.BROADBAND), dict(W.HOM)])):
        b, c, n = W._fill(buckets, 1e-3, n_mp)
        run = W.Run(ring, res, b, c, n, seed=3, turns=K, precision=W.PREC_MIXED, name=name)
        out = {"case": name}
        stream = torch.cuda.current_stream()
        for mode in ("resident", "per-turn kernels"):
            tr = pkg.tracker_for_run(run, record_turns=max(K, 64))
            tr.init_particles(stream)
            if mode == "resident":
                tr.track_resident(max(3, args.warmup), stream)
            else:
                tr.set_graph(min(K, GRAPH_TURNS))
                tr.track(min(K, GRAPH_TURNS) * 2, stream)
            tr.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if mode == "resident":
                tr.track_resident(K, stream)
            else:
                tr.track(K, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            tr.sync()
            out[mode + " us_per_turn"] = e0.elapsed_time(e1) * 1e3 / K
            if mode == "resident":
                out["cluster"], out["per_cta"] = tr.resident_shape()
            tr.close()
        cases.append(out)
    print(json.dumps({"workload": "cluster-resident tracking", "turns": K, "cases": cases}), flush=True)
    return 0


def three_f64_bench(args, rank, local):
    """Three bunches x 1e5 macro-particles, broadband + HOM, on the FP64
    tracker: throughput, and the FP64 push's time per launch.  The FP64 path
    is bound by the FP64 pipe; its utilisation comes from the ncu counters
    (sm__inst_executed_pipe_fp64), not from a byte count."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    run = W.three_bunches(seed=1)
    K, Wm, KR = min(args.steps, 2000), max(args.warmup, 3), 300
    stream = torch.cuda.current_stream()
    tr = pkg.tracker_for_run(run, record_turns=K + Wm + 2 * GRAPH_TURNS + KR + 16)
    tr.init_particles(stream)
    tr.set_graph(GRAPH_TURNS)
    tr.track(max(Wm, GRAPH_TURNS), stream)
    tr.sync()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        tr.track(K, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    tr.sync()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    tr.set_timing(True)
    tr.track(KR, stream)
    tr.sync()
    push_ms, post_ms, launches = tr.timing()
    tr.set_timing(False)
    n = run.n_particles
    line = {"metric": "macro-particle-turns/s (3 bunches, FP64 tracker)", "value": n * K / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": run.name, "turns_timed": K, "l2": "state 4.8 MB: L2-resident (FP64-pipe bound)"},
            "roofline": {"bound": "fp64 pipe", "kernel": "k_push_f64", "unit_count": n,
                         "push_us": push_ms / max(1, launches) * 1e3, "post_us": post_ms / max(1, launches) * 1e3,
                         "utilisation": "ncu counter sm__inst_executed_pipe_fp64"},
            "gpu_launches": 2 * K, "clocks": clocks}
    print(json.dumps(line), flush=True)
    tr.close()
    return 0


FP64_FLOPS_PER_MP_TURN = 182   # FP64 flops of the FP64 push per macro-particle-turn (ncu count: 71 DFMA, 21 DADD, 19 DMUL)


def fill390_f64_bench(args, rank, local):
    """The 390-bunch fill on the plain FP64 tracker (tau and delta FP64, every
    step in FP64), beside the mixed-precision path on the same fill: both
    timed as K graph-replayed turns with CUDA events; the FP64 push against
    the GPU's measured DFMA throughput (mbt_probe_fp64_fma)."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    K, Wm = min(args.steps, 200), max(args.warmup, 3)
    G = max(1, min(GRAPH_TURNS, K))
    stream = torch.cuda.current_stream()
    peak, sms = pkg.probe_fp64_fma(stream=stream)

    def timed(prec):
        run = W.fill_390(seed=1, precision=prec)
        tr = pkg.tracker_for_run(run, record_turns=K + Wm + 2 * G + 64)
        tr.init_particles(stream)
        tr.set_graph(G)
        tr.track(max(Wm, G), stream)
        tr.sync()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            ev0.record(stream)
            tr.track(K, stream)
            ev1.record(stream)
            torch.cuda.synchronize()
        tr.sync()
        ms = ev0.elapsed_time(ev1)
        tr.set_timing(True)
        tr.track(min(K, 50), stream)
        tr.sync()
        push_ms, post_ms, launches = tr.timing()
        tr.close()
        return run, ms, push_ms / max(1, launches), post_ms / max(1, launches), clk.summary()

    run, ms64, push64, post64, clocks = timed(W.PREC_F64)
    _, msmx, pushmx, _, _ = timed(W.PREC_MIXED)
    n = run.n_particles
    achieved = FP64_FLOPS_PER_MP_TURN * n / (push64 * 1e-3)
    line = {"metric": "macro-particle-turns/s (390-bunch fill, FP64 tracker)", "value": n * K / (ms64 * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": ms64 / K, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": run.name + ", FP64 tracker", "turns_timed": K,
                       "l2": "state 624 MB > 129 MB L2 (no flush needed)"},
            "roofline": {"bound": "fp64 pipe", "kernel": "k_push_f64", "achieved": achieved, "peak": peak,
                         "unit": "FLOP/s", "frac": achieved / peak,
                         "peak_source": f"measured: DFMA throughput probe, 8 CTAs x {sms} SMs x 256 threads, "
                                        f"CUDA events", "flops_per_unit": FP64_FLOPS_PER_MP_TURN,
                         "unit_count": n, "push_us": push64 * 1e3, "post_us": post64 * 1e3},
            "mixed_same_fill": {"value": n * K / (msmx * 1e-3), "ms_per_step": msmx / K, "push_us": pushmx * 1e3,
                                "speedup_over_f64": ms64 / msmx},
            "gpu_launches": 2 * K, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def state_bench(args, rank, local):
    """Profiling helper for the 390-bunch fill at a chosen beam state: if
    --state-file does not exist yet, track the fill from its matched start
    for --at-turn turns and save the state there; then load that state into
    a fresh tracker and track --steps turns with plain launches (so that a
    profiler run of this command sees only a few launches before the push it
    captures)."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    run = fill390t_run()[0] if args.transverse else W.fill_390(seed=1)
    path = args.state_file
    made = False
    if not os.path.exists(path):
        tr = pkg.tracker_for_run(run, record_turns=64)
        tr.init_particles()
        tr.set_graph(GRAPH_TURNS)
        tr.track(args.at_turn)
        tr.sync()
        blob = tr.save_state()
        tr.close()
        with open(path, "wb") as f:
            f.write(blob)
        made = True
    with open(path, "rb") as f:
        blob = f.read()
    tr = pkg.tracker_for_run(run, record_turns=64)
    tr.load_state(blob)
    turn0 = tr.info["turn"]
    tr.track(args.steps)
    tr.sync()
    rec = tr.moments(turn0 + args.steps - 1, 1)[0]
    tr.close()
    print(json.dumps({"workload": run.name, "state_file": path, "saved_now": made, "turn_loaded": turn0,
                      "turns_tracked": args.steps,
                      "outside_mesh_fraction": float(np.mean(rec[:, 5]) / run.n_mp[0]),
                      "centroid_rms_ps": float(np.sqrt(np.mean(rec[:, 0] ** 2)) * 1e12)}), flush=True)
    return 0


def fill390t_run():
    """The 390-bunch fill with a horizontal plane (beta 10 m, tune 0.31,
    chromaticity 1.5, 1 nm) and a transverse HOM (200 kOhm/m, 1.5 GHz, Q 2e4,
    short and long range)."""
    base = W.fill_390(precision=W.PREC_MIXED)
    tplane = dict(beta_m=10.0, alpha=0.0, tune=0.31, chromaticity=1.5, emittance_m=1e-9,
                  resonators=[dict(Rs_ohm=2e5, fr_Hz=1.5e9, Q=2e4, range=W.RANGE_BOTH)])
    return W.Run(**{**base.__dict__, "transverse": tplane, "name": base.name + " + transverse plane"}), tplane


def fill390t_bench(args, rank, local):
    """The 390-bunch fill with a transverse plane: throughput and push roofline."""
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local)
    import paper_1809_00391_gb300 as pkg
    pkg.build()
    run, tplane = fill390t_run()
    K, Wm = min(args.steps, 5000), max(args.warmup, 3)
    stream = torch.cuda.current_stream()
    tr = pkg.tracker_for_run(run, record_turns=K + Wm + GRAPH_TURNS + 17 * (AUTOTUNE_TURNS + 2) + 600)
    tr.init_particles(stream)
    if args.tile > 0:
        tr.set_tile(args.tile)
        tile = args.tile
    else:
        tile = tr.autotune(AUTOTUNE_TURNS)
    tr.set_graph(GRAPH_TURNS)
    tr.track(max(Wm, GRAPH_TURNS), stream)
    tr.sync()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        tr.track(K, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    tr.sync()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.summary()
    KR = 500
    tr.set_timing(True)
    tr.track(KR, stream)
    tr.sync()
    push_ms, post_ms, launches = tr.timing()
    tr.set_timing(False)
    n = run.n_particles
    bpp = 40
    push_s = push_ms / max(1, launches) * 1e-3
    peak, kind = measured_peak_hbm()
    achieved = bpp * n / push_s / 1e9
    line = {"metric": "macro-particle-turns/s (390-bunch fill with a transverse plane)", "value": n * K / (ms * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": run.name, "transverse": {k: v for k, v in tplane.items() if k != "resonators"},
                       "transverse_resonator": tplane["resonators"][0], "turns_timed": K, "push_tile": tile},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": kind, "kernel": "k_push_mixed_t",
                         "bytes_per_unit": bpp, "unit_count": n, "push_us": push_s * 1e6,
                         "post_us": post_ms / max(1, launches) * 1e3},
            "gpu_launches": 2 * K, "clocks": clocks}
    print(json.dumps(line), flush=True)
    tr.close()
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload == "serving":
        return serving_bench(args, rank, local)
    if args.workload == "l5scan":
        return l5scan_bench(args, rank, local)
    if args.workload == "rwscan":
        return rwscan_bench(args, rank, local)
    if args.workload == "hcscan":
        return hcscan_bench(args, rank, local)
    if args.workload == "three_f64":
        return three_f64_bench(args, rank, local)
    if args.workload == "fill390t":
        return fill390t_bench(args, rank, local)
    if args.workload == "fill390_f64":
        return fill390_f64_bench(args, rank, local)
    if args.workload == "state":
        return state_bench(args, rank, local)
    if args.workload == "resident":
        return resident_bench(args, rank, local)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_1809_00391_gb300 as pkg
    pkg.build()

    run = replica_run(rank)
    K, Wm = args.steps, args.warmup
    G = max(1, min(GRAPH_TURNS, K))
    stream = torch.cuda.current_stream()
    tr = pkg.tracker_for_run(run, record_turns=max(K + Wm + G + 17 * (AUTOTUNE_TURNS + 2), 16))
    tr.init_particles(stream)
    if args.tile > 0:
        tr.set_tile(args.tile)
        tile = args.tile
    else:
        tile = tr.autotune(AUTOTUNE_TURNS)  # push-tile autotuner: its trial turns are real warm-up turns
    tr.set_graph(G)
    tr.track(max(Wm, G), stream)       # warm-up; also captures the G-turn graph
    tr.sync()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: K turns replayed from the captured graph (programmatic
    # dependent launch between the kernels), CUDA events on the tracking stream
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        tr.track(K, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    tr.sync()
    clocks = clk.summary()

    t_max = max_over_ranks(elapsed_ms, dist)
    n_part = run.n_particles
    value = weak_scaling_value(n_part, K, world, t_max)

    # ---- roofline of the dominant kernel (push): a second timed region of KR
    # turns with CUDA events around every launch (ordinary launches), right
    # after the headline region (the same beam state)
    def timed_push(turns):
        tr.set_timing(True)
        tr.track(turns, stream)
        tr.sync()
        push_ms, post_ms, launches = tr.timing()
        tr.set_timing(False)
        return push_ms / max(1, launches) * 1e-3, post_ms / max(1, launches) * 1e-3, launches

    KR = max(1, min(K, ROOFLINE_TURNS))
    turn_a = tr.info["turn"]
    push_avg_s, post_avg_s, launches = timed_push(KR)
    achieved = BYTES_PER_MP_TURN * n_part / push_avg_s / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = recorded_traffic(n_part)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "kernel": "k_push_stream", "bytes_per_unit": BYTES_PER_MP_TURN, "unit_count": n_part,
                "timed_launches": launches, "push_us": push_avg_s * 1e6, "post_us": post_avg_s * 1e6,
                "region": f"turns {turn_a}..{turn_a + KR - 1}, right after the headline region, CUDA events around "
                          f"each push launch"}
    # the same kernel once the coupled-bunch instability has saturated (from
    # turn ~1000 on most particles lie outside the mesh and skip the deposit)
    if args.saturated_turn > 0:
        now = tr.info["turn"]
        if now < args.saturated_turn:
            tr.track(args.saturated_turn - now, stream)
            tr.sync()
        turn_b = tr.info["turn"]
        ps, qs, ls = timed_push(SATURATED_TURNS)
        a_s = BYTES_PER_MP_TURN * n_part / ps / 1e9
        out_frac = float(np.mean(tr.moments(tr.info["turn"] - 1, 1)[0, :, 5]) / run.n_mp[0])
        roofline["saturated"] = {"achieved": a_s, "frac": a_s / peak, "push_us": ps * 1e6, "post_us": qs * 1e6,
                                 "timed_launches": ls, "outside_mesh_fraction": out_frac,
                                 "region": f"turns {turn_b}..{turn_b + ls - 1}"}

    # ---- end to end through the C ABI with host buffers: a fresh job (new
    # particle state from page-locked host arrays, K turns, all K turns of
    # moments back to the host) on a tracker whose turn graph is captured
    e2e = None
    if not args.no_e2e:
        rng = np.random.default_rng(100 + rank)
        n = run.n_particles
        # tau in FP32, the precision the mixed path keeps it in (mbt_set_particles_all_f32)
        host_tau = torch.from_numpy(rng.normal(0.0, 13.2e-12, n).astype(np.float32)).pin_memory()
        host_del = torch.from_numpy(rng.normal(0.0, 9e-4, n)).pin_memory()
        tr2 = pkg.tracker_for_run(run, record_turns=max(K, 16))
        tr2.set_tile(tile)
        tr2.set_graph(G)
        tr2.init_particles(stream)
        tr2.track(G, stream)             # captures the turn graph
        tr2.init_particles(stream)       # turn counter, wakes and phasors back to zero
        tr2.sync()
        barrier()
        t0 = time.perf_counter()
        tr2.set_particles_all(host_tau, host_del, stream)
        tr2.track(K, stream)
        mom = tr2.moments(0, K)
        torch.cuda.synchronize()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
        h2d = host_tau.numel() * host_tau.element_size() + host_del.numel() * host_del.element_size()
        d2h = mom.nbytes
        e2e = {"value": n_part * K * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": d2h / K, "ms": e2e_s * 1e3,
               "note": "host clock around: tau (FP32) and delta (FP64) of every bunch from page-locked host "
                       "memory (mbt_set_particles_all_f32), K turns, all K turns of moments read to the host"}
        tr2.close()

    # ---- a bounded sample of the serving workload (Poisson requests at about
    # the server's capacity, so that the latencies are service times, not a
    # growing queue); the full-stream figures come from --workload serving
    serving = None
    if rank == 0 and args.serving_requests > 0:
        tr.close()
        mean_work = float(np.mean([rq.run.turns * rq.run.n_particles
                                   for rq in W.serving_stream(200, rate_hz=1.0, seed=7)]))
        rate = 0.9 * value / mean_work
        lat, queue, work, stats, span = serving_sample(args.serving_requests, rate, lanes=LANES["serving"])
        serving = {"requests": args.serving_requests, "rate_hz": rate,
                   "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                   "queue_p99_s": float(np.percentile(queue, 99)), "delivered": float(work.sum() / span),
                   "unit": UNIT, "span_s": span, "max_active_seen": stats["max_active_seen"],
                   "stream": "Poisson, seed 7: 1-484 bunches, 1e4-2e5 mp per bunch, 0.1-5 mA, HOM 1-3 GHz, "
                             "2000-2e4 turns; 16 active, 200 turns per step; rate = 0.9 x this run's "
                             "throughput / mean request work"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(run)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
                "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": run.name, "bunches": run.nb, "mp_per_bunch": int(run.n_mp[0]),
                           "turns_timed": K, "precision": "tau f32, delta f64-accumulated, wake bf16x2 on tcgen05 "
                           "(fp32 accumulate), phasor scan + moments f64",
                           "l2": "state 468 MB > 129 MB L2 (no flush needed)",
                           "push": "persistent, one 1024-thread CTA per SM, equal per-SM shares of each run",
                           "parallelism": f"{world} independent fill(s), one per GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "serving": serving, "gpu_launches": 2 * K,
                "launch_mode": f"CUDA graph of {G} turns, programmatic dependent launch between kernels",
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if serving is None:
        tr.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
