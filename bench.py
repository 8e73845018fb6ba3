#!/usr/bin/env python3
"""Benchmark: UT decode + Compass events/s on one GB300.

A step is one pass of the whole path (raw-bank decoding with the per-sector
sort, window search, tracklet finding, q/p fit) over one batch of seeded
synthetic events whose shapes follow the paper's workloads (the LHCb
minbias samples themselves are not available).  Default workload: 1000
events, 4 planes x 256 sectors, 4000 hits and 200 VELO tracks per event.
Default form: the persistent decode + Compass kernel (one launch replayed
from a CUDA graph) with its launch shape picked by the autotuner; --form
fused (sorted decode, then compass_find) and --form plain (decode, sort,
find, fit) time the per-kernel forms.

Timing: W untimed warm-up steps, then K steps timed with CUDA events on the
launching stream, the L2 flushed (256 MB write) before every step, bracketed
by a barrier and a device synchronise; max over ranks.  One JSON line.

--impl reference times the CPU oracle (the plain C statement of the
method) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "UT decode+Compass events/s on 1 GB300, % HBM roofline, p99 batch latency"
WORKLOADS = {
    "plain": dict(name="plain", n_events=1000, n_sectors=256, tracks=200, hits=4000, seed=2),
    "batched": dict(name="batched", n_events=20000, n_sectors=256, tracks=None, hits="lognormal", seed=3),
    "tiny": dict(name="tiny", n_events=16, n_sectors=64, tracks=100, hits=1500, seed=1),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain", choices=list(WORKLOADS))
    ap.add_argument("--events", type=int, default=None,
                    help="first N events of the workload's generator (smaller cases for profiling)")
    ap.add_argument("--form", default="batched", choices=["batched", "fused", "plain"])
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched form: use --tracks-per-warp/--block instead of the autotuner's pick")
    ap.add_argument("--x-cap", type=int, default=8192)
    ap.add_argument("--tracks-per-warp", type=int, default=8)
    ap.add_argument("--block", type=int, default=None,
                    help="threads per block (default: 800 at 8 tracks per warp, else 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the uneven-workload form comparison, serving and alignment measurements")
    ap.add_argument("--physics", action="store_true",
                    help="also run the sectors x candidates physics sweep and the kick-map workload")
    ap.add_argument("--only", default=None,
                    choices=["sector_groups", "alignment", "uneven_workload", "serving"],
                    help="run only this variant measurement and print its detail line (profiling)")
    return ap.parse_args()


def max_over_ranks(value, dist=None, device="cuda"):
    """The largest `value` over all ranks (the job's time is its slowest
    rank's); `value` itself without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_events_per_s(world, events_per_rank, steps, seconds):
    """Whole-job throughput: every rank processes its own `events_per_rank`
    per step (weak scaling), the time is the slowest rank's."""
    return world * events_per_rank * steps / seconds


def make_batch(wl, rank, n_events=None):
    import synth
    c = dict(WORKLOADS[wl])
    c.pop("name")
    if n_events is not None:
        c["n_events"] = n_events
    c["seed"] = c["seed"] + 1000 * rank
    return synth.generate(**c)


def workload_config(wl, batch, form, extra=None):
    c = WORKLOADS[wl]
    cfg = {"workload": f"{wl}: {batch.n_events} events, 4x{c['n_sectors']} sectors, "
                       f"hits/event {c['hits']}, tracks/event {c['tracks'] or '0.05*hits'}",
           "n_events": batch.n_events, "hits_per_event": round(batch.n_hits / batch.n_events, 1),
           "tracks_per_event": round(batch.n_tracks / batch.n_events, 1),
           "n_sectors_searched": 5, "n_candidates": 8, "form": form,
           "l2": "flushed before every step (256 MB write)"}
    if extra:
        cfg.update(extra)
    return cfg


class Clocks:
    """SM clock and clock-event reasons sampled during the timed region.

    NVML is read directly (libnvidia-ml through ctypes, read-only queries)
    from a thread polling about every millisecond, so that a timed region of
    a few milliseconds still gets samples; nvidia-smi's 100 ms loop is the
    fallback where NVML cannot be opened."""

    # NVML clocks event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        import ctypes
        import threading
        import torch
        self.p = None
        self.samples = []
        self.stop_flag = threading.Event()
        self.t = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            h = ctypes.c_void_p()
            # the CUDA device's own GPU (CUDA_VISIBLE_DEVICES may renumber):
            # by UUID, else by PCI bus id, else by index
            props = torch.cuda.get_device_properties(index)
            uuid = getattr(props, "uuid", None)
            ok = False
            if uuid is not None:
                u = str(uuid)
                ok = nv.nvmlDeviceGetHandleByUUID((u if u.startswith("GPU-") else "GPU-" + u).encode(),
                                                  ctypes.byref(h)) == 0
            if not ok and hasattr(props, "pci_bus_id"):
                bus = "%08x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id,
                                            getattr(props, "pci_device_id", 0))
                ok = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
            if not ok and nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                raise OSError("nvmlDeviceGetHandle")
            self.handle_by = "uuid/pci" if ok else "index"
            mx = ctypes.c_uint()
            nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # 1 = NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
            get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons

            def poll():
                clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
                while not self.stop_flag.is_set():
                    if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                        r = rs.value if get_reasons(h, ctypes.byref(rs)) == 0 else 0
                        self.samples.append((float(clk.value), int(r)))
                    time.sleep(0.001)

            self.t = threading.Thread(target=poll, daemon=True)
            self.t.start()
            t0 = time.perf_counter()
            while not self.samples and time.perf_counter() - t0 < 2.0:  # sampling before the region starts
                time.sleep(0.001)
            self.samples.clear()
            self.how = "nvml"
        except Exception:  # no NVML library or device: nvidia-smi
            self.t = None
            self._smi(index)

    def _smi(self, index):
        self.how = "nvidia-smi"
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.t is not None:
            self.stop_flag.set()
            self.t.join(timeout=2)
            if not self.samples:
                return None
            reasons = set()
            for _, r in self.samples:
                reasons |= {n for bit, n in self.REASONS.items() if r & bit}
            return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                    "reasons": sorted(reasons), "samples": len(self.samples), "source": f"nvml ({self.handle_by}), ~1 ms polling"}
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 100 ms loop"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# The sources each measured kernel is built and launched from: its .cu
# file, the device headers it includes, the ABI header, and the host code
# that fills its arguments (make_find_args in compass.cu) or sizes its grid
# (the context in ctx.cu).
KERNEL_SOURCES = {
    "ut_run_batched": ("batched.cu", "compass.cu", "compass_track.cuh", "decode_event.cuh", "common.cuh",
                       "ctx.cu", "../../include/ut_compass.h"),
    "compass_find": ("compass.cu", "compass_track.cuh", "common.cuh", "ctx.cu", "../../include/ut_compass.h"),
    "ut_decode": ("decode.cu", "decode_event.cuh", "common.cuh", "ctx.cu", "../../include/ut_compass.h"),
}


def source_digest(kernel):
    """sha256 over the sources of one measured kernel (KERNEL_SOURCES)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2002_11529_gb300", "csrc")
    for rel in sorted(KERNEL_SOURCES[kernel]):
        path = os.path.normpath(os.path.join(csrc, rel))
        h.update(os.path.basename(path).encode())
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(kernel, workload):
    """DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)
    recorded in profiles/traffic.json for this kernel and workload, or None
    when absent or taken on other sources than the current ones."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(f"{kernel}|{workload}")
    except (OSError, ValueError):
        return None
    if not rec or kernel not in KERNEL_SOURCES or rec.get("source_sha256") != source_digest(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


def _time_oracle(batch, params, threads, min_seconds):
    """Events/s of the oracle (decode + Compass) over repeated passes of
    `batch` for at least min_seconds; (events/s, passes, seconds)."""
    import oracle
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.run_batch(batch, params, n_threads=threads)
        n += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            return n * batch.n_events / el, n, el


def cpu_baseline(batch, params, min_seconds=8.0):
    """The oracle as it stands: OpenMP over events on all host threads on
    the bench workload (the reported value), plus one thread on a bounded
    sample of it, the tiny workload in full and the first 2000 events of
    the uneven 20000-event workload on all threads."""
    import oracle
    import synth
    threads = oracle.max_threads()
    v, n, el = _time_oracle(batch, params, threads, min_seconds)
    out = {"value": v, "unit": "events/s", "cores": threads, "kind": "oracle",
           "sample": f"the full {batch.n_events}-event workload x{n} ({el:.1f} s), decode+sort+windows+"
                     f"tracklets+float and double fits"}
    sub = synth.subset(batch, 0, min(batch.n_events, 100))
    v1, n1, el1 = _time_oracle(sub, params, 1, 3.0)
    out["single_thread"] = {"value": round(v1, 1), "cores": 1, "sample": f"first {sub.n_events} events x{n1}"}
    tiny = make_batch("tiny", 0)
    vt, nt, _ = _time_oracle(tiny, params, threads, 1.0)
    out["tiny"] = {"value": round(vt, 1), "cores": threads, "sample": f"all {tiny.n_events} events x{nt}"}
    unev = make_batch("batched", 0, 2000)
    vu, nu, _ = _time_oracle(unev, params, threads, 3.0)
    out["uneven"] = {"value": round(vu, 1), "cores": threads,
                     "sample": f"first 2000 of the 20000 uneven events x{nu}"}
    return out


def run_reference(args):
    import synth
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    batch = make_batch(args.workload, 0)
    params = synth.CompassParams()
    sample_events = min(batch.n_events, 200)
    sub = synth.subset(batch, 0, sample_events)
    threads = oracle.max_threads()
    for _ in range(args.warmup):
        oracle.run_batch(sub, params, n_threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run_batch(sub, params, n_threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = sample_events * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(args.workload, batch, "cpu-oracle",
                                      {"sample_events_per_step": sample_events}),
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": threads, "kind": "oracle",
                             "sample": f"first {sample_events} events of the workload per step"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_forms_on_uneven_workload(g, params, flush, steps=5):
    """Form comparison on the 20000-event uneven workload: the batched
    persistent form (one graph-replayed launch, autotuned shape) against
    the plain per-kernel form (decode, sort, find, fit)."""
    import torch
    batch = make_batch("batched", 0)
    ctx = g.Context(batch.geom)
    pipe = g.Pipeline(ctx, batch, params)
    from paper_2002_11529_gb300 import autotune
    cfg, _ = autotune.autotune(pipe, reps=2, flush=flush)
    runner = g.GraphRunner(pipe, cfg)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            flush.zero_()
            fn()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    ms_b = timed(runner.replay)
    blk_p = 800 if cfg.tracks_per_warp == 8 else 256   # compass_find's best block at that width
    ms_p = timed(lambda: pipe.run_plain(stream, cfg.tracks_per_warp, blk_p))
    E = batch.n_events
    # decode alone (sorted and bank order) against the measured HBM bandwidth
    dec = {}
    hbm, _ = peaks()
    algo = algorithmic_bytes(batch)["ut_decode"]
    for name, srt in (("sorted", True), ("bank_order", False)):
        ms = timed(lambda: g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, E, pipe.hits_a, srt,
                                       pipe.workspace, stream))
        gbs = algo / (ms / 1e3) / 1e9
        dec[name] = {"ms": round(ms, 4), "gbs": round(gbs, 1), "frac": round(gbs / hbm, 4)}
    ctx.check(stream, "uneven workload")
    out = {"workload": f"{E} events, hits/event lognormal (median 3000, sigma 0.6, 500-15000), "
                       f"tracks/event 0.05*hits, 4x256 sectors",
           "batched_form": {"ms": round(ms_b, 4), "events_per_s": E / ms_b * 1e3,
                            "launch": {"tracks_per_warp": cfg.tracks_per_warp, "block": cfg.block,
                                       "graph": True, "kernels_per_step": 1}},
           "plain_form": {"ms": round(ms_p, 4), "events_per_s": E / ms_p * 1e3, "kernels_per_step": 4,
                          "compass_find_block": blk_p},
           "batched_over_plain": ms_p / ms_b,
           "decode_only": dict(dec, algorithmic_bytes=algo)}
    ctx.close()
    return out


def measure_serving(g, params, cfg=None, loads=(0.5, 0.8, 0.95), runs_per_level=5):
    """Serving: requests of 64-4096 events (log-uniform, plain-workload
    occupancy) through the continuous-batching engine, 40 GB budget,
    8 stream slots, persistent launch shape `cfg`: sustained peak (all
    submitted at once), then Poisson arrivals at fractions of that peak
    (runs_per_level runs of 96 requests per level, after an untimed
    open-loop pass); p50/p99 request latency as the median over the runs,
    and the largest p99 of the runs."""
    import numpy as np
    import synth
    from paper_2002_11529_gb300 import serve
    rng = np.random.default_rng(55)
    sizes = np.exp(rng.uniform(np.log(64), np.log(4096), 24)).astype(int)
    batches = [synth.generate(n_events=int(n), n_sectors=256, tracks=200, hits=4000, seed=7000 + i)
               for i, n in enumerate(sizes)]
    reqs = [serve.HostRequest.from_batch(b) for b in batches]
    res = {"requests_per_level": 4 * len(reqs), "events_per_request": "64-4096 log-uniform",
           "budget_bytes": 40 << 30, "slots": 8,
           "launch": None if cfg is None else {"tracks_per_warp": cfg.tracks_per_warp, "block": cfg.block}}
    with serve.Server(batches[0].geom, params, budget_bytes=40 << 30, n_slots=8, cfg=cfg) as sv:
        serve.run_closed_loop(sv, reqs)            # warm-up
        peak, _ = serve.run_closed_loop(sv, reqs * 4)
        res["peak_events_per_s"] = peak["events_per_s"]
        res["peak_p99_ms"] = peak["p99_ms"]
        serve.run_open_loop(sv, reqs, events_per_s=0.5 * peak["events_per_s"], seed=1)  # warm-up
        for f in loads:
            runs = [serve.run_open_loop(sv, reqs * 4, events_per_s=f * peak["events_per_s"],
                                        seed=int(f * 100) + 7 * k)[0] for k in range(runs_per_level)]
            p50 = [r["p50_ms"] for r in runs]
            p99 = [r["p99_ms"] for r in runs]
            res[f"load_{int(round(f * 100))}"] = {
                "events_per_s": statistics.median(r["events_per_s"] for r in runs),
                "p50_ms": statistics.median(p50), "p99_ms": statistics.median(p99),
                "p99_ms_max": max(p99), "p99_ms_runs": [round(v, 3) for v in p99],
                "errors": sum(len(r["errors"]) for r in runs)}
        res["arena_peak_bytes"] = sv.stats()["arena_peak"]
    return res


def measure_alignment(g, params, reps=10):
    """Alignment on the 100k-track, 4 x 256-sector set (3072 parameters):
    device times of one chi2 + adjoint pass (gradients and Gauss-Newton
    blocks), one refit, one reduced Hessian-vector product, and the 20-step
    solve (ut_align_solve: the whole loop on the device; CUDA events, L2
    flushed before each timed call)."""
    import numpy as np
    import torch
    import synth
    from paper_2002_11529_gb300 import align
    a = synth.generate_alignment(100_000, 256, seed=4)
    b = a.batch
    ctx = g.Context(b.geom)
    raw, ev = g.upload_raw(b.raw, b.ev_off)
    nw = int(b.ev_off[-1])
    hits = g.HitBuffers.allocate(2 * nw, b.n_events, b.geom.n_sectors)
    g.ut_decode(ctx, raw, nw, ev, b.n_events, hits, sorted_=False)
    t = lambda arr, dt: torch.from_numpy(np.ascontiguousarray(arr).view(dt)).cuda()
    velo = g.VeloBuffers(t(a.x, np.float32), t(a.y, np.float32), t(a.tx, np.float32), t(a.ty, np.float32),
                         torch.zeros(a.n_tracks, dtype=torch.uint8, device="cuda"),
                         torch.zeros(2, dtype=torch.int32, device="cuda"))
    prob = align.AlignmentProblem(ctx, hits, t(a.track_hits, np.int32), velo, params)
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    al = torch.from_numpy(a.align_true().astype(np.float32)).cuda()
    th = prob.refit(al)
    v = torch.ones((4 * b.geom.n_sectors, 3), dtype=torch.float64, device="cuda")

    def timed(fn, n=reps):
        ms = []
        for _ in range(n + 1):
            flush.add_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms[1:]))

    res = {"tracks": a.n_tracks, "parameters": 3 * 4 * b.geom.n_sectors,
           "chi2_and_adjoint_ms": timed(lambda: prob.chi2(th, al, grads=True)),
           "refit_ms": timed(lambda: prob.refit(al)),
           "hvp_ms": timed(lambda: prob.hvp(th, al, v))}
    align.solve_alignment(prob, steps=20)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    est, hist = align.solve_alignment(prob, steps=20)
    e1.record()
    e1.synchronize()
    hist = hist.tolist()
    c_true = prob.chi2(prob.refit(al), al)[0].item()
    res["solve_20_steps_ms"] = e0.elapsed_time(e1)
    res["chi2_per_track"] = {"start": hist[0] / a.n_tracks, "after_20_steps": hist[-1] / a.n_tracks,
                             "truth": c_true / a.n_tracks}
    ctx.check(what="alignment")
    return res


def physics_sweep(g, batch, params, reps=5):
    """The paper's trade-off table on the synthetic workload: for
    n_sectors in {1, 3, 5} and n_candidates in {1, 2, 4, 8, 16}, the track
    finding efficiency and fake rate on generator truth, and the events/s
    of the sorted decode + compass_find (8 tracks per warp, 800 threads, L2
    flushed)."""
    import numpy as np
    import torch
    from paper_2002_11529_gb300 import physics
    ctx = g.Context(batch.geom)
    pipe = g.Pipeline(ctx, batch, params)
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    E = batch.n_events
    out = []
    for n_sec in (1, 3, 5):
        for n_cand in (1, 2, 4, 8, 16):
            p = params.replace(n_sectors=n_sec, n_candidates=n_cand)
            ms = []
            for r in range(reps + 1):
                flush.add_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, E, pipe.hits_a, True, pipe.workspace)
                g.compass_find(ctx, pipe.hits_a, pipe.velo, E, p, pipe.tracks, tracks_per_warp=8, block=800)
                e1.record()
                e1.synchronize()
                if r:
                    ms.append(e0.elapsed_time(e1))
            ctx.check(what="physics sweep")
            ev = physics.evaluate(batch, g.tracks_to_numpy(pipe.tracks, batch.n_tracks))
            out.append({"n_sectors": n_sec, "n_candidates": n_cand, "events_per_s": E / float(np.median(ms)) * 1e3,
                        "efficiency": ev["efficiency"], "fake_rate": ev["fake_rate"], "clone_rate": ev["clone_rate"]})
    return {"workload": "the bench workload; efficiency on generator truth (Sec. II-C definitions)",
            "reconstructible": ev["reconstructible"], "table": out}


def measure_kick_map(g, params, cfg, reps=10):
    """The field look-up table of the kick (row f4) on the fieldmap workload
    (the plain workload's shapes, hits made with a direction-dependent
    field): the persistent form's events/s (graph replay, L2 flushed) with
    the field's 17 x 17 map and with the constant kick, and for each the
    efficiency, fake rate and the median |q/p / true q/p - 1| of the
    found 4-hit tracks of the particles they were made from."""
    import numpy as np
    import torch
    import synth
    from paper_2002_11529_gb300 import physics
    b = synth.generate_config("fieldmap")
    ctx = g.Context(b.geom)
    pipe = g.Pipeline(ctx, b, params)
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    truth = b.qop_true.astype(np.float64)
    res = {"workload": "fieldmap: 1000 events, 4x256 sectors, hits/event 4000, tracks/event 200, "
                       "kick = field_kick(tx, ty) (KICK_K x [0.8, 1.4])",
           "launch": {"tracks_per_warp": cfg.tracks_per_warp, "block": cfg.block}}
    for name, km in (("map_17x17", synth.kick_map()), ("constant_kick", None)):
        ctx.set_kick_map(km)
        runner = g.GraphRunner(pipe, cfg)
        ms = []
        for r in range(reps + 1):
            flush.add_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            runner.replay()
            e1.record()
            e1.synchronize()
            if r:
                ms.append(e0.elapsed_time(e1))
        ctx.check(what="kick map")
        tr = g.tracks_to_numpy(pipe.tracks, b.n_tracks)
        ev = physics.evaluate(b, tr)
        own = physics.own_track(b, tr)
        sel = (tr["nhits"] == 4) & own
        res[name] = {"events_per_s": b.n_events / float(np.median(ms)) * 1e3,
                     "efficiency": ev["efficiency"], "fake_rate": ev["fake_rate"],
                     "qop_median_rel_err": float(np.median(np.abs(tr["qop"][sel] / truth[sel] - 1.0)))}
        del runner
    ctx.close()
    return res


def measure_sector_groups(g, reps=10, tol_y=5.0):
    """Row f2 on 1000 events of a detector with 48 columns x 4 rows of
    sensors per plane and 84 groups (200 tracks, 4000 hits per event):
    device time of the bank-order decode, of the group pass
    (ut_sector_groups) and of the group search (compass_find_groups, y
    windows of +-tol_y), CUDA events, L2 flushed; each pass's algorithmic
    bytes against the measured HBM bandwidth (group pass: id read, six
    4-byte fields written per hit, group offsets written)."""
    import numpy as np
    import torch
    import synth
    from synth.grouped import generate_grouped
    b = generate_grouped(1000, n_columns=48, rows=4, n_groups=84, tracks=200, hits=4000, seed=21)
    gg = b.geom
    ctx = g.Context(gg.raw_geometry())
    raw_d, ev_d = g.upload_raw(b.raw, b.ev_off)
    nw = int(b.ev_off[-1])
    E = b.n_events
    hits = g.HitBuffers.allocate(2 * nw + 8, E, gg.n_columns * gg.rows)
    out = g.GroupHitBuffers.allocate(2 * nw + 8, E, gg.n_groups)
    ws = torch.empty((g.decode_workspace_size(E) + 15) // 16 * 4, dtype=torch.int32, device="cuda")
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda")
    velo = g.upload_velo(b)
    tracks = g.TrackBuffers.allocate(b.n_tracks)
    params = synth.CompassParams()
    t_dec, t_grp, t_find = [], [], []
    for r in range(reps + 1):
        flush.add_(1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        g.ut_decode(ctx, raw_d, nw, ev_d, E, hits, False, ws)
        ev[1].record()
        g.ut_sector_groups(ctx, hits, E, gg, out)
        ev[2].record()
        g.compass_find_groups(ctx, out, gg, velo, E, params, tracks, tol_y)
        ev[3].record()
        ev[3].synchronize()
        if r:
            t_dec.append(ev[0].elapsed_time(ev[1]))
            t_grp.append(ev[1].elapsed_time(ev[2]))
            t_find.append(ev[2].elapsed_time(ev[3]))
    ctx.check(what="sector groups")
    n = int(b.bank_n.sum())
    T = b.n_tracks
    alg = n * (4 + 24) + (E * 4 * gg.n_groups + 1) * 4 + 2 * E * 4
    # group search: hit x (staged once per event), group offsets, VELO state
    # and trk_off read, track slots written
    alg_find = 4 * n + (E * 4 * gg.n_groups + 1) * 4 + 17 * T + 4 * (E + 1) + 34 * T
    ms, ms_d, ms_f = (float(np.median(v)) for v in (t_grp, t_dec, t_find))
    peak, _ = peaks()
    found = int(tracks.found[:T].sum().item())
    ctx.close()
    return {"workload": "1000 events, 4 planes x 48 columns x 4 rows of sensors, 84 groups, hits/event 4000, "
                        "tracks/event 200",
            "hits": n, "decode_bank_order_ms": ms_d, "sector_groups_ms": ms,
            "algorithmic_bytes": alg, "achieved_gbs": alg / ms / 1e6, "frac": alg / ms / 1e6 / peak,
            "group_search": {"tol_y_mm": tol_y, "ms": ms_f, "found": found, "algorithmic_bytes": alg_find,
                             "achieved_gbs": alg_find / ms_f / 1e6, "frac": alg_find / ms_f / 1e6 / peak},
            "events_per_s": E / (ms_d + ms + ms_f) * 1e3,
            "events_per_s_what": "decode (bank order) + sector groups + group search"}


def measure_consolidation(g, ctx, pipe, batch, flush, reps=10):
    """ut_consolidate on the tracks of the last step: device time and the
    fraction of the measured HBM bandwidth of its algorithmic bytes (found
    flags and trk_off read, the found tracks' fields read and written)."""
    import numpy as np
    import torch
    E, T = batch.n_events, batch.n_tracks
    n = int(pipe.tracks.found[:T].sum().item())
    out = g.CompactTracks.allocate(n)
    off = torch.empty(E + 1, dtype=torch.int32, device="cuda")
    ws = g.ut_consolidate(ctx, pipe.velo.trk_off, E, pipe.tracks, out, off)
    ms = []
    for _ in range(reps + 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.ut_consolidate(ctx, pipe.velo.trk_off, E, pipe.tracks, out, off, ws)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctx.check(what="consolidation")
    m = float(np.median(ms[1:]))
    algo = T + 4 * (E + 1) + n * 33 + n * 37 + 4 * (E + 1)
    hbm, _ = peaks()
    return {"found_tracks": n, "ms": m, "algorithmic_bytes": algo, "achieved_gbs": algo / (m / 1e3) / 1e9,
            "frac": algo / (m / 1e3) / 1e9 / hbm}


def e2e_through_server(g, batch, params, cfg, steps, n_slots=4):
    """End to end through the serving engine: every step is one request of
    the whole batch (host inputs in page-locked memory copied in, one
    persistent launch, track slots copied out); up to n_slots requests are
    in flight on their own streams, so one request's copies overlap another
    one's kernel.  Host wall clock over `steps` requests after a warm-up."""
    import time as _t
    from paper_2002_11529_gb300 import serve
    reqs = [serve.HostRequest.from_batch(batch) for _ in range(n_slots)]
    h2d = sum(t.numel() * t.element_size() for t in reqs[0].bufs.values())
    d2h = sum(t.numel() * t.element_size() for t in reqs[0].out.values())
    with serve.Server(batch.geom, params, budget_bytes=8 << 30, n_slots=n_slots, cfg=cfg) as sv:
        def run(n):
            free = list(range(n_slots))
            inflight = {}
            sent = done = 0
            while done < n:
                while free and sent < n:
                    i = free.pop()
                    inflight[sv.submit(reqs[i])] = i
                    sent += 1
                for r in sv.poll(wait=True):
                    if r["status"] != 0:
                        raise RuntimeError(f"serving request failed: {r['status']} at {r['where']}")
                    free.append(inflight.pop(r["id"]))
                    done += 1
        run(2 * n_slots)
        t0 = _t.perf_counter()
        run(steps)
        wall = _t.perf_counter() - t0
    return wall, h2d, d2h


def summarize_variants(d):
    """The compact summary of the variant measurements kept at the end of
    the bench line (the full figures are printed on the detail lines)."""
    r = lambda v, n=4: None if v is None else round(float(v), n)
    out = {}
    u = d.get("uneven_workload")
    if u:
        out["uneven_20000"] = {"batched_ev_s": r(u["batched_form"]["events_per_s"], 0),
                               "plain_ev_s": r(u["plain_form"]["events_per_s"], 0),
                               "batched_over_plain": r(u["batched_over_plain"], 3),
                               "decode_sorted_frac": u["decode_only"]["sorted"]["frac"],
                               "decode_bank_order_frac": u["decode_only"]["bank_order"]["frac"]}
    sv = d.get("serving")
    if sv:
        out["serving"] = {"peak_ev_s": r(sv["peak_events_per_s"], 0)}
        for k in ("load_50", "load_80", "load_95"):
            if k in sv:
                out["serving"][k] = {"p50_ms": r(sv[k]["p50_ms"], 3), "p99_ms": r(sv[k]["p99_ms"], 3),
                                     "p99_ms_max": r(sv[k]["p99_ms_max"], 3)}
    a = d.get("alignment")
    if a:
        out["alignment"] = {"solve_20_ms": r(a["solve_20_steps_ms"], 3),
                            "chi2_per_track": [r(a["chi2_per_track"][k], 3)
                                               for k in ("start", "after_20_steps", "truth")]}
    c = d.get("consolidation")
    if c:
        out["consolidation"] = {"ms": r(c["ms"]), "frac": r(c["frac"])}
    sg = d.get("sector_groups")
    if sg:
        out["sector_groups"] = {"layout_frac": r(sg["frac"]), "search_ms": r(sg["group_search"]["ms"]),
                                "ev_s": r(sg["events_per_s"], 0)}
    return out


def algorithmic_bytes(batch):
    """Minimum bytes each kernel must move for one batch."""
    E, B, H, T = batch.n_events, batch.geom.n_banks, batch.n_hits, batch.n_tracks
    raw = 4 * int(batch.ev_off[-1]) + 8 * (E + 1)
    decode = raw + 4 * (E * B + 1) + 15 * H
    # find: hit x of the searched banks (<= all hits), offsets, VELO state, outputs
    find = 4 * H + 4 * (E * B + 1) + 17 * T + 4 * (E + 1) + 34 * T
    sort_b = 2 * 15 * H + 4 * (E * B + 1)
    fit = 17 * T + 16 * T + 16 * T + 4 * 4 * T
    # one persistent kernel: decode traffic + VELO in + track slots out
    # (the search reads the event's hits from shared memory)
    batched = decode + 17 * T + 4 * (E + 1) + 34 * T
    return {"ut_decode": decode, "compass_find": find, "ut_sort_hits": sort_b, "compass_fit": fit,
            "ut_run_batched": batched}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import synth
    import paper_2002_11529_gb300 as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    g.build.build()

    params = synth.CompassParams()
    if args.only is not None:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
        fn = {"sector_groups": lambda: measure_sector_groups(g), "alignment": lambda: measure_alignment(g, params),
              "uneven_workload": lambda: time_forms_on_uneven_workload(g, params, flush),
              "serving": lambda: measure_serving(g, params)}[args.only]
        print(f"detail {args.only} {json.dumps(fn())}", flush=True)
        return
    batch = make_batch(args.workload, rank, args.events)
    ctx = g.Context(batch.geom)
    pipe = g.Pipeline(ctx, batch, params)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    tpw = args.tracks_per_warp
    blk = args.block if args.block is not None else (800 if tpw == 8 else 256)
    E = batch.n_events

    kern = {"plain": ["ut_decode", "ut_sort_hits", "compass_find", "compass_fit"],
            "fused": ["ut_decode", "compass_find"],
            "batched": ["ut_run_batched"]}[args.form]
    cfg = g.LaunchConfig(tpw, blk, args.x_cap, 8192)
    tune_table = None
    if args.form == "batched" and not args.no_autotune:
        from paper_2002_11529_gb300 import autotune
        cfg, tune_table = autotune.autotune(pipe, reps=3, flush=flush)
    runner = g.GraphRunner(pipe, cfg) if args.form == "batched" else None

    def step(ev=None):
        """One pass; ev: list of (start, end) event pairs per kernel."""
        def mark(i, which):
            if ev is not None:
                ev[i][which].record(stream)
        if args.form == "batched":
            mark(0, 0)
            runner.replay()
            mark(0, 1)
        elif args.form == "plain":
            mark(0, 0)
            g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, E, pipe.hits_a, False, pipe.workspace, stream)
            mark(0, 1); mark(1, 0)
            g.ut_sort_hits(ctx, pipe.hits_a, pipe.hits_b, E, stream=stream)
            pipe.hits_b.hit_off = pipe.hits_a.hit_off
            mark(1, 1); mark(2, 0)
            g.compass_find(ctx, pipe.hits_b, pipe.velo, E, params, pipe.tracks, tracks_per_warp=tpw,
                           block=blk, stream=stream)
            mark(2, 1); mark(3, 0)
            g.compass_fit(ctx, pipe.hits_b, pipe.velo, params, pipe.tracks, stream=stream)
            mark(3, 1)
        else:
            mark(0, 0)
            g.ut_decode(ctx, pipe.raw, pipe.n_words, pipe.ev_off, E, pipe.hits_a, True, pipe.workspace, stream)
            mark(0, 1); mark(1, 0)
            g.compass_find(ctx, pipe.hits_a, pipe.velo, E, params, pipe.tracks, tracks_per_warp=tpw,
                           block=blk, stream=stream)
            mark(1, 1)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ctx.check(stream, "warm-up")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-timed region -------------------------------------------------
    nk = len(kern)
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(nk)]
           for _ in range(args.steps)]
    step_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    clocks = Clocks(local) if rank == 0 else None
    barrier()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        step_ev[k][0].record(stream)
        step(evs[k])
        step_ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop() if clocks else None
    ctx.check(stream, "timed region")
    step_ms = [step_ev[k][0].elapsed_time(step_ev[k][1]) for k in range(args.steps)]
    kern_ms = {kern[i]: [evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(args.steps)] for i in range(nk)}
    tot_ms = max_over_ranks(sum(step_ms), dist)
    value = job_events_per_s(world, E, args.steps, tot_ms / 1e3)

    # ---- end to end through host buffers ------------------------------------
    h_raw = pipe.raw.cpu().pin_memory()
    h_ev = pipe.ev_off.cpu().pin_memory()
    h_velo = [getattr(pipe.velo, n).cpu().pin_memory() for n in ("x", "y", "tx", "ty", "flags", "trk_off")]
    d_velo = [getattr(pipe.velo, n) for n in ("x", "y", "tx", "ty", "flags", "trk_off")]
    outs = [pipe.tracks.hit, pipe.tracks.qop, pipe.tracks.chi2, pipe.tracks.x, pipe.tracks.tx,
            pipe.tracks.nhits, pipe.tracks.found]
    h_outs = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
    h2d = sum(t.numel() * t.element_size() for t in [h_raw, h_ev] + h_velo)
    d2h = sum(t.numel() * t.element_size() for t in h_outs)

    def e2e_step():
        pipe.raw.copy_(h_raw, non_blocking=True)
        pipe.ev_off.copy_(h_ev, non_blocking=True)
        for d, h in zip(d_velo, h_velo):
            d.copy_(h, non_blocking=True)
        step()
        for h, d in zip(h_outs, outs):
            h.copy_(d, non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.zero_()
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    barrier()
    e2e_ms = max_over_ranks(e2e_ms, dist)
    ctx.check(stream, "e2e")
    e2e_serial = job_events_per_s(world, E, args.steps, e2e_ms / 1e3)
    e2e = {"value": e2e_serial, "unit": "events/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "how": "copy in, step, copy out on one stream, one step at a time (CUDA events)"}
    if args.form == "batched":
        # the persistent form through the serving engine: steps overlap
        wall, sh2d, sd2h = e2e_through_server(g, batch, params, cfg, args.steps)
        wall = max_over_ranks(wall, dist)
        e2e = {"value": job_events_per_s(world, E, args.steps, wall), "unit": "events/s", "h2d_bytes_per_step": sh2d,
               "d2h_bytes_per_step": sd2h,
               "how": "ut_server: each step one request of the whole batch from page-locked host memory, "
                      "up to 4 in flight on 4 stream slots; host wall clock",
               "serial": {"value": e2e_serial, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                          "how": e2e["how"]}}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- roofline of each kernel (algorithmic bytes / mean launch time) -----
    hbm, peak_kind = peaks()
    algo = algorithmic_bytes(batch)
    kinfo = {}
    for name in kern:
        ms = statistics.mean(kern_ms[name])
        gbs = algo[name] / (ms / 1e3) / 1e9
        kinfo[name] = {"ms": round(ms, 5), "algorithmic_bytes": algo[name], "achieved_gbs": round(gbs, 1),
                       "frac": round(gbs / hbm, 4), "share": round(ms / (tot_ms / args.steps), 3)}
    dom = max(kern, key=lambda n: kinfo[n]["ms"])
    roof = {"kernel": dom, "bound": "hbm", "achieved": kinfo[dom]["achieved_gbs"], "peak": hbm,
            "unit": "GB/s", "frac": kinfo[dom]["frac"], "traffic": measured_traffic(dom, args.workload),
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback 6.8 TB/s"}
    lat = sorted(step_ms)
    p = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded generator standing in for the LHCb minbias sample)",
        "config": workload_config(args.workload, batch, args.form,
                                  {"tracks_per_warp": cfg.tracks_per_warp, "block": cfg.block,
                                   "x_cap": cfg.x_cap, "graph": args.form == "batched",
                                   "autotuned": tune_table is not None,
                                   "parallelism": f"events sharded, {world} independent replicas" if world > 1
                                   else "single GPU"}),
        "latency_ms": {"p50": p(0.5), "p99": p(0.99), "what": "one step = one batch"},
        "roofline": roof,
        "kernels": kinfo,
        "e2e": e2e,
        "gpu_launches": nk * args.steps,
        "autotune": None if tune_table is None else [
            {"tracks_per_warp": c.tracks_per_warp, "block": c.block, "x_cap": c.x_cap, "ms": round(m, 4)}
            for c, m in tune_table],
        "clocks": clk,
        "wall_s": wall,
    }
    detail = {"autotune": line.pop("autotune")}
    if not args.no_variants and world == 1:
        detail["uneven_workload"] = time_forms_on_uneven_workload(g, params, flush)
        detail["serving"] = measure_serving(g, params, cfg if args.form == "batched" else None)
        detail["alignment"] = measure_alignment(g, params)
        detail["consolidation"] = measure_consolidation(g, ctx, pipe, batch, flush)
        detail["sector_groups"] = measure_sector_groups(g)
        if args.physics:
            detail["physics_sweep"] = physics_sweep(g, batch, params)
            detail["kick_map"] = measure_kick_map(g, params,
                                                  cfg if args.form == "batched" else g.LaunchConfig(8, 512))
        line["variants"] = summarize_variants(detail)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(batch, params)
    # full measurements first (lines that are not JSON objects), then the
    # bench line, whose last keys hold the compact summary
    for k, v in detail.items():
        if v is not None:
            print(f"detail {k} {json.dumps(v)}", flush=True)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
