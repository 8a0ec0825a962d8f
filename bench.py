#!/usr/bin/env python
"""Throughput benchmark of the 3D degridding hot path; prints one JSON line.

A step is one degrid_execute over the whole workload: 64 subgrids of
512 x 512 x 4 complex64 samples with 250,000 visibilities each on random
lines (16M visibilities), Kaiser-Bessel G_uv (support 8, oversampling 16384)
and G_w (support 4, oversampling 128).  Inputs are resident in HBM when the
timed region starts; L2 is flushed (256 MB write, outside the step events)
before every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank degrids its own copy of the workload on its
own GPU (independent subgrid shards, no collective on the data path); the
step time is the maximum over ranks and `value` counts all ranks' work.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "degridded visibilities/s on 1 GB300: FP32 vs BF16/FP16 subgrids at stated error"
UNIT = "visibilities/s"
WORKLOAD = "lines64_250k"
WORKLOAD_DESC = ("64 subgrids of 512x512x4 complex64 (i.i.d. complex Gaussian), 250,000 "
                 "visibilities per subgrid on a random line each (16,000,000 total); "
                 "separable Kaiser-Bessel G_uv support 8 oversampling 16384, G_w support 4 "
                 "oversampling 128")
FLOP_PER_VIS = 1024          # 256 footprint points x complex*real FMA (2 FMA = 4 flop)
# DRAM bytes (read + write) per visibility of degrid_kernel<DG_C64>, from one ncu capture
# of the 4,000,000-visibility case lines16_250k (the traffic is uvw, output and footprints,
# all proportional to the visibilities).  Valid only for the kernel sources it was taken
# on: the bench reports null traffic once they change.
TRAFFIC_KERNEL_SOURCES = ("paper_2102_12739_gb300/csrc/degrid.cu",
                          "paper_2102_12739_gb300/csrc/pipeline.cuh",
                          "paper_2102_12739_gb300/csrc/internal.cuh")
TRAFFIC_SHA = "a15f6785f22862b7"
TRAFFIC_BYTES_PER_VIS = (98.424320e6 + 11.519232e6) / 4_000_000
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20
# (chunk, warps per CTA, CTAs per SM, direct-arm threshold) tried on the headline workload
HEADLINE_CANDIDATES = [(256, 8, 0, 33), (512, 8, 0, 33), (256, 4, 0, 33), (512, 4, 0, 33)]


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="named workload (paper_2102_12739_gb300.synth.workload); the "
                         "default is the throughput configuration, others serve profiling")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--sweep-steps", type=int, default=500)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-scatter", action="store_true")
    ap.add_argument("--no-table2d", action="store_true")
    ap.add_argument("--no-predict", action="store_true")
    ap.add_argument("--aux-steps", type=int, default=50,
                    help="timed steps of the batched and adjoint sections")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        cmd = ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + ",".join(self.FIELDS),
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        self.out.close()
        os.unlink(self.out.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 8:
                continue
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for n, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_query_id(torch, dev) -> str:
    try:
        p = torch.cuda.get_device_properties(dev)
        return "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return str(dev.index)


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------

def oracle_pairs(subgrids) -> np.ndarray:
    """complex subgrids -> the FP64 (re, im) pairs the oracle works on
    (exact), so that the timed oracle calls do not include the conversion."""
    sub = np.asarray(subgrids)
    return np.ascontiguousarray(np.stack([sub.real, sub.imag], axis=-1), dtype=np.float64)


# the reference arm's whole run (warm-up and timed steps) is sized to about
# this much CPU time: each step degrids as many whole subgrids of the
# workload as fit, all 64 when the run has few steps
REFERENCE_RUN_SECONDS = 60.0


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_2102_12739_gb300 import synth
    g_uv, g_w = synth.default_tables()
    w = synth.workload(WORKLOAD)
    # probe: one subgrid's list, to size the step
    probe = oracle_pairs(w.subgrid(0)[None])
    lo1 = int(w.vis_offsets[1])
    t0 = time.perf_counter()
    oracle.degrid(g_uv, g_w, probe, w.uvw[:lo1], w.vis_offsets[:2])
    per_subgrid = time.perf_counter() - t0
    m = int(REFERENCE_RUN_SECONDS / max(args.steps + args.warmup, 1) / max(per_subgrid, 1e-6))
    m = max(1, min(w.n_subgrids, m))
    hi = int(w.vis_offsets[m])
    sub = oracle_pairs(w.subgrids()[:m]) if m > 1 else probe
    uvw = w.uvw[:hi]
    offs = w.vis_offsets[:m + 1]
    for _ in range(args.warmup):
        oracle.degrid(g_uv, g_w, sub, uvw, offs)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.degrid(g_uv, g_w, sub, uvw, offs)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * hi / total
    cores = oracle.max_threads()
    whole = m == w.n_subgrids
    sample = ("the whole workload (%d visibilities) per step" % hi if whole else
              "subgrids 0..%d of the workload (%d of its %d visibilities) per step, sized so that "
              "the %d steps end in about %.0f s" % (m - 1, hi, w.n_vis, args.steps + args.warmup,
                                                    REFERENCE_RUN_SECONDS))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD + ": " + WORKLOAD_DESC, "n_vis": w.n_vis,
                   "subgrid_storage": "complex64",
                   "step": "FP64 CPU oracle over " + sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu": cpu_model(), "nproc": os.cpu_count(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def cpu_model() -> str:
    """Host CPU model (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline(g_uv, g_w, reps=3):
    """The FP64 oracle, as it stands, on the host cores: degridding on the
    single-line, headline and batched workloads and gridding on the
    differentiation workload, each the median of `reps` runs (inputs
    prepared outside the timing).  The batched workload's sample is every
    8th of its 512 subgrids (64 lists, all count decades), so that the whole
    baseline stays within about a minute."""
    import oracle
    from paper_2102_12739_gb300 import synth

    def timed(fn):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    def forward(w, pick=None):
        ids = np.arange(w.n_subgrids) if pick is None else np.asarray(pick)
        rows = np.concatenate([np.arange(w.vis_offsets[s], w.vis_offsets[s + 1]) for s in ids])
        uvw = np.ascontiguousarray(w.uvw[rows])
        offs = synth.offsets_from_counts(w.counts()[ids])
        sub = oracle_pairs(np.stack([w.subgrid(int(s)) for s in ids]))
        t = timed(lambda: oracle.degrid(g_uv, g_w, sub, uvw, offs))
        return {"visibilities": int(offs[-1]), "subgrids": int(len(ids)), "median_s": t,
                "value": offs[-1] / t, "unit": UNIT}

    per = {}
    per["line1_20k"] = forward(synth.workload("line1_20k"))
    per[WORKLOAD] = forward(synth.workload(WORKLOAD))
    wb = synth.workload("batched512")
    per["batched512 (every 8th subgrid)"] = forward(wb, np.arange(0, wb.n_subgrids, 8))
    wd = synth.workload("diff32_100k")
    y = synth.adjoint_vis(wd.n_vis)
    t = timed(lambda: oracle.grid(g_uv, g_w, wd.shape, wd.n_subgrids, wd.uvw, wd.vis_offsets, y))
    per["diff32_100k gridding (adjoint)"] = {"visibilities": wd.n_vis, "subgrids": wd.n_subgrids,
                                             "median_s": t, "value": wd.n_vis / t,
                                             "unit": "gridded visibilities/s"}
    head = per[WORKLOAD]
    return {"value": head["value"], "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "cpu": cpu_model(), "nproc": os.cpu_count(),
            "sample": "the whole %s workload (%d visibilities), median of %d runs; per_config "
                      "adds the other workloads" % (WORKLOAD, head["visibilities"], reps),
            "per_config": per}


def oracle_reference(w, g_uv, g_w, subgrid_of, group=8):
    """The FP64 oracle's value of every visibility of w, complex128 [N]
    (subgrid_of(s) gives subgrid s in any complex type)."""
    import oracle
    out = np.empty(w.n_vis, dtype=np.complex128)
    for s0 in range(0, w.n_subgrids, group):
        s1 = min(s0 + group, w.n_subgrids)
        lo, hi = int(w.vis_offsets[s0]), int(w.vis_offsets[s1])
        if hi > lo:
            sub = oracle_pairs(np.stack([subgrid_of(s) for s in range(s0, s1)]))
            out[lo:hi], _ = oracle.degrid(g_uv, g_w, sub, w.uvw[lo:hi], w.vis_offsets[s0:s1 + 1] - lo)
    return out


def error_vs(got, ref):
    """Relative L2 and max-abs error of got against ref over every visibility."""
    d = np.asarray(got, dtype=np.complex128) - ref
    return float(np.linalg.norm(d) / np.linalg.norm(ref)), float(np.max(np.abs(d)))


def warm_up(torch, call, flush_buf, steps, min_seconds=1.0):
    """At least `steps` (>= 3) untimed steps, and at least `min_seconds` of them,
    so that clocks have ramped up before the timed region."""
    t0 = time.perf_counter()
    done = 0
    while done < max(steps, 3) or time.perf_counter() - t0 < min_seconds:
        flush_buf.zero_()
        call()
        done += 1
        if done % 50 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()


def warm_kernel_ms(torch, plan, call, steps):
    """Median main-kernel time with warm caches (no flush between calls)."""
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    plan.kernel_times_ms(1)
    for _ in range(steps):
        call()
    ms = sorted(plan.kernel_times_ms(steps))
    return ms[len(ms) // 2]


def time_steps(torch, plan, call, steps, flush_buf, stream):
    """Run `steps` calls with an L2 flush before each; return per-step event
    times (ms) and per-launch main-kernel times (ms)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        flush_buf.zero_()
        ev[i][0].record(stream)
        call()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = plan.kernel_times_ms(steps)
    return step_ms, kern_ms


def batched_section(torch, dg, synth, dev, flush, steps):
    """512 subgrids with log-uniform counts in [1e3, 1e6] (segments and arcs):
    for each storage type autotuned, captured once in a CUDA graph and
    replayed."""
    w = synth.workload("batched512")
    sub = synth.subgrid_stack_on_device(w.n_subgrids, dev, w.shape)
    uvw = torch.from_numpy(w.uvw).to(dev)
    offs = torch.from_numpy(w.vis_offsets).to(dev)
    out = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)
    res = {}
    for dt in ("c64", "f16", "bf16"):
        codes, scale = (sub, None) if dt == "c64" else dg.pack_subgrids(sub, dt)
        with dg.DegridPlan(dtype=dt, device=dev) as plan:
            tuned = dg.autotune(plan, codes, uvw, offs, scale=scale, use_cache=False)
            plan.degrid(codes, uvw, offs, scale=scale, out=out)
            torch.cuda.synchronize()
            assert plan.status() == 0
            graph = torch.cuda.CUDAGraph()
            cap = torch.cuda.Stream(device=dev)
            with torch.cuda.stream(cap):
                with torch.cuda.graph(graph, stream=cap):
                    plan.degrid(codes, uvw, offs, scale=scale, out=out)
            stream = torch.cuda.current_stream(dev)
            warm_up(torch, graph.replay, flush, 3, min_seconds=0.3)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                graph.replay()
                b.record(stream)
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in ev)
            del graph
        med = ms[len(ms) // 2]
        res[dt] = {"value": w.n_vis / (med * 1e-3), "ms_per_step": med, "tuning": tuned["tuning"],
                   "autotune_candidates": len(tuned["timings"])}
        if dt != "c64":
            del codes, scale
    counts = w.counts()
    return {"workload": "batched512: 512 subgrids 512x512x4, visibility counts "
                        "log-uniform in [1e3, 1e6] (%d..%d, %d total), lists of 1-8 segments "
                        "or arcs; subgrid values from a seeded on-device generator"
                        % (counts.min(), counts.max(), w.n_vis),
            "value": res["c64"]["value"], "unit": UNIT, "ms_per_step": res["c64"]["ms_per_step"],
            "steps": steps, "cuda_graph": True, "tuning": res["c64"]["tuning"],
            "autotune_candidates": res["c64"]["autotune_candidates"], "by_storage": res}


def scatter_section(torch, dg, synth, dev, flush, steps, l2_gbs):
    """Sparse coverage: every visibility has its own footprint (no reuse), the
    regime where subgrid bytes, and so the storage type, matter.  Each storage
    type is autotuned over the summing arms, then timed.  The no-reuse bound
    is the footprint bytes (256 elements of 8 B complex64 or 4 B FP16/BF16 per
    visibility) at the measured L2 read bandwidth."""
    import oracle
    w = synth.workload("scatter16_250k")
    sub_np = w.subgrids()
    sub = torch.from_numpy(sub_np).to(dev)
    uvw = torch.from_numpy(w.uvw).to(dev)
    offs = torch.from_numpy(w.vis_offsets).to(dev)
    out = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)
    g_uv, g_w = synth.default_tables()
    ref = oracle_reference(w, g_uv, g_w, lambda s: sub_np[s])
    cands = [(256, 8, 0, 33, 0), (256, 8, 0, 9, 0), (512, 4, 0, 33, 0), (512, 4, 0, 9, 0),
             (128, 8, 0, 33, 1), (256, 8, 0, 33, 1), (512, 8, 0, 33, 1)]
    res = {}
    for dt in ("c64", "f16", "bf16"):
        codes, scale = (sub, None) if dt == "c64" else dg.pack_subgrids(sub, dt)
        with dg.DegridPlan(dtype=dt, device=dev) as plan:
            tuned = dg.autotune(plan, codes, uvw, offs, scale=scale, candidates=cands,
                                use_cache=False)
            plan.enable_timing(steps)

            def step():
                plan.degrid(codes, uvw, offs, scale=scale, out=out)
            warm_up(torch, step, flush, 3, min_seconds=0.2)
            s_ms, k_ms = time_steps(torch, plan, step, steps, flush, torch.cuda.current_stream(dev))
            err = error_vs(out.cpu().numpy(), ref)
        ms = sorted(s_ms)[len(s_ms) // 2]
        kms = sorted(k_ms)[len(k_ms) // 2]
        gather_ms = w.n_vis * 256 * (8 if dt == "c64" else 4) / (l2_gbs * 1e9) * 1e3
        res[dt] = {"value": w.n_vis / (ms * 1e-3), "ms_per_step": ms,
                   "kernel_ms": kms, "l2_gather_bound_ms": gather_ms,
                   "frac_of_l2_gather_bound": gather_ms / kms, "rel_l2": err[0],
                   "error_sample": "all",
                   "arm": ("gather" if tuned["tuning"]["gather"] else
                           "direct" if tuned["tuning"]["direct_runs"] < 33 else "footprint cache"),
                   "tuning": tuned["tuning"]}
        del codes, scale
    # gridding (the adjoint) of the same coverage: the run-accumulating kernel
    # (atomic adds at every run end) and the tensor reduce-add kernel
    y = torch.from_numpy(synth.adjoint_vis(w.n_vis)).to(dev)
    grid_out = torch.empty((w.n_subgrids,) + w.shape, dtype=torch.complex64, device=dev)
    gridding = {}
    for gather in (False, True):
        with dg.DegridPlan(device=dev, gather=gather) as plan:
            plan.enable_timing(steps)
            warm_up(torch, lambda: plan.grid(y, uvw, offs, w.n_subgrids, out=grid_out), flush, 3,
                    min_seconds=0.3)
            for _ in range(steps):
                flush.zero_()
                plan.grid(y, uvw, offs, w.n_subgrids, out=grid_out)
            k_ms = sorted(plan.kernel_times_ms(steps))
            assert plan.status() == 0
        kms = k_ms[len(k_ms) // 2]
        gridding["tensor reduce-add" if gather else "run accumulation + atomics"] = {
            "kernel_ms": kms, "value": w.n_vis / (kms * 1e-3), "unit": "gridded visibilities/s"}
    # the reduce-add kernel's bound: every visibility adds its 2 KB footprint
    # tile, at the measured rate of the copy engines' tensor reduce-adds
    red_gbs = dg.measure_l2_reduce_bw(dev.index)
    red = gridding["tensor reduce-add"]
    red["reduce_bound_ms"] = w.n_vis * 2048 / (red_gbs * 1e9) * 1e3
    red["frac_of_reduce_bound"] = red["reduce_bound_ms"] / red["kernel_ms"]
    red["l2_reduce_gbs_measured"] = red_gbs
    return {"workload": "scatter16_250k: 16 subgrids 512x512x4, 250,000 visibilities each "
                        "scattered uniformly over the valid box (no footprint shared by "
                        "consecutive visibilities)", "unit": UNIT, "steps": steps,
            "l2_read_gbs_measured": l2_gbs, "by_storage": res, "gridding": gridding}


def latency_section(torch, dg, synth, dev, steps):
    """The smallest configuration (1 subgrid, 20,000 visibilities on a line):
    time of one degrid_execute call, schedule included, inputs in HBM."""
    w = synth.workload("line1_20k")
    sub = torch.from_numpy(synth.subgrid_stack(1)).to(dev)
    uvw = torch.from_numpy(w.uvw).to(dev)
    offs = torch.from_numpy(w.vis_offsets).to(dev)
    out = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    with dg.DegridPlan(device=dev) as plan:
        t0 = time.perf_counter()            # clocks ramped up first (at least 0.3 s of calls)
        done = 0
        while done < 20 or time.perf_counter() - t0 < 0.3:
            plan.degrid(sub, uvw, offs, out=out)
            done += 1
            if done % 200 == 0:
                torch.cuda.synchronize()
        torch.cuda.synchronize()

        def timed(prefill):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            if prefill:
                # a spin kernel holds the stream while the host queues every
                # call, so each event pair brackets only that call's GPU work
                torch.cuda._sleep(20_000_000)
            for a, b in ev:
                a.record(stream)
                plan.degrid(sub, uvw, offs, out=out)
                b.record(stream)
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in ev)
            return ms[len(ms) // 2] * 1e3

        paced_us = timed(False)
        device_us = timed(True) if hasattr(torch.cuda, "_sleep") else None
        assert plan.status() == 0
    call_us = device_us if device_us is not None else paced_us
    return {"workload": "line1_20k: 1 subgrid 512x512x4, 20,000 visibilities on one line",
            "call_us": call_us, "value": w.n_vis / (call_us * 1e-6),
            "unit": UNIT, "steps": steps,
            "call_us_host_paced": paced_us,
            "timing": "call_us: GPU time of one call with the queue filled ahead (events on the "
                      "stream, medians); call_us_host_paced: calls issued back to back as the host "
                      "enqueues them, so the host's own enqueue time can show",
            "call_includes": "one scheduling launch (offset validation, chunk scan and chunk "
                             "table) and the degridding kernel"}


def table2d_section(torch, dg, synth, dev, flush, steps, sub, sub_np, uvw, offs, w):
    """The headline workload with a non-separable G_uv: a circular
    Kaiser-Bessel table [64][64][8][8] (weights read per visibility from L2)."""
    import oracle
    G2 = synth.default_table_2d()
    out = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)
    with dg.DegridPlan(device=dev, g_uv2=G2) as plan:
        plan.enable_timing(steps)

        def step():
            plan.degrid(sub, uvw, offs, out=out)
        warm_up(torch, step, flush, 3, min_seconds=0.3)
        s_ms, k_ms = time_steps(torch, plan, step, steps, flush, torch.cuda.current_stream(dev))
        assert plan.status() == 0
    got = out.cpu().numpy()
    _, g_w = synth.default_tables()
    ref = np.empty(w.n_vis, dtype=np.complex128)
    for s0 in range(0, w.n_subgrids, 8):
        lo, hi = int(w.vis_offsets[s0]), int(w.vis_offsets[min(s0 + 8, w.n_subgrids)])
        ref[lo:hi], _ = oracle.degrid_2d(G2, g_w, oracle_pairs(sub_np[s0:s0 + 8]), w.uvw[lo:hi],
                                         w.vis_offsets[s0:s0 + 9] - lo)
    ms = sorted(s_ms)[len(s_ms) // 2]
    return {"workload": WORKLOAD + " with a non-separable G_uv: circular Kaiser-Bessel table, "
                        "oversampling 64 ([64][64][8][8] FP32, 1 MiB)",
            "value": w.n_vis / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "kernel_ms": sorted(k_ms)[len(k_ms) // 2],
            "rel_l2_vs_oracle": error_vs(got, ref)[0], "error_sample": "all",
            "steps": steps}


def predict_section(torch, dg, synth, dev, flush, steps, hbm_gbs, plan=None, uvw=None, offs=None):
    """The step upstream of degridding: 64 subgrids of 512 x 512 x 4 made from
    a 512 x 512 model sky (the w-plane grids of improved w-stacking, 4 planes
    per subgrid, 256 planes in all), then, with the headline plan, those
    subgrids degridded at the headline workload's 16M visibilities: sky image
    to visibilities in one step."""
    from oracle import predict as P
    n, S, per_pass = 512, 64, 32
    img_np, tp_np = synth.sky_image(n), synth.image_taper(n)
    uv_np, w_np = synth.predict_offsets(S)
    img = torch.from_numpy(img_np).to(dev)
    tp = torch.from_numpy(tp_np).to(dev)
    uv = torch.from_numpy(uv_np).to(dev)
    w = torch.from_numpy(w_np).to(dev)
    out = torch.empty((S, n, n, 4), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        warm_up(torch, fn, flush, 3, min_seconds=0.3)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        t = sorted(a.elapsed_time(b) for a, b in ev)
        return t[len(t) // 2]

    res = {}
    with dg.SubgridPredictor(n, 4, per_pass, device=dev) as pr:
        def produce():
            pr.predict(img, synth.PREDICT_THETA, uv, w, taper=tp, out=out)
        ms = timed(produce)
        got = out.cpu().numpy()
        s_w = int(offs.shape[0]) - 1 if offs is not None else 0
        if plan is not None and 0 < s_w <= S:
            vis = torch.empty(uvw.shape[0], dtype=torch.complex64, device=dev)

            def sky_to_vis():
                produce()
                plan.degrid(out[:s_w], uvw, offs, out=vis)
            pipe_ms = timed(sky_to_vis)
            assert plan.status() == 0
            res["sky_to_visibilities"] = {
                "value": uvw.shape[0] / (pipe_ms * 1e-3), "unit": UNIT, "ms_per_step": pipe_ms,
                "step": "64 subgrids made from the sky image, then %d visibilities degridded from the "
                        "first %d of them (the headline plan and coordinates)" % (uvw.shape[0], s_w)}
    ref = P.predict(img_np, synth.PREDICT_THETA, np.concatenate([uv_np, w_np], axis=1), nz=4, taper=tp_np)
    err = error_vs(got.reshape(-1), ref.reshape(-1))
    out_bytes = S * n * n * 4 * 8
    in_bytes = n * n * (8 + 4)
    bound_ms = (out_bytes + in_bytes) / (hbm_gbs * 1e9) * 1e3
    res.update({
        "workload": "64 subgrids 512x512x4 (complex64) from a 512x512 model sky (300 point sources + "
                    "background), image width 0.1 direction cosines, tapered; w-stacks of 4 planes "
                    "100 wavelengths apart covering -12800..12800 wavelengths",
        "value": S / (ms * 1e-3), "unit": "subgrids/s", "ms_per_call": ms, "steps": steps,
        "subgrids_per_pass": per_pass,
        "kernels": "screen_kernel (tapered image x w-phase screens), batched 512x512 C2C FFT (cuFFT), "
                   "window_kernel (cell window, sign, [y][x][c] interleave)",
        "hbm_bytes_compulsory": out_bytes + in_bytes, "hbm_bound_ms": bound_ms,
        "hbm_frac": bound_ms / ms,
        "rel_l2_vs_oracle": err[0], "max_abs_vs_oracle": err[1], "error_sample": "all"})
    return res


def adjoint_section(torch, dg, synth, dev, flush, steps):
    """Gridding (the adjoint) of 32 subgrids x 100,000 random-line visibilities.
    The gridding call is timed over at least 150 L2-flushed calls (medians):
    its kernel time varies by about 2% between groups of 50."""
    w = synth.workload("diff32_100k")
    steps = max(steps, 150)
    uvw = torch.from_numpy(w.uvw).to(dev)
    offs = torch.from_numpy(w.vis_offsets).to(dev)
    y = torch.from_numpy(synth.adjoint_vis(w.n_vis)).to(dev)
    out = torch.empty((w.n_subgrids,) + w.shape, dtype=torch.complex64, device=dev)
    with dg.DegridPlan(device=dev) as plan:
        plan.enable_timing(steps)
        # as for every timed section: clocks ramped up first (the workload's
        # generation on the host leaves the GPU idle for about a second)
        warm_up(torch, lambda: plan.grid(y, uvw, offs, w.n_subgrids, out=out), flush, 3, min_seconds=0.3)
        stream = torch.cuda.current_stream(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            plan.grid(y, uvw, offs, w.n_subgrids, out=out)
            b.record(stream)
        torch.cuda.synchronize()
        call_ms = sorted(a.elapsed_time(b) for a, b in ev)
        kern_ms = sorted(plan.kernel_times_ms(steps))
        assert plan.status() == 0
        # the same workload forward (degridding) and as one autograd step:
        # forward, loss ||D s - y||^2, backward (gridding of 2 (D s - y))
        sub = synth.subgrid_stack_on_device(w.n_subgrids, dev, w.shape)
        vis = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)

        def fwd():
            plan.degrid(sub, uvw, offs, out=vis)

        s_req = sub.clone().requires_grad_(True)

        def train_step():
            s_req.grad = None
            v = dg.DegridFn.apply(s_req, uvw, offs, plan)
            (v - y).abs().pow(2).sum().backward()

        def time_fn(fn):
            warm_up(torch, fn, flush, 3, min_seconds=0.3)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(steps)]
            for a, b in evs:
                flush.zero_()
                a.record(stream)
                fn()
                b.record(stream)
            torch.cuda.synchronize()
            t = sorted(a.elapsed_time(b) for a, b in evs)
            return t[len(t) // 2]
        fwd_ms = time_fn(fwd)
        step_ms = time_fn(train_step)
        assert plan.status() == 0
    return {"workload": "diff32_100k: 32 subgrids 512x512x4, 100,000 random-line visibilities each",
            "visibilities": w.n_vis,
            "value": w.n_vis / (call_ms[len(call_ms) // 2] * 1e-3), "unit": "gridded visibilities/s",
            "ms_per_call": call_ms[len(call_ms) // 2], "kernel_ms": kern_ms[len(kern_ms) // 2],
            "call_includes": "zeroing the 256 MB output stack, scheduling kernels, gridding kernel",
            "forward_ms": fwd_ms, "forward_value": w.n_vis / (fwd_ms * 1e-3),
            "autograd_step_ms": step_ms,
            "autograd_step": "DegridFn forward, loss ||D s - y||^2 in torch, backward = gridding",
            "steps": steps}


def kernel_sources_sha():
    """Hash of the kernel sources' device code (comments and whitespace
    removed, so that documentation edits keep the measured traffic valid; of
    the shared header only the part before the plan object and of degrid.cu
    only the part before its host-side launch code, so that host-side changes
    do not invalidate it; without the index checks of the bounds-checking
    build)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in TRAFFIC_KERNEL_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            src = fh.read()
        if f.endswith("internal.cuh"):
            src = src.split("struct degrid_plan {")[0]
        if f.endswith("degrid.cu"):
            src = src.split("\nsize_t smem_bytes(")[0]
        # the index checks exist only in the bounds-checking build
        src = re.sub(r"#ifdef DEGRID_BOUNDS_CHECK.*?#endif", " ", src, flags=re.S)
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def measured_traffic(n_vis):
    """DRAM bytes per launch from the ncu capture, or None if the kernel changed since."""
    try:
        if kernel_sources_sha() != TRAFFIC_SHA:
            return None
    except OSError:
        return None
    return TRAFFIC_BYTES_PER_VIS * n_vis


def run_ours(args, rank, world):
    import torch
    import paper_2102_12739_gb300 as dg
    from paper_2102_12739_gb300 import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks, peaks_src = measured_peaks()

    g_uv, g_w = synth.default_tables()
    if world > 1 and args.workload == WORKLOAD:
        # weak scaling: the job has 64 subgrids per GPU; this rank builds and
        # degrids only the subgrids it owns (no data-path collective)
        from paper_2102_12739_gb300 import shard
        per = 250_000
        owned = shard.partition_subgrids([per] * (64 * world), world)[rank]
        w = synth.lines_workload("%s shard %d/%d" % (WORKLOAD, rank, world), [per] * len(owned),
                                 ids=owned)
    else:
        w = synth.workload(args.workload)
    sub_np = w.subgrids()
    sub = torch.from_numpy(sub_np).to(dev)
    uvw = torch.from_numpy(w.uvw).to(dev)
    offs = torch.from_numpy(w.vis_offsets).to(dev)
    out = torch.empty(w.n_vis, dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    plan = dg.DegridPlan(device=dev)

    def step():
        plan.degrid(sub, uvw, offs, out=out)

    # clocks up first, then the autotuner picks chunk size and warps per CTA
    # on this workload (the footprint-cache arm: dense lines), then timing
    warm_up(torch, step, flush, args.warmup)
    tuned = dg.autotune(plan, sub, uvw, offs, candidates=HEADLINE_CANDIDATES, use_cache=False)
    plan.enable_timing(max(args.steps, args.sweep_steps, 16))
    warm_up(torch, step, flush, args.warmup, min_seconds=0.2)
    assert plan.status() == 0

    sampler = ClockSampler(gpu_query_id(torch, dev)) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    wall0 = time.perf_counter()
    step_ms, kern_ms = time_steps(torch, plan, step, args.steps, flush, stream)
    wall = time.perf_counter() - wall0
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None

    mean_step = sum(step_ms) / len(step_ms)
    mean_kern = sum(kern_ms) / len(kern_ms)
    if world > 1:
        t = torch.tensor([mean_step, mean_kern], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        mean_step, mean_kern = float(t[0]), float(t[1])
    value = world * w.n_vis / (mean_step * 1e-3)

    # end to end through the C-ABI call on HOST buffers (degrid_execute_host),
    # on every rank: the step's inputs cross the host link inside the timing
    e2e = None
    if not args.no_e2e:
        h_sub = torch.empty(sub.shape, dtype=sub.dtype, pin_memory=True)
        h_sub.copy_(torch.from_numpy(sub_np))
        h_uvw = torch.empty(uvw.shape, dtype=uvw.dtype, pin_memory=True)
        h_uvw.copy_(torch.from_numpy(w.uvw))
        h_offs = torch.from_numpy(w.vis_offsets).pin_memory()
        h_out = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)

        def e2e_run():
            ts = []
            for i in range(args.e2e_steps + 2):
                flush.zero_()                   # no host line left in L2 from the last step
                torch.cuda.synchronize()
                if world > 1:
                    torch.distributed.barrier()
                t0 = time.perf_counter()
                plan.degrid_host(h_sub, h_uvw, h_offs, out=h_out)
                if i >= 2:
                    ts.append(time.perf_counter() - t0)
            assert plan.status() == 0
            med = statistics.median(ts)
            if world > 1:                       # the slowest rank sets the job's time
                t = torch.tensor([med], dtype=torch.float64, device=dev)
                torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
                med = float(t[0])
            return world * w.n_vis / med

        # pinned buffers: the kernel reads them in place over the host link
        e2e_value = e2e_run()
        e2e_out = h_out.numpy().copy()
        # the same call made to copy the inputs in subgrid groups instead
        plan.set_host_direct(False)
        h_out.zero_()
        copy_value = e2e_run()
        copy_out = h_out.numpy().copy()
        plan.set_host_direct(True)
        e2e = (h_sub, h_uvw, h_offs, h_out, e2e_value, copy_value, e2e_out, copy_out)

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    out_np = out.cpu().numpy()
    # the FP64 oracle's value of every visibility: the reference of every
    # error below
    ref_all = oracle_reference(w, g_uv, g_w, lambda s: sub_np[s])
    err_c64 = error_vs(out_np, ref_all)

    props = torch.cuda.get_device_properties(dev)
    sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    analytic_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    # the FP32 peak measured on this GPU (FFMA2 and FFMA chain kernels), the higher of the two
    measured_fp32 = {"ffma2": dg.measure_fp32_peak(local, packed=True),
                     "ffma": dg.measure_fp32_peak(local, packed=False)}
    peak_tflops = max(measured_fp32.values())
    achieved = w.n_vis * FLOP_PER_VIS / (mean_kern * 1e-3) / 1e12
    # the other bound of the direct method: compulsory DRAM bytes (coordinates,
    # output, every touched subgrid element once) against the measured copy rate
    import oracle
    touched = int(oracle.touched(w.shape, w.n_subgrids, w.uvw, w.vis_offsets).sum())
    hbm_bytes = w.n_vis * (24 + 8) + touched * 8
    hbm_ms = hbm_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3
    alu_ms = w.n_vis * FLOP_PER_VIS / (peak_tflops * 1e12) * 1e3
    roofline = {"bound": "alu" if alu_ms >= hbm_ms else "hbm", "achieved": achieved,
                "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": measured_traffic(w.n_vis),
                "kernel": "degrid_kernel<DG_C64>",
                "peak_source": "measured: the faster of FFMA2 and FFMA chain kernels filling "
                               "every SM (degrid_measure_fp32_peak), TFLOP/s %s" % (
                                   {k: round(v, 2) for k, v in measured_fp32.items()},),
                "peak_analytic": analytic_tflops,
                "peak_analytic_source": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} "
                                        f"FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                "kernel_ms": mean_kern,
                # the other bound: compulsory DRAM bytes at the measured copy rate
                # over the kernel's time (1.0 = the kernel moves its bytes at that rate)
                "hbm_frac": hbm_ms / mean_kern,
                "bounds_ms": {"alu": alu_ms, "hbm": hbm_ms,
                              "hbm_bytes": hbm_bytes, "hbm_gbs": peaks["hbm_gbs"],
                              "touched_subgrid_elements": touched},
                "warm_kernel_ms": warm_kernel_ms(torch, plan, step, 200)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (WORKLOAD + ": " + WORKLOAD_DESC) if args.workload == WORKLOAD
                   else args.workload, "n_vis": w.n_vis,
                   "subgrid_storage": "complex64",
                   "reduction": "compensated" if plan.compensated else "plain",
                   "l2": "flushed before every step (256 MB write outside the step events)",
                   "parallelism": ("%d GPUs, each degrids its own 64 of %d subgrids (greedy "
                                   "partition by visibility count, no data-path collective)"
                                   % (world, 64 * world)) if world > 1 else "1 GPU",
                   "tuning": plan.tuning(), "autotuned_over": len(tuned["timings"]),
                   "peaks": peaks_src},
        "roofline": roofline,
        # per step: the schedule kernel (two kernels above 4096 subgrids) and the sums
        "gpu_launches": (2 if w.n_subgrids <= 4096 else 3) * args.steps,
        "clocks": clocks,
        "accuracy": {"rel_l2_vs_oracle": err_c64[0], "max_abs_vs_oracle": err_c64[1],
                     "sample": "all", "bound": 2e-6},
        "wall_s_timed_region": wall,
    }

    # the single-GPU diagnostics (storage sweep, other workloads, the CPU
    # oracle) run at N = 1 only: at N > 1 they would hold every GPU meanwhile
    solo = world == 1
    if solo and not args.no_sweep:
        # config 3: each storage type, plain and with the compensated reduction; errors
        # against the FP64 oracle on the original complex64 subgrids (quantisation
        # included) and, for FP16/BF16, on the values the kernel reads (kernel error)
        # every entry, the plain complex64 one included, is timed the same way
        # (its own autotuned plan, sweep_steps L2-flushed steps), so the
        # storage types compare like for like
        sweep = {}
        for dt in ("c64", "f16", "bf16"):
            if dt == "c64":
                codes, scale, ref_q = sub, None, None
            else:
                codes, scale = dg.pack_subgrids(sub, dt)
                import oracle
                qc, qs = oracle.quantize(sub_np, dt)
                # the oracle on the stored (dequantised, exact) values
                ref_q = oracle_reference(w, g_uv, g_w,
                                         lambda s_: oracle.dequantize(qc[s_:s_ + 1], qs[s_:s_ + 1], dt)[0])
                del qc, qs
            for comp in (False, True):
                with dg.DegridPlan(dtype=dt, device=dev, compensated=comp) as p2:
                    # tuned like the headline plan, over the same candidates
                    dg.autotune(p2, codes, uvw, offs, scale=scale, candidates=HEADLINE_CANDIDATES,
                                use_cache=False)
                    p2.enable_timing(args.sweep_steps)
                    o2 = torch.empty_like(out)

                    def step2():
                        p2.degrid(codes, uvw, offs, scale=scale, out=o2)
                    warm_up(torch, step2, flush, args.warmup, min_seconds=0.3)
                    s_ms, k_ms = time_steps(torch, p2, step2, args.sweep_steps, flush, stream)
                    o2_np = o2.cpu().numpy()
                    e = error_vs(o2_np, ref_all)
                    ek = error_vs(o2_np, ref_q) if ref_q is not None else e
                ms = sum(s_ms) / len(s_ms)
                kms = sum(k_ms) / len(k_ms)
                elem = 8 if dt == "c64" else 4
                sweep[dt + ("_compensated" if comp else "")] = {
                    "value": w.n_vis / (ms * 1e-3), "kernel_ms": kms,
                    "rel_l2": e[0], "max_abs": e[1], "rel_l2_vs_stored_values": ek[0],
                    "bound": {"c64": 2e-6, "f16": 1e-3, "bf16": 8e-3}[dt], "error_sample": "all",
                    "compensated": comp,
                    "roofline_frac": w.n_vis * FLOP_PER_VIS / (kms * 1e-3) / 1e12 / peak_tflops,
                    "hbm_bound_ms": (w.n_vis * 32 + touched * elem) / (peaks["hbm_gbs"] * 1e9) * 1e3}
            del codes, scale, ref_q
        line["precision_sweep"] = sweep

    if e2e is not None:
        h_sub, h_uvw, h_offs, h_out, e2e_value, copy_value, e2e_out, copy_out = e2e
        e2e_err = error_vs(e2e_out, ref_all)
        copy_err = error_vs(copy_out, ref_all)
        bi = world * (h_sub.numel() * h_sub.element_size() + h_uvw.numel() * 8 + h_offs.numel() * 8)
        bo = world * h_out.numel() * h_out.element_size()
        line["e2e"] = {"value": e2e_value, "unit": UNIT,
                       "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
                       "rel_l2_vs_oracle": e2e_err[0],
                       "path": "degrid_execute_host on pinned host buffers, read in place: the "
                               "kernel loads the coordinates (%d B) and the footprint rows it "
                               "uses (%d touched elements, %d B of the %d B stack) over the host "
                               "link and stores the visibilities there; the offsets are copied. "
                               "h2d_bytes_per_step counts every input the call is given (all "
                               "ranks); the value is all ranks' visibilities over the slowest "
                               "rank's median step"
                               % (h_uvw.numel() * 8, touched, touched * 8,
                                  h_sub.numel() * h_sub.element_size()),
                       "copy_path": {"value": copy_value, "rel_l2_vs_oracle": copy_err[0],
                                     "path": "the same call copying the inputs: subgrid groups of "
                                             "64 MB copied in, summed and copied out on three "
                                             "overlapping streams"},
                       "l2": "flushed before every step (outside the timing)",
                       "host_link": "about 211 GB/s host to device on this box, for copies "
                                    "and for kernel loads alike"}

    if solo and not args.no_adjoint:
        adj = adjoint_section(torch, dg, synth, dev, flush, args.aux_steps)
        # the same 1024-flop roofline as the degridding kernel (Eq. 1's sum, transposed)
        adj["roofline_frac"] = adj["visibilities"] * FLOP_PER_VIS / (adj["kernel_ms"] * 1e-3) / 1e12 / peak_tflops
        adj["roofline_peak_tflops"] = peak_tflops
        line["adjoint"] = adj

    if solo and not args.no_predict:
        line["predict"] = predict_section(torch, dg, synth, dev, flush, args.aux_steps, peaks["hbm_gbs"],
                                          plan=plan, uvw=uvw, offs=offs)

    if solo:
        line["latency"] = latency_section(torch, dg, synth, dev, args.aux_steps)

    if solo and not args.no_table2d:
        line["table2d"] = table2d_section(torch, dg, synth, dev, flush, args.aux_steps, sub, sub_np,
                                          uvw, offs, w)

    if solo and not args.no_scatter:
        line["scatter"] = scatter_section(torch, dg, synth, dev, flush, args.aux_steps,
                                          dg.measure_l2_read_bw(local))

    if solo and not args.no_batched:
        del sub_np
        line["batched"] = batched_section(torch, dg, synth, dev, flush, args.aux_steps)

    if solo and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g_uv, g_w)

    print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
