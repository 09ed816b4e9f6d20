#!/usr/bin/env python3
"""Benchmark of the multilevel hot path on one B300 (or N replicas).

A step is one multilevel measurement of the 24^3 x 8 FP32 workload (beta 0.98,
slabs of 2, 100 sub-updates, r = 2..12, six field components at offsets
0..8 for every r): k0 = 10 full compound sweeps, 100 slab sub-updates each
followed by the accumulation of T^(2) and TO^(2), and the cross-slab products
(Algorithm 1 of arXiv:1309.3859).  The lattice is thermalised (200 compound
sweeps) before the warm-up steps.

Metric: link updates per second over whole steps (every heatbath and
overrelaxation link update of the step, divided by the step's device time),
with multilevel measurements per second beside it.  The K timed steps are one
call of K measurements (CUDA events around it), so each measurement's
products overlap the next one's sweeps as in any run of measurements; L2 is
flushed (a 512 MB write) before that call, and the slab sums the step streams
through (1.05 GB) are larger than L2.  `isolated_ms_per_step` is one
measurement per call with L2 flushed before each.  With --gpus N > 1 (torchrun) every rank runs
its own lattice (independent Markov chains, weak scaling) and the value is the
sum over ranks divided by the slowest rank's time.

The same JSON line carries the other configured workloads: the 8^3 x 4 FP64
plain multilevel run (its 5 measurements) and one 48^3 x 16 two-level
measurement (20 outer x 200 inner sub-updates) under `configs`, each with its
kernel classes, roofline and the oracle beside it (truncated for 48^3 x 16);
the 64-lattice batch (`batched`); and serving (10 000 seeded requests with
Poisson arrivals at 80% of the measured capacity, p50/p99 latency per lattice
size, `serving`).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (one sub-update per step) on the host cores.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1309_3859_b300 import workloads  # noqa: E402

METRIC = "multilevel link-updates/s"  # with HBM fraction (roofline) and serving p50/p99 beside it
UNIT = "link-updates/s"
L2_FLUSH_BYTES = 512 << 20


def link_updates_per_step(w) -> int:
    """Heatbath + overrelaxation link updates of one measurement step."""
    V = w.V
    sweeps = 1 + w.n_or

    def slab_links(d):  # temporal links always move; spatial ones on t = 0 mod d are frozen
        return V + 3 * V * (d - 1) // d

    n = w.k_between * 4 * V * sweeps
    if w.outer_slab:
        n += w.n_sub_outer * (slab_links(w.outer_slab) + w.n_sub * slab_links(w.slab)) * sweeps
    else:
        n += w.n_sub * slab_links(w.slab) * sweeps
    return n


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- peaks
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ----------------------------------------------------------------------------- CPU baseline
def oracle_sample(w, steps=1, threads=None):
    """Time the FP64 oracle on a bounded sample of the workload: ``steps``
    slab sub-updates with their accumulation and the cross-slab products."""
    import oracle

    threads = threads or os.cpu_count()
    po = oracle.Params(L=w.L, Nt=w.Nt, beta=w.beta, seed=w.seed, n_or=w.n_or, slab=w.slab, n_sub=steps,
                       k_between=0, r=w.r, rf=w.rf, probes=w.probes, comp_mask=w.comp_mask, threads=threads)
    th = oracle.hot_start(po)
    t0 = time.perf_counter()
    oracle.measure(po, th, 0, 1)
    dt = time.perf_counter() - t0
    V = w.V
    updates = steps * (V + 3 * V * (w.slab - 1) // w.slab) * (1 + w.n_or)
    return updates / dt, threads, dt, updates


def cpu_baseline(w):
    rate, cores, dt, updates = oracle_sample(w, steps=6)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"six slab sub-updates (compound sweep + T/TO accumulation + products) of {w.name}: "
                      f"{updates} link updates in {dt:.1f} s, FP64, OpenMP link updates"}


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    rates = []
    for _ in range(args.warmup):
        oracle_sample(w, steps=1)
    t0 = time.perf_counter()
    tot_updates, tot_time, cores = 0, 0.0, None
    for _ in range(args.steps):
        rate, cores, dt, upd = oracle_sample(w, steps=1)
        tot_updates += upd
        tot_time += dt
        rates.append(rate)
    value = tot_updates / tot_time
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_time / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (hot start from the Philox stream)",
            "config": {"workload": w.name, "L": w.L, "Nt": w.Nt, "beta": w.beta, "sample": "1 sub-update per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one slab sub-update with accumulation and products per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def kernel_classes(ml, lat, w, ms_step):
    """Per-launch device time of each kernel class (ml_kernel_timing) and its
    share of a measurement step: the k0 full sweeps run as one launch of
    k_between compound sweeps; a slab sub-update is one launch of the sweep
    kernel with the record fused (the resident kernel runs a ring buffer of
    sub-updates per launch and its folds overlap on the SMs it leaves free, so
    shares can sum past 1)."""
    nB = lat.batch_slots
    n_outer = w.n_sub_outer if w.outer_slab else 1
    per_step = {
        "subupdate": (ml.ML_K_SUBUPDATE, w.n_sub * n_outer),
        "full_sweeps": (ml.ML_K_FULLSWEEP, w.k_between),
        "accumulate": (ml.ML_K_ACCUMULATE, n_outer * -(-w.n_sub // nB)),
        "products": (ml.ML_K_PRODUCTS, 1),
    }
    kms = {name: lat.kernel_ms(kid, reps=20 if name != "products" else 3) for name, (kid, _) in per_step.items()}
    share = {name: kms[name] * per_step[name][1] / ms_step for name in per_step}
    return kms, share


def hbm_roofline(ml, lat, w, kms, share, peak, peak_kind):
    """HBM roofline of the step's dominant kernel class (sub-updates or folds):
    algorithmic bytes per launch over the event-timed launch."""
    nB = lat.batch_slots
    dominant = max(("subupdate", "accumulate"), key=share.get)
    resident = lat.sweep_mode == ml.ML_SWEEP_RESIDENT
    per_launch = nB if (dominant == "subupdate" and resident) else 1  # sub-updates per launch
    nbytes = algorithmic_bytes(w, "sweep" if dominant == "subupdate" else dominant, nB) * per_launch
    launch_ms = kms[dominant] * per_launch
    achieved = nbytes / (launch_ms * 1e-3) / 1e9
    impl = ["k_sweeps_table (persistent, record fused)", "k_pass_table + k_record_table",
            "k_sweeps_resident (cluster-resident slabs, record fused)"][lat.sweep_mode]
    return {"kernel": {"subupdate": impl, "accumulate": "k_accum_T_table + k_accum_O_table"}[dominant],
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_kind, "traffic": None, "algorithmic_bytes_per_launch": nbytes,
            "launch_ms": launch_ms, "sub_updates_per_launch": per_launch, "batch_slots": nB}


def config_point(ml, w, n_meas, warmup, peak, peak_kind):
    """One configured workload: n_meas measurements in one call after warm-up
    (L2 flushed before), link updates/s, measurements/s, kernel classes and
    the roofline of the dominant one."""
    import torch

    p = ml.Params.from_workload(w)
    with ml.Lattice(p) as lat:
        lat.thermalize(w.n_therm)
        rec = torch.empty((n_meas, lat.rec_len), dtype=torch.float64, device=lat.device)
        for _ in range(warmup):
            lat.measure_device(1, rec[:1])
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=lat.device)
        with torch.cuda.stream(lat.stream):
            flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        lat.measure_device(n_meas, rec)
        e1.record(lat.stream)
        lat.sync()
        ms = e0.elapsed_time(e1) / n_meas
        del flush
        kms, share = kernel_classes(ml, lat, w, ms)
        roof = hbm_roofline(ml, lat, w, kms, share, peak, peak_kind)
        mode = ["persistent", "per-pass", "resident"][lat.sweep_mode]
    upd = link_updates_per_step(w)
    return {"workload": w.name, "dtype": "f64" if w.fp64 else "f32 links; f64 slab sums, products, reductions",
            "ms_per_measurement": ms, "measurements_per_s": 1e3 / ms, "link_updates_per_s": upd / (ms * 1e-3),
            "link_updates_per_measurement": upd, "measurements_timed": n_meas, "sweep_impl": mode,
            "kernel_ms": kms, "kernel_share": share, "roofline": roof}


def oracle_small_point(w):
    """The oracle on the whole 8^3 x 4 FP64 workload: thermalisation, then its
    n_meas measurements timed."""
    import oracle

    po = oracle.Params(L=w.L, Nt=w.Nt, beta=w.beta, seed=w.seed, n_or=w.n_or, slab=w.slab, n_sub=w.n_sub,
                       k_between=w.k_between, r=w.r, rf=w.rf, probes=w.probes, comp_mask=w.comp_mask,
                       threads=os.cpu_count())
    th = oracle.hot_start(po)
    c = oracle.thermalize(po, th, 0, w.n_therm)
    t0 = time.perf_counter()
    oracle.measure(po, th, c, w.n_meas)
    dt = time.perf_counter() - t0
    upd = link_updates_per_step(w) * w.n_meas
    return {"kind": "oracle", "cores": os.cpu_count(), "ms_per_measurement": 1e3 * dt / w.n_meas,
            "link_updates_per_s": upd / dt, "sample": f"the whole workload: {w.n_meas} measurements"}


def oracle_large_point(w):
    """The oracle on the 48^3 x 16 two-level workload, truncated: one slab
    sub-update (a compound sweep with the inner mask), extrapolated to a whole
    measurement by its link updates (the oracle's accumulations, whose slab
    sums for this workload's probe set would hold 6.6 GB, are left out, so
    the extrapolation is a lower bound on the oracle's time)."""
    import oracle

    po = oracle.Params(L=w.L, Nt=w.Nt, beta=w.beta, seed=w.seed, n_or=w.n_or, draws=1, slab=w.slab, n_sub=1,
                       k_between=0, r=w.r, threads=os.cpu_count())
    th = oracle.hot_start(po)
    t0 = time.perf_counter()
    oracle.compound_sweep(po, th, 0, w.slab)
    dt = time.perf_counter() - t0
    V = w.V
    upd = (V + 3 * V * (w.slab - 1) // w.slab) * (1 + w.n_or)
    rate = upd / dt
    return {"kind": "oracle", "cores": os.cpu_count(), "link_updates_per_s": rate,
            "ms_per_measurement_extrapolated": 1e3 * link_updates_per_step(w) / rate,
            "sample": f"truncated: one slab sub-update of the 48^3 x 16 lattice ({dt:.1f} s), extrapolated to a "
                      "whole measurement by its link updates, accumulations left out (a lower bound)"}


def pass_bytes(V, mu, d, tsz):
    """Bytes one (mu, parity) pass must move at minimum.

    Without frozen links (d = 0) a pass updates V/2 links: it reads U_mu at
    both parities (V angles; the staples reach the other parity), the three
    other directions everywhere (3V) and writes V/2: 4.5 V angles.  With the
    slab mask d a temporal pass is the same; a spatial pass updates the links
    on d - 1 of every d time slices (V (d - 1) / (2d) of them) and reads U_mu
    everywhere (its staples reach the frozen slices at t +- 1), the other two
    spatial directions on the updated slices only and U_0 at t and t - 1 (all
    slices): 2 V + 2.5 V (d - 1) / d angles (3.25 V for d = 2)."""
    if d == 0 or mu == 0:
        return 4.5 * V * tsz
    if d == 1:
        return 0.0  # every spatial link is frozen: the pass moves nothing
    return (2.0 * V + 2.5 * V * (d - 1) / d) * tsz


def sweep_bytes(V, d, n_or, tsz):
    """Compound sweep: 1 + n_or sweeps of the four directions at both parities."""
    return (1 + n_or) * 2 * sum(pass_bytes(V, mu, d, tsz) for mu in range(4))


def algorithmic_bytes(w, kernel, n_batch=1, d=None):
    """Bytes one launch of a kernel class must move at minimum.

    sweep: the compound sweep's passes (pass_bytes) with the slab mask d
    (default: the workload's inner slab).  fold: every slab accumulator (16
    bytes per complex sum) is read and written once (32 bytes) and every
    record of the batch is read once."""
    tsz = 8 if w.fp64 else 4
    Ns, V = w.L ** 3, w.V
    nslab = w.Nt // w.slab
    nR = len(set(w.r) | set(w.rf))
    nc = bin(w.comp_mask).count("1")
    if kernel == "sweep":
        return int(sweep_bytes(V, w.slab if d is None else d, w.n_or, tsz))
    if kernel == "accumulate":
        acc_o = nslab * len(w.rf) * len(w.probes) * nc * 2 * Ns
        acc_t = nslab * nR * Ns
        records = n_batch * nslab * Ns * (1 + nc * 2) * tsz
        return 32 * (acc_o + acc_t) + records
    raise ValueError(kernel)


# Warp instructions per link update of the global-memory pass kernel
# (k_update_pass_pair<float, KIND>, ncu on a 64^4 FP32 lattice): heatbath 622
# and overrelaxation 233 per 32 links.  The cluster-resident kernel runs the
# same link update on shared memory; these counts give its issue bound.
INSTR_PER_LINK = {"heatbath": 622 / 32, "overrelax": 233 / 32}


def l2_note(w):
    """How the timed steps treat L2: flushed before the timed call, and
    whether the step's slab sums (16 bytes per complex value) exceed L2."""
    nslab, Ns, nc = w.Nt // w.slab, w.L ** 3, 6
    sums = 16 * nslab * Ns * (len(w.r) + len(w.rf) * len(w.probes) * nc * 2)
    size = f"{sums / 1e9:.2f} GB" if sums >= 1e8 else f"{sums / 1e6:.1f} MB"
    rel = "larger than L2" if sums > 126e6 else "within L2; the flush makes each timed call start cold"
    return (f"flushed ({L2_FLUSH_BYTES >> 20} MB write) before the timed call of K measurements; the step's "
            f"slab sums ({size}) are {rel}")


def issue_roofline(w, launch_ms, sub_updates, sms, sm_mhz):
    """Issue bound of the cluster-resident sub-updates: warp instructions of
    the launch's link updates over (SMs x 4 schedulers x clock)."""
    V, d = w.V, w.slab
    links = V + 3 * V * (d - 1) // d  # per sweep: temporal links all, spatial on d - 1 of d slices
    instr = sub_updates * links * (INSTR_PER_LINK["heatbath"] + w.n_or * INSTR_PER_LINK["overrelax"])
    bound_ms = instr / (sms * 4 * sm_mhz * 1e6) * 1e3
    return {"bound": "issue", "kernel": "k_sweeps_resident", "warp_instructions_per_launch": instr,
            "instr_per_link": INSTR_PER_LINK, "sms": sms, "sm_mhz": sm_mhz, "issue_bound_ms": bound_ms,
            "launch_ms": launch_ms, "frac": bound_ms / launch_ms,
            "source": "instruction counts of k_update_pass_pair<float> (ncu, 64^4 FP32); SMs = 16-CTA clusters x slabs"}


def _timed_passes(ml, lat, mu, kind, reps=10):
    """Average event time of `reps` unmasked (mu, even) passes through
    ml_update_pass (one kernel launch each)."""
    import torch

    lat.update_pass(mu, 0, 0, 10 ** 6, kind)
    lat.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    for i in range(reps):
        lat.update_pass(mu, 0, 0, 10 ** 6 + i, kind)
    e1.record(lat.stream)
    lat.sync()
    return e0.elapsed_time(e1) / reps


def hbm_sweep_point(ml, peak):
    """A 64^4 FP32 lattice (268 MB of angles, beyond L2): the compound sweep
    without frozen links (as in thermalisation), its heatbath and
    overrelaxation passes separately, and the slab-masked sweep with the bytes
    its passes need (pass_bytes)."""
    p = ml.Params(L=64, Nt=64, beta=0.98, seed=5, fp64=False, slab=2, n_sub=1, r=(1,))
    with ml.Lattice(p) as lat:
        lat.thermalize(2)
        ms_full = lat.kernel_ms(ml.ML_K_FULLSWEEP, reps=5)
        ms_masked = lat.kernel_ms(ml.ML_K_SWEEP, reps=5)
        passes = {(kind, mu): _timed_passes(ml, lat, mu, kind) for kind in (0, 1) for mu in (0, 1)}
    V = p.V
    full_bytes = sweep_bytes(V, 0, 3, 4)
    masked_bytes = sweep_bytes(V, 2, 3, 4)
    pb = pass_bytes(V, 0, 0, 4)
    gbs = lambda nbytes, ms: nbytes / (ms * 1e-3) / 1e9  # noqa: E731
    out = {"workload": "sweep-64x64x64x64-fp32", "angle_bytes": 16 * V,
           "full_sweep_ms": ms_full, "full_sweep_link_updates_per_s": 16 * V / (ms_full * 1e-3),
           "sweep_achieved_gbs": gbs(full_bytes, ms_full), "sweep_frac": gbs(full_bytes, ms_full) / peak,
           "masked_sweep_ms": ms_masked, "masked_sweep_gbs": gbs(masked_bytes, ms_masked),
           "masked_sweep_frac": gbs(masked_bytes, ms_masked) / peak,
           "note": "sweep_frac: unmasked compound sweep (1 heatbath + 3 overrelaxation sweeps), 4.5 V angles per "
                   "pass; masked: slab mask 2, spatial passes charged 3.25 V"}
    for (kind, mu), ms in passes.items():
        name = ("hb" if kind == 0 else "or") + f"_pass_mu{mu}"
        out[name + "_ms"] = ms
        out[name + "_frac"] = gbs(pb, ms) / peak
    return out


def batch_params(ml, n=64):
    """The batched workload: 64 lattices, L from {12,16,20,24}, N_t from
    {4,...,12}, beta in [0.94, 0.99], FP32, slabs of 2, 50 sub-updates,
    P(r) r = 1..L/2, E_x on the mid-plane at r = L/4, offsets 0..L/4."""
    out = []
    for (L, Nt, beta, seed) in workloads.batch_mix(n):
        out.append(ml.Params(L=L, Nt=Nt, beta=beta, seed=seed, fp64=False, slab=2, n_sub=50, k_between=10,
                             r=tuple(range(1, L // 2 + 1)), rf=(L // 4,),
                             probes=tuple((d, 0) for d in range(L // 4 + 1)), comp_mask=workloads.COMP_EX))
    return out


def batched_point(ml, steps=3, warmup=1):
    """The 64-lattice batch in the autotuned sweep implementation, and each
    implementation forced (the same chains: the implementations are
    bit-identical), ms per measurement of every lattice."""
    import torch

    ps = batch_params(ml)
    names = ["persistent", "per-pass", "resident"]
    forced = {}
    with ml.Batch(ps) as b:
        b.thermalize(200)
        auto = b.sweep_mode

        def timed():
            for _ in range(warmup):
                b.measure_device(1)
            b.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            for _ in range(steps):
                b.measure_device(1)
            e1.record(b.stream)
            b.sync()
            return e0.elapsed_time(e1) / steps

        ms = timed()
        for mode in (ml.ML_SWEEP_PERSISTENT, ml.ML_SWEEP_PASSES, ml.ML_SWEEP_RESIDENT):
            try:
                b.sweep_mode = mode
            except ml.MLError:
                continue
            forced[names[mode]] = timed()
        b.sweep_mode = auto
    upd = 0
    for p in ps:
        V = p.L ** 3 * p.Nt
        upd += (p.k_between * 4 * V + p.n_sub * (V + 3 * V * (p.slab - 1) // p.slab)) * (1 + p.n_or)
    return {"workload": "batched-64-lattices-fp32", "lattices": len(ps), "ms_per_step": ms,
            "link_updates_per_s": upd / (ms * 1e-3), "measurements_per_s": len(ps) / (ms * 1e-3),
            "sweep_impl": names[auto], "ms_per_step_by_impl": forced,
            "step": "one measurement of every lattice"}


def step_breakdown(ml, w, n_meas=20):
    """Where the step goes, from the public API: streamed ms per measurement
    of the workload, without the k0 sweeps, without the field insertions
    (no rf, probes or components), and without both."""
    import torch

    variants = {"step": {}, "no_k0": dict(k_between=0), "no_field": dict(rf=(), probes=(), comp_mask=0),
                "no_k0_no_field": dict(k_between=0, rf=(), probes=(), comp_mask=0)}
    out = {}
    for name, kw in variants.items():
        p = ml.Params.from_workload(w, **kw)
        with ml.Lattice(p) as lat:
            lat.thermalize(50)
            recs = torch.empty((n_meas, lat.rec_len), dtype=torch.float64, device=lat.device)
            lat.measure_device(3, recs[:3])
            lat.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(lat.stream)
            lat.measure_device(n_meas, recs)
            e1.record(lat.stream)
            lat.sync()
            out[name + "_ms"] = e0.elapsed_time(e1) / n_meas
    out["k0_sweeps_ms"] = out["step_ms"] - out["no_k0_ms"]
    out["field_insertions_ms"] = out["step_ms"] - out["no_field_ms"]
    out["note"] = "streamed measurements (one call of 20); differences of whole steps, so overlap is accounted"
    return out


def serving_request(ml, L, Nt, beta, seed):
    """One serving request: thermalise 100 sweeps, one measurement of 50 slab
    sub-updates, P(r) r = 1..L/2, E_x at r = L/4 over offsets 0..L/4."""
    return ml.Params(L=L, Nt=Nt, beta=beta, seed=seed, fp64=False, slab=2, n_sub=50, k_between=0,
                     r=tuple(range(1, L // 2 + 1)), rf=(max(1, L // 4),),
                     probes=tuple((d, 0) for d in range(L // 4 + 1)), comp_mask=workloads.COMP_EX)


def serving_point(ml, n_requests=1000, load=0.8, budget_gb=160):
    """Poisson arrivals at `load` x the measured capacity; latency per size class."""
    with ml.Server(budget_bytes=int(budget_gb) << 30, fp64=False) as srv:
        # capacity: a burst of requests submitted at once
        cal = workloads.request_stream(200, 1.0, seed=11)
        t0 = time.perf_counter()
        jobs = [srv.submit(serving_request(ml, L, Nt, beta, 10 ** 6 + sd), 100, 1) for (_, L, Nt, beta, sd) in cal]
        for j in jobs:
            srv.wait(j, 600)
        capacity = len(jobs) / (time.perf_counter() - t0)
        for j in jobs:
            srv.release(j)
        rate = load * capacity
        stream = workloads.request_stream(n_requests, rate, seed=7)
        start = time.perf_counter()
        sub = []
        for (t_arr, L, Nt, beta, sd) in stream:
            delay = start + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            sub.append((srv.submit(serving_request(ml, L, Nt, beta, sd), 100, 1), L, Nt))
        lat, by_L, upd = [], {}, 0
        for (j, L, Nt) in sub:
            srv.wait(j, 600)
            t_s, t_a, t_d = srv.times(j)
            lat.append(t_d - t_s)
            by_L.setdefault(L, []).append(t_d - t_s)
            V = L ** 3 * Nt
            upd += (100 * 4 * V + 50 * (V + 3 * V // 2)) * 4
        span = time.perf_counter() - start
        stats = srv.stats()
    q = lambda a, f: float(np.percentile(np.asarray(a), f))  # noqa: E731
    return {"workload": "serving-poisson-fp32", "requests": n_requests, "load": load,
            "capacity_req_per_s": capacity, "arrival_rate_per_s": rate, "throughput_req_per_s": n_requests / span,
            "link_updates_per_s": upd / span, "latency_s": {"p50": q(lat, 50), "p99": q(lat, 99)},
            "latency_by_L_s": {str(L): {"n": len(v), "p50": q(v, 50), "p99": q(v, 99)} for L, v in sorted(by_L.items())},
            # link updates x 36 B (the unmasked per-pass bytes of an FP32 update): an upper bound on the sweeps'
            # algorithmic traffic, as a fraction of the measured HBM bandwidth
            "sweep_gbs_at_36B": 36 * upd / span / 1e9, "sweep_frac_at_36B": 36 * upd / span / 1e9 / measured_peaks()[0],
            "budget_gb": budget_gb, "ticks": stats["ticks"], "lanes": 3,
            "request": "100 thermalisation sweeps + 1 measurement (50 sub-updates), L in 12..32, Nt in 4..12"}


def multihit_point(ml, w, n_meas=40):
    """The step's workload with Section II.C's analytic multihit for P(r)
    against the plain estimator on the same chain (same seed): time per step
    and the jackknife error of every P(r) entry, so the error reduction per
    unit of device time can be read off."""
    import torch

    from paper_1309_3859_b300.stats import jackknife

    out = {"workload": w.name + "-multihit", "measurements": n_meas}
    errs = {}
    for mh in (0, 1):
        p = ml.Params.from_workload(w, seed=w.seed + 7, multihit=mh)
        with ml.Lattice(p) as lat:
            lat.thermalize(w.n_therm)
            rec = torch.empty((n_meas, lat.rec_len), dtype=torch.float64, device=lat.device)
            lat.measure_device(1, rec[:1])
            lat.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(lat.stream)
            lat.measure_device(n_meas, rec)
            e1.record(lat.stream)
            lat.sync()
            ms = e0.elapsed_time(e1) / n_meas
            P = ml.split_record(p, rec.cpu().numpy())["P"][:, :, 0]
        errs[mh] = np.array([jackknife(P[:, a])[1] for a in range(P.shape[1])])
        out["ms_per_step" if mh else "plain_ms_per_step"] = ms
    ratio = errs[0] / errs[1]
    out["error_ratio_plain_over_multihit"] = {f"r={r}": float(x) for r, x in zip(w.r, ratio)}
    # (error ratio)^2 x (time ratio): measurements needed for equal error, per unit time
    out["efficiency_gain_median"] = float(np.median(ratio ** 2) * out["plain_ms_per_step"] / out["ms_per_step"])
    return out


def fp64_point(ml, w, steps=3):
    """The same workload on the FP64 GPU path (FP64 angles, update arithmetic
    and slab sums): measurements/s of the single-lattice FP64 path against
    which the FP32 path is compared."""
    import torch

    p = ml.Params.from_workload(w, fp64=True)
    with ml.Lattice(p) as lat:
        lat.thermalize(w.n_therm)
        rec = torch.empty((1, lat.rec_len), dtype=torch.float64, device=lat.device)
        lat.measure_device(1, rec)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        for _ in range(steps):
            lat.measure_device(1, rec)
        e1.record(lat.stream)
        lat.sync()
        ms = e0.elapsed_time(e1) / steps
        mode = ["persistent", "per-pass", "resident"][lat.sweep_mode]
    return {"workload": w.name.replace("fp32", "fp64"), "ms_per_step": ms,
            "measurements_per_s": 1e3 / ms, "link_updates_per_s": link_updates_per_step(w) / (ms * 1e-3),
            "sweep_impl": mode}


def pair_sums_point(ml, w, steps=5):
    """The step's workload with float-pair slab sums (ml_params.pair_sums = 1)
    instead of double-precision ones, on the same chain: the device-time cost
    of keeping the slab sums in FP64 on this GPU's double-precision pipe."""
    import torch

    p = ml.Params.from_workload(w, pair_sums=1)
    with ml.Lattice(p) as lat:
        lat.thermalize(w.n_therm)
        rec = torch.empty((1, lat.rec_len), dtype=torch.float64, device=lat.device)
        for _ in range(2):
            lat.measure_device(1, rec)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        for _ in range(steps):
            lat.measure_device(1, rec)
        e1.record(lat.stream)
        lat.sync()
        ms = e0.elapsed_time(e1) / steps
        fold_ms = lat.kernel_ms(ml.ML_K_ACCUMULATE, reps=20)
        prod_ms = lat.kernel_ms(ml.ML_K_PRODUCTS, reps=3)
    return {"workload": w.name + "-pair-sums", "ms_per_step": ms, "fold_ms": fold_ms, "products_ms": prod_ms,
            "link_updates_per_s": link_updates_per_step(w) / (ms * 1e-3),
            "slab_sums": "float pairs (about 47 bits), products and reductions in double"}


def replay_point(ml, w, steps=3):
    """The step's workload with the field insertions by replay: the inner
    loop runs twice, and no per-site insertion sums are kept."""
    import torch

    p = ml.Params.from_workload(w, seed=w.seed + 11, replay=1)
    with ml.Lattice(p) as lat:
        lat.thermalize(w.n_therm)
        rec = torch.empty((1, lat.rec_len), dtype=torch.float64, device=lat.device)
        lat.measure_device(1, rec)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        for _ in range(steps):
            lat.measure_device(1, rec)
        e1.record(lat.stream)
        lat.sync()
        ms = e0.elapsed_time(e1) / steps
    nslab = w.Nt // w.slab
    direct_bytes = nslab * len(w.rf) * len(w.probes) * bin(w.comp_mask).count("1") * 2 * w.L ** 3 * 16
    upd = link_updates_per_step(w)
    return {"workload": w.name + "-replay", "ms_per_step": ms, "link_updates_per_s": upd / (ms * 1e-3),
            "insertion_sums_bytes_direct": direct_bytes, "insertion_sums_bytes_replay": 0,
            "note": "link updates of the chain; the replay executes the inner loop's updates twice"}


def run_gpu(args, w, rank, world):
    import torch

    from paper_1309_3859_b300 import ml

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl")

    p = ml.Params.from_workload(w, seed=w.seed + 1000 * rank)
    lat = ml.Lattice(p)
    if args.sweep_mode == "resident":  # full sweeps in the persistent kernel
        lat.sweep_mode = SWEEP_MODES["persistent"]
    if args.sweep_mode != "auto":
        lat.sweep_mode = SWEEP_MODES[args.sweep_mode]
    st = lat.stream
    lat.thermalize(w.n_therm)
    rec = torch.empty((1, lat.rec_len), dtype=torch.float64, device=lat.device)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=lat.device)
    for _ in range(args.warmup):
        lat.measure_device(1, rec)
    lat.sync()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # The K timed steps run as one call of K measurements, as a run of
    # measurements streams on the device: each measurement's products (on the
    # accumulation stream) overlap the next one's sweeps.  L2 is flushed
    # before the call; the step's working set (the slab sums, about 1 GB at
    # 24^3 x 8) is larger than L2.  With --profile each step is one call
    # bracketed for the profiler.
    recs = torch.empty((args.steps, lat.rec_len), dtype=torch.float64, device=lat.device)
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    launches0 = ml.kernel_launches()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_wall0 = time.perf_counter()
        with torch.cuda.stream(st):
            flush.fill_(0.0)
        if args.profile:
            e_start.record(st)
            for k in range(args.steps):
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStart()
                lat.measure_device(1, recs[k:k + 1])
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStop()
            e_end.record(st)
        else:
            e_start.record(st)
            lat.measure_device(args.steps, recs)
            e_end.record(st)
        lat.sync()
        barrier()
        t_wall = time.perf_counter() - t_wall0
    launches = ml.kernel_launches() - launches0
    ms = e_start.elapsed_time(e_end)
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=lat.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    upd = link_updates_per_step(w)
    value = world * upd * args.steps / (ms * 1e-3)

    # one measurement per call, L2 flushed before each (nothing overlaps the
    # products): reported beside the streamed step time
    iso = []
    for k in range(3):
        with torch.cuda.stream(st):
            flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lat.measure_device(1, rec)
        e1.record(st)
        lat.sync()
        iso.append(e0.elapsed_time(e1))
    kms, share = kernel_classes(ml, lat, w, ms / args.steps)
    peak, peak_kind = measured_peaks()
    roof = hbm_roofline(ml, lat, w, kms, share, peak, peak_kind)
    hbm_point = hbm_sweep_point(ml, peak) if rank == 0 and not args.no_extra else None
    batch_point = batched_point(ml) if rank == 0 and not args.no_extra else None
    mh_point = multihit_point(ml, w) if rank == 0 and not args.no_extra else None
    rp_point = replay_point(ml, w) if rank == 0 and not args.no_extra and not w.outer_slab else None
    f64_point = fp64_point(ml, w) if rank == 0 and not args.no_extra and not w.fp64 else None
    pair_point = pair_sums_point(ml, w) if rank == 0 and not args.no_extra and not w.fp64 else None
    breakdown = step_breakdown(ml, w) if rank == 0 and not args.no_extra else None
    tl = step_timeline(ml, lat, w) if rank == 0 and not args.no_extra else None
    rprof = resident_profile_point(ml, lat, w) if rank == 0 and not args.no_extra else None

    # end to end through the public API with host buffers: upload this
    # step's configuration from pinned memory, measure, read the record
    theta_host = torch.from_numpy(lat.get_angles()).pin_memory()
    out_host = np.zeros((1, lat.rec_len))
    e2e_steps = max(1, min(args.steps, 5))
    lat.set_angles(theta_host.numpy())
    lat.measure(1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.set_angles(theta_host.numpy())
        out_host[:] = lat.measure(1)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * upd * e2e_steps / e2e_s

    clocks = clk.summary()
    roof_issue = None
    if lat.sweep_mode == ml.ML_SWEEP_RESIDENT and clocks["sm_mhz"]:
        nslab = w.Nt // w.slab
        roof_issue = issue_roofline(w, kms["subupdate"] * lat.batch_slots, lat.batch_slots, 16 * nslab,
                                    clocks["sm_mhz"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)
    # the other configured workloads: 8^3 x 4 FP64 plain multilevel and the
    # 48^3 x 16 two-level measurement, each with the oracle beside it
    configs = None
    if rank == 0 and not args.no_configs:
        small = config_point(ml, workloads.SMALL_FP64, workloads.SMALL_FP64.n_meas, 1, peak, peak_kind)
        large = config_point(ml, workloads.LARGE_48, 1, 1, peak, peak_kind)
        large["fold_share"] = large["kernel_share"]["accumulate"]
        if world == 1 and not args.no_cpu_baseline:
            small["oracle"] = oracle_small_point(workloads.SMALL_FP64)
            large["oracle"] = oracle_large_point(workloads.LARGE_48)
        configs = {"plain-8x8x8x4-fp64": small, "two-level-48x48x48x16-fp32": large}
    serving = None
    if rank == 0 and args.serving_requests > 0:
        serving = serving_point(ml, n_requests=args.serving_requests)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if w.fp64 else "f32 links and update; f64 slab sums, averages, products and reductions",
        "data": "synthetic (hot start from the Philox stream, thermalised)",
        "config": {"workload": w.name, "L": w.L, "Nt": w.Nt, "beta": w.beta, "n_sub": w.n_sub,
                   "k_between": w.k_between, "n_or": w.n_or, "r": f"{w.r[0]}..{w.r[-1]}",
                   "field_r": f"{w.rf[0]}..{w.rf[-1]}", "probes": len(w.probes), "components": 6,
                   "link_updates_per_step": upd,
                   "l2": l2_note(w),
                   "parallelism": f"{world} independent lattice(s)"},
        "measurements_per_s": world * args.steps / (ms * 1e-3),
        "isolated_ms_per_step": float(np.median(iso)),
        "roofline": roof,
        "roofline_issue": roof_issue,
        "kernel_ms": kms, "kernel_share": share,
        "sweep_hbm_point": hbm_point,
        "batched": batch_point,
        "multihit": mh_point,
        "replay": rp_point,
        "fp64_path": f64_point,
        "pair_sums": pair_point,
        "step_breakdown": breakdown,
        "timeline": tl,
        "resident_profile": rprof,
        "vs_fp64_path": (f64_point["ms_per_step"] / (ms / args.steps)) if f64_point else None,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(theta_host.numel() * 8),
                "d2h_bytes_per_step": int(lat.rec_len * 8), "steps": e2e_steps},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "configs": configs,
        "serving": serving,
        "wall_s": t_wall,
    }
    lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


SWEEP_MODES = {"persistent": 0, "passes": 1, "resident": 2}


def resident_profile_point(ml, lat, w):
    """Where one cluster-resident launch spends its time (ml_resident_profile:
    SM clock cycles per phase, thread 0 of each CTA), in microseconds at the
    GPU's maximum SM clock (the bench's clock samples show it is held), and
    each phase's share of a sub-update."""
    if lat.sweep_mode != ml.ML_SWEEP_RESIDENT:
        return None
    pr = lat.resident_profile()
    mhz = 2032.0
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=10).stdout.split()
        mhz = float(out[0])
    except Exception:  # noqa: BLE001 - the bench also runs where nvidia-smi is absent
        pass
    us = {k: v / mhz for k, v in pr.items() if k not in ("sub_updates", "ctas")}
    n_or = w.n_or
    counts = {"heatbath_t": 2, "heatbath_s": 6, "overrelax_t": 2 * n_or, "overrelax_s": 6 * n_or}
    per_sub = {"update": sum(counts[c] * us["update_" + c] for c in counts),
               "exchange": sum(counts[c] * us["exchange_" + c] for c in counts), "record": us["record"]}
    total = sum(per_sub.values())
    return {"us_per_pass": {k: round(v, 3) for k, v in us.items() if k.startswith(("update_", "exchange_"))},
            "us_per_sub_update": {k: round(v, 2) for k, v in per_sub.items()},
            "share_of_sub_update": {k: round(v / total, 3) for k, v in per_sub.items()},
            "launch_us": round(us["launch"], 1), "setup_us": round(us["setup"], 1),
            "write_back_us": round(us["write_back"], 1), "sub_updates_per_launch": pr["sub_updates"],
            "sm_mhz_assumed": mhz,
            "note": "timed variant of the launch (thread 0 of each CTA reads the SM clock; a block barrier splits "
                    "each pass into own updates and exchange); pass classes: heatbath/overrelaxation, t = temporal "
                    "links (both slices), s = spatial links (inner slice)"}


def step_timeline(ml, lat, w, n_meas=4):
    """Launch timeline of n_meas streamed measurements (ml_timeline_read):
    mean durations of the full sweeps, the sub-update groups (a whole ring
    buffer), the folds and the products, and how much of the span the main
    stream's work covers (the step's critical path: full sweeps, then
    sub-updates)."""
    import torch

    rec = torch.empty((n_meas, lat.rec_len), dtype=torch.float64, device=lat.device)
    lat.timeline_enable(64 * n_meas)
    lat.measure_device(n_meas, rec)
    marks = lat.timeline()
    lat.timeline_enable(0)
    spans = {}
    open_at = {}
    for tag, ms in marks:
        kind, end = tag // 2, tag % 2
        if not end:
            open_at[kind] = ms
        elif kind in open_at:
            spans.setdefault(kind, []).append(ms - open_at.pop(kind))
    names = {0: "full_sweeps", 1: "sub_update_group", 2: "fold", 3: "products"}
    main = [ms for tag, ms in marks if tag // 2 in (0, 1)]
    span = main[-1] - main[0] if len(main) > 1 else 0.0
    busy = sum(spans.get(0, [])) + sum(spans.get(1, []))
    nB = lat.batch_slots
    full_groups = [d for i, d in enumerate(spans.get(1, [])) if (i + 1) % -(-w.n_sub // nB) != 0]
    return {"measurements": n_meas, "ms_per_measurement": span / n_meas if n_meas else None,
            **{names[k] + "_ms": float(np.mean(v)) for k, v in spans.items()},
            "full_ring_group_ms": float(np.mean(full_groups)) if full_groups else None,
            "sub_updates_per_group": nB, "main_stream_busy_frac": busy / span if span else None,
            "note": "CUDA events around each launch group (ml_timeline_read); main stream: full sweeps and "
                    "sub-update groups back to back; accumulation stream: folds and products beside them"}


def fold_case(impl, reps=3):
    """The fold of the two-level 48^3 workload's field insertions (probes at y
    offsets 0..12, six components) on a 48^3 x 8 lattice with one field
    separation: the same blocks and tiles as the 48^3 x 16 workload with 1.1
    GB of slab sums instead of 6.6 GB.  Prints one JSON line."""
    from paper_1309_3859_b300 import ml

    w = workloads.LARGE_48
    p = ml.Params(L=w.L, Nt=8, beta=w.beta, seed=w.seed, fp64=False, slab=w.slab, n_sub=32, k_between=1, r=(2, 4),
                  rf=(16,), probes=w.probes, comp_mask=w.comp_mask)
    with ml.Lattice(p) as lat:
        lat.thermalize(1)
        lat.fold_mode = ml.ML_FOLD_TILE if impl == "tile" else ml.ML_FOLD_SITE
        nslab, nrf, nq = p.Nt // p.slab, 1, 2 * bin(w.comp_mask).count("1")
        print(json.dumps({"workload": "fold-48x48x48x8-fp32", "fold": impl,
                          "slab_sum_bytes": nslab * nrf * len(w.probes) * nq * w.L ** 3 * 16,
                          "fold_ms": lat.kernel_ms(ml.ML_K_ACCUMULATE, reps=reps)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=workloads.SINGLE_24.name, choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 64^4 HBM sweep point and the batch")
    ap.add_argument("--profile", action="store_true",
                    help="bracket the first timed step with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--sweep-mode", default="auto", choices=["auto", "persistent", "passes", "resident"],
                    help="force the single lattice's sweep implementation (default: autotuned; resident: "
                         "sub-updates cluster-resident, full sweeps persistent)")
    ap.add_argument("--serving-requests", type=int, default=10000,
                    help="requests of the serving measurement (0 skips it)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 8^3 x 4 FP64 and 48^3 x 16 two-level workloads")
    ap.add_argument("--fold-case", choices=["tile", "site"],
                    help="only time the fold of the two-level workload's probes on a 48^3 x 8 lattice (one "
                         "field separation, 1.1 GB of sums) in the given implementation, and exit; a small case "
                         "for profiling the 48^3 folds")
    args = ap.parse_args()
    if args.fold_case:
        return fold_case(args.fold_case)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    w = workloads.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, rank, world)
    return run_gpu(args, w, rank, world)


if __name__ == "__main__":
    sys.exit(main())
