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
with multilevel measurements per second beside it.  L2 is flushed (a 512 MB
write) before every timed step.  With --gpus N > 1 (torchrun) every rank runs
its own lattice (independent Markov chains, weak scaling) and the value is the
sum over ranks divided by the slowest rank's time.

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
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
def algorithmic_bytes(w, kernel, n_batch=1):
    """Bytes one launch of a kernel class must move at minimum.

    update pass: a (mu, parity) pass reads U_mu at both parities (V angles),
    the other three directions everywhere (3V) and writes V/2: 4.5 V angles;
    the persistent kernel runs 4 (1 + n_or) ... = 8 (1 + n_or) passes per
    compound sweep.  fold: every slab accumulator (16 bytes per complex sum:
    two doubles, or two float pairs) is read and written once (32 bytes) and
    every record of the batch is read once."""
    tsz = 8 if w.fp64 else 4
    Ns, V = w.L ** 3, w.V
    nslab = w.Nt // w.slab
    nR = len(set(w.r) | set(w.rf))
    nc = bin(w.comp_mask).count("1")
    if kernel == "pass":
        return int(4.5 * V * tsz)
    if kernel == "sweep":
        return int(8 * (1 + w.n_or) * 4.5 * V * tsz)
    if kernel == "accumulate":
        acc_o = nslab * len(w.rf) * len(w.probes) * nc * 2 * Ns
        acc_t = nslab * nR * Ns
        records = n_batch * nslab * Ns * (1 + nc * 2) * tsz
        return 32 * (acc_o + acc_t) + records
    raise ValueError(kernel)


def hbm_sweep_point(ml, peak):
    """Persistent compound sweep on a 64^4 FP32 lattice (268 MB of angles,
    beyond L2): link updates/s and effective bandwidth against HBM."""
    p = ml.Params(L=64, Nt=64, beta=0.98, seed=5, fp64=False, slab=2, n_sub=1, r=(1,))
    with ml.Lattice(p) as lat:
        lat.thermalize(2)
        ms_sweep = lat.kernel_ms(ml.ML_K_SWEEP, reps=5)
        ms_or = lat.kernel_ms(ml.ML_K_OVERRELAX, reps=10)
        ms_hb = lat.kernel_ms(ml.ML_K_HEATBATH, reps=10)
    V = p.V
    # slab mask 2: temporal links all move, spatial links on half the slices
    moved = (V + 3 * V // 2) * 4
    pass_bytes = 4.5 * V * 4
    return {"workload": "sweep-64x64x64x64-fp32", "angle_bytes": 16 * V,
            "compound_sweep_ms": ms_sweep, "link_updates_per_s": moved / (ms_sweep * 1e-3),
            "sweep_achieved_gbs": 32 * pass_bytes / (ms_sweep * 1e-3) / 1e9,
            "sweep_frac": 32 * pass_bytes / (ms_sweep * 1e-3) / 1e9 / peak,
            "or_pass_ms": ms_or, "or_pass_gbs": pass_bytes / (ms_or * 1e-3) / 1e9,
            "hb_pass_ms": ms_hb, "hb_pass_gbs": pass_bytes / (ms_hb * 1e-3) / 1e9}


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
    import torch

    ps = batch_params(ml)
    with ml.Batch(ps) as b:
        b.thermalize(200)
        for _ in range(warmup):
            b.measure_device(1)
        b.sync()
        st = b.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            b.measure_device(1)
        e1.record(st)
        b.sync()
        ms = e0.elapsed_time(e1) / steps
        mode = b.sweep_mode
    upd = 0
    for p in ps:
        V = p.L ** 3 * p.Nt
        upd += (p.k_between * 4 * V + p.n_sub * (V + 3 * V * (p.slab - 1) // p.slab)) * (1 + p.n_or)
    return {"workload": "batched-64-lattices-fp32", "lattices": len(ps), "ms_per_step": ms,
            "link_updates_per_s": upd / (ms * 1e-3), "measurements_per_s": len(ps) / (ms * 1e-3),
            "sweep_impl": ["persistent", "per-pass", "resident"][mode], "step": "one measurement of every lattice"}


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
            "budget_gb": budget_gb, "ticks": stats["ticks"],
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

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    launches0 = ml.kernel_launches()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(st):
                flush.fill_(float(k))
            if args.profile and k == 0:
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStart()
            starts[k].record(st)
            lat.measure_device(1, rec)
            ends[k].record(st)
            if args.profile and k == 0:
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStop()
        lat.sync()
        barrier()
        t_wall = time.perf_counter() - t_wall0
    launches = ml.kernel_launches() - launches0
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=lat.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    upd = link_updates_per_step(w)
    value = world * upd * args.steps / (ms * 1e-3)

    # kernel classes: per-launch device time and launches per step
    nB = lat.batch_slots
    n_folds = -(-w.n_sub // nB)
    # the k0 full sweeps run as one launch of k_between compound sweeps; a
    # slab sub-update is one launch of the sweep kernel with the record fused
    # (the resident kernel runs a ring buffer of nB sub-updates per launch and
    # its folds overlap on the SMs it leaves free, so shares can sum past 1)
    per_step = {
        "subupdate": (ml.ML_K_SUBUPDATE, w.n_sub),
        "full_sweeps": (ml.ML_K_FULLSWEEP, w.k_between),
        "accumulate": (ml.ML_K_ACCUMULATE, n_folds),
        "products": (ml.ML_K_PRODUCTS, 1),
    }
    kms = {name: lat.kernel_ms(kid, reps=20 if name != "products" else 3) for name, (kid, _) in per_step.items()}
    share = {name: kms[name] * per_step[name][1] / (ms / args.steps) for name in per_step}
    dominant = max(("subupdate", "accumulate"), key=share.get)
    peak, peak_kind = measured_peaks()
    resident = lat.sweep_mode == ml.ML_SWEEP_RESIDENT
    per_launch = nB if (dominant == "subupdate" and resident) else 1  # sub-updates per launch
    nbytes = algorithmic_bytes(w, "sweep" if dominant == "subupdate" else dominant, nB) * per_launch
    launch_ms = kms[dominant] * per_launch
    achieved = nbytes / (launch_ms * 1e-3) / 1e9
    impl = ["k_sweeps_table (persistent, record fused)", "k_pass_table + k_record_table",
            "k_sweeps_resident (cluster-resident slabs, record fused)"][lat.sweep_mode]
    roof = {"kernel": {"subupdate": impl, "accumulate": "k_accum_T_table + k_accum_O_table"}[dominant], "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_kind, "traffic": None, "algorithmic_bytes_per_launch": nbytes,
            "launch_ms": launch_ms, "sub_updates_per_launch": per_launch, "batch_slots": nB}
    hbm_point = hbm_sweep_point(ml, peak) if rank == 0 and not args.no_extra else None
    batch_point = batched_point(ml) if rank == 0 and not args.no_extra else None
    mh_point = multihit_point(ml, w) if rank == 0 and not args.no_extra else None
    rp_point = replay_point(ml, w) if rank == 0 and not args.no_extra and not w.outer_slab else None
    f64_point = fp64_point(ml, w) if rank == 0 and not args.no_extra and not w.fp64 else None

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

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)
    serving = None
    if rank == 0 and args.serving_requests > 0:
        serving = serving_point(ml, n_requests=args.serving_requests)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if w.fp64 else "f32 (float-pair slab sums, FP64 products)",
        "data": "synthetic (hot start from the Philox stream, thermalised)",
        "config": {"workload": w.name, "L": w.L, "Nt": w.Nt, "beta": w.beta, "n_sub": w.n_sub,
                   "k_between": w.k_between, "n_or": w.n_or, "r": f"{w.r[0]}..{w.r[-1]}",
                   "field_r": f"{w.rf[0]}..{w.rf[-1]}", "probes": len(w.probes), "components": 6,
                   "link_updates_per_step": upd, "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": f"{world} independent lattice(s)"},
        "measurements_per_s": world * args.steps / (ms * 1e-3),
        "roofline": roof,
        "kernel_ms": kms, "kernel_share": share,
        "sweep_hbm_point": hbm_point,
        "batched": batch_point,
        "multihit": mh_point,
        "replay": rp_point,
        "fp64_path": f64_point,
        "vs_fp64_path": (f64_point["ms_per_step"] / (ms / args.steps)) if f64_point else None,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(theta_host.numel() * 8),
                "d2h_bytes_per_step": int(lat.rec_len * 8), "steps": e2e_steps},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
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
    ap.add_argument("--serving-requests", type=int, default=1000,
                    help="requests of the serving measurement (0 skips it)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    w = workloads.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, rank, world)
    return run_gpu(args, w, rank, world)


if __name__ == "__main__":
    sys.exit(main())
