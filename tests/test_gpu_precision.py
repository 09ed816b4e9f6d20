"""Precision of the device measurement where it matters: full-size lattices,
long inner loops and large separations, where the cross-slab products are
far smaller than the per-site values they are summed from (Section II.C:
P(r) falls as exp(-V(r) Nt)).

For each precision mode (FP64 lattices; FP32 lattices with double-precision
slab sums, the default; FP32 lattices with float-pair slab sums) one handle
measures with ml_measure, and the same handle, put back to the same
configuration and sweep counter, replays the measurement's chain one
sub-update at a time (the sweep implementations give bit-identical chains),
handing each configuration to the oracle, which measures exactly those
configurations in double precision.  Every P(r), field-separation P, field
insertion W, vacuum, naive and plaquette value is compared relative to its
own magnitude.  The printed table is the per-observable error of each mode
against the FP64 oracle.
"""

import numpy as np
import pytest

import oracle
from paper_1309_3859_b300 import ml, workloads

pytestmark = pytest.mark.gpu


def _oracle_params(pm: ml.Params) -> oracle.Params:
    return oracle.Params(L=pm.L, Nt=pm.Nt, beta=pm.beta, seed=pm.seed, n_or=pm.n_or, draws=0 if pm.fp64 else 1,
                         slab=pm.slab, n_sub=pm.n_sub, outer_slab=pm.outer_slab, n_sub_outer=pm.n_sub_outer,
                         k_between=0, r=pm.r, rf=pm.rf, probes=pm.probes, comp_mask=pm.comp_mask)


def measure_and_replay(pm: ml.Params, n_therm: int, with_oracle: bool = True):
    """(device record, oracle record or None) of one measurement."""
    po = _oracle_params(pm)
    with ml.Lattice(pm) as lat:
        lat.thermalize(n_therm)
        th0 = lat.get_angles()
        n0 = lat.sweep
        rec = lat.measure(1)[0]
        if not with_oracle:
            return rec, None
        lat.set_angles(th0)
        lat.sweep = n0
        with oracle.Accumulator(po) as acc:
            acc.begin(th0)
            for _ in range(pm.n_sub_outer if pm.outer_slab else 1):
                if pm.outer_slab:
                    lat.compound_sweeps(1, pm.outer_slab)
                for _ in range(pm.n_sub):
                    lat.compound_sweeps(1, pm.slab)
                    acc.add(lat.get_angles())
                if pm.outer_slab:
                    acc.end_outer()
            ref = acc.finish()
    return rec, ref


def _cplx(a):
    return a[..., 0] + 1j * a[..., 1]


def relative_errors(pm, rec, ref):
    """Largest |device - oracle| / |oracle| per observable block (complex
    values; W over the selected components)."""
    g, o = ml.split_record(pm, rec), ml.split_record(pm, ref)
    out = {}
    for key in ("P", "Pf", "naive"):
        d, r = _cplx(g[key]), _cplx(o[key])
        out[key] = float(np.max(np.abs(d - r) / np.abs(r)))
    sel = [c for c in range(6) if (pm.comp_mask >> c) & 1]
    d, r = _cplx(g["W"])[:, :, sel], _cplx(o["W"])[:, :, sel]
    out["W"] = float(np.max(np.abs(d - r) / np.abs(r)))
    out["vac"] = float(np.max(np.abs(g["vac"] - o["vac"])[sel] / np.abs(o["vac"][sel, 0])[:, None]))
    out["plaq"] = float(abs(g["plaq"] - o["plaq"]) / abs(o["plaq"]))
    out["min |P|"] = float(np.min(np.abs(_cplx(o["P"]))))
    out["min |W|"] = float(np.min(np.abs(r)))
    return out


# Bounds on the relative error of each block.  FP64: the device and the
# oracle differ by rounding only.  FP32 lattices: the per-sub-update phases
# and plaquettes are single-precision values (a few 1e-7 absolute each: the
# angle sums, their difference and the hardware sine and cosine); the slab
# averages, products and sums over sites are double precision, so P(r) and W
# keep that relative error down to the smallest values measured here (|P|
# about 1e-6 at 24^3 x 8, r = 12, and 4e-10 at 48^3 x 16, r = 24).  Measured
# (one B300): FP64 P 4.5e-15, W 8.3e-14; FP32 P 8.5e-7 (24^3 x 8) and 2.8e-6
# (48^3 x 16), W 1.3e-5 and 7.1e-6, vacuum 5.6e-8, plaquette 2e-10; the
# naive correlator and plaquette are double-precision sums of the single-
# precision angles.  The bounds are about ten times those.
BOUNDS = {
    "fp64": {"P": 1e-12, "Pf": 1e-12, "naive": 1e-12, "W": 1e-11, "vac": 1e-12, "plaq": 1e-13},
    "fp32": {"P": 3e-5, "Pf": 3e-5, "naive": 1e-12, "W": 2e-4, "vac": 1e-6, "plaq": 1e-8},
}

_tables = {}


def _report(name, errs):
    _tables[name] = errs
    print("\n" + name + ": " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))


def _workload_24():
    w = workloads.SINGLE_24
    return dict(L=w.L, Nt=w.Nt, beta=w.beta, seed=w.seed, slab=w.slab, n_sub=w.n_sub, k_between=0,
                r=tuple(w.r), rf=tuple(w.rf), probes=tuple(w.probes), comp_mask=w.comp_mask)


def test_precision_single_24_fp64():
    """24^3 x 8, beta 0.98, 100 sub-updates, r = 2..12, every field
    separation, probe and component: FP64 lattice against the oracle."""
    pm = ml.Params(fp64=True, **_workload_24())
    rec, ref = measure_and_replay(pm, 200)
    errs = relative_errors(pm, rec, ref)
    _report("24^3x8 fp64", errs)
    for k, b in BOUNDS["fp64"].items():
        assert errs[k] < b, (k, errs)


def test_precision_single_24_fp32_modes():
    """The same workload on FP32 lattices: double-precision slab sums (the
    default) and float-pair slab sums share one chain and one oracle
    reference."""
    kw = _workload_24()
    pm = ml.Params(fp64=False, **kw)
    rec, ref = measure_and_replay(pm, 200)
    rec_pair, _ = measure_and_replay(ml.Params(fp64=False, pair_sums=1, **kw), 200, with_oracle=False)
    for name, r in (("24^3x8 fp32 (f64 sums)", rec), ("24^3x8 fp32 (pair sums)", rec_pair)):
        errs = relative_errors(pm, r, ref)
        _report(name, errs)
        for k, b in BOUNDS["fp32"].items():
            assert errs[k] < b, (name, k, errs)


def test_precision_two_level_48_fp32():
    """48^3 x 16 two-level (outer slabs of 4, inner of 2), beta 0.99, r =
    2..24, the field at r = 8, 16, 24 over two probes: FP32 lattice with
    double-precision sums against the oracle; the inner and outer loops are
    shortened (20 inner x 4 outer sub-updates) to keep the oracle's share to
    about a minute."""
    w = workloads.LARGE_48
    pm = ml.Params(fp64=False, L=w.L, Nt=w.Nt, beta=w.beta, seed=w.seed, slab=w.slab, n_sub=20,
                   outer_slab=w.outer_slab, n_sub_outer=4, k_between=0, r=tuple(w.r), rf=tuple(w.rf),
                   probes=((0, 0), (6, 0)), comp_mask=w.comp_mask)
    rec, ref = measure_and_replay(pm, 100)
    errs = relative_errors(pm, rec, ref)
    _report("48^3x16 two-level fp32 (f64 sums)", errs)
    for k, b in BOUNDS["fp32"].items():
        assert errs[k] < b, (k, errs)
