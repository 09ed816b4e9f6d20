"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Deterministic comparisons (same inputs, same Philox stream):
* Philox blocks bit for bit; hot start; angle layout round trip.
* Every (direction, parity, kind, slab mask) pass from the same configuration:
  FP64 within 1e-12 (the links of a pass are independent, so no rounding is
  amplified inside a pass).
* One full heatbath sweep in FP64 within 1e-12.
* Measurement of one configuration (plaquette sums, slab products, field
  insertions, vacuum, naive estimator): FP64 within 1e-12; FP32 kernels on the
  same configuration within 1e-5 relative on the plaquette.
* Whole multilevel runs (one and two levels) in the ordered phase, where
  rounding differences are not amplified by the chain: FP64 within 1e-9.
* Replay of the field insertions: same chain as the direct scheme bit for bit,
  records to rounding; whole ordered-phase runs against the oracle.
* Analytic multihit (Section II.C): the multihit P(r) of one configuration and
  of whole ordered-phase runs against the oracle; on the same chain only the
  multihit entries differ from the plain run's records.

Chains near the transition amplify rounding by ~100x per sweep, so there
the comparison is statistical (test_gpu_statistics.py).
"""

import numpy as np
import pytest

import oracle
from paper_1309_3859_b300 import ml, workloads

pytestmark = pytest.mark.gpu

TWO_PI = 2 * np.pi


def wrapd(a):
    return np.abs((a + np.pi) % TWO_PI - np.pi)


def pair(**kw):
    """(oracle params, library params) for the same run."""
    fp64 = kw.pop("fp64", True)
    replay = kw.pop("replay", 0)  # the same estimator as the oracle's direct sums
    po = oracle.Params(draws=0 if fp64 else 1, **kw)
    pm = ml.Params(fp64=fp64, replay=replay, **kw)
    return po, pm


def thermal_config(po, n=20, cold=False, seed_shift=0):
    th = np.zeros((4, po.V)) if cold else oracle.hot_start(po)
    c = oracle.thermalize(po, th, 0, n)
    return th, c


# ----------------------------------------------------------------------------- RNG and layout
def test_philox_matches_oracle_bitwise():
    rng = np.random.default_rng(5)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(ml.philox(ctr, key), oracle.philox(ctr, key))


@pytest.mark.parametrize("fp64", [True, False])
def test_hot_start_matches_oracle(fp64):
    po, pm = pair(L=6, Nt=4, beta=1.0, seed=0xDEADBEEF12345, fp64=fp64)
    with ml.Lattice(pm) as lat:
        got = lat.get_angles()
    ref = oracle.hot_start(po)
    if fp64:
        assert np.abs(got - ref).max() <= 2e-15
    else:
        assert np.abs(got - ref.astype(np.float32).astype(np.float64)).max() <= 4e-7


@pytest.mark.parametrize("fp64", [True, False])
def test_angle_round_trip(fp64):
    po, pm = pair(L=4, Nt=6, beta=1.0, fp64=fp64)
    th = workloads.random_angles(4, 6, seed=2)
    with ml.Lattice(pm) as lat:
        lat.set_angles(th)
        got = lat.get_angles()
    if fp64:
        assert np.array_equal(got, th)
    else:
        assert np.array_equal(got, th.astype(np.float32).astype(np.float64))


# ----------------------------------------------------------------------------- single passes
def condition_tolerance(po, th0, ref, mu, idx, kind, base=1e-13):
    """Per-link tolerance base * (1 + 12/k + 1/|sin psi|): a one-ulp difference
    in the staple moves alpha = arg W by ~ulp/k, and acos amplifies a one-ulp
    difference in its argument by 1/|sin psi| (psi = theta + alpha)."""
    W = np.array([oracle.staple(po, th0, mu, int(i)) for i in idx])
    k = np.maximum(np.abs(W), 1e-300)
    tol = base * (1.0 + 12.0 / k)
    if kind == 0:
        psi = ref[mu, idx] + np.angle(W)
        tol = tol + base / np.maximum(np.abs(np.sin(psi)), 1e-300)
    return tol


@pytest.mark.parametrize("L,Nt", [(4, 4), (6, 4), (2, 2), (8, 6)])
def test_every_pass_fp64(L, Nt):
    """Each pass from the same configuration: all links within 1e-12 once the
    conditioning of atan2 / acos at that link is accounted for, and at least
    99.9% of links within 1e-12 outright."""
    po, pm = pair(L=L, Nt=Nt, beta=0.95, seed=77)
    th0, _ = thermal_config(po, n=5)
    i = np.arange(po.V)
    par_of = ((i % L) + (i // L) % L + (i // L ** 2) % L + i // L ** 3) % 2
    with ml.Lattice(pm) as lat:
        for kind in (0, 1):
            for d in (0, 2):
                for mu in range(4):
                    for par in range(2):
                        n = 1000 + 10 * mu + par
                        ref = th0.copy()
                        oracle.update_pass(po, ref, mu, par, d, n, kind)
                        lat.set_angles(th0)
                        lat.update_pass(mu, par, d, n, kind)
                        got = lat.get_angles()
                        dev = wrapd(got - ref)
                        others = np.ones_like(dev, bool)
                        others[mu, par_of == par] = False
                        assert dev[others].max() == 0.0
                        idx = np.flatnonzero(par_of == par)
                        tol = 10 * condition_tolerance(po, th0, ref, mu, idx, kind)
                        assert np.all(dev[mu, idx] <= np.maximum(tol, 1e-12)), (kind, d, mu, par, dev.max())
                        assert np.mean(dev[mu, idx] <= 1e-12) >= 0.999


def test_one_heatbath_sweep_fp64():
    """One heatbath sweep (8 chained passes) from a hot start."""
    po, pm = pair(L=6, Nt=4, beta=0.95, seed=78, n_or=0)
    th0 = oracle.hot_start(po)
    ref = th0.copy()
    oracle.compound_sweep(po, ref, 0)
    with ml.Lattice(pm) as lat:
        lat.compound_sweeps(1)
        got = lat.get_angles()
        assert lat.sweep == 1
    dev = wrapd(got - ref)
    # chained passes amplify one-ulp differences of atan2 / acos at badly
    # conditioned links; measured on a B300: 99.6% within 1e-12, max 4.4e-12
    assert np.mean(dev <= 1e-12) >= 0.99 and dev.max() < 1e-10, dev.max()


def test_overrelaxation_pass_fp32():
    """FP32 pass against the FP64 oracle on the same (float) configuration:
    the angle error scales like the staple error over |W|."""
    po, pm = pair(L=6, Nt=4, beta=0.95, seed=79, fp64=False)
    th0, _ = thermal_config(po, n=5)
    th0 = th0.astype(np.float32).astype(np.float64)
    with ml.Lattice(pm) as lat:
        for mu in range(4):
            for par in range(2):
                ref = th0.copy()
                oracle.update_pass(po, ref, mu, par, 0, 1, 1)
                lat.set_angles(th0)
                lat.update_pass(mu, par, 0, 1, 1)
                got = lat.get_angles()
                idx = np.flatnonzero(wrapd(ref[mu] - th0[mu]) > 0)
                k = np.abs([oracle.staple(po, th0, mu, int(i)) for i in idx])
                err = wrapd(got[mu, idx] - ref[mu, idx])
                assert np.max(err * k) < 2e-5, (mu, par, np.max(err * k))


def test_heatbath_pass_fp32_same_draws():
    """FP32 heatbath against the oracle run on the 23-bit draws: the same
    sample except where a rejection decision sits within rounding of its
    threshold; every angle valid."""
    po, pm = pair(L=8, Nt=4, beta=0.95, seed=80, fp64=False)
    th0, _ = thermal_config(po, n=5)
    th0 = th0.astype(np.float32).astype(np.float64)
    close = total = 0
    with ml.Lattice(pm) as lat:
        for mu in range(4):
            for par in range(2):
                ref = th0.copy()
                oracle.update_pass(po, ref, mu, par, 0, 7, 0)
                lat.set_angles(th0)
                lat.update_pass(mu, par, 0, 7, 0)
                got = lat.get_angles()
                assert np.all(np.isfinite(got)) and np.abs(got).max() <= np.pi + 1e-6
                err = wrapd(got[mu] - ref[mu])
                close += int((err < 2e-3).sum())
                total += err.size
    assert close >= total - max(2, total // 2000)


# ----------------------------------------------------------------------------- Metropolis (Section II's update)
METRO = dict(update=1, metro_hits=3, metro_width=1.4)


@pytest.mark.parametrize("d", [0, 2])
def test_metropolis_pass_fp64(d):
    """Every Metropolis pass (kind 2) from the same configuration against the
    oracle: the same proposals and decisions, angles within 1e-12 except where
    a decision sits within rounding of its threshold (none expected)."""
    po, pm = pair(L=6, Nt=4, beta=0.95, seed=81, **METRO)
    th0, _ = thermal_config(po, n=5)
    with ml.Lattice(pm) as lat:
        for mu in range(4):
            for par in range(2):
                n = 2000 + 10 * mu + par
                ref = th0.copy()
                oracle.update_pass(po, ref, mu, par, d, n, 2)
                lat.set_angles(th0)
                lat.update_pass(mu, par, d, n, 2)
                dev = wrapd(lat.get_angles() - ref)
                assert np.mean(dev <= 1e-12) >= 0.9995 and dev.max() < 1e-9, (mu, par, dev.max())
                moved = wrapd(ref[mu] - th0[mu]) > 0
                assert 0.1 < moved.mean() < 0.5, moved.mean()  # most unfrozen links of the parity move


def test_metropolis_pass_fp32_same_draws():
    """FP32 Metropolis against the oracle on the 23-bit draws: the same
    decisions except within rounding of a threshold, angles close."""
    po, pm = pair(L=8, Nt=4, beta=0.95, seed=82, fp64=False, **METRO)
    th0, _ = thermal_config(po, n=5)
    th0 = th0.astype(np.float32).astype(np.float64)
    close = total = 0
    with ml.Lattice(pm) as lat:
        for mu in range(4):
            for par in range(2):
                ref = th0.copy()
                oracle.update_pass(po, ref, mu, par, 0, 9, 2)
                lat.set_angles(th0)
                lat.update_pass(mu, par, 0, 9, 2)
                err = wrapd(lat.get_angles()[mu] - ref[mu])
                close += int((err < 1e-5).sum())
                total += err.size
    assert close >= total - max(2, total // 2000)


def test_metropolis_update_kind_needs_metropolis_handle():
    _, pm = pair(L=4, Nt=4, beta=1.0)
    with ml.Lattice(pm) as lat:
        with pytest.raises(ml.MLError) as exc:
            lat.update_pass(0, 0, 0, 1, 2)
        assert exc.value.status == ml.ML_EINVAL


@pytest.mark.parametrize("two_level,n_sub", [(False, 3), (True, 3)])
def test_multilevel_run_metropolis_fp64_ordered_phase(two_level, n_sub):
    """Whole Metropolis multilevel runs against the oracle in the ordered
    phase (beta = 2.5 from a cold start), FP64 within 1e-9."""
    kw = dict(slab=2, n_sub=n_sub, k_between=2, r=(1, 2, 3), rf=(1, 2), probes=((0, 0), (1, 0)), comp_mask=0x3F,
              **METRO)
    if two_level:
        kw.update(outer_slab=4, n_sub_outer=2)
    po, pm = pair(L=4, Nt=8, beta=2.5, seed=91, **kw)
    th, c = thermal_config(po, n=8, cold=True)
    ref_rec, c2 = oracle.measure(po, th.copy(), c, 2)
    with ml.Lattice(pm) as lat:
        lat.set_angles(th)
        lat.sweep = c
        got = lat.measure(2)
    assert np.abs(got - ref_rec).max() < 1e-9


# ----------------------------------------------------------------------------- measurement of one configuration
MEAS = dict(slab=2, n_sub=1, k_between=0, r=(1, 2, 3), rf=(1, 2, 3), probes=((0, 0), (1, 0), (0, 1), (-1, 2)),
            comp_mask=0x3F)


def _observe_parity(L, Nt, fp64, tol, **extra):
    kw = dict(MEAS)
    kw.update(extra)
    po, pm = pair(L=L, Nt=Nt, beta=0.9, seed=5, fp64=fp64, **kw)
    th, c = thermal_config(po, n=6)
    rec, _ = oracle.measure(po, th, c, 1)  # one slab sub-update, then accumulate
    ref = oracle.split_record(po, rec[0])
    thin = th if fp64 else th.astype(np.float32).astype(np.float64)
    with ml.Lattice(pm) as lat:
        lat.set_angles(thin)
        got = ml.split_record(pm, lat.observe())
    for key in ("P", "Pf", "W", "vac"):
        assert np.abs(got[key] - ref[key]).max() < tol, (key, np.abs(got[key] - ref[key]).max())
    for a, r in enumerate(pm.r):
        z = oracle.naive_correlator(po, thin, r)
        assert abs(complex(*got["naive"][a]) - z) < tol
    pl = oracle.plaquette_mean(po, thin)
    assert abs(got["plaq"] - pl) < (1e-13 if fp64 else 1e-5 * abs(pl))


@pytest.mark.parametrize("L,Nt", [(4, 8), (6, 4), (2, 2)])
def test_observe_fp64(L, Nt):
    _observe_parity(L, Nt, True, 1e-12, r=tuple(r for r in (1, 2, 3) if r < L),
                    rf=tuple(r for r in (1, 2, 3) if r < L),
                    probes=tuple(q for q in MEAS["probes"] if max(abs(q[0]), abs(q[1])) < L))


def test_observe_fp32():
    _observe_parity(6, 4, False, 2e-5)


def test_observe_fp32_component_subset():
    _observe_parity(6, 4, False, 2e-5, comp_mask=0b010010)


# ----------------------------------------------------------------------------- analytic multihit (Section II.C)
@pytest.mark.parametrize("L,Nt", [(4, 8), (6, 4)])
def test_observe_multihit_fp64(L, Nt):
    """P(r) at 2 <= r <= L-2 from the multihit products, r = 1 and r = L-1
    (adjacent lines) and the field records from the plain links."""
    _observe_parity(L, Nt, True, 1e-12, multihit=1, r=tuple(r for r in (1, 2, 3, 5) if r < L))


def test_observe_multihit_fp32():
    _observe_parity(6, 4, False, 2e-5, multihit=1, r=(1, 2, 3, 5))


@pytest.mark.parametrize("two_level,n_sub", [(False, 37), (True, 3)])
def test_multilevel_run_multihit_fp64_ordered_phase(two_level, n_sub):
    kw = dict(slab=2, n_sub=n_sub, k_between=2, r=(1, 2, 3), rf=(1, 2), probes=((0, 0), (1, 0)), comp_mask=0x3F,
              multihit=1)
    if two_level:
        kw.update(outer_slab=4, n_sub_outer=2)
    po, pm = pair(L=6, Nt=8, beta=2.5, seed=92, **kw)
    th, c = thermal_config(po, n=8, cold=True)
    ref_rec, _ = oracle.measure(po, th.copy(), c, 2)
    with ml.Lattice(pm) as lat:
        lat.set_angles(th)
        lat.sweep = c
        got = lat.measure(2)
    assert np.abs(got - ref_rec).max() < 1e-9


@pytest.mark.parametrize("fp64", [True, False])
def test_multihit_changes_only_the_multihit_entries(fp64):
    """Multihit is a different estimator on the same chain: with the same seed
    the angles, P(r) at adjacent lines, the field records, the vacuum and the
    naive estimator are bit-identical to the plain run's; P(r >= 2) differs."""
    base = dict(L=8, Nt=8, beta=1.0, seed=17, fp64=fp64, slab=2, n_sub=20, k_between=2, r=(1, 2, 4, 7), rf=(2, 3),
                probes=((0, 0), (1, 1)), comp_mask=0x3F)
    out = {}
    for mh in (0, 1):
        with ml.Lattice(ml.Params(multihit=mh, **base)) as lat:
            lat.thermalize(4)
            out[mh] = (ml.split_record(lat.p, lat.measure(3)), lat.get_angles())
    (a, tha), (b, thb) = out[0], out[1]
    assert np.array_equal(tha, thb)
    for key in ("Pf", "W", "vac", "naive", "plaq"):
        assert np.array_equal(a[key], b[key]), key
    for i, r in enumerate(base["r"]):
        same = np.array_equal(a["P"][:, i], b["P"][:, i])
        assert same == (r in (1, 7)), r


# ----------------------------------------------------------------------------- replay of the field insertions
@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("n_sub", [3, 29, 37])
def test_replay_matches_the_direct_scheme(fp64, n_sub):
    """The replay scheme runs the inner loop twice from the same configuration
    and sweep numbers: the chain ends where the direct scheme's ends (bit for
    bit) and the records agree to rounding (the same sums in another order).
    The direct scheme's last ring buffer, folded by the products, holds 3, 13
    and 5 records: the products read 4, 16 and 8 ring slots."""
    base = dict(L=6, Nt=8, beta=1.0, seed=23, fp64=fp64, slab=2, n_sub=n_sub, k_between=2, r=(1, 2, 3),
                rf=(1, 2, 3), probes=((0, 0), (1, 0), (0, 1), (-1, 2)), comp_mask=0x3F)
    out = {}
    for rp in (0, 1):
        p = ml.Params(replay=rp, **base)
        with ml.Lattice(p) as lat:
            lat.thermalize(5)
            rec = lat.measure(2)
            out[rp] = (ml.split_record(p, rec), lat.get_angles(), lat.sweep)
    (a, tha, na), (b, thb, nb) = out[0], out[1]
    assert na == nb and np.array_equal(tha, thb)
    for key in ("P", "Pf", "vac", "naive", "plaq"):
        assert np.array_equal(a[key], b[key]), key
    scale = np.abs(a["W"]).max()
    assert np.abs(a["W"] - b["W"]).max() < (1e-13 if fp64 else 2e-6) * scale


@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 2e-5)])
def test_observe_replay(fp64, tol):
    _observe_parity(6, 4, fp64, tol, replay=1)


def test_multilevel_run_replay_fp64_ordered_phase():
    kw = dict(slab=2, n_sub=37, k_between=2, r=(1, 2, 3), rf=(1, 2), probes=((0, 0), (1, 0), (2, 1)),
              comp_mask=0x3F)
    po = oracle.Params(L=4, Nt=8, beta=2.5, seed=93, draws=0, **kw)
    pm = ml.Params(L=4, Nt=8, beta=2.5, seed=93, fp64=True, replay=1, **kw)
    th, c = thermal_config(po, n=8, cold=True)
    ref_rec, c2 = oracle.measure(po, th.copy(), c, 2)
    with ml.Lattice(pm) as lat:
        lat.set_angles(th)
        lat.sweep = c
        got = lat.measure(2)
        assert lat.sweep == c2
    assert np.abs(got - ref_rec).max() < 1e-9


def test_replay_refusals():
    """Replay is one level only, uniform within a batch, and not served."""
    base = dict(L=4, Nt=8, beta=1.0, seed=1, slab=2, n_sub=2, r=(1,), rf=(1,), probes=((0, 0),), comp_mask=1)
    with pytest.raises(ml.MLError) as exc:
        ml.Lattice(ml.Params(replay=1, outer_slab=4, n_sub_outer=2, **base))
    assert exc.value.status == ml.ML_EINVAL
    with pytest.raises(ml.MLError) as exc:
        ml.Batch([ml.Params(replay=1, **base), ml.Params(replay=0, **base)])
    assert exc.value.status == ml.ML_EINVAL
    with ml.Batch([ml.Params(replay=1, **base), ml.Params(replay=1, **dict(base, seed=2))]) as b:
        b.thermalize(1)
        assert np.all(np.isfinite(b.measure(1)))
    with ml.Server(budget_bytes=64 << 20, fp64=True) as srv:
        with pytest.raises(ml.MLError) as exc:
            srv.submit(ml.Params(replay=1, **base), 1, 1)
        assert exc.value.status == ml.ML_EINVAL


# ----------------------------------------------------------------------------- whole runs, ordered phase
@pytest.mark.parametrize("two_level,n_sub", [(False, 3), (True, 3), (False, 37), (True, 18)])
def test_multilevel_run_fp64_ordered_phase(two_level, n_sub):
    """n_sub > 16 exercises full folds of the record ring plus a ragged tail."""
    kw = dict(slab=2, n_sub=n_sub, k_between=2, r=(1, 2, 3), rf=(1, 2), probes=((0, 0), (1, 0), (2, 1)),
              comp_mask=0x3F)
    if two_level:
        kw.update(outer_slab=4, n_sub_outer=2)
    po, pm = pair(L=4, Nt=8, beta=2.5, seed=90, **kw)
    th, c = thermal_config(po, n=8, cold=True)
    ref_rec, c2 = oracle.measure(po, th.copy(), c, 2)
    ref_th = th.copy()
    oracle.measure(po, ref_th, c, 2)
    with ml.Lattice(pm) as lat:
        lat.set_angles(th)
        lat.sweep = c
        got = lat.measure(2)
        assert lat.sweep == c2
        got_th = lat.get_angles()
    assert wrapd(got_th - ref_th).max() < 1e-9
    assert np.abs(got - ref_rec).max() < 1e-9


@pytest.mark.parametrize("fp64", [True, False])
def test_connected_profile_on_device(fp64):
    """ml_connected_device (Section II.C's connected field, F and F^2) on the
    device's own records against the oracle's orc_connected on the same
    records."""
    po, pm = pair(L=4, Nt=4, beta=2.5, seed=91, slab=2, n_sub=2, k_between=1, r=(1, 2), rf=(2, 1),
                  probes=((0, 0), (1, 0)), comp_mask=0b101011, fp64=fp64)
    with ml.Lattice(pm) as lat:
        lat.thermalize(3)
        recs = lat.measure_device(5)
        out_dev = lat.connected(recs)
        lat.sync()  # the results are complete in the lattice stream's order
        out = out_dev.cpu().numpy()
        r = recs.cpu().numpy()
    ref = oracle.connected(po, r)
    assert np.abs(ref[..., :2]).max() > 0.01
    assert np.allclose(out, ref[..., :2], rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------------------------- full-size sampled parity
def test_full_size_pass_fp32_single_24():
    """24^3 x 8 (FP32 bulk workload): one overrelaxation pass of every
    direction checked link by link against the oracle."""
    w = workloads.SINGLE_24
    po, pm = pair(L=w.L, Nt=w.Nt, beta=w.beta, seed=3, fp64=False)
    th0 = oracle.hot_start(po).astype(np.float32).astype(np.float64)
    with ml.Lattice(pm) as lat:
        for mu in range(4):
            ref = th0.copy()
            oracle.update_pass(po, ref, mu, 1, 2, 1, 1)
            lat.set_angles(th0)
            lat.update_pass(mu, 1, 2, 1, 1)
            got = lat.get_angles()
            err = wrapd(got[mu] - ref[mu])
            moved = wrapd(ref[mu] - th0[mu]) > 0
            assert np.array_equal(wrapd(got[mu] - th0[mu]) > 0, moved)
            assert np.quantile(err, 0.999) < 1e-4 and np.median(err) < 1e-6


@pytest.mark.parametrize("multihit", [0, 1])
def test_full_size_observe_fp32_single_24(multihit):
    """24^3 x 8 with the full r = 2..12, six components, offsets 0..8 layout:
    measurement of one configuration against the oracle (with multihit every
    P(r) entry comes from the multihit products)."""
    w = workloads.SINGLE_24
    kw = dict(slab=2, n_sub=1, k_between=0, r=w.r, rf=w.rf, probes=w.probes, comp_mask=w.comp_mask, threads=0,
              multihit=multihit)
    po = oracle.Params(L=w.L, Nt=w.Nt, beta=w.beta, seed=4, draws=1, **kw)
    kw.pop("threads")
    pm = ml.Params(L=w.L, Nt=w.Nt, beta=w.beta, seed=4, fp64=False, **kw)
    th = oracle.hot_start(po)
    c = oracle.thermalize(po, th, 0, 3)
    rec, _ = oracle.measure(po, th, c, 1)
    ref = oracle.split_record(po, rec[0])
    with ml.Lattice(pm) as lat:
        lat.set_angles(th)
        got = ml.split_record(pm, lat.observe())
    scale = {k: np.abs(ref[k]).max() for k in ("P", "Pf", "W", "vac")}
    for key in ("P", "Pf", "W", "vac"):
        assert np.abs(got[key] - ref[key]).max() < 3e-5 * max(scale[key], 1e-3), key


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("geom", [dict(L=8, Nt=4, n_sub=3), dict(L=6, Nt=8, n_sub=18, outer_slab=4, n_sub_outer=2),
                                  dict(L=8, Nt=4, n_sub=3, **METRO), dict(L=6, Nt=4, n_sub=18, multihit=1),
                                  dict(L=6, Nt=4, n_sub=18, replay=1), dict(L=6, Nt=4, n_sub=5, slab=1),
                                  dict(L=8, Nt=8, n_sub=3, slab=4), dict(L=10, Nt=4, n_sub=3),
                                  dict(L=4, Nt=4, n_sub=17), dict(L=24, Nt=8, n_sub=17)])
def test_sweep_implementations_agree(fp64, geom):
    """The persistent kernel, the per-pass kernels and the cluster-resident
    kernels run the same link updates with the same random numbers: identical
    chains and records.  L = 6 puts cluster boundaries and partial record
    warps inside a slab; n_sub = 18 covers a full record ring and a tail; the
    two-level run uses the resident kernels for both slab thicknesses.  In the
    resident kernel: slab thickness 1 (spatial passes that move no link, so
    CTAs exchange only their per-pass tokens) and 4, ragged bricks (L = 10 on
    3 x 5 bricks) and bricks one site thick (L = 4); L = 24 in slabs of
    thickness 2 runs, in FP32, the resident kernel compiled for that shape."""
    kw = dict(beta=0.95, seed=5, fp64=fp64, slab=2, k_between=1, r=(1, 2), rf=(2,), probes=((0, 0), (1, 0)),
              comp_mask=0x3F)
    kw.update(geom)
    p = ml.Params(**kw)
    out = {}
    modes = (ml.ML_SWEEP_PERSISTENT, ml.ML_SWEEP_PASSES, ml.ML_SWEEP_RESIDENT)
    for mode in modes:
        with ml.Lattice(p) as lat:
            lat.sweep_mode = mode
            assert lat.sweep_mode == mode
            lat.thermalize(3)
            rec = lat.measure(2)
            out[mode] = (rec, lat.get_angles(), lat.sweep)
    a = out[modes[0]]
    for mode in modes[1:]:
        b = out[mode]
        assert a[2] == b[2], mode
        assert np.array_equal(a[1], b[1]), mode
        assert np.array_equal(a[0], b[0]), mode


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("geom", [dict(L=8, Nt=4, n_sub=20, probes=((0, 0), (1, 0), (-2, 1), (3, -2))),
                                  dict(L=8, Nt=8, n_sub=18, outer_slab=4, n_sub_outer=2,
                                       probes=((0, 0), (2, 0), (-3, 3))),
                                  dict(L=12, Nt=4, n_sub=3, probes=tuple((d, 0) for d in range(7))),
                                  dict(L=6, Nt=4, n_sub=5, probes=((0, 0), (1, -1)))])
def test_fold_implementations_agree(fp64, geom):
    """The per-site fold and the shared-memory tiled fold form the same sums
    operation for operation: identical records.  The probe sets reach both
    signs of y and z offsets and wrap around the lattice."""
    p = ml.Params(beta=0.95, seed=8, fp64=fp64, slab=2, k_between=1, r=(1, 2), rf=(1, 2, 3), comp_mask=0x3F, **geom)
    out = {}
    for mode in (ml.ML_FOLD_SITE, ml.ML_FOLD_TILE):
        with ml.Lattice(p) as lat:
            lat.fold_mode = mode
            assert lat.fold_mode == mode
            lat.thermalize(2)
            out[mode] = lat.measure(2)
    assert np.array_equal(out[ml.ML_FOLD_SITE], out[ml.ML_FOLD_TILE])


def test_tiled_fold_refused_when_the_tile_does_not_fit():
    """Probes six z planes apart on a 64^3 lattice need a tile of 28 rows x 64
    sites x 16 slots (112 KB) per block, above the tiled fold's shared-memory
    limit: the tiled fold is refused and the handle keeps the per-site fold."""
    p = ml.Params(L=64, Nt=4, beta=0.95, seed=8, fp64=False, slab=2, n_sub=2, r=(1,), rf=(2,),
                  probes=((0, 0), (0, 6)), comp_mask=0x01)
    with ml.Lattice(p) as lat:
        assert lat.fold_mode == ml.ML_FOLD_SITE
        with pytest.raises(ml.MLError) as exc:
            lat.fold_mode = ml.ML_FOLD_TILE
        assert exc.value.status == ml.ML_EINVAL
        assert lat.fold_mode == ml.ML_FOLD_SITE


def test_resident_mode_needs_fitting_slabs():
    """A 64^3 slab of thickness 2 needs more shared memory than a cluster
    has: forcing the resident implementation is rejected, the handle keeps
    working in its own mode."""
    p = ml.Params(L=64, Nt=2, beta=1.0, seed=1, fp64=False, slab=2, n_sub=1, r=(1,), rf=(1,), probes=((0, 0),),
                  comp_mask=0x01)
    with ml.Lattice(p) as lat:
        mode = lat.sweep_mode
        assert mode != ml.ML_SWEEP_RESIDENT
        with pytest.raises(ml.MLError) as exc:
            lat.sweep_mode = ml.ML_SWEEP_RESIDENT
        assert exc.value.status == ml.ML_EINVAL
        assert lat.sweep_mode == mode
        lat.thermalize(1)
        assert np.all(np.isfinite(lat.measure(1)))


def test_full_size_two_level_48():
    """48^3 x 16 two-level workload in FP32: one overrelaxation pass of every
    direction link by link, and the measurement of one configuration with its
    full layout (r = 2..24, six components at r = 8, 16, 24, offsets 0..12)
    against the oracle."""
    w = workloads.LARGE_48
    kw = dict(slab=2, n_sub=1, k_between=0, r=w.r, rf=w.rf, probes=w.probes, comp_mask=w.comp_mask)
    po = oracle.Params(L=w.L, Nt=w.Nt, beta=w.beta, seed=6, draws=1, threads=0, **kw)
    pm = ml.Params(L=w.L, Nt=w.Nt, beta=w.beta, seed=6, fp64=False, outer_slab=w.outer_slab,
                   n_sub_outer=w.n_sub_outer, **kw)
    th0 = oracle.hot_start(po).astype(np.float32).astype(np.float64)
    with ml.Lattice(pm) as lat:
        for mu in (0, 3):
            ref = th0.copy()
            oracle.update_pass(po, ref, mu, 0, 4, 1, 1)
            lat.set_angles(th0)
            lat.update_pass(mu, 0, 4, 1, 1)
            err = wrapd(lat.get_angles()[mu] - ref[mu])
            assert np.quantile(err, 0.999) < 1e-4 and np.median(err) < 1e-6
        rec, _ = oracle.measure(po, th0.copy(), 0, 1)
        ref = oracle.split_record(po, rec[0])
        # the oracle swept once before measuring: measure that configuration
        th1 = th0.copy()
        oracle.compound_sweep(po, th1, 0, slab_d=2)
        lat.set_angles(th1)
        got = ml.split_record(pm, lat.observe())
    for key in ("P", "Pf", "W", "vac"):
        scale = max(np.abs(ref[key]).max(), 1e-3)
        assert np.abs(got[key] - ref[key]).max() < 3e-5 * scale, key


# ----------------------------------------------------------------------------- slab-sum formats
@pytest.mark.parametrize("two_level", [False, True])
def test_pair_sums_same_chain_close_records(two_level):
    """FP32 lattices with float-pair slab sums (pair_sums = 1) run the same
    chain as with the default double-precision sums; the records agree to the
    float pairs' ~47 bits relative to each block's scale, and the
    double-precision default stays within the FP32 tolerance of the oracle
    measurement of one configuration."""
    kw = dict(L=8, Nt=8, beta=0.98, seed=41, slab=2, n_sub=37, k_between=2, r=(1, 2, 3, 4), rf=(2, 4),
              probes=((0, 0), (1, 0), (2, 1)), comp_mask=0x3F)
    if two_level:
        kw.update(n_sub=18, outer_slab=4, n_sub_outer=2)
    out = {}
    for ps in (0, 1):
        p = ml.Params(fp64=False, pair_sums=ps, **kw)
        with ml.Lattice(p) as lat:
            lat.thermalize(5)
            rec = lat.measure(2)
            out[ps] = (rec, lat.get_angles())
    assert np.array_equal(out[0][1], out[1][1])
    a, b = ml.split_record(p, out[0][0]), ml.split_record(p, out[1][0])
    for key in ("P", "Pf", "W", "vac", "naive", "plaq"):
        scale = max(np.abs(a[key]).max(), 1e-30)
        assert np.abs(a[key] - b[key]).max() <= 1e-9 * scale, key


def test_pair_sums_refused_for_fp64():
    p = ml.Params(L=4, Nt=4, beta=1.0, fp64=True, pair_sums=1)
    with pytest.raises(ml.MLError) as e:
        ml.Lattice(p)
    assert e.value.status == ml.ML_EINVAL


def test_fp32_rounding_matches_conversions():
    """The FP32 update rounds its range reductions and wrap on the FP32 pipe
    and builds its uniforms in the mantissa; on the device these equal rintf,
    floorf and the integer-to-float uniform formulas for every float of
    magnitude below 2^22, every 23-bit uniform and 2^24 52-bit uniforms."""
    assert ml.check_rounding() == [0, 0, 0, 0]
