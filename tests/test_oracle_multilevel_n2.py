"""Pins of the oracle's multilevel averages at n2 > 1 (Section II.C, the
equations for <P+P>, <P+P O>, T^(4) and TO^(4); Algorithm 1).

The estimators are multilinear in the slab averages:
    P(r) = (1/Ns) sum_x prod_s [T]_s,
    W    = (1/(Ns Nt)) sum_x sum_s [TO]_s prod_{s' != s} [T]_{s'},
and at two levels each outer average is the mean over outer iterations of
products of inner averages.  If the sub-update configurations differ only in
the links that a sub-update of ONE slab moves (its temporal links and its
interior spatial links), every other slab's average is that of a single
configuration, and multilinearity makes the multilevel record exactly the
mean over the configurations of the single-configuration record.  That record
is fixed by the n2 = 1 identity: P(x)^* P(x + r) and P^* P sum_t O(x0, t)
from Polyakov loops (``ml_identity``).  At two levels the same holds when,
within each outer iteration, one inner slab varies per sub-update and the
other inner slab of the same outer slab (with the spatial links between the
two) varies only per outer iteration.

Every normalisation and slab index of the estimators enters these
identities, so each plausible mistake planted in a copy of the oracle (a
missing or doubled 1/n on [TO], a wrong slab in the product over the other
slabs, the wrong inner average or a dropped term in TO^(4), a missing 1/n2
in the level combination) fails them; the last test builds those copies and
checks exactly that.  A statistical check compares multilevel W at n2 = 10
with the naive estimator.
"""

import numpy as np
import pytest

import oracle
from ml_identity import _identity_expectation
from paper_1309_3859_b300.stats import jackknife

BASE = dict(L=4, Nt=8, beta=0.9, seed=3, slab=2, r=(1, 2, 3), rf=(1, 2, 3),
            probes=((0, 0), (1, 0), (0, 1), (-1, 2)), comp_mask=0x3F)


def _randomise(th, p, rng, temporal_times=(), spatial_times=()):
    """Copy of th with the temporal links at temporal_times and the spatial
    links at spatial_times drawn uniformly from [-pi, pi)."""
    out = th.copy()
    Ns = p.Ns
    for t in temporal_times:
        out[0, t * Ns:(t + 1) * Ns] = rng.uniform(-np.pi, np.pi, Ns)
    for t in spatial_times:
        out[1:, t * Ns:(t + 1) * Ns] = rng.uniform(-np.pi, np.pi, (3, Ns))
    return out


def _slab_interior(t0, d):
    """(temporal, spatial) times a sub-update of the slab [t0, t0 + d) moves."""
    return tuple(range(t0, t0 + d)), tuple(range(t0 + 1, t0 + d))


def one_level_case(s0, n2=3, seed=7):
    """(params, first configuration, sub-update configurations)."""
    p = oracle.Params(n_sub=n2, **BASE)
    rng = np.random.default_rng(seed)
    base = oracle.hot_start(p)
    oracle.thermalize(p, base, 0, 2)
    tt, st = _slab_interior(s0 * p.slab, p.slab)
    return p, base, [_randomise(base, p, rng, tt, st) for _ in range(n2)]


def two_level_case(S0, n2=3, n4=2, seed=9):
    p = oracle.Params(n_sub=n2, outer_slab=4, n_sub_outer=n4, **BASE)
    rng = np.random.default_rng(seed)
    base = oracle.hot_start(p)
    oracle.thermalize(p, base, 0, 2)
    a0 = S0 * p.outer_slab  # first time of inner slab a; inner slab b follows it
    b0 = a0 + p.slab
    ta, sa = _slab_interior(a0, p.slab)
    tb, sb = _slab_interior(b0, p.slab)
    cfgs = []
    for _ in range(n4):
        outer = _randomise(base, p, rng, tb, sb + (b0,))  # slab b and the spatial links between a and b
        for _ in range(n2):
            cfgs.append(_randomise(outer, p, rng, ta, sa))
    return p, base, cfgs


def deviation(p, base, cfgs):
    """Largest difference between the oracle's record from the
    configurations and the mean of their single-configuration records, over
    P, Pf, W (relative to their scale) and the vacuum sums."""
    rec = oracle.split_record(p, oracle.measure_configs(p, base, cfgs))
    ids = [_identity_expectation(p, th) for th in cfgs]
    P = np.mean([a for a, _ in ids], axis=0)
    W = np.mean([b for _, b in ids], axis=0)
    Pf = P[[p.r.index(r) for r in p.rf]]
    got_P = rec["P"][:, 0] + 1j * rec["P"][:, 1]
    got_Pf = rec["Pf"][:, 0] + 1j * rec["Pf"][:, 1]
    got_W = rec["W"][..., 0] + 1j * rec["W"][..., 1]
    vac = np.mean([oracle.plaquette_field(p, th).mean(axis=2) for th in cfgs], axis=0)
    dev = [np.abs(got_P - P).max() / np.abs(P).max(), np.abs(got_Pf - Pf).max() / np.abs(Pf).max(),
           np.abs(got_W - W).max() / np.abs(W).max(), np.abs(rec["vac"] - vac).max()]
    return max(dev)


@pytest.mark.parametrize("s0", [0, 2])
def test_one_level_one_slab_varied_is_mean_of_single_records(s0):
    p, base, cfgs = one_level_case(s0)
    assert deviation(p, base, cfgs) < 1e-13


@pytest.mark.parametrize("S0", [0, 1])
def test_two_level_one_inner_slab_varied_is_mean_of_single_records(S0):
    p, base, cfgs = two_level_case(S0)
    assert deviation(p, base, cfgs) < 1e-13


def test_measure_configs_reproduces_measure():
    """The caller-supplied path is the same arithmetic as orc_measure's own
    chain (one and two levels)."""
    for kw in (dict(n_sub=3), dict(n_sub=2, outer_slab=4, n_sub_outer=2)):
        p = oracle.Params(k_between=0, **BASE, **kw)
        th = oracle.hot_start(p)
        c = oracle.thermalize(p, th, 0, 2)
        first = th.copy()
        cfgs, t, cc = [], th.copy(), c
        for o in range(p.n_sub_outer if p.outer_slab else 1):
            if p.outer_slab:
                cc = oracle.compound_sweep(p, t, cc, p.outer_slab)
            for j in range(p.n_sub):
                cc = oracle.compound_sweep(p, t, cc, p.slab)
                cfgs.append(t.copy())
        rec, _ = oracle.measure(p, th, c, 1)
        assert np.array_equal(rec[0], oracle.measure_configs(p, first, cfgs))


# Plausible mistakes, each planted in a copy of the oracle source: (name,
# text in the W products or level combination, replacement).
MUTANTS = [
    ("missing 1/n on [TO]",
     "cplx term = T_O(S, sl, a, b, c, k, xs);\n                term.re *= inv;\n                term.im *= inv;",
     "cplx term = T_O(S, sl, a, b, c, k, xs);"),
    ("doubled 1/n on [TO]",
     "cplx term = T_O(S, sl, a, b, c, k, xs);\n                term.re *= inv;\n                term.im *= inv;",
     "cplx term = T_O(S, sl, a, b, c, k, xs);\n                term.re *= inv * inv;\n"
     "                term.im *= inv * inv;"),
    ("wrong slab left out of prod_{s' != s}", "if (s2 == sl) continue;",
     "if (s2 == (sl + 1) % S->nslab) continue;"),
    ("no slab left out of prod_{s' != s}", "if (s2 == sl) continue;", ""),
    ("TO^(4) with the inserted slab's own average", "if (jj == j) continue;", "if (jj != j) continue;"),
    ("TO^(4) without its second term", "for (int j = 0; j < q; ++j) {\n                cplx term = T_O(in,",
     "for (int j = 0; j < 1; ++j) {\n                cplx term = T_O(in,"),
    ("missing 1/n2 on [TO] in the level combination",
     "cplx term = T_O(in, q * so + j, a, b, c, k, xs);\n                term.re *= inv;\n                term.im *= inv;",
     "cplx term = T_O(in, q * so + j, a, b, c, k, xs);"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_fail_the_pins(tmp_path, name, old, new):
    src = oracle.source()
    assert src.count(old) == 1, name
    path = oracle.build_variant(src.replace(old, new), str(tmp_path / "liborc_variant.so"))
    cases = [one_level_case(0), two_level_case(1)]
    with oracle.using_library(path):
        devs = [deviation(*case) for case in cases]
    assert max(devs) > 1e-6, (name, devs)


def test_multilevel_field_insertion_agrees_with_naive():
    """Multilevel W at n2 = 10 against the naive estimator
    (1/(Ns Nt)) sum_x P(x)^* P(x + r) sum_t O(x0, t) on the measurements'
    first configurations, within 3 combined jackknife errors, on the entries
    whose naive mean is resolved."""
    p = oracle.Params(L=4, Nt=4, beta=1.1, seed=31, slab=2, n_sub=10, k_between=0, r=(1,), rf=(1,),
                      probes=((0, 0), (1, 0)), comp_mask=0x3F, threads=4)
    th = oracle.hot_start(p)
    c = oracle.thermalize(p, th, 0, 40)
    ml_w, naive_w = [], []
    for _ in range(160):
        c = oracle.thermalize(p, th, c, 2)
        naive_w.append(_identity_expectation(p, th)[1].real)
        rec, c = oracle.measure(p, th, c, 1)
        ml_w.append(oracle.split_record(p, rec[0])["W"][..., 0])
    ml_w, naive_w = np.array(ml_w), np.array(naive_w)
    checked = 0
    for idx in np.ndindex(ml_w.shape[1:]):
        mn, en = jackknife(naive_w[(slice(None),) + idx])
        if abs(mn) < 4 * en:
            continue  # no resolved signal to compare
        mm, em = jackknife(ml_w[(slice(None),) + idx])
        assert abs(mm - mn) < 3 * np.hypot(em, en), (idx, mm, em, mn, en)
        checked += 1
    assert checked >= 4
