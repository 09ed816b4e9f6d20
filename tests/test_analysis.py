"""Host analysis (paper_1309_3859_b300/analysis.py) against closed forms.

* Cornell fit of -log P(r)/Nt recovers (V0, sigma, gamma) from synthetic
  measurements, with jackknife errors that cover the truth.
* Sommer scale: exact r0 = sqrt((1.65 - gamma)/sigma) for a potential whose
  Coulomb part is the continuum 1/r (geometric rbar) or the lattice
  propagator (tree-level rbar); the tree-level rbar tends to sqrt(r (r-1)).
* Width: a Gaussian profile e^{-x^2/s} has w^2 = s; the ansatz fit recovers
  its parameters; the measured-profile width of sampled Gaussian points.
* Dedekind eta: eta(i) = Gamma(1/4) / (2 pi^{3/4}) and eta(i/t) = sqrt(t) eta(i t).
* Width law: the zero- and high-temperature limits of the tree-level formula,
  and the fit recovering (sigma, rho0).
* Connected field from records: the ratio estimator against a direct
  computation on synthetic records.
"""

import math

import numpy as np
import pytest

from paper_1309_3859_b300 import analysis as an
from paper_1309_3859_b300 import ml


def test_cornell_fit_recovers_parameters():
    rng = np.random.default_rng(1)
    r = np.arange(2, 9)
    v0, sigma, gamma, Nt = 0.3, 0.18, 0.25, 8
    truth = an.cornell(r, v0, sigma, gamma)
    pp = np.exp(-Nt * truth)[None, :] * (1.0 + 0.02 * rng.standard_normal((400, r.size)))
    (f, df) = an.fit_potential_jackknife(pp, r, Nt)
    for got, err, want in zip(f, df, (v0, sigma, gamma)):
        assert abs(got - want) < 4 * err + 1e-6, (got, err, want)
    v, dv = an.potential(pp, Nt)
    assert np.all(np.abs(v - truth) < 4 * dv + 1e-6)


@pytest.mark.parametrize("sigma,gamma", [(0.18, 0.26), (0.05, 0.3)])
def test_sommer_scale_exact_for_continuum_coulomb(sigma, gamma):
    r = np.arange(1, 12)
    v = an.cornell(r, 0.1, sigma, gamma)
    r0 = an.sommer_r0(r, v, rbar="geometric")
    assert abs(r0 - math.sqrt((1.65 - gamma) / sigma)) < 1e-12


def test_sommer_scale_exact_for_lattice_coulomb():
    sigma, gamma = 0.12, 0.28
    r = np.arange(1, 10)
    v = np.array([0.2 + sigma * ri - gamma * 4 * math.pi * an.lattice_coulomb_g(int(ri)) for ri in r])
    r0 = an.sommer_r0(r, v, rbar="tree")
    assert abs(r0 - math.sqrt((1.65 - gamma) / sigma)) < 1e-9


def test_tree_level_distance_tends_to_continuum():
    for r, tol in ((6, 0.02), (10, 0.006), (14, 0.003)):  # lattice corrections fall like 1/r^2
        assert abs(an.rbar_tree(r) / math.sqrt(r * (r - 1)) - 1) < tol
    assert an.rbar_tree(2) < math.sqrt(2)  # lattice force stronger at short distance


def test_gaussian_width_and_profile_fit():
    s = 3.7
    assert abs(an.width_squared(lambda x: math.exp(-x * x / s), s_hint=s) - s) < 1e-8
    x = np.linspace(0, 6, 25)
    par = (0.8, 0.4, 0.2, 2.5)
    f = an.profile_ansatz(x, *par)
    got = an.fit_profile(x, f, p0=(0.7, 0.3, 0.1, 2.0))
    assert np.allclose(got, par, rtol=1e-5, atol=1e-6)
    probes = [(dy, dz) for dy in range(0, 7) for dz in range(0, 3)]
    xs = an.transverse_distances(probes)
    w2, _ = an.profile_width(xs, 1.3 * np.exp(-xs ** 2 / s))
    assert abs(w2 - s) < 1e-4 * s


def test_dedekind_eta():
    assert abs(an.dedekind_eta_imag(1.0) - math.gamma(0.25) / (2 * math.pi ** 0.75)) < 1e-14
    for t in (0.3, 0.7, 2.0):
        assert abs(an.dedekind_eta_imag(1 / t) - math.sqrt(t) * an.dedekind_eta_imag(t)) < 1e-13


def test_width_law_limits_and_fit():
    sigma, rho0 = 0.18, 0.6
    r = np.array([4.0, 6.0, 8.0])
    # zero temperature: the eta term vanishes
    zero = an.width_tree_level(r, sigma, rho0, T=1e-4)
    assert np.allclose(zero, 2 / (2 * math.pi * sigma) * np.log(r / rho0), rtol=0, atol=1e-9)
    # high temperature (T r >> 1): logarithm of 1/(4 T rho0) plus the linear term
    T = 0.5
    r_hot = np.array([12.0, 16.0])
    hot = an.width_tree_level(r_hot, sigma, rho0, T)
    lim = 2 / (2 * math.pi * sigma) * math.log(1 / (4 * T * rho0)) + 2 / (4 * sigma) * T * r_hot
    assert np.allclose(hot, lim, rtol=0, atol=1e-6)
    w2 = an.width_tree_level(np.arange(3, 12), sigma, rho0, T=1 / 8)
    got = an.fit_width_law(np.arange(3, 12), w2, T=1 / 8)
    assert np.allclose(got, (sigma, rho0), rtol=1e-6)


def test_connected_field_from_records():
    rng = np.random.default_rng(3)
    p = ml.Params(L=8, Nt=4, beta=1.1, r=(1,), rf=(2, 4), probes=((0, 0), (1, 0), (0, 2)), comp_mask=0x3F)
    n = 50
    rec = rng.normal(size=(n, ml.record_len(p)))
    s = ml.split_record(p, rec)
    s["Pf"][..., 0] = 1.0 + 0.1 * rng.random((n, 2))
    (F, dF), (F2, dF2) = an.connected_field(s, p.beta)
    m = {k: v.mean(axis=0) for k, v in s.items()}
    wantF = math.sqrt(p.beta) * (m["W"][..., 1, 0] / m["Pf"][:, None, None, 0] - m["vac"][None, None, :, 1])
    wantF2 = -2 * p.beta * (m["W"][..., 0, 0] / m["Pf"][:, None, None, 0] - m["vac"][None, None, :, 0])
    assert np.allclose(F, wantF, rtol=1e-12, atol=1e-12) and np.allclose(F2, wantF2, rtol=1e-12, atol=1e-12)
    assert np.all(dF > 0) and np.all(dF2 > 0)
