"""Pins of the oracle's random-number layer against published values and laws.

* Philox4x32-10 against the known-answer vectors of Salmon et al. (SC'11).
* The open-interval uniform maps at their exact end points.
* The Best-Fisher von Mises sampler against its density
  exp(kappa cos psi) / (2 pi I0(kappa)) by a binned chi-squared test, in both
  draw schemes (52-bit uniforms for the FP64 stream, 23-bit for FP32).
"""

import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp
import scipy.stats as st

import oracle


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(w, 16) for w in line.split()])
    return np.array(rows, dtype=np.uint64).astype(np.uint32)


def test_philox_known_answers(golden_dir):
    kat = _kat(golden_dir)
    out = oracle.philox(kat[:, 0:4], kat[:, 4:6])
    assert np.array_equal(out, kat[:, 6:10])


def test_philox_words_uniform():
    n = 1 << 16
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 1] = 7
    key = np.tile(np.array([12345, 678], dtype=np.uint32), (n, 1))
    words = oracle.philox(ctr, key).ravel()
    counts = np.bincount(words >> 24, minlength=256)
    assert st.chisquare(counts).pvalue > 1e-4


def test_uniform_map_end_points():
    assert oracle.uniform52(0, 0) == 2.0 ** -53
    assert oracle.uniform52(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.uniform52(0, 1 << 12) == 3 * 2.0 ** -53
    assert oracle.uniform52(1, 0) == (2 ** 20 + 0.5) * 2.0 ** -52
    assert oracle.uniform23(0) == 2.0 ** -24
    assert oracle.uniform23(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.uniform23(1 << 9) == 3 * 2.0 ** -24
    # 23-bit draws are exact binary32 values
    u = oracle.uniform23(0x9E3779B9)
    assert float(np.float32(u)) == u


def _vm_bin_probs(kappa, edges):
    norm = 2 * np.pi * sp.i0e(kappa)

    def dens(x):
        return np.exp(kappa * (np.cos(x) - 1.0)) / norm

    return np.array([si.quad(dens, a, b, epsabs=1e-13, epsrel=1e-12)[0] for a, b in zip(edges[:-1], edges[1:])])


@pytest.mark.parametrize("draws", [0, 1])
@pytest.mark.parametrize("kappa", [0.0, 1e-4, 0.1, 1.0, 3.0, 6.0])
def test_vonmises_sampler_chi_squared(kappa, draws):
    n = 200_000
    x = oracle.vonmises_samples(kappa, n, seed=11 + draws, draws=draws)
    assert np.all(x > -np.pi) and np.all(x <= np.pi)
    edges = np.linspace(-np.pi, np.pi, 65)
    counts, _ = np.histogram(x, bins=edges)
    probs = _vm_bin_probs(kappa, edges)
    assert abs(probs.sum() - 1.0) < 1e-9
    chi2 = ((counts - n * probs) ** 2 / (n * probs)).sum()
    pval = st.chi2.sf(chi2, df=len(counts) - 1)
    assert pval > 1e-4, (kappa, draws, chi2)
    # first moment against the closed form I1/I0
    m = np.cos(x).mean()
    expect = sp.i1e(kappa) / sp.i0e(kappa)
    assert abs(m - expect) < 5 * np.sqrt(0.5 / n) + 1e-12
