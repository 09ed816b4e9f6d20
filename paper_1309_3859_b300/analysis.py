"""Host analysis of multilevel measurements (arXiv:1309.3859, Sections I, III).

From the per-measurement records of ``ml_measure`` to the paper's derived
quantities, with jackknife errors over measurements (Section III.C):

* the static potential V(r) = -log<P+P>(r) / Nt and its fit
  V(r) = V0 + sigma r - gamma / r (Section I, potential equation), giving the
  string tension sigma;
* the Sommer scale r0 from r0^2 F(r0) = 1.65 with the local force
  interpolation F(r) = f1 + f2 / rbar^2 through two consecutive differences
  V(r) - V(r-1), at the tree-level improved distance rbar built from the
  lattice Coulomb propagator G(r) (Section II.A, Sommer scale);
* the connected field-squared profile on the mediator plane and its fit to
  the ansatz C1 e^{-x^2/s} (1 + C2 e^{-x^2/s}) / (1 + C3 e^{-x^2/s})
  (Section III, width determination), and the squared width
  w^2 = int d^2x x^2 f / int d^2x f of the fitted profile (Section II.B,
  profile equation);
* the effective-string width law at tree level with the Dedekind eta function
  (Section I, tree-level width equation) and its fit for sigma and rho0.

Everything here runs on the host with numpy and scipy; nothing is on the hot
path.
"""

from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

from .stats import jackknife

SOMMER_R0_FORCE = 1.65  # r0^2 F(r0) (Section II.A)


# ----------------------------------------------------------------------------- potential
def potential(pp: np.ndarray, Nt: int) -> tuple[np.ndarray, np.ndarray]:
    """V(r) = -log <P+P>(r) / Nt with jackknife errors.

    ``pp`` is [n_meas][nr] of the real parts of the per-measurement P(r)
    (the record's P[..., 0])."""
    pp = np.asarray(pp, dtype=np.float64)
    return jackknife(pp, lambda m: -np.log(m) / Nt)


def cornell(r, v0, sigma, gamma):
    """V0 + sigma r - gamma / r (Section I, potential equation)."""
    r = np.asarray(r, dtype=np.float64)
    return v0 + sigma * r - gamma / r


def fit_potential(r, v, dv=None) -> np.ndarray:
    """Weighted least-squares fit of the Cornell form; returns (V0, sigma, gamma)."""
    r = np.asarray(r, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    w = np.ones_like(v) if dv is None else 1.0 / np.maximum(np.asarray(dv, dtype=np.float64), 1e-300)
    A = np.stack([np.ones_like(r), r, -1.0 / r], axis=1) * w[:, None]
    coef, *_ = np.linalg.lstsq(A, v * w, rcond=None)
    return coef


def fit_potential_jackknife(pp: np.ndarray, r, Nt: int):
    """Cornell fit of every jackknife sample of the measurements: means and
    errors of (V0, sigma, gamma)."""
    pp = np.asarray(pp, dtype=np.float64)
    _, dv = potential(pp, Nt)
    return jackknife(pp, lambda m: fit_potential(r, -np.log(m) / Nt, dv))


# ----------------------------------------------------------------------------- Sommer scale
def lattice_coulomb_g(r: int, n: int = 96) -> float:
    """Lattice Coulomb propagator G(r) = int_{BZ} d^3k/(2 pi)^3 cos(k1 r) /
    (4 sum_j sin^2(k_j/2)) (-> 1/(4 pi r) at large r), by the midpoint rule on
    an n^3 grid (the grid avoids k = 0; the integrable singularity cancels in
    the differences G(r-1) - G(r) the scale uses)."""
    k = (np.arange(n) + 0.5) * (2 * np.pi / n) - np.pi
    s = np.sin(k / 2) ** 2
    den = 4.0 * (s[:, None, None] + s[None, :, None] + s[None, None, :])
    num = np.cos(k * r)[:, None, None]
    return float((num / den).mean())


def rbar_tree(r: int, n: int = 96) -> float:
    """Tree-level improved distance of the force V(r) - V(r-1):
    rbar = [4 pi (G(r-1) - G(r))]^(-1/2), so that the lattice Coulomb force
    equals 1 / rbar^2 (-> sqrt(r (r-1)) at large r)."""
    d = lattice_coulomb_g(r - 1, n) - lattice_coulomb_g(r, n)
    return float((4.0 * math.pi * d) ** -0.5)


def sommer_r0(r, v, rbar: str = "tree", n: int = 96) -> float:
    """r0 from r0^2 (f1 + f2 / r0^2) = 1.65, with (f1, f2) through the two
    consecutive forces F(rbar_r) = V(r) - V(r-1) that bracket the crossing of
    rbar^2 F(rbar) = 1.65.  rbar: "tree" (lattice Coulomb propagator),
    "midpoint" (r - 1/2) or "geometric" (sqrt(r (r-1)), exact for a continuum
    1/r term).  NaN when the data never reach 1.65."""
    r = np.asarray(r, dtype=np.int64)
    v = np.asarray(v, dtype=np.float64)
    order = np.argsort(r)
    r, v = r[order], v[order]
    pts = []
    for a in range(1, len(r)):
        if r[a] - r[a - 1] != 1:
            continue
        ra = int(r[a])
        if rbar == "tree":
            rb = rbar_tree(ra, n)
        elif rbar == "midpoint":
            rb = ra - 0.5
        else:
            rb = math.sqrt(ra * (ra - 1.0))
        pts.append((rb, v[a] - v[a - 1]))
    for (r1, f1v), (r2, f2v) in zip(pts, pts[1:]):
        if (r1 * r1 * f1v - SOMMER_R0_FORCE) * (r2 * r2 * f2v - SOMMER_R0_FORCE) <= 0:
            # f1 + f2 / rb^2 = F at both points
            f2 = (f1v - f2v) / (1.0 / r1 ** 2 - 1.0 / r2 ** 2)
            f1 = f1v - f2 / r1 ** 2
            return math.sqrt((SOMMER_R0_FORCE - f2) / f1)
    return float("nan")


# ----------------------------------------------------------------------------- field profile and width
def profile_ansatz(x, c1, c2, c3, s):
    """C1 e^{-x^2/s} (1 + C2 e^{-x^2/s}) / (1 + C3 e^{-x^2/s}) (Section III)."""
    e = np.exp(-np.asarray(x, dtype=np.float64) ** 2 / s)
    return c1 * e * (1.0 + c2 * e) / (1.0 + c3 * e)


def fit_profile(x, f, df=None, p0=None) -> np.ndarray:
    """Fit of the profile ansatz; returns (C1, C2, C3, s)."""
    x = np.asarray(x, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    if p0 is None:
        p0 = (float(f.max()) if f.max() > 0 else 1.0, 0.0, 0.0, max(1.0, float((x ** 2 * np.abs(f)).sum() /
                                                                                 max(np.abs(f).sum(), 1e-300))))
    popt, _ = optimize.curve_fit(profile_ansatz, x, f, p0=p0, sigma=df, absolute_sigma=df is not None,
                                 bounds=([-np.inf, -0.99, -0.99, 1e-6], [np.inf, np.inf, np.inf, np.inf]),
                                 maxfev=20000)
    return popt


def width_squared(fn, x_max: float | None = None, s_hint: float = 1.0) -> float:
    """w^2 = int d^2x x^2 f(|x|) / int d^2x f(|x|) over the transverse plane
    (Section II.B, profile equation), for a radial profile function fn."""
    top = x_max if x_max is not None else 30.0 * math.sqrt(s_hint)
    num, _ = integrate.quad(lambda x: x ** 3 * fn(x), 0.0, top, limit=200)
    den, _ = integrate.quad(lambda x: x * fn(x), 0.0, top, limit=200)
    return num / den


def profile_width(x, f, df=None) -> tuple[float, np.ndarray]:
    """Fit the ansatz to a measured profile and integrate it: (w^2, parameters)."""
    par = fit_profile(x, f, df)
    return width_squared(lambda t: profile_ansatz(t, *par), s_hint=par[3]), par


def connected_field(split, beta: float):
    """Connected field and squared field at every (field separation, probe,
    component) from split records (``ml.split_record`` of [n_meas][record]),
    with jackknife errors over measurements (Section II.C, electromagnetic
    field):  F = sqrt(beta) (<W_Im> / <Pf> - <vac_Im>),
    F^2 = -2 beta (<W_Re> / <Pf> - <vac_Re>), the real parts of the
    insertion sums W[..., k, 0] with k = 0 (Re P_c) and 1 (Im P_c).
    Returns ((F, dF), (F2, dF2)), each [nrf][nprobe][6]."""
    pf = split["Pf"][..., 0]                  # [n][nrf]
    w = split["W"][..., 0]                    # [n][nrf][np][6][2]
    vac = split["vac"]                        # [n][6][2]
    n = pf.shape[0]
    nrf, npb = w.shape[1], w.shape[2]
    flat = np.concatenate([pf.reshape(n, -1), w.reshape(n, -1), vac.reshape(n, -1)], axis=1)

    def unpack(m):
        mpf = m[:nrf]
        mw = m[nrf:nrf + nrf * npb * 12].reshape(nrf, npb, 6, 2)
        mv = m[nrf + nrf * npb * 12:].reshape(6, 2)
        F = math.sqrt(beta) * (mw[..., 1] / mpf[:, None, None] - mv[None, None, :, 1])
        F2 = -2.0 * beta * (mw[..., 0] / mpf[:, None, None] - mv[None, None, :, 0])
        return np.concatenate([F.ravel(), F2.ravel()])

    val, err = jackknife(flat, unpack)
    h = nrf * npb * 6
    shape = (nrf, npb, 6)
    return (val[:h].reshape(shape), err[:h].reshape(shape)), (val[h:].reshape(shape), err[h:].reshape(shape))


def transverse_distances(probes) -> np.ndarray:
    """|x_perp| of the probe offsets (dy, dz) on the mediator plane."""
    return np.array([math.hypot(dy, dz) for dy, dz in probes])


# ----------------------------------------------------------------------------- effective string width
def log_dedekind_eta_imag(tau: float) -> float:
    """log eta(i tau), tau > 0: -pi tau / 12 + sum_n log(1 - q^n), q = e^{-2 pi tau},
    after the modular transform eta(i tau) = eta(i / tau) / sqrt(tau) when
    tau < 1, so the product always converges fast."""
    shift = 0.0
    if tau < 1.0:
        shift = -0.5 * math.log(tau)
        tau = 1.0 / tau
    q = math.exp(-2.0 * math.pi * tau)
    acc, qn = 0.0, 1.0
    while True:
        qn *= q
        if qn < 1e-18:
            break
        acc += math.log1p(-qn)
    return -math.pi * tau / 12.0 + acc + shift


def dedekind_eta_imag(tau: float) -> float:
    """Dedekind eta at i tau (tau > 0)."""
    return math.exp(log_dedekind_eta_imag(tau))


def width_tree_level(r, sigma, rho0, T, d: int = 4):
    """w^2(r/2) = (d-2)/(2 pi sigma) log(r/rho0) + (d-2)/(pi sigma)
    log(eta(2iu) / eta(iu)^2), u = 1/(2 T r) (Section I, tree-level width)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    out = np.empty_like(r)
    for i, ri in enumerate(r):
        u = 1.0 / (2.0 * T * ri)
        out[i] = ((d - 2) / (2 * math.pi * sigma) * math.log(ri / rho0) +
                  (d - 2) / (math.pi * sigma) * (log_dedekind_eta_imag(2 * u) - 2 * log_dedekind_eta_imag(u)))
    return out


def fit_width_law(r, w2, T, dw2=None, d: int = 4, p0=(0.2, 0.5)) -> np.ndarray:
    """Fit of the tree-level width law for (sigma, rho0) at temperature T = 1/Nt."""
    popt, _ = optimize.curve_fit(lambda rr, s, rho: width_tree_level(rr, s, rho, T, d), np.asarray(r, float),
                                 np.asarray(w2, float), p0=p0, sigma=dw2, absolute_sigma=dw2 is not None,
                                 bounds=([1e-6, 1e-6], [np.inf, np.inf]), maxfev=20000)
    return popt
