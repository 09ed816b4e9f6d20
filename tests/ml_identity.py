"""Single-configuration values of the multilevel records from Polyakov loops.

With one sub-update (n2 = 1) the slab two-link operators of a configuration
multiply to P(x)^* P(x + r xhat) and the field-insertion sum to that times
the time sum of the plaquette at the probe (Section II.C, the product of the
two-link operators): computed here from the oracle's Polyakov loops and
plaquette field with numpy shifts, a different code path from the oracle's
slab sums.
"""

import numpy as np

import oracle


def _spatial(a, L, Nt):
    """[..., V] -> [..., Nt, z, y, x]"""
    return a.reshape(a.shape[:-1] + (Nt, L, L, L))


def _identity_expectation(p, th):
    """P and W records of one configuration from Polyakov loops and the
    plaquette field, with numpy shifts for the separations and probes."""
    L, Nt = p.L, p.Nt
    P = oracle.polyakov(p, th).reshape(L, L, L)  # [z, y, x]
    f = _spatial(oracle.plaquette_field(p, th), L, Nt)  # [c, k, t, z, y, x]
    ft = f.sum(axis=2)  # time sum of Re / Im P_c
    Pexp = []
    for r in p.r:
        Pexp.append((np.conj(P) * np.roll(P, -r, axis=2)).mean())
    W = np.zeros((len(p.rf), len(p.probes), 6, 2), dtype=complex)
    for a, rf in enumerate(p.rf):
        pp = np.conj(P) * np.roll(P, -rf, axis=2)
        for b, (dy, dz) in enumerate(p.probes):
            for c in range(6):
                if not (p.comp_mask >> c) & 1:
                    continue
                for k in range(2):
                    o = np.roll(ft[c, k], shift=(-dz, -dy, -(rf // 2)), axis=(0, 1, 2))
                    W[a, b, c, k] = (pp * o).sum() / (p.Ns * Nt)
    return np.array(Pexp), W
