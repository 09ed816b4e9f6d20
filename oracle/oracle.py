"""ctypes front end of the FP64 CPU oracle (``ml_oracle.c``).

Test infrastructure only: the test-suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The oracle follows the
multilevel method of Amado, Cardoso & Bicudo (arXiv:1309.3859), Section II
and Algorithm 1; see ``ml_oracle.c`` for the passage each function restates.

Angles use the canonical layout ``theta[mu, i]`` with
``i = x + L*(y + L*(z + L*t))`` and ``mu`` = 0 (t), 1 (x), 2 (y), 3 (z).
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ml_oracle.c")
_LIB = os.path.join(_HERE, "libml_oracle.so")

COMPONENTS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


def build(force: bool = False) -> str:
    """Compile ``ml_oracle.c`` into ``libml_oracle.so`` (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _declare(_lib)
    return _lib


def source() -> str:
    """Text of ``ml_oracle.c`` (the tests compile copies with planted mistakes)."""
    with open(_SRC) as f:
        return f.read()


def build_variant(text: str, path: str) -> str:
    """Compile C source ``text`` (a modified copy of ``ml_oracle.c``) into the
    shared library ``path``, with the oracle's own flags."""
    c = path + ".c"
    with open(c, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", "-o", path, c,
                    "-lm"], check=True)
    return path


@contextlib.contextmanager
def using_library(path: str):
    """Run every oracle function against another build (``build_variant``)."""
    global _lib
    saved = _lib
    L = ctypes.CDLL(path)
    _declare(L)
    _lib = L
    try:
        yield
    finally:
        _lib = saved


class _Params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int), ("Nt", ctypes.c_int), ("beta", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("n_or", ctypes.c_int), ("draws", ctypes.c_int), ("slab", ctypes.c_int), ("n_sub", ctypes.c_int),
        ("outer_slab", ctypes.c_int), ("n_sub_outer", ctypes.c_int), ("k_between", ctypes.c_int),
        ("nr", ctypes.c_int), ("r", ctypes.POINTER(ctypes.c_int)),
        ("nrf", ctypes.c_int), ("rf", ctypes.POINTER(ctypes.c_int)),
        ("nprobe", ctypes.c_int), ("probe_dy", ctypes.POINTER(ctypes.c_int)),
        ("probe_dz", ctypes.POINTER(ctypes.c_int)),
        ("comp_mask", ctypes.c_uint), ("threads", ctypes.c_int),
        ("update", ctypes.c_int), ("metro_hits", ctypes.c_int), ("metro_width", ctypes.c_double),
        ("multihit", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U64 = ctypes.POINTER(ctypes.c_uint64)
_P = ctypes.POINTER(_Params)


def _declare(L):
    L.orc_bessel_i0.argtypes = [ctypes.c_double]
    L.orc_bessel_i0.restype = ctypes.c_double
    L.orc_bessel_i1.argtypes = [ctypes.c_double]
    L.orc_bessel_i1.restype = ctypes.c_double
    L.orc_multihit_link.argtypes = [_P, _D, ctypes.c_int64, _D]
    L.orc_philox_batch.argtypes = [ctypes.c_int64, _U32, _U32, _U32]
    L.orc_uniform52.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    L.orc_uniform52.restype = ctypes.c_double
    L.orc_uniform23.argtypes = [ctypes.c_uint32]
    L.orc_uniform23.restype = ctypes.c_double
    L.orc_vonmises_samples.argtypes = [_P, ctypes.c_double, ctypes.c_int64, _D]
    L.orc_staple.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, ctypes.c_int64, _D, _D]
    L.orc_plaquette_mean.argtypes = [ctypes.c_int, ctypes.c_int, _D]
    L.orc_plaquette_mean.restype = ctypes.c_double
    L.orc_action.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
    L.orc_action.restype = ctypes.c_double
    L.orc_plaquette_field.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
    L.orc_hot_start.argtypes = [_P, _D]
    L.orc_update_pass.argtypes = [_P, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int]
    L.orc_compound_sweep.argtypes = [_P, _D, ctypes.c_int, _U64]
    L.orc_thermalize.argtypes = [_P, _D, _U64, ctypes.c_int]
    L.orc_polyakov.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
    L.orc_naive_correlator.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _D, _D]
    L.orc_record_len.argtypes = [_P]
    L.orc_record_len.restype = ctypes.c_int64
    L.orc_validate.argtypes = [_P]
    L.orc_measure.argtypes = [_P, _D, _U64, ctypes.c_int, _D]
    L.orc_acc_create.argtypes = [_P]
    L.orc_acc_create.restype = ctypes.c_void_p
    L.orc_acc_free.argtypes = [ctypes.c_void_p]
    L.orc_acc_begin.argtypes = [ctypes.c_void_p, _D]
    L.orc_acc_add.argtypes = [ctypes.c_void_p, _D]
    L.orc_acc_end_outer.argtypes = [ctypes.c_void_p]
    L.orc_acc_finish.argtypes = [ctypes.c_void_p, _D]
    L.orc_connected.argtypes = [_P, _D, ctypes.c_int, _D]


@dataclass
class Params:
    """Run parameters (mirrors the oracle's C struct)."""

    L: int
    Nt: int
    beta: float
    seed: int = 1
    n_or: int = 3
    draws: int = 0          # 0: 52-bit uniforms (FP64 stream), 1: 23-bit (FP32 stream)
    slab: int = 2
    n_sub: int = 1
    outer_slab: int = 0
    n_sub_outer: int = 0
    k_between: int = 0
    r: tuple = (1,)
    rf: tuple = ()
    probes: tuple = ()      # ((dy, dz), ...)
    comp_mask: int = 0
    threads: int = 0
    update: int = 0         # first sweep of a compound sweep: 0 heatbath, 1 Metropolis
    metro_hits: int = 1     # Metropolis hits per link visit
    metro_width: float = 1.0  # Metropolis proposal half-width (radians)
    multihit: int = 0       # 1: P(r >= 2) from multihit temporal links
    _keep: list = field(default_factory=list, repr=False)

    @property
    def V(self) -> int:
        return self.L ** 3 * self.Nt

    @property
    def Ns(self) -> int:
        return self.L ** 3

    def c(self) -> _Params:
        r = (ctypes.c_int * max(1, len(self.r)))(*self.r)
        rf = (ctypes.c_int * max(1, len(self.rf)))(*self.rf)
        dy = (ctypes.c_int * max(1, len(self.probes)))(*[p[0] for p in self.probes])
        dz = (ctypes.c_int * max(1, len(self.probes)))(*[p[1] for p in self.probes])
        self._keep[:] = [r, rf, dy, dz]
        return _Params(self.L, self.Nt, float(self.beta), int(self.seed) & (2**64 - 1), self.n_or, self.draws,
                       self.slab, self.n_sub, self.outer_slab, self.n_sub_outer, self.k_between,
                       len(self.r), r, len(self.rf), rf, len(self.probes), dy, dz, self.comp_mask, self.threads,
                       self.update, self.metro_hits, float(self.metro_width), self.multihit)


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


# ----------------------------------------------------------------------------- RNG
def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 blocks for counters ``ctr[n, 4]`` and keys ``key[n, 2]`` (uint32)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    assert ctr.shape[0] == key.shape[0]
    out = np.empty_like(ctr)
    lib().orc_philox_batch(ctr.shape[0], ctr.ctypes.data_as(_U32), key.ctypes.data_as(_U32),
                           out.ctypes.data_as(_U32))
    return out


def uniform52(a: int, b: int) -> float:
    return lib().orc_uniform52(a, b)


def uniform23(a: int) -> float:
    return lib().orc_uniform23(a)


def vonmises_samples(kappa: float, n: int, seed: int = 1, draws: int = 0) -> np.ndarray:
    p = Params(L=2, Nt=2, beta=0.0, seed=seed, draws=draws)
    out = np.empty(n, dtype=np.float64)
    st = lib().orc_vonmises_samples(ctypes.byref(p.c()), kappa, n, _dp(out))
    if st != 0:
        raise RuntimeError(f"von Mises sampler hit its trial cap (status {st})")
    return out


# ----------------------------------------------------------------------------- configurations
def hot_start(p: Params) -> np.ndarray:
    th = np.empty((4, p.V), dtype=np.float64)
    lib().orc_hot_start(ctypes.byref(p.c()), _dp(th))
    return th


def staple(p: Params, th: np.ndarray, mu: int, i: int) -> complex:
    wr, wi = ctypes.c_double(), ctypes.c_double()
    lib().orc_staple(p.L, p.Nt, _dp(th), mu, i, ctypes.byref(wr), ctypes.byref(wi))
    return complex(wr.value, wi.value)


def update_pass(p: Params, th: np.ndarray, mu: int, parity: int, slab_d: int, n: int, kind: int) -> int:
    """One heatbath (kind 0), overrelaxation (kind 1) or Metropolis (kind 2) pass, in place."""
    return lib().orc_update_pass(ctypes.byref(p.c()), _dp(th), mu, parity, slab_d, n, kind)


def compound_sweep(p: Params, th: np.ndarray, counter: int, slab_d: int = 0) -> int:
    """One update sweep (heatbath or Metropolis) + n_or overrelaxation sweeps in place; returns the new sweep
    counter."""
    c = ctypes.c_uint64(counter)
    st = lib().orc_compound_sweep(ctypes.byref(p.c()), _dp(th), slab_d, ctypes.byref(c))
    if st != 0:
        raise RuntimeError(f"oracle sweep failed with status {st}")
    return c.value


def thermalize(p: Params, th: np.ndarray, counter: int, n: int) -> int:
    c = ctypes.c_uint64(counter)
    st = lib().orc_thermalize(ctypes.byref(p.c()), _dp(th), ctypes.byref(c), n)
    if st != 0:
        raise RuntimeError(f"oracle thermalize failed with status {st}")
    return c.value


# ----------------------------------------------------------------------------- observables
def plaquette_mean(p: Params, th: np.ndarray) -> float:
    return lib().orc_plaquette_mean(p.L, p.Nt, _dp(th))


def action(p: Params, th: np.ndarray) -> float:
    return lib().orc_action(p.L, p.Nt, p.beta, _dp(th))


def plaquette_field(p: Params, th: np.ndarray) -> np.ndarray:
    """Re/Im of the six field plaquettes at every site: ``out[c, k, i]``."""
    out = np.empty((6, 2, p.V), dtype=np.float64)
    lib().orc_plaquette_field(p.L, p.Nt, _dp(th), _dp(out))
    return out


def polyakov(p: Params, th: np.ndarray) -> np.ndarray:
    re = np.empty(p.Ns)
    im = np.empty(p.Ns)
    lib().orc_polyakov(p.L, p.Nt, _dp(th), _dp(re), _dp(im))
    return re + 1j * im


def naive_correlator(p: Params, th: np.ndarray, r: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_naive_correlator(p.L, p.Nt, _dp(th), r, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def record_len(p: Params) -> int:
    return lib().orc_record_len(ctypes.byref(p.c()))


def validate(p: Params) -> int:
    return lib().orc_validate(ctypes.byref(p.c()))


def measure(p: Params, th: np.ndarray, counter: int, n_meas: int):
    """``n_meas`` multilevel measurements (Algorithm 1) in place on ``th``.

    Returns ``(records, counter)``; ``records[m]`` has ``record_len(p)`` doubles,
    split by :func:`split_record`.
    """
    n = record_len(p)
    rec = np.zeros((n_meas, n), dtype=np.float64)
    c = ctypes.c_uint64(counter)
    st = lib().orc_measure(ctypes.byref(p.c()), _dp(th), ctypes.byref(c), n_meas, _dp(rec))
    if st != 0:
        raise RuntimeError(f"oracle measure failed with status {st}")
    return rec, c.value


class Accumulator:
    """One multilevel measurement from configurations the caller supplies
    (Algorithm 1's accumulation, level combination and cross-slab products,
    without its sweeps): ``begin(th_first)``, then ``add(th)`` for each
    sub-update configuration (two levels: ``end_outer()`` after every n_sub of
    them), then ``finish()`` returns the record.  ``measure`` runs the same
    functions on its own chain."""

    def __init__(self, p: Params):
        self.p = p
        self._cp = p.c()
        self.h = lib().orc_acc_create(ctypes.byref(self._cp))
        if not self.h:
            raise RuntimeError("oracle accumulator: invalid parameters or out of memory")

    def close(self):
        if self.h:
            lib().orc_acc_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        self.close()

    @staticmethod
    def _th(th):
        return np.ascontiguousarray(th, dtype=np.float64).reshape(4, -1)

    def begin(self, th_first: np.ndarray):
        t = self._th(th_first)
        lib().orc_acc_begin(self.h, _dp(t))

    def add(self, th: np.ndarray):
        t = self._th(th)
        lib().orc_acc_add(self.h, _dp(t))

    def end_outer(self):
        st = lib().orc_acc_end_outer(self.h)
        if st != 0:
            raise RuntimeError("end_outer: one level, or not n_sub configurations since the last call")

    def finish(self) -> np.ndarray:
        rec = np.zeros(record_len(self.p), dtype=np.float64)
        st = lib().orc_acc_finish(self.h, _dp(rec))
        if st != 0:
            raise RuntimeError("finish: the configurations added do not complete a measurement")
        return rec


def measure_configs(p: Params, th_first: np.ndarray, configs) -> np.ndarray:
    """One record from ``th_first`` (naive estimator and plaquette) and the
    sub-update configurations ``configs`` in order (two levels: n_sub_outer
    groups of n_sub)."""
    with Accumulator(p) as acc:
        acc.begin(th_first)
        for k, th in enumerate(configs):
            acc.add(th)
            if p.outer_slab and (k + 1) % p.n_sub == 0:
                acc.end_outer()
        return acc.finish()


def connected(p: Params, recs: np.ndarray) -> np.ndarray:
    """Connected field profile (Section II.C) from records ``recs[n_meas, record_len]``:
    ``out[nrf, nprobe, 6, 4]`` = (F, F^2, jackknife error of F, of F^2)."""
    recs = np.ascontiguousarray(recs, dtype=np.float64).reshape(-1, record_len(p))
    out = np.zeros((max(1, len(p.rf)), max(1, len(p.probes)), 6, 4))
    st = lib().orc_connected(ctypes.byref(p.c()), _dp(recs), recs.shape[0], _dp(out))
    if st != 0:
        raise RuntimeError(f"oracle connected failed with status {st}")
    return out[:len(p.rf), :len(p.probes)]


def split_record(p: Params, rec: np.ndarray) -> dict:
    """Views of a record array ``[..., record_len]``: P, Pf, W, vac, naive, plaq."""
    nr, nrf, npb = len(p.r), len(p.rf), len(p.probes)
    o = 0
    P = rec[..., o:o + 2 * nr].reshape(rec.shape[:-1] + (nr, 2))
    o += 2 * nr
    Pf = rec[..., o:o + 2 * nrf].reshape(rec.shape[:-1] + (nrf, 2))
    o += 2 * nrf
    W = rec[..., o:o + nrf * npb * 24].reshape(rec.shape[:-1] + (nrf, npb, 6, 2, 2))
    o += nrf * npb * 24
    vac = rec[..., o:o + 12].reshape(rec.shape[:-1] + (6, 2))
    o += 12
    naive = rec[..., o:o + 2 * nr].reshape(rec.shape[:-1] + (nr, 2))
    o += 2 * nr
    plaq = rec[..., o]
    return {"P": P, "Pf": Pf, "W": W, "vac": vac, "naive": naive, "plaq": plaq}


def bessel_i0(x: float) -> float:
    return lib().orc_bessel_i0(float(x))


def bessel_i1(x: float) -> float:
    return lib().orc_bessel_i1(float(x))


def multihit_link(p: Params, th: np.ndarray, i: int) -> complex:
    """Multihit mean e^{-i alpha} I1(beta k) / I0(beta k) of the temporal link at site i."""
    out = np.zeros(2)
    lib().orc_multihit_link(ctypes.byref(p.c()), _dp(th), int(i), _dp(out))
    return complex(out[0], out[1])
