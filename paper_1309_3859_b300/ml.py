"""Python binding of ``libml.so`` (include/ml.h): argument marshalling only.

Every step of the multilevel path runs in the library's CUDA kernels; this
module converts Python arguments to the C ABI, supplies PyTorch's caching
allocator and a PyTorch stream, and raises :class:`MLError` on a non-zero
status.  There is no CPU fallback: without the built library or a CUDA
device the calls fail.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

ML_OK, ML_EINVAL, ML_ENOMEM, ML_ECUDA, ML_ETIMEOUT, ML_EREJECT, ML_EBUSY, ML_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
ML_FP64, ML_FP32 = 0, 1
ML_SWEEP_PERSISTENT, ML_SWEEP_PASSES, ML_SWEEP_RESIDENT = 0, 1, 2
ML_FOLD_SITE, ML_FOLD_TILE = 0, 1
ML_UPDATE_HEATBATH, ML_UPDATE_METROPOLIS = 0, 1
ML_PART_LINKS, ML_PART_SLAB_SUMS, ML_PART_VACUUM, ML_PART_W_SUMS = 0, 1, 2, 3
(ML_K_HEATBATH, ML_K_OVERRELAX, ML_K_RECORD, ML_K_ACCUMULATE, ML_K_PRODUCTS, ML_K_SWEEP, ML_K_SUBUPDATE,
 ML_K_FULLSWEEP) = range(8)
(ML_TL_FULL_BEGIN, ML_TL_FULL_END, ML_TL_SUB_BEGIN, ML_TL_SUB_END, ML_TL_FOLD_BEGIN, ML_TL_FOLD_END,
 ML_TL_PROD_BEGIN, ML_TL_PROD_END) = range(8)
COMPONENTS = ("Ex", "Ey", "Ez", "Bx", "By", "Bz")


class MLError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib.ml_error_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


class _Offset(ctypes.Structure):
    _fields_ = [("dy", ctypes.c_int), ("dz", ctypes.c_int)]


class _Params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int), ("Nt", ctypes.c_int), ("beta", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("prec", ctypes.c_int), ("n_or", ctypes.c_int), ("slab", ctypes.c_int), ("n_sub", ctypes.c_int),
        ("outer_slab", ctypes.c_int), ("n_sub_outer", ctypes.c_int), ("k_between", ctypes.c_int),
        ("nr", ctypes.c_int), ("r", ctypes.POINTER(ctypes.c_int)),
        ("nrf", ctypes.c_int), ("rf", ctypes.POINTER(ctypes.c_int)),
        ("nprobe", ctypes.c_int), ("probe", ctypes.POINTER(_Offset)),
        ("comp_mask", ctypes.c_uint32),
        ("update", ctypes.c_int), ("metro_hits", ctypes.c_int), ("metro_width", ctypes.c_double),
        ("multihit", ctypes.c_int), ("replay", ctypes.c_int), ("pair_sums", ctypes.c_int),
    ]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


_D = ctypes.POINTER(ctypes.c_double)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_H = ctypes.c_void_p

# name -> (restype, argtypes) for every entry point declared in include/ml.h
SIGNATURES = {
    "ml_create": (ctypes.c_int, [ctypes.POINTER(_Params), ctypes.POINTER(_Allocator), ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_void_p)]),
    "ml_destroy": (ctypes.c_int, [_H]),
    "ml_thermalize": (ctypes.c_int, [_H, ctypes.c_int]),
    "ml_measure": (ctypes.c_int, [_H, ctypes.c_int, _D, ctypes.c_size_t]),
    "ml_measure_device": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "ml_record_len": (ctypes.c_int, [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_size_t)]),
    "ml_connected_device": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "ml_get_angles": (ctypes.c_int, [_H, _D, ctypes.c_size_t]),
    "ml_set_angles": (ctypes.c_int, [_H, _D, ctypes.c_size_t]),
    "ml_get_sweep": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_uint64)]),
    "ml_set_sweep": (ctypes.c_int, [_H, ctypes.c_uint64]),
    "ml_update_pass": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int]),
    "ml_compound_sweeps": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int]),
    "ml_observe": (ctypes.c_int, [_H, _D, ctypes.c_size_t]),
    "ml_sync": (ctypes.c_int, [_H]),
    "ml_philox": (ctypes.c_int, [_U32, _U32, ctypes.c_size_t, _U32]),
    "ml_check_rounding": (ctypes.c_int, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "ml_kernel_timing": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "ml_timeline_enable": (ctypes.c_int, [_H, ctypes.c_int]),
    "ml_resident_profile": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "ml_timeline_read": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ml_batch_slots": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int)]),
    "ml_sweep_mode": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int)]),
    "ml_set_sweep_mode": (ctypes.c_int, [_H, ctypes.c_int]),
    "ml_fold_mode": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int)]),
    "ml_set_fold_mode": (ctypes.c_int, [_H, ctypes.c_int]),
    "ml_naive_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "ml_batch_create": (ctypes.c_int, [ctypes.POINTER(_Params), ctypes.c_int, ctypes.POINTER(_Allocator),
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "ml_batch_destroy": (ctypes.c_int, [_H]),
    "ml_batch_size": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int)]),
    "ml_batch_thermalize": (ctypes.c_int, [_H, ctypes.c_int]),
    "ml_batch_result_len": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "ml_batch_record_offset": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "ml_batch_measure": (ctypes.c_int, [_H, ctypes.c_int, _D, ctypes.c_size_t]),
    "ml_batch_measure_device": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "ml_batch_get_angles": (ctypes.c_int, [_H, ctypes.c_int, _D, ctypes.c_size_t]),
    "ml_batch_sync": (ctypes.c_int, [_H]),
    "ml_batch_sweep_mode": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int)]),
    "ml_batch_set_sweep_mode": (ctypes.c_int, [_H, ctypes.c_int]),
    "ml_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "ml_submit": (ctypes.c_int, [_H, ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_uint64)]),
    "ml_poll": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), _D, ctypes.c_size_t]),
    "ml_wait": (ctypes.c_int, [_H, ctypes.c_uint64, ctypes.c_double]),
    "ml_job_times": (ctypes.c_int, [_H, ctypes.c_uint64, _D, _D, _D]),
    "ml_job_release": (ctypes.c_int, [_H, ctypes.c_uint64]),
    "ml_server_stats": (ctypes.c_int, [_H, ctypes.c_void_p]),
    "ml_server_destroy": (ctypes.c_int, [_H]),
    "ml_set_time_range": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int]),
    "ml_part_size": (ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "ml_part_copy": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_int]),
    "ml_measure_inner": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
    "ml_measure_products": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "ml_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ml_kernel_launches": (ctypes.c_uint64, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load ``libml.so`` (building it with nvcc first when it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing and _build.stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is not built; run paper_1309_3859_b300.build.build()")
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != ML_OK:
        raise MLError(status, what)


@dataclass
class Params:
    """Run parameters of one lattice (mirrors ``ml_params``)."""

    L: int
    Nt: int
    beta: float
    seed: int = 1
    fp64: bool = True
    n_or: int = 3
    slab: int = 2
    n_sub: int = 1
    outer_slab: int = 0
    n_sub_outer: int = 0
    k_between: int = 0
    r: tuple = (1,)
    rf: tuple = ()
    probes: tuple = ()
    comp_mask: int = 0
    update: int = 0           # ML_UPDATE_HEATBATH or ML_UPDATE_METROPOLIS
    metro_hits: int = 1
    metro_width: float = 1.0
    multihit: int = 0         # 1: P(r) at 2 <= r <= L-2 from multihit temporal links
    replay: int = 0           # 1: field insertions by replay of the inner loop (one level)
    pair_sums: int = 0        # 1 (FP32 only): float-pair slab sums instead of double precision
    _keep: list = field(default_factory=list, repr=False, compare=False)

    @property
    def V(self) -> int:
        return self.L ** 3 * self.Nt

    @property
    def Ns(self) -> int:
        return self.L ** 3

    def c(self) -> _Params:
        r = (ctypes.c_int * max(1, len(self.r)))(*self.r)
        rf = (ctypes.c_int * max(1, len(self.rf)))(*self.rf)
        pr = (_Offset * max(1, len(self.probes)))(*[_Offset(int(a), int(b)) for a, b in self.probes])
        self._keep[:] = [r, rf, pr]
        return _Params(self.L, self.Nt, float(self.beta), int(self.seed) & (2 ** 64 - 1),
                       ML_FP64 if self.fp64 else ML_FP32, self.n_or, self.slab, self.n_sub, self.outer_slab,
                       self.n_sub_outer, self.k_between, len(self.r), r, len(self.rf), rf, len(self.probes), pr,
                       self.comp_mask, self.update, self.metro_hits, float(self.metro_width), self.multihit,
                       self.replay, self.pair_sums)

    @classmethod
    def from_workload(cls, w, **kw) -> "Params":
        d = dict(L=w.L, Nt=w.Nt, beta=w.beta, seed=w.seed, fp64=w.fp64, n_or=w.n_or, slab=w.slab, n_sub=w.n_sub,
                 outer_slab=w.outer_slab, n_sub_outer=w.n_sub_outer, k_between=w.k_between, r=tuple(w.r),
                 rf=tuple(w.rf), probes=tuple(w.probes), comp_mask=w.comp_mask)
        d.update(kw)
        return cls(**d)


def record_len(p: Params) -> int:
    n = ctypes.c_size_t()
    _check(lib().ml_record_len(ctypes.byref(p.c()), ctypes.byref(n)), "ml_record_len")
    return n.value


def split_record(p: Params, rec: np.ndarray) -> dict:
    """Views of records ``[..., record_len]`` by block: P, Pf, W, vac, naive, plaq."""
    nr, nrf, npb = len(p.r), len(p.rf), len(p.probes)
    sizes = [("P", 2 * nr, (nr, 2)), ("Pf", 2 * nrf, (nrf, 2)), ("W", 24 * nrf * npb, (nrf, npb, 6, 2, 2)),
             ("vac", 12, (6, 2)), ("naive", 2 * nr, (nr, 2)), ("plaq", 1, ())]
    out, o = {}, 0
    lead = rec.shape[:-1]
    for name, n, shape in sizes:
        out[name] = rec[..., o:o + n].reshape(lead + shape)
        o += n
    return out


def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 blocks evaluated on the device."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    _check(lib().ml_philox(ctr.ctypes.data_as(_U32), key.ctypes.data_as(_U32), ctr.shape[0],
                           out.ctypes.data_as(_U32)), "ml_philox")
    return out


def check_rounding() -> list:
    """Mismatch counts of the FP32 update's own rounding and uniforms against
    the conversions they replace (ml_check_rounding): rint, floor, 23-bit and
    52-bit uniforms."""
    out = (ctypes.c_ulonglong * 4)()
    _check(lib().ml_check_rounding(out), "ml_check_rounding")
    return [int(v) for v in out]


def kernel_launches() -> int:
    return int(lib().ml_kernel_launches())


class Lattice:
    """One lattice resident on the GPU (``ml_create`` ... ``ml_destroy``).

    Device memory comes from PyTorch's caching allocator and all work runs on
    a dedicated PyTorch stream (``self.stream``)."""

    def __init__(self, p: Params, stream=None, device=None):
        import torch

        self.p = p
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        # high priority: the sweeps own the critical path, folds fill the SMs they leave
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device, priority=-100)
        self._cb, self._alloc = _torch_allocator(torch, self.device, self.stream)
        st = self.stream
        self._cp = p.c()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().ml_create(ctypes.byref(self._cp), ctypes.byref(self._alloc),
                                   ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)), "ml_create")
        self.h = h
        self.rec_len = record_len(p)

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            _check(lib().ml_destroy(self.h), "ml_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- Algorithm 1
    def thermalize(self, n: int):
        _check(lib().ml_thermalize(self.h, int(n)), "ml_thermalize")

    def measure(self, n_meas: int) -> np.ndarray:
        out = np.zeros((n_meas, self.rec_len), dtype=np.float64)
        _check(lib().ml_measure(self.h, int(n_meas), out.ctypes.data_as(_D), out.size), "ml_measure")
        return out

    def measure_device(self, n_meas: int, out=None):
        """Enqueue measurements whose records stay in a device tensor.

        The work runs on ``self.stream``; wait for it (``sync()`` or
        ``torch.cuda.current_stream().wait_stream(self.stream)``) before
        reading the tensor on another stream."""
        torch = self._torch
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty((n_meas, self.rec_len), dtype=torch.float64, device=self.device)
        assert out.is_cuda and out.dtype == torch.float64 and out.is_contiguous()
        _check(lib().ml_measure_device(self.h, int(n_meas), ctypes.c_void_p(out.data_ptr()), out.numel()),
               "ml_measure_device")
        return out

    def connected(self, records_dev):
        """Connected F and F^2 profile [nrf][nprobe][6][2] from device records."""
        torch = self._torch
        with torch.cuda.stream(self.stream):
            out = torch.empty((len(self.p.rf), len(self.p.probes), 6, 2), dtype=torch.float64, device=self.device)
        _check(lib().ml_connected_device(self.h, ctypes.c_void_p(records_dev.data_ptr()), records_dev.shape[0],
                                         ctypes.c_void_p(out.data_ptr()), out.numel()), "ml_connected_device")
        return out

    def observe(self) -> np.ndarray:
        out = np.zeros(self.rec_len, dtype=np.float64)
        _check(lib().ml_observe(self.h, out.ctypes.data_as(_D), out.size), "ml_observe")
        return out

    # -- configuration access
    def get_angles(self) -> np.ndarray:
        out = np.empty((4, self.p.V), dtype=np.float64)
        _check(lib().ml_get_angles(self.h, out.ctypes.data_as(_D), out.size), "ml_get_angles")
        return out

    def set_angles(self, theta: np.ndarray):
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(4, self.p.V)
        _check(lib().ml_set_angles(self.h, th.ctypes.data_as(_D), th.size), "ml_set_angles")

    @property
    def sweep(self) -> int:
        n = ctypes.c_uint64()
        _check(lib().ml_get_sweep(self.h, ctypes.byref(n)), "ml_get_sweep")
        return n.value

    @sweep.setter
    def sweep(self, n: int):
        _check(lib().ml_set_sweep(self.h, int(n)), "ml_set_sweep")

    def update_pass(self, mu: int, parity: int, slab_d: int, n: int, kind: int):
        _check(lib().ml_update_pass(self.h, mu, parity, slab_d, int(n), kind), "ml_update_pass")

    def compound_sweeps(self, n: int, slab_d: int = 0):
        _check(lib().ml_compound_sweeps(self.h, int(n), int(slab_d)), "ml_compound_sweeps")

    def resident_profile(self) -> dict:
        """SM clock cycles of one cluster-resident launch by phase
        (ml_resident_profile): own updates and exchange per pass of each
        class, record per sub-update, set-up, write-back, whole launch."""
        n = 14
        out = (ctypes.c_double * n)()
        _check(lib().ml_resident_profile(self.h, out, n), "ml_resident_profile")
        cls = ("heatbath_t", "heatbath_s", "overrelax_t", "overrelax_s")
        d = {f"update_{c}": out[i] for i, c in enumerate(cls)}
        d.update({f"exchange_{c}": out[4 + i] for i, c in enumerate(cls)})
        d.update(record=out[8], setup=out[9], write_back=out[10], launch=out[11], sub_updates=int(out[12]),
                 ctas=int(out[13]))
        return d

    def timeline_enable(self, capacity: int):
        """Record up to `capacity` launch marks of the measurement schedule
        (ml_timeline_enable; 0 turns it off)."""
        _check(lib().ml_timeline_enable(self.h, int(capacity)), "ml_timeline_enable")

    def timeline(self, cap: int = 1 << 16) -> list:
        """The marks recorded so far as (ML_TL_* tag, ms after the first mark),
        in recording order (ml_timeline_read); they are then discarded."""
        tags = (ctypes.c_int * cap)()
        ms = (ctypes.c_float * cap)()
        n = ctypes.c_int()
        _check(lib().ml_timeline_read(self.h, tags, ms, int(cap), ctypes.byref(n)), "ml_timeline_read")
        return [(tags[i], ms[i]) for i in range(n.value)]

    def kernel_ms(self, kernel: int, reps: int = 20) -> float:
        """Average event-timed duration of one kernel class (ml_kernel_timing)."""
        ms = ctypes.c_double()
        _check(lib().ml_kernel_timing(self.h, int(kernel), int(reps), ctypes.byref(ms)), "ml_kernel_timing")
        return ms.value

    @property
    def sweep_mode(self) -> int:
        m = ctypes.c_int()
        _check(lib().ml_sweep_mode(self.h, ctypes.byref(m)), "ml_sweep_mode")
        return m.value

    @sweep_mode.setter
    def sweep_mode(self, mode: int):
        _check(lib().ml_set_sweep_mode(self.h, int(mode)), "ml_set_sweep_mode")

    @property
    def fold_mode(self) -> int:
        m = ctypes.c_int()
        _check(lib().ml_fold_mode(self.h, ctypes.byref(m)), "ml_fold_mode")
        return m.value

    @fold_mode.setter
    def fold_mode(self, mode: int):
        _check(lib().ml_set_fold_mode(self.h, int(mode)), "ml_set_fold_mode")

    @property
    def batch_slots(self) -> int:
        n = ctypes.c_int()
        _check(lib().ml_batch_slots(self.h, ctypes.byref(n)), "ml_batch_slots")
        return n.value

    def sync(self):
        _check(lib().ml_sync(self.h), "ml_sync")

    # -- time-slab partition (ml_set_time_range ... ml_measure_products)
    def set_time_range(self, t_lo: int, t_hi: int):
        _check(lib().ml_set_time_range(self.h, int(t_lo), int(t_hi)), "ml_set_time_range")

    def part_size(self, what: int) -> int:
        n = ctypes.c_size_t()
        _check(lib().ml_part_size(self.h, int(what), ctypes.byref(n)), "ml_part_size")
        return n.value

    def part_read(self, what: int, begin: int, count: int, mu: int = 0, parity: int = 0):
        """Units [begin, begin + count) of a partition block as a new uint8 device tensor."""
        torch = self._torch
        with torch.cuda.stream(self.stream):
            buf = torch.empty(count * self.part_size(what), dtype=torch.uint8, device=self.device)
        _check(lib().ml_part_copy(self.h, int(what), int(mu), int(parity), int(begin), int(count),
                                  ctypes.c_void_p(buf.data_ptr()), 0), "ml_part_copy")
        # the copy is on the lattice's stream: work the caller queues on its
        # current stream waits for it, and the memory is kept until then
        cur = torch.cuda.current_stream(self.device)
        cur.wait_stream(self.stream)
        buf.record_stream(cur)
        return buf

    def part_write(self, what: int, begin: int, count: int, buf, mu: int = 0, parity: int = 0):
        """Copy a uint8 device tensor into units [begin, begin + count) of a partition block."""
        assert buf.is_cuda and buf.is_contiguous() and buf.numel() == count * self.part_size(what)
        self.stream.wait_stream(self._torch.cuda.current_stream(self.device))
        buf.record_stream(self.stream)  # its memory is not reused before the copy is done
        _check(lib().ml_part_copy(self.h, int(what), int(mu), int(parity), int(begin), int(count),
                                  ctypes.c_void_p(buf.data_ptr()), 1), "ml_part_copy")

    def measure_inner(self, rec):
        assert rec.is_cuda and rec.dtype == self._torch.float64 and rec.numel() >= self.rec_len
        _check(lib().ml_measure_inner(self.h, ctypes.c_void_p(rec.data_ptr()), rec.numel()), "ml_measure_inner")

    def measure_products(self, w_in=None, w_out=None, rec=None):
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        if w_in is not None:
            self.stream.wait_stream(self._torch.cuda.current_stream(self.device))
            w_in.record_stream(self.stream)
        _check(lib().ml_measure_products(self.h, ptr(w_in), ptr(w_out), ptr(rec),
                                         rec.numel() if rec is not None else 0), "ml_measure_products")


def _torch_allocator(torch, dev, st):
    def _alloc(size, ctx):
        return torch.cuda.caching_allocator_alloc(int(size), dev, st)

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    cb = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    return cb, _Allocator(cb[0], cb[1], None)


class Batch:
    """Independent lattices advanced together (``ml_batch_*``).

    All parameter sets must share one schedule (precision, n_or, slab,
    outer_slab, n_sub, n_sub_outer, k_between)."""

    def __init__(self, params, stream=None, device=None):
        import torch

        self.params = list(params)
        self._torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        # high priority: the sweeps own the critical path, folds fill the SMs they leave
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device, priority=-100)
        self._cb, self._alloc = _torch_allocator(torch, self.device, self.stream)
        arr = (_Params * len(self.params))(*[p.c() for p in self.params])
        self._arr = arr
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().ml_batch_create(arr, len(self.params), ctypes.byref(self._alloc),
                                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "ml_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _check(lib().ml_batch_destroy(self.h), "ml_batch_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.params)

    def thermalize(self, n: int):
        _check(lib().ml_batch_thermalize(self.h, int(n)), "ml_batch_thermalize")

    def result_len(self, n_meas: int) -> int:
        n = ctypes.c_size_t()
        _check(lib().ml_batch_result_len(self.h, int(n_meas), ctypes.byref(n)), "ml_batch_result_len")
        return n.value

    def offsets(self, n_meas: int):
        out = []
        for i in range(len(self.params)):
            o = ctypes.c_size_t()
            _check(lib().ml_batch_record_offset(self.h, i, int(n_meas), ctypes.byref(o)), "ml_batch_record_offset")
            out.append(o.value)
        return out

    def split(self, flat: np.ndarray, n_meas: int):
        """Per-lattice record arrays [n_meas][record_len] from a batch output."""
        offs = self.offsets(n_meas) + [flat.shape[-1]]
        return [flat[..., offs[i]:offs[i + 1]].reshape(flat.shape[:-1] + (n_meas, -1))
                for i in range(len(self.params))]

    def measure(self, n_meas: int):
        flat = np.zeros(self.result_len(n_meas), dtype=np.float64)
        _check(lib().ml_batch_measure(self.h, int(n_meas), flat.ctypes.data_as(_D), flat.size), "ml_batch_measure")
        return self.split(flat, n_meas)

    def measure_device(self, n_meas: int, out=None):
        torch = self._torch
        if out is None:
            with torch.cuda.stream(self.stream):
                out = torch.empty(self.result_len(n_meas), dtype=torch.float64, device=self.device)
        _check(lib().ml_batch_measure_device(self.h, int(n_meas), ctypes.c_void_p(out.data_ptr()), out.numel()),
               "ml_batch_measure_device")
        return out

    def get_angles(self, i: int) -> np.ndarray:
        p = self.params[i]
        out = np.empty((4, p.V), dtype=np.float64)
        _check(lib().ml_batch_get_angles(self.h, int(i), out.ctypes.data_as(_D), out.size), "ml_batch_get_angles")
        return out

    @property
    def sweep_mode(self) -> int:
        m = ctypes.c_int()
        _check(lib().ml_batch_sweep_mode(self.h, ctypes.byref(m)), "ml_batch_sweep_mode")
        return m.value

    @sweep_mode.setter
    def sweep_mode(self, mode: int):
        _check(lib().ml_batch_set_sweep_mode(self.h, int(mode)), "ml_batch_set_sweep_mode")

    def sync(self):
        _check(lib().ml_batch_sync(self.h), "ml_batch_sync")


class _ServerConfig(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("n_or", ctypes.c_int), ("budget_bytes", ctypes.c_size_t),
                ("max_active", ctypes.c_int), ("lanes", ctypes.c_int)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("active", ctypes.c_int), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("ticks", ctypes.c_uint64), ("budget_bytes", ctypes.c_size_t),
                ("used_bytes", ctypes.c_size_t)]


class Server:
    """Request server with continuous batching (``ml_server_*``, ``ml_submit``)."""

    def __init__(self, budget_bytes: int, fp64: bool = False, n_or: int = 3, max_active: int = 0, lanes: int = 0):
        import torch

        torch.cuda.init()
        cfg = _ServerConfig(ML_FP64 if fp64 else ML_FP32, n_or, int(budget_bytes), int(max_active), int(lanes))
        h = ctypes.c_void_p()
        _check(lib().ml_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ml_server_create")
        self.h = h
        self._params = {}

    def submit(self, p: Params, n_therm: int, n_meas: int) -> int:
        job = ctypes.c_uint64()
        _check(lib().ml_submit(self.h, ctypes.byref(p.c()), int(n_therm), int(n_meas), ctypes.byref(job)),
               "ml_submit")
        self._params[job.value] = (p, n_meas)
        return job.value

    def poll(self, job: int):
        """(done, records or None)"""
        p, n_meas = self._params[job]
        out = np.zeros((n_meas, record_len(p)), dtype=np.float64)
        done = ctypes.c_int()
        _check(lib().ml_poll(self.h, job, ctypes.byref(done), out.ctypes.data_as(_D), out.size), "ml_poll")
        return (True, out) if done.value else (False, None)

    def wait(self, job: int, timeout_s: float = 600.0):
        _check(lib().ml_wait(self.h, job, float(timeout_s)), "ml_wait")
        return self.poll(job)[1]

    def times(self, job: int):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().ml_job_times(self.h, job, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "ml_job_times")
        return a.value, b.value, c.value

    def release(self, job: int):
        _check(lib().ml_job_release(self.h, job), "ml_job_release")
        self._params.pop(job, None)

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().ml_server_stats(self.h, ctypes.byref(st)), "ml_server_stats")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            _check(lib().ml_server_destroy(self.h), "ml_server_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
