"""Time-slab partition of one lattice over the processes of a
``torch.distributed`` group (one GPU each).

Section II.C of arXiv:1309.3859: with the spatial links on the slab
boundaries frozen, the sub-updates of different time slabs are independent.
So each of R processes owns a contiguous range of time slices (a whole number
of top-level slabs), holds a copy of the whole lattice, and moves only its own
links.  One measurement (Algorithm 1) runs as:

1. k0 full compound sweeps pass by pass, from a halo refreshed in every
   direction (the previous measurement's sub-updates moved the neighbours'
   boundary links); after every (direction, parity) pass each process sends
   the moved links of its first and last slice to its two neighbours, which
   need them in the staples of their boundary links;
2. the owned slices of every process are gathered into every copy;
3. ``ml_measure_inner``: the naive correlator and plaquette of that
   configuration, then the slab sub-updates, records and folds of the owned
   slabs with no communication at all;
4. the top-level [T] slab sums of all processes gathered into every copy
   (each process's products multiply by the other slabs' averages), the
   vacuum block sums into the last process;
5. ``ml_measure_products`` in process order: each adds its slabs' field
   insertions to the per-site sums it receives and sends them on; the last
   completes the record, which is then broadcast.

The records equal those of one process bit for bit (the library adds the same
terms in the same order).  Every exchange goes through ``torch.distributed``:
with the gloo backend the buffers are staged through host memory, with NCCL
they stay on the device.  No kernel of one process waits on another process;
all waiting is on the host.

The lattice object only needs the methods of ``ml.Lattice`` used below, so
the communication plan can be exercised on the CPU with a stand-in.
"""

from __future__ import annotations

import numpy as np

from . import ml


class SlabPartition:
    """One lattice split by time slices over the ranks of ``group``.

    ``lat`` is this rank's copy of the whole lattice (an ``ml.Lattice`` made
    from ``p``); the constructor restricts it to the rank's slices."""

    def __init__(self, lat, p: ml.Params, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.p = p
        self.lat = lat
        top = p.outer_slab or p.slab
        if p.Nt % (self.world * top) != 0:
            raise ValueError(f"Nt = {p.Nt} is not a multiple of {self.world} ranks x slab thickness {top}")
        per = p.Nt // self.world
        self.t_lo, self.t_hi = self.rank * per, (self.rank + 1) * per
        self.top = top
        self.n_top = p.Nt // top                 # top-level slabs
        self.n_inner = p.Nt // p.slab            # inner slabs
        self.staged = self.world > 1 and dist.get_backend(group) == "gloo"
        if self.world > 1:
            lat.set_time_range(self.t_lo, self.t_hi)

    # ------------------------------------------------------------------ comm
    def _out(self, t):
        """A tensor as the backend sends it (gloo: host memory)."""
        self.lat.sync()
        return t.cpu() if self.staged else t

    def _buffer(self, like_bytes):
        import torch

        dev = "cpu" if self.staged else self.lat.device
        return torch.empty(like_bytes, dtype=torch.uint8, device=dev)

    def _in(self, t):
        """A received tensor as the lattice takes it (its device)."""
        return t.to(self.lat.device) if self.staged else t

    def _global(self, r):
        return self.dist.get_global_rank(self.group, r) if self.group is not None else r

    # ------------------------------------------------------------------ sweeps
    def _exchange_halo(self, mu: int, parity: int):
        """After pass (mu, parity): the moved links of the first and last owned
        slice go to the neighbouring ranks, whose boundary staples read them;
        this rank's halo slices t_lo - 1 and t_hi come back."""
        if self.world == 1:
            return
        lat, L = self.lat, ml.ML_PART_LINKS
        Nt = self.p.Nt
        lower, upper = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        first = self._out(lat.part_read(L, self.t_lo, 1, mu, parity))
        last = self._out(lat.part_read(L, self.t_hi - 1, 1, mu, parity))
        from_lower, from_upper = self._buffer(first.numel()), self._buffer(first.numel())
        reqs = [self.dist.isend(first, self._global(lower), group=self.group, tag=0),
                self.dist.isend(last, self._global(upper), group=self.group, tag=1),
                self.dist.irecv(from_upper, self._global(upper), group=self.group, tag=0),
                self.dist.irecv(from_lower, self._global(lower), group=self.group, tag=1)]
        for r in reqs:
            r.wait()
        lat.part_write(L, (self.t_lo - 1) % Nt, 1, self._in(from_lower), mu, parity)
        lat.part_write(L, self.t_hi % Nt, 1, self._in(from_upper), mu, parity)

    def refresh_halo(self):
        """The neighbours' boundary slices of every direction and parity.  The
        per-pass exchange keeps them current only through sweeps; the slab
        sub-updates of a measurement move the neighbours' boundary links
        (temporal links, spatial links inside their slabs) without any
        exchange, so the next sweeps start from a refreshed halo."""
        for mu in range(4):
            for parity in (0, 1):
                self._exchange_halo(mu, parity)

    def sweeps(self, n: int):
        """n full compound sweeps (one update sweep + n_or overrelaxation
        sweeps, no frozen links), the halo exchanged after every pass."""
        if n > 0:
            self.refresh_halo()
        for _ in range(n):
            nsw = self.lat.sweep + 1  # heatbath sweep number of this compound sweep
            for kind in [0] + [1] * self.p.n_or:
                for mu in range(4):
                    for parity in (0, 1):
                        self.lat.update_pass(mu, parity, 0, nsw, kind)
                        self._exchange_halo(mu, parity)
            self.lat.sweep = nsw

    def gather_configuration(self):
        """Every copy receives the owned slices of every rank."""
        if self.world == 1:
            return
        import torch

        lat, L = self.lat, ml.ML_PART_LINKS
        per = self.t_hi - self.t_lo
        own = torch.cat([lat.part_read(L, self.t_lo, per, mu, parity) for mu in range(4) for parity in (0, 1)])
        own = self._out(own)
        parts = [self._buffer(own.numel()) for _ in range(self.world)]
        self.dist.all_gather(parts, own, group=self.group)
        unit = own.numel() // 8
        for r, blob in enumerate(parts):
            if r == self.rank:
                continue
            blob = self._in(blob)
            for k, (mu, parity) in enumerate((m, q) for m in range(4) for q in (0, 1)):
                lat.part_write(L, r * per, per, blob[k * unit:(k + 1) * unit].contiguous(), mu, parity)

    # ------------------------------------------------------------------ measurement
    def _gather(self, what: int, units_per_rank: int, everywhere: bool):
        """Units of block `what` owned by each rank into every copy
        (everywhere) or into the last rank's."""
        lat = self.lat
        own = self._out(lat.part_read(what, self.rank * units_per_rank, units_per_rank))
        parts = [self._buffer(own.numel()) for _ in range(self.world)]
        self.dist.all_gather(parts, own, group=self.group)
        if everywhere or self.rank == self.world - 1:
            for r, blob in enumerate(parts):
                if r != self.rank:
                    lat.part_write(what, r * units_per_rank, units_per_rank, self._in(blob))

    def measure(self, n_meas: int) -> np.ndarray:
        """n_meas measurements; every rank returns the records [n_meas][rec_len]."""
        import torch

        lat = self.lat
        out = np.zeros((n_meas, lat.rec_len))
        for m in range(n_meas):
            self.sweeps(self.p.k_between)
            self.gather_configuration()
            with torch.cuda.stream(lat.stream):
                rec = torch.zeros(lat.rec_len, dtype=torch.float64, device=lat.device)
            lat.measure_inner(rec)
            if self.world == 1:
                lat.measure_products(rec=rec)
                lat.sync()
                out[m] = rec.cpu().numpy()
                continue
            # every rank's products take the other slabs' [T] (prod over s' != s)
            self._gather(ml.ML_PART_SLAB_SUMS, self.n_top // self.world, everywhere=True)
            self._gather(ml.ML_PART_VACUUM, self.n_inner // self.world, everywhere=False)
            nbytes = lat.part_size(ml.ML_PART_W_SUMS)
            w_in = None
            if self.rank > 0:
                buf = self._buffer(nbytes)
                self.dist.recv(buf, self._global(self.rank - 1), group=self.group)
                w_in = self._in(buf)
            if self.rank < self.world - 1:
                with torch.cuda.stream(lat.stream):
                    w_out = torch.empty(nbytes, dtype=torch.uint8, device=lat.device)
                lat.measure_products(w_in=w_in, w_out=w_out)
                self.dist.send(self._out(w_out), self._global(self.rank + 1), group=self.group)
            else:
                lat.measure_products(w_in=w_in, rec=rec)
            lat.sync()
            r = rec.cpu() if self.staged else rec
            self.dist.broadcast(r, self._global(self.world - 1), group=self.group)
            out[m] = r.cpu().numpy()
        return out
