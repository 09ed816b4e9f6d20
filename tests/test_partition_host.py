"""The communication plan of the time-slab partition on the CPU: two gloo
ranks driving a stand-in lattice must end with the same records and the same
configuration as one rank.

The stand-in keeps a small float64 array per (direction, parity, time slice)
and mimics the dependencies of the real lattice: a link update reads links
of other directions on the neighbouring slices t - 1 and t + 1 (so a missing
or misplaced halo exchange changes the chain), slab sub-updates read only
their own slices and the frozen boundary slice above them, the slab sums and
vacuum block sums are per slab, and the products add per-slab terms to
per-site sums in slab order, taking every slab's [T] sums.  Any mistake in
which slice goes to which neighbour, in the gather offsets or in the
pipeline order changes the result.
"""

import os
import socket

import numpy as np
import pytest
import torch

from paper_1309_3859_b300 import ml

S = 5  # values per slice of one (direction, parity) array


class FakeLattice:
    device = "cpu"
    stream = None

    def __init__(self, p):
        self.p = p
        self.Nt = p.Nt
        self.top = p.outer_slab or p.slab
        self.n_top = p.Nt // self.top
        self.n_inner = p.Nt // p.slab
        i = torch.arange(4 * 2 * p.Nt * S, dtype=torch.float64).reshape(4, 2, p.Nt, S)
        self.links = torch.sin(0.37 * i + 0.1)
        self.t_lo, self.t_hi = 0, p.Nt
        self.sweep = 0
        self.T = torch.zeros(self.n_top, S, dtype=torch.float64)
        self.vac = torch.zeros(self.n_inner, 2, dtype=torch.float64)
        self.rec_len = 4

    # -- the interface the partition uses
    def sync(self):
        pass

    def set_time_range(self, lo, hi):
        self.t_lo, self.t_hi = lo, hi

    def _new(self, mu, parity, t, n, kind):
        a = self.links[(mu + 1) % 4, 1 - parity, (t - 1) % self.Nt]
        b = self.links[(mu + 2) % 4, parity, (t + 1) % self.Nt]
        return torch.cos(0.5 * a - 0.25 * b + 0.01 * (n + 3 * kind + 7 * mu + 11 * t))

    def update_pass(self, mu, parity, slab_d, n, kind):
        for t in range(self.t_lo, self.t_hi):
            if slab_d and mu != 0 and t % slab_d == 0:
                continue
            self.links[mu, parity, t] = self._new(mu, parity, t, n, kind)

    def part_size(self, what):
        return {ml.ML_PART_LINKS: S * 8, ml.ML_PART_SLAB_SUMS: S * 8, ml.ML_PART_VACUUM: 2 * 8,
                ml.ML_PART_W_SUMS: S * 8}[what]

    def _block(self, what, mu, parity):
        return {ml.ML_PART_LINKS: lambda: self.links[mu, parity], ml.ML_PART_SLAB_SUMS: lambda: self.T,
                ml.ML_PART_VACUUM: lambda: self.vac}[what]()

    def part_read(self, what, begin, count, mu=0, parity=0):
        return self._block(what, mu, parity)[begin:begin + count].contiguous().view(torch.uint8).reshape(-1).clone()

    def part_write(self, what, begin, count, buf, mu=0, parity=0):
        self._block(what, mu, parity)[begin:begin + count] = buf.view(torch.float64).reshape(count, -1)

    def _slab_sweep(self, d, n):
        """A slab sub-update: every link of the owned slabs of thickness d,
        spatial links on t = 0 mod d frozen, reading only the slab's own
        slices and its frozen upper boundary."""
        for s0 in range(self.t_lo, self.t_hi, d):
            for t in range(s0, s0 + d):
                for mu in range(4):
                    if mu != 0 and t % d == 0:
                        continue
                    up = (s0 + d) % self.Nt  # the next slab's first slice: its spatial links are frozen
                    above = self.links[1 + mu % 3, 0, t + 1 if t + 1 < s0 + d else up]
                    self.links[mu, 1, t] = torch.cos(0.3 * self.links[mu, 0, t] + 0.2 * above + 0.01 * (n + mu + t))

    def measure_inner(self, rec):
        rec.zero_()
        rec[0] = self.links.sum()  # "naive": a function of the whole configuration
        self.vac.zero_()
        p = self.p
        inner_T = torch.zeros(self.n_inner, S, dtype=torch.float64)
        for o in range(p.n_sub_outer if p.outer_slab else 1):
            if p.outer_slab:
                self.sweep += 1
                self._slab_sweep(p.outer_slab, self.sweep)
            inner_T.zero_()
            for _ in range(p.n_sub):
                self.sweep += 1
                self._slab_sweep(p.slab, self.sweep)
                for s in range(self.n_inner):  # every slab: the others' are stale and replaced later
                    t = s * p.slab
                    inner_T[s] += self.links[0, 1, t] * (1.0 + 0.1 * s)
                    self.vac[s, 0] += self.links[1, 1, t].sum()
                    self.vac[s, 1] += self.links[2, 0, t].sum()
            if p.outer_slab:
                q = p.outer_slab // p.slab
                if o == 0:
                    self.T.zero_()
                for S_ in range(self.n_top):
                    self.T[S_] += torch.prod(inner_T[q * S_:q * S_ + q], dim=0)
            else:
                self.T[:] = inner_T

    def measure_products(self, w_in=None, w_out=None, rec=None):
        w = torch.zeros(S, dtype=torch.float64) if w_in is None else w_in.view(torch.float64).clone()
        lo, hi = self.t_lo // self.top, self.t_hi // self.top
        run = torch.ones(S, dtype=torch.float64)
        for s in range(self.n_top):
            if lo <= s < hi:  # this slab's term times every other slab's [T]
                rest = torch.prod(torch.cat([self.T[:s], self.T[s + 1:]]), dim=0)
                w = w + (1.0 + 0.5 * self.T[s]) * rest
            run = run * self.T[s]
        if w_out is not None:
            w_out.view(torch.float64)[:] = w
            return
        rec[1] = run.sum()  # "P": every slab's [T]
        rec[2] = w.sum()    # "W": the per-site sums through every process
        rec[3] = self.vac.sum()


CASES = [dict(L=4, Nt=8, beta=1.0, slab=2, n_sub=3, k_between=2),
         dict(L=4, Nt=8, beta=1.0, slab=2, n_sub=2, outer_slab=4, n_sub_outer=2, k_between=1)]


def run(kw, n_meas):
    from paper_1309_3859_b300.partition import SlabPartition

    p = ml.Params(**kw)
    lat = FakeLattice(p)
    part = SlabPartition(lat, p)
    recs = part.measure(n_meas)
    return recs, lat.links.numpy().copy(), part.t_lo, part.t_hi


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, kw, out_dir):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        recs, links, lo, hi = run(kw, 2)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), recs=recs, links=links, lo=lo, hi=hi)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kw", CASES, ids=["one-level", "two-level"])
def test_two_gloo_ranks_match_one_rank(kw, tmp_path):
    import torch.multiprocessing as mp

    mp.start_processes(_rank_main, args=(2, _free_port(), kw, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    ref, links_ref, _, _ = run(kw, 2)
    assert np.all(np.isfinite(ref)) and np.abs(ref).max() > 0
    for rank in range(2):
        d = np.load(tmp_path / f"rank{rank}.npz")
        assert np.array_equal(d["recs"], ref), (rank, d["recs"], ref)
        own = slice(int(d["lo"]), int(d["hi"]))
        assert np.array_equal(d["links"][:, :, own], links_ref[:, :, own]), rank


def test_uneven_split_refused():
    from paper_1309_3859_b300.partition import SlabPartition

    import torch.distributed as dist

    assert not dist.is_initialized()
    p = ml.Params(L=4, Nt=6, beta=1.0, slab=2)
    SlabPartition(FakeLattice(p), p)  # one rank takes every slab
    q = ml.Params(L=4, Nt=6, beta=1.0, slab=4)  # slabs of 4 do not tile 6 slices
    with pytest.raises(ValueError):
        SlabPartition(FakeLattice(q), q)
