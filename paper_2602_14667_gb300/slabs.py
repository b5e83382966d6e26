"""Row-slab decomposition of one periodic lattice.

The fused step shards along y: each slab (an MHD_HALO lattice) owns a band
of rows plus a ghost row on either side, and one exchange per step carries
across every slab boundary the post-collision populations whose velocity
crosses it (pull streaming: the first row of a slab pulls its c_y = +1
populations from the row below, its last row the c_y = -1 ones from the row
above).  This module holds the host-side bookkeeping -- the partition, the
populations that cross a boundary, the exchange schedule and the
combination of the slabs' totals -- and SlabGroup, which runs the slabs of
one lattice on the current device through the library's calls
(mhd_advance, mhd_slab_exchange, mhd_get_totals).  With one slab per GPU the
same schedule drives peer copies (or NCCL send / receive of the crossing
rows) and an all-reduce of the totals.

Population order (library planes and oracle arrays alike): f_0 .. f_8 in
the paper's D2Q9 order, then g_{j,a} at 9 + 2 j + a (D2Q5, a = x, y).
"""
from __future__ import annotations

import math

import numpy as np

from ._abi import Lattice, SlabSteps, slab_exchange

# c_y of the 19 populations: D2Q9 (the paper's order) and D2Q5 (each twice)
_CY_F = (0, 1, 0, -1, -1, -1, 0, 1, 1)
_CY_G = (0, 0, -1, 0, 1)
CY = _CY_F + tuple(c for c in _CY_G for _ in range(2))
CROSS_UP = tuple(p for p, c in enumerate(CY) if c == 1)      # f_1, f_7, f_8, g_4 (x, y)
CROSS_DOWN = tuple(p for p, c in enumerate(CY) if c == -1)   # f_3, f_4, f_5, g_2 (x, y)


def partition(ny: int, nslabs: int):
    """Row ranges [y0, y1) of nslabs slabs of an ny-row lattice, as equal as
    they can be (the first ny % nslabs slabs get one row more)."""
    if nslabs < 1 or nslabs > ny:
        raise ValueError("need 1 <= nslabs <= ny")
    base, extra = divmod(ny, nslabs)
    out, y = [], 0
    for s in range(nslabs):
        h = base + (1 if s < extra else 0)
        out.append((y, y + h))
        y += h
    return out


def exchange_schedule(nslabs: int):
    """The boundaries of a periodic y axis as (lower, upper) slab pairs:
    slab s lies just below slab s + 1, and the last just below the first."""
    return [(s, (s + 1) % nslabs) for s in range(nslabs)]


SUMS = ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y")
MEANS = ("e_kin", "e_mag", "cross_hel")
MAXIMA = ("divb_max", "jz_max", "omega_max")


def combine_totals(parts, nx: int, wall_x: bool = False) -> dict:
    """Totals of the whole lattice from those of its slabs: parts is a list
    of (totals, rows).  Sums add, means are weighted by the slab's nodes,
    maxima take the largest, and the rms of div b is weighted by the nodes
    whose stencil is valid (all rows of a slab; on an x-walled lattice every
    column but the first and the last)."""
    n = sum(nx * rows for _, rows in parts)
    nvalid = [(nx - 2 if wall_x else nx) * rows for _, rows in parts]
    out = {k: sum(t[k] for t, _ in parts) for k in SUMS}
    out.update({k: sum(t[k] * nx * rows for t, rows in parts) / n for k in MEANS})
    out.update({k: max(t[k] for t, _ in parts) for k in MAXIMA})
    sq = sum(t["divb_rms"] ** 2 * v for (t, _), v in zip(parts, nvalid))
    out["divb_rms"] = math.sqrt(sq / sum(nvalid)) if sum(nvalid) else 0.0
    out["step"] = parts[0][0]["step"]
    return out


def allreduce_totals(totals: dict, rows: int, nx: int, wall_x: bool = False, group=None) -> dict:
    """The whole lattice's totals when each rank of a torch.distributed
    group holds one slab (its own totals and row count): combine_totals as
    two FP64 all-reduces, one SUM (the sums, the node-weighted means, the
    weighted squares of the rms of div b and the node counts) and one MAX
    (the maxima)."""
    import torch
    import torch.distributed as dist
    nodes = nx * rows
    nvalid = (nx - 2 if wall_x else nx) * rows
    s = torch.tensor([float(totals[k]) for k in SUMS] + [totals[k] * nodes for k in MEANS]
                     + [totals["divb_rms"] ** 2 * nvalid, float(nodes), float(nvalid)], dtype=torch.float64)
    m = torch.tensor([float(totals[k]) for k in MAXIMA], dtype=torch.float64)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
    s, m = s.tolist(), m.tolist()
    ns, nm = len(SUMS), len(MEANS)
    out = dict(zip(SUMS, s[:ns]))
    out.update({k: s[ns + i] / s[-2] for i, k in enumerate(MEANS)})
    out.update(zip(MAXIMA, m))
    out["divb_rms"] = math.sqrt(s[ns + nm] / s[-1]) if s[-1] else 0.0
    out["step"] = totals["step"]
    return out


class SlabGroup:
    """The slabs of one nx x ny lattice with a periodic y axis, all on the
    current device and one stream: every step advances each slab and then
    exchanges every boundary -- through the library's slab group
    (mhd_slab_group_advance: one exchange kernel per round, 64-round CUDA
    graphs), or, with stepwise=True, one mhd_advance per slab and one
    mhd_slab_exchange per boundary and step.  Fields, populations and totals
    are those of the whole lattice."""

    def __init__(self, nx, ny, nslabs, tau_f, tau_m, precision="fp32", rows=None, stream=None, **kw):
        self.nx, self.ny = int(nx), int(ny)
        self.rows = list(rows) if rows is not None else partition(ny, nslabs)
        if self.rows[0][0] != 0 or self.rows[-1][1] != ny or any(
                a[1] != b[0] for a, b in zip(self.rows, self.rows[1:])):
            raise ValueError("row ranges must tile [0, ny)")
        self.wall_x = bool(kw.get("wall_x", False))
        self.slabs = [Lattice(nx, y1 - y0, tau_f, tau_m, precision=precision, halo_y=True, stream=stream, **kw)
                      for y0, y1 in self.rows]
        self.schedule = exchange_schedule(len(self.slabs))
        self._steps = None

    def close(self):
        if self._steps is not None:
            self._steps.close()
            self._steps = None
        for s in self.slabs:
            s.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def kernel_config(self):
        return self.slabs[0].kernel_config

    @kernel_config.setter
    def kernel_config(self, v):
        for s in self.slabs:
            s.kernel_config = v

    def exchange(self, all_planes=False):
        for lo, up in self.schedule:
            slab_exchange(self.slabs[lo], self.slabs[up], all_planes)

    def set_fields(self, ux, uy, bx, by, rho=None):
        for s, (y0, y1) in zip(self.slabs, self.rows):
            s.set_fields(*(np.ascontiguousarray(a[y0:y1]) for a in (ux, uy, bx, by)),
                         rho=None if rho is None else np.ascontiguousarray(rho[y0:y1]))
        self.exchange()

    def set_populations(self, f, g):
        for s, (y0, y1) in zip(self.slabs, self.rows):
            s.set_populations(np.ascontiguousarray(f[:, y0:y1]), np.ascontiguousarray(g[:, :, y0:y1]))
        self.exchange()

    def advance(self, nsteps: int, stepwise: bool = False):
        if stepwise:
            for _ in range(int(nsteps)):
                for s in self.slabs:
                    s.advance(1)
                self.exchange()
            return
        if self._steps is None:
            self._steps = SlabSteps(self.slabs)
        self._steps.advance(nsteps)

    def get_fields(self) -> dict:
        parts = [s.get_fields() for s in self.slabs]
        return {k: np.concatenate([p[k] for p in parts], axis=0) for k in parts[0]}

    def get_populations(self):
        parts = [s.get_populations() for s in self.slabs]
        return (np.concatenate([p[0] for p in parts], axis=1), np.concatenate([p[1] for p in parts], axis=2))

    def get_totals(self) -> dict:
        self.exchange(all_planes=True)   # the stencil at the edge rows reads the ghost rows' moments
        return combine_totals([(s.get_totals(), y1 - y0) for s, (y0, y1) in zip(self.slabs, self.rows)],
                              self.nx, self.wall_x)
