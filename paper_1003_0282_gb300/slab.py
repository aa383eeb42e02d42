"""z-slab decomposition of one axisymmetric domain (cut faces, AXLBM_Z_HALO).

A long pipe (the periodic pipes of Sec. IV A) is cut across z into slabs,
each advanced by its own handle whose cut faces are ``z_lo`` / ``z_hi =
"halo"``.  After every lattice step each cut face hands the populations that
cross it to the neighbouring slab (``axlbm_halo_send`` -> the neighbour's
``axlbm_halo_recv``; slab A above slab B pairs A's lo face with B's hi face,
and a periodic domain pairs the top slab's hi face with the bottom slab's lo
face).  The slabs together then advance exactly the undivided domain.

Two drivers share the pairing rules:

* :class:`LocalSlabs` holds every slab in this process (one GPU, messages in
  device buffers on one stream);
* :class:`RankSlab` holds one slab per rank of a ``torch.distributed`` group
  and stages each message through host memory (send and receive over the
  group, e.g. gloo), so that no GPU-to-GPU path is needed.  Only the halo
  exchange crosses ranks; the residual and the check values are reduced over
  the group.

The arithmetic of every step runs in the CUDA library; this module only
splits the problem and moves the messages.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

from . import inputs as I

LO, HI = 2, 3  # AXLBM_FACE_LO, AXLBM_FACE_HI
# message tags by the receiving face (a pair of ranks may trade both faces in a periodic domain of two slabs)
_TAG = {LO: 11, HI: 12}


def split_rows(nz: int, nslabs: int) -> List[Tuple[int, int]]:
    """Row ranges [k0, k1) of nslabs slabs of nearly equal height (each >= 2 rows)."""
    if nslabs < 1 or nz < 2 * nslabs:
        raise ValueError(f"cannot cut {nz} rows into {nslabs} slabs of at least 2 rows")
    edges = [round(s * nz / nslabs) for s in range(nslabs + 1)]
    return [(edges[s], edges[s + 1]) for s in range(nslabs)]


def slab_problems(pb: I.Problem, nslabs: int) -> List[I.Problem]:
    """The slabs of pb: the same problem on rows [k0, k1), cut faces where a
    neighbour slab lies (every axial face of a periodic domain)."""
    if pb.z_lo in (I.NEE, I.HALO) or pb.z_hi in (I.NEE, I.HALO):
        raise ValueError("slabs need non-wet, uncut axial faces on the whole domain")
    periodic = pb.z_lo == I.PERIODIC
    out = []
    for s, (k0, k1) in enumerate(split_rows(pb.nz, nslabs)):
        z_lo = pb.z_lo if (s == 0 and not periodic) else I.HALO
        z_hi = pb.z_hi if (s == nslabs - 1 and not periodic) else I.HALO
        keep = lambda d: {f: v for f, v in d.items() if not ((f == "lo" and z_lo == I.HALO) or
                                                              (f == "hi" and z_hi == I.HALO))}
        out.append(dataclasses.replace(pb, nz=k1 - k0, z_lo=z_lo, z_hi=z_hi, omega=keep(pb.omega),
                                       t_wall=keep(pb.t_wall), name=f"{pb.name} slab {s} rows {k0}:{k1}"))
    return out


def neighbours(s: int, nslabs: int, periodic: bool) -> Tuple[Optional[int], Optional[int]]:
    """(slab below, slab above) of slab s, None at a domain end."""
    below = s - 1 if s > 0 else (nslabs - 1 if periodic else None)
    above = s + 1 if s < nslabs - 1 else (0 if periodic else None)
    return below, above


class LocalSlabs:
    """Every slab of one domain on the current CUDA device, exchanged through
    device buffers on the current stream."""

    def __init__(self, pb: I.Problem, nslabs: int, precision: str = "fp32"):
        import torch

        from . import axlbm as B

        self.pb = pb
        self.parts = slab_problems(pb, nslabs)
        self.rows = split_rows(pb.nz, nslabs)
        self.periodic = pb.z_lo == I.PERIODIC
        self.doms = [B.Domain(p, precision) for p in self.parts]
        nbytes = max(d.halo_bytes() for d in self.doms)
        self._buf = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]

    def close(self) -> None:
        for d in self.doms:
            d.close()

    @property
    def time(self) -> int:
        return self.doms[0].time

    def exchange(self) -> None:
        n = len(self.doms)
        for s in range(n):
            _, above = neighbours(s, n, self.periodic)
            if above is None:
                continue
            lower, upper = self.doms[s], self.doms[above]
            upper.halo_send(LO, self._buf[0])
            lower.halo_recv(HI, self._buf[0])
            lower.halo_send(HI, self._buf[1])
            upper.halo_recv(LO, self._buf[1])

    def step(self, n: int) -> None:
        for _ in range(int(n)):
            for d in self.doms:
                d.step(1)
            self.exchange()

    def set_residual_lag(self, lag: int) -> None:
        for d in self.doms:
            d.set_residual_lag(lag)

    def residual(self):
        """(max residual, total mass, total budget) of the slabs' last check steps."""
        rs = [d.residual() for d in self.doms]
        return max(r[0] for r in rs), sum(r[1] for r in rs), sum(r[2] for r in rs)

    def set_populations(self, f, g=None, h=None, time: int = 0) -> None:
        cut = lambda a, k0, k1: None if a is None else a[:, k0:k1]
        for d, (k0, k1) in zip(self.doms, self.rows):
            d.set_populations(cut(f, k0, k1), cut(g, k0, k1), cut(h, k0, k1), time=time)

    def get_populations(self):
        parts = [d.get_populations() for d in self.doms]
        join = lambda i: None if parts[0][i] is None else np.concatenate([p[i] for p in parts], axis=1)
        return join(0), join(1), join(2)

    def moments(self, mask: int) -> np.ndarray:
        return np.concatenate([d.moments(mask) for d in self.doms], axis=1)


class RankSlab:
    """One slab per rank of a torch.distributed group; messages staged
    through host memory.  `solver` (for tests) replaces the slab's Domain: an
    object with step(n), halo_bytes(), halo_send(face, out) and
    halo_recv(face, msg) on uint8 host arrays."""

    def __init__(self, pb: I.Problem, precision: str = "fp32", group=None, solver=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.periodic = pb.z_lo == I.PERIODIC
        self.part = slab_problems(pb, self.world)[self.rank]
        self.rows = split_rows(pb.nz, self.world)[self.rank]
        if solver is None:
            from . import axlbm as B

            solver = B.Domain(self.part, precision)
        self.dom = solver
        self.below, self.above = neighbours(self.rank, self.world, self.periodic)
        nbytes = self.dom.halo_bytes()
        self._out = {LO: np.empty(nbytes, np.uint8), HI: np.empty(nbytes, np.uint8)}
        self._in = {LO: np.empty(nbytes, np.uint8), HI: np.empty(nbytes, np.uint8)}

    def _peer(self, face: int) -> Optional[int]:
        return self.below if face == LO else self.above

    def exchange(self) -> None:
        import torch

        faces = [f for f in (LO, HI) if self._peer(f) is not None]
        for f in faces:
            self.dom.halo_send(f, self._out[f])
        if self.world == 1:  # a periodic domain in one slab: its faces pair with each other
            for f in faces:
                self._in[f][:] = self._out[LO if f == HI else HI]
        else:
            reqs = []
            for f in faces:
                peer = self.group_rank(self._peer(f))
                # what leaves through my face f arrives at the peer's opposite face
                reqs.append(self.dist.isend(torch.from_numpy(self._out[f]), peer, group=self.group,
                                            tag=_TAG[HI if f == LO else LO]))
                reqs.append(self.dist.irecv(torch.from_numpy(self._in[f]), peer, group=self.group, tag=_TAG[f]))
            for r in reqs:
                r.wait()
        for f in faces:
            self.dom.halo_recv(f, self._in[f])

    def group_rank(self, r: int) -> int:
        """Global rank of group rank r (point-to-point calls take global ranks)."""
        if self.group is None:
            return r
        return self.dist.get_global_rank(self.group, r)

    def step(self, n: int) -> None:
        for _ in range(int(n)):
            self.dom.step(1)
            self.exchange()

    def residual(self):
        """(max residual, total mass, total budget) over the ranks' slabs."""
        import torch

        res, mass, budget = self.dom.residual()
        t = torch.tensor([res], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        s = torch.tensor([mass, budget], dtype=torch.float64)
        self.dist.all_reduce(s, group=self.group)
        return float(t[0]), float(s[0]), float(s[1])
