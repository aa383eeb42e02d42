"""Host side of the z-slab decomposition (slab.py), on CPU.

The splitting rules (row ranges, cut faces, neighbours) and the exchange over
a torch.distributed gloo group with two and three ranks.  The GPU slab is
replaced by a small stand-in with the same contract -- after every step each
cut face sends what crossed it and stores what its neighbour sent -- a
three-velocity lattice along z (rest, up, down) with a linear collision,
periodic or bounce-back ends.  The slabs run on the ranks must reproduce the
undivided lattice bit for bit; the residual and mass reductions are checked
too.  The same exchange drives the CUDA slabs in tests/test_gpu_slabs.py.
"""
import os
import socket

import numpy as np
import pytest

from paper_1003_0282_gb300 import inputs as I
from paper_1003_0282_gb300 import slab as SL

LO, HI = SL.LO, SL.HI


class ToySlab:
    """Rest / up / down populations on rows [0, nz); ends: 'periodic', 'wall'
    (bounce-back) or 'halo' (a cut: what leaves is sent, what arrives is
    received).  A whole domain is a ToySlab with no cut."""

    W = np.array([4 / 6, 1 / 6, 1 / 6])

    def __init__(self, rho, u, lo, hi, omega=1.3):
        self.f = np.stack([self.W[a] * rho * (1 + 3 * e * u) for a, e in enumerate((0, 1, -1))])
        self.lo, self.hi, self.omega = lo, hi, omega
        self.out = {LO: np.zeros(1), HI: np.zeros(1)}
        self.prev = None
        self.t = 0

    def speed(self):
        rho = self.f.sum(axis=0)
        return np.abs((self.f[1] - self.f[2]) / rho)

    def step(self, n):
        for _ in range(n):
            self.prev = self.speed()
            f = self.f
            rho = f.sum(axis=0)
            u = (f[1] - f[2]) / rho
            feq = np.stack([self.W[a] * rho * (1 + 3 * e * u + 4.5 * (e * u) ** 2 - 1.5 * u * u)
                            for a, e in enumerate((0, 1, -1))])
            post = f + self.omega * (feq - f) + 1e-4 * np.sin(0.1 * self.t)  # a time-dependent source
            new = post.copy()
            new[1] = np.roll(post[1], 1)
            new[2] = np.roll(post[2], -1)
            nz = f.shape[1]
            # up population leaving through the top, down leaving through the bottom
            up_out, down_out = post[1, nz - 1], post[2, 0]
            if self.hi == "wall":
                new[2, nz - 1] = up_out
            if self.lo == "wall":
                new[1, 0] = down_out
            if self.hi == "halo":
                self.out[HI] = np.array([up_out])
            if self.lo == "halo":
                self.out[LO] = np.array([down_out])
            self.f = new
            self.t += 1

    def halo_bytes(self):
        return 8

    def halo_send(self, face, out):
        out[:] = self.out[face].view(np.uint8)

    def halo_recv(self, face, msg):
        v = np.frombuffer(msg.tobytes(), dtype=np.float64)[0]
        if face == LO:
            self.f[1, 0] = v          # the neighbour below sent its up population
        else:
            self.f[2, -1] = v         # the neighbour above sent its down population

    def residual(self):
        return float(np.max(np.abs(self.speed() - self.prev))), float(self.f.sum()), 0.0


def test_split_rows_and_slab_problems():
    assert SL.split_rows(10, 3) == [(0, 3), (3, 7), (7, 10)]
    with pytest.raises(ValueError):
        SL.split_rows(5, 3)
    pipe = I.hagen_poiseuille(nr=8, nz=12)
    parts = SL.slab_problems(pipe, 3)
    assert [p.nz for p in parts] == [4, 4, 4]
    assert all(p.z_lo == "halo" and p.z_hi == "halo" for p in parts)
    cav = I.rotating_lid_cavity(nr=16, aspect=1.5, re=100.0)
    parts = SL.slab_problems(cav, 2)
    assert (parts[0].z_lo, parts[0].z_hi, parts[1].z_lo, parts[1].z_hi) == ("wall", "halo", "halo", "wall")
    assert parts[1].omega_of("hi") == cav.omega_of("hi") and "hi" not in parts[0].omega
    assert SL.neighbours(0, 3, True) == (2, 1) and SL.neighbours(2, 3, False) == (1, None)
    assert SL.neighbours(0, 1, True) == (0, 0) and SL.neighbours(0, 1, False) == (None, None)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


NZ = 23


def _fields():
    k = np.arange(NZ)
    return 1.0 + 0.01 * np.cos(2 * np.pi * k / NZ), 0.02 * np.sin(4 * np.pi * k / NZ) + 0.005


def _worker(rank, world, port, ends, nsteps, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pb = I.Problem(nr=4, nz=NZ, tau=0.8, z_lo=ends, z_hi=ends)
        k0, k1 = SL.split_rows(NZ, world)[rank]
        part = SL.slab_problems(pb, world)[rank]
        rho, u = _fields()
        toy = ToySlab(rho[k0:k1], u[k0:k1], part.z_lo, part.z_hi)
        rs = SL.RankSlab(pb, group=None, solver=toy)
        rs.step(nsteps)
        res, mass, _ = rs.residual()
        q.put((rank, k0, toy.f.copy(), res, mass))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("ends", ["periodic", "wall"])
def test_slabs_on_gloo_ranks_equal_the_undivided_lattice(world, ends):
    import torch.multiprocessing as mp
    nsteps = 41
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ends, nsteps, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=120) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rho, u = _fields()
    whole = ToySlab(rho, u, ends, ends)
    whole.step(nsteps)
    got = np.concatenate([o[2] for o in out], axis=1)
    assert np.array_equal(got, whole.f)
    res, mass, _ = whole.residual()
    assert all(o[3] == res for o in out)                     # max over ranks
    assert all(abs(o[4] - mass) <= 1e-12 * mass for o in out)  # sum over ranks


def test_one_periodic_slab_exchanges_with_itself():
    class G:  # a one-rank group stand-in
        pass
    rho, u = _fields()
    toy = ToySlab(rho, u, "halo", "halo")
    rs = SL.RankSlab.__new__(SL.RankSlab)
    rs.dom, rs.world, rs.rank, rs.periodic = toy, 1, 0, True
    rs.below, rs.above = SL.neighbours(0, 1, True)
    rs._out = {LO: np.empty(8, np.uint8), HI: np.empty(8, np.uint8)}
    rs._in = {LO: np.empty(8, np.uint8), HI: np.empty(8, np.uint8)}
    rs.step(17)
    whole = ToySlab(rho, u, "periodic", "periodic")
    whole.step(17)
    assert np.array_equal(toy.f, whole.f)
