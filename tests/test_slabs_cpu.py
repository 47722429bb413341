"""Slab decomposition on CPU: the exchange logic of slabs.DistSlab over two
gloo ranks, with each slab stepped by the FP64 oracle, equals one lattice
stepped whole, bit for bit, through a dam break whose cells convert across
the cut.  (The library's own pack/unpack kernels run in the GPU tests.)

The oracle-backed lattice below implements the part of the library's
interface that the slab driver uses: set_owned, halo_bytes, halo_pack,
halo_unpack, step and total_mass, with the state (flags, post-collision
populations, interface mass, fill levels) held on the host.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LIQ, IFC = 1, 2


class OracleLattice:
    """One lattice whose steps are the oracle's (from post-collision state)."""

    def __init__(self, case):
        from oracle.oracle import F_POST, MASS, PHI, Oracle
        self._F_POST, self._MASS, self._PHI = F_POST, MASS, PHI
        self.dims = tuple(case["dims"])
        self.o = Oracle.from_case(case)
        self.lost = 0.0
        self.own = ((0, 0, 0), self.dims)
        self._read()

    def _read(self):
        o = self.o
        self.flags = o.flags().copy()
        self.f = o.get(self._F_POST).copy()
        self.m = np.where(self.flags == IFC, o.get(self._MASS), 0.0)
        self.phi = o.get(self._PHI).copy()

    def step(self, n=1):
        for _ in range(int(n)):
            assert self.o.step_from_post(self.flags, self.f, self.m, self.phi) == 0
            self._read()
            self.lost += self.o.total_mass()[1]

    def _sel(self, lo, hi):
        nx, ny, nz = self.dims
        idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
        return idx[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].reshape(-1)

    def sync(self):
        pass

    def set_owned(self, lo, hi):
        self.own = (tuple(lo), tuple(hi))

    def halo_bytes(self, lo, hi):
        return int(self._sel(lo, hi).size) * (1 + 8 + 8 + 19 * 8)

    def halo_pack(self, lo, hi, buf):
        i = self._sel(lo, hi)
        parts = [self.flags[i].astype(np.uint8).view(np.uint8), self.m[i].view(np.uint8),
                 self.phi[i].view(np.uint8), np.ascontiguousarray(self.f[:, i]).reshape(-1).view(np.uint8)]
        buf.numpy()[:] = np.concatenate(parts)

    def halo_unpack(self, lo, hi, buf):
        i = self._sel(lo, hi)
        n = i.size
        b = buf.numpy()
        self.flags[i] = b[:n]
        self.m[i] = b[n:9 * n].view(np.float64)
        self.phi[i] = b[9 * n:17 * n].view(np.float64)
        self.f[:, i] = b[17 * n:].view(np.float64).reshape(19, n)

    def total_mass(self):
        """sum_liquid rho + sum_interface m over the owned cells (the
        oracle's lost ledger covers ghost cells too, so it is left out)."""
        i = self._sel(*self.own)
        fl = self.flags[i]
        rho = self.f[:, i].sum(axis=0)
        M = float(np.where(fl == LIQ, rho, 0.0).sum() + np.where(fl == IFC, self.m[i], 0.0).sum())
        return M, 0.0

    def owned_state(self):
        i = self._sel(*self.own)
        return self.flags[i], self.f[:, i], self.m[i], self.phi[i]


AXIS = 2


def _case():
    """A ragged surface at the cut (z = 20 of 40) in fast motion: cells fill,
    empty and appear on both sides of the cut every few steps."""
    from paper_1409_5645_gb300 import cases
    return cases.churn(nx=5, ny=4, nz=40, base=20.0, plant=False, u_amp=0.05)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


STEPS = 60


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    try:
        import torch
        import torch.distributed as dist
        from paper_1409_5645_gb300 import slabs
        dist.init_process_group("gloo", rank=rank, world_size=ws)
        c = _case()
        s = slabs.Slab(c["dims"], AXIS, ws, rank)
        lat = OracleLattice(slabs.slice_case(c, AXIS, s.lo, s.hi))
        run = slabs.DistSlab(lat, s, torch.device("cpu"))
        whole = OracleLattice(c)
        M0, _ = run.total_mass()
        converted = 0
        for t in range(STEPS):
            run.step(1)
            whole.step(1)
            converted += int(whole.o.counters()[0][0] + whole.o.counters()[0][1])
        Mw, _ = whole.total_mass()  # the whole lattice's sum_liquid rho + sum_interface m
        mine = lat.owned_state()
        lo, hi = [0, 0, 0], list(c["dims"])
        lo[AXIS], hi[AXIS] = s.o0, s.o1
        whole.set_owned(lo, hi)
        ref = whole.owned_state()
        same = all(np.array_equal(a, b) for a, b in zip(mine, ref))
        M1, _ = run.total_mass()
        q.put((rank, same, converted, Mw, M1))
        dist.destroy_process_group()
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, repr(e), 0, 0.0, 0.0))


def test_two_gloo_ranks_match_one_lattice_bit_for_bit():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, same, converted, Mw, M1 in out:
        assert same is True, (rank, same)
        assert converted > 0
        # the FP64 sum over the ranks of their owned masses is the whole's
        assert M1 == pytest.approx(Mw, rel=1e-13)


def _owned_matches(run, whole_states, c):
    for t, W in enumerate(whole_states):
        run.step(1)
        for s, lat in zip(run.slabs, run.lats):
            lo, hi = [0, 0, 0], list(c["dims"])
            lo[AXIS], hi[AXIS] = s.o0, s.o1
            i = lat._sel(*s.owned_box())
            gi = lat._sel.__func__(type("D", (), {"dims": c["dims"]})(), lo, hi)
            if not (np.array_equal(lat.flags[i], W[0][gi]) and np.array_equal(lat.f[:, i], W[1][:, gi])
                    and np.array_equal(lat.m[i], W[2][gi])):
                return t + 1
    return None


def test_ghost_band_thinner_than_the_reach_breaks_parity():
    """The same scenario with slabs in one process: 8 ghost layers match the
    whole lattice for 60 steps; 1 and 2 layers (less than the cells one step
    reaches) do not: the comparison sees the cut."""
    from paper_1409_5645_gb300 import slabs
    c = _case()
    whole = OracleLattice(c)
    W = []
    for _ in range(STEPS):
        whole.step(1)
        W.append((whole.flags.copy(), whole.f.copy(), whole.m.copy()))
    for G, expect_ok in ((1, False), (2, False), (slabs.GHOST, True)):
        run = slabs.LocalSlabs(c, 2, axis=AXIS, ghost=G, make=OracleLattice, device="cpu")
        bad = _owned_matches(run, W, c)
        assert (bad is None) == expect_ok, (G, bad)


def test_slab_geometry():
    """Owned ranges tile the axis, held ranges add GHOST layers at each cut,
    and the boxes of an exchange pair up: what slab k sends to k+1 is the
    global range k+1 receives."""
    from paper_1409_5645_gb300 import slabs
    dims = (37, 29, 50)
    for parts in (2, 3, 4):
        S = [slabs.Slab(dims, 2, parts, k) for k in range(parts)]
        assert S[0].o0 == 0 and S[-1].o1 == 50
        for a, b in zip(S, S[1:]):
            assert a.o1 == b.o0 and a.hi == a.o1 + slabs.GHOST and b.lo == b.o0 - slabs.GHOST
            send = [box for nb, box, _ in a.neighbours() if nb == b.k][0]
            recv = [box for nb, _, box in b.neighbours() if nb == a.k][0]
            g_send = (send[0][2] + a.lo, send[1][2] + a.lo)
            g_recv = (recv[0][2] + b.lo, recv[1][2] + b.lo)
            assert g_send == g_recv == (b.lo, b.o0)
            send = [box for nb, box, _ in b.neighbours() if nb == a.k][0]
            recv = [box for nb, _, box in a.neighbours() if nb == b.k][0]
            assert (send[0][2] + b.lo, send[1][2] + b.lo) == (recv[0][2] + a.lo, recv[1][2] + a.lo) == (a.o1, a.hi)
    with pytest.raises(ValueError):
        slabs.bounds(12, 3, 0)  # slabs thinner than the ghost band
