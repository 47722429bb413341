"""Slab decomposition of a lattice: one library handle per slab, the ghost
layers beside each cut refilled once per time step from the neighbouring
slabs' owned cells.

Host logic only (which boxes go where, and in what order); the state moves
through the library's fslbm_halo_pack / fslbm_halo_unpack kernels, and
between GPUs or processes through torch.distributed (NCCL on GPUs, gloo on
CPUs).  A step of a cell reads the state of time t within 7 cells of it, so
with GHOST >= 7 ghost layers every owned cell is exact after a step and one
exchange restores the ghost layers (see include/fslbm.h).  The lattice must
not be periodic along the split axis, and a periodic x wrap with a z shift
is not split.
"""
from __future__ import annotations

import numpy as np

GHOST = 8  # ghost layers per cut (>= the step's reach of 7 cells)


def bounds(n: int, parts: int, k: int, ghost: int = GHOST):
    """Global index ranges of slab k of `parts` along an axis of n cells:
    (held_lo, held_hi, own_lo, own_hi).  Slabs own near-equal ranges."""
    if not 0 <= k < parts:
        raise ValueError("slab index out of range")
    o0, o1 = (k * n) // parts, ((k + 1) * n) // parts
    if o1 - o0 < ghost:
        raise ValueError(f"a slab of {o1 - o0} cells is thinner than the {ghost} ghost layers")
    lo = o0 - ghost if k > 0 else o0
    hi = o1 + ghost if k < parts - 1 else o1
    return lo, hi, o0, o1


def slice_case(case, axis: int, lo: int, hi: int):
    """The sub-lattice [lo, hi) along `axis` of a case (flags, rho, u, phi,
    noise, wall link fractions; the same parameters)."""
    from .cases import Case

    nx, ny, nz = case["dims"]
    if case["params"]["periodic"][axis]:
        raise ValueError("the split axis must not be periodic")
    if case["params"].get("zshift", 0) and axis != 1:
        raise ValueError("a periodic x wrap with a z shift couples x and z: split along y only")
    sl = [slice(None)] * 3
    sl[2 - axis] = slice(lo, hi)  # arrays are [z][y][x]
    sl = tuple(sl)

    def cut(a, comps=None):
        if a is None:
            return None
        a = np.asarray(a)
        if comps is None:
            return np.ascontiguousarray(a.reshape(nz, ny, nx)[sl]).reshape(-1)
        if a.shape[0] == comps:  # [comps][N]
            return np.ascontiguousarray(a.reshape(comps, nz, ny, nx)[(slice(None),) + sl]).reshape(comps, -1)
        return np.ascontiguousarray(a.reshape(nz, ny, nx, comps)[sl]).reshape(-1, comps)  # [N][comps]

    dims = [nx, ny, nz]
    dims[axis] = hi - lo
    return Case(dims=tuple(dims), params=dict(case["params"]), flags=cut(case["flags"]), rho=cut(case["rho"]),
                u=cut(case["u"], 3), phi=cut(case["phi"]), noise=cut(case.get("noise"), 19),
                wall_delta=cut(case.get("wall_delta"), 19))


class Slab:
    """Geometry of slab k of a lattice of `dims` split into `parts` along
    `axis`: the held range, the owned range, and the four boxes of an
    exchange in the slab's own (local) coordinates."""

    def __init__(self, dims, axis: int, parts: int, k: int, ghost: int = GHOST):
        self.dims, self.axis, self.parts, self.k, self.ghost = tuple(dims), axis, parts, k, ghost
        self.lo, self.hi, self.o0, self.o1 = bounds(dims[axis], parts, k, ghost)
        self.local_dims = list(dims)
        self.local_dims[axis] = self.hi - self.lo
        self.local_dims = tuple(self.local_dims)

    def _box(self, a, b):
        """Local box of the global range [a, b) along the axis, whole along the others."""
        lo, hi = [0, 0, 0], list(self.local_dims)
        lo[self.axis], hi[self.axis] = a - self.lo, b - self.lo
        return tuple(lo), tuple(hi)

    def owned_box(self):
        return self._box(self.o0, self.o1)

    def neighbours(self):
        """[(neighbour slab, send box, receive box)] for the lower and the
        upper cut: send my owned layers next to the cut, receive that
        neighbour's into my ghost layers."""
        out = []
        g = self.ghost
        if self.k > 0:
            out.append((self.k - 1, self._box(self.o0, self.o0 + g), self._box(self.lo, self.o0)))
        if self.k < self.parts - 1:
            out.append((self.k + 1, self._box(self.o1 - g, self.o1), self._box(self.o1, self.hi)))
        return out


def _buffer(nbytes, device):
    import torch
    # 16-byte aligned (the caching allocator aligns to 512 bytes)
    return torch.empty(int(nbytes), dtype=torch.uint8, device=device)


class LocalSlabs:
    """Every slab in this process, each with its own lattice object (on one
    GPU or several); exchanges are device copies through pack buffers."""

    def __init__(self, case, parts: int, axis: int = 1, precision="f64", ghost: int = GHOST, make=None,
                 device=None):
        from . import fslbm
        self.slabs = [Slab(case["dims"], axis, parts, k, ghost) for k in range(parts)]
        make = make or (lambda c: fslbm.Lattice.from_case(c, precision=precision))
        self.lats = []
        for s in self.slabs:
            lat = make(slice_case(case, axis, s.lo, s.hi))
            lat.set_owned(*s.owned_box())
            self.lats.append(lat)
        import torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.bufs = {}

    def _sync(self):
        import torch
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)

    def exchange(self):
        """Refill every ghost layer from the neighbour's owned cells: all
        packs first (owned cells), then all unpacks (ghost cells)."""
        for k, (s, lat) in enumerate(zip(self.slabs, self.lats)):
            for nb, send, _ in s.neighbours():
                key = (k, nb)
                if key not in self.bufs:
                    self.bufs[key] = _buffer(lat.halo_bytes(*send), self.device)
                lat.halo_pack(*send, self.bufs[key])
        self._sync()
        for k, (s, lat) in enumerate(zip(self.slabs, self.lats)):
            for nb, _, recv in s.neighbours():
                lat.halo_unpack(*recv, self.bufs[(nb, k)])
        self._sync()

    def step(self, n: int = 1):
        for _ in range(int(n)):
            for lat in self.lats:
                lat.step(1)
            self.exchange()

    def total_mass(self):
        """Sum over the slabs of their owned mass and lost ledgers (FP64)."""
        M = L = 0.0
        for lat in self.lats:
            m, l = lat.total_mass()
            M += m
            L += l
        return M, L

    def owned_fields(self, mask):
        """Fields of the owned cells, reassembled on the global lattice."""
        parts = []
        for s, lat in zip(self.slabs, self.lats):
            st = lat.get(mask)
            lo, hi = s.owned_box()
            parts.append({k: _crop(v, s.local_dims, lo, hi, s.axis) for k, v in st.items()})
        return {k: _join([p[k] for p in parts], k, self.slabs[0]) for k in parts[0]}


def _crop(a, dims, lo, hi, axis):
    """Owned part of a field of a slab, as an array [..][z][y][x] cut to the box."""
    nx, ny, nz = dims
    sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    if a.ndim == 1:
        return a.reshape(nz, ny, nx)[sl]
    if a.shape[0] == 19:
        return a.reshape(19, nz, ny, nx)[(slice(None),) + sl]
    return a.reshape(nz, ny, nx, a.shape[1])[sl]


def _join(pieces, key, slab):
    ax = 2 - slab.axis  # array axis of the split in [z][y][x]
    if pieces[0].ndim == 3:
        return np.concatenate(pieces, axis=ax).reshape(-1)
    if key == "f":
        return np.concatenate(pieces, axis=ax + 1).reshape(19, -1)
    return np.concatenate(pieces, axis=ax).reshape(-1, pieces[0].shape[-1])


class DistSlab:
    """This rank's slab of a lattice split over a torch.distributed group:
    rank k owns slab k.  exchange() packs the two sides, swaps them with the
    neighbouring ranks (batched point-to-point), unpacks; total_mass() sums
    the owned masses over the group in FP64."""

    def __init__(self, lat, slab: Slab, device, group=None):
        self.lat, self.slab, self.device, self.group = lat, slab, device, group
        lat.set_owned(*slab.owned_box())
        self.send = {nb: _buffer(lat.halo_bytes(*box), device) for nb, box, _ in slab.neighbours()}
        self.recv = {nb: _buffer(lat.halo_bytes(*box), device) for nb, _, box in slab.neighbours()}
        self.bytes_per_exchange = sum(int(b.numel()) for b in self.send.values())

    def exchange(self):
        import torch
        import torch.distributed as dist
        s = self.slab
        for nb, box, _ in s.neighbours():
            self.lat.halo_pack(*box, self.send[nb])
        self.lat.sync()  # the packs are done (the lattice's own stream)
        ops = []
        for nb, _, _ in s.neighbours():
            ops.append(dist.P2POp(dist.isend, self.send[nb], nb, group=self.group))
            ops.append(dist.P2POp(dist.irecv, self.recv[nb], nb, group=self.group))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        if self.device.type == "cuda":
            torch.cuda.current_stream(self.device).synchronize()  # the receives have landed
        for nb, _, box in s.neighbours():
            self.lat.halo_unpack(*box, self.recv[nb])

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.lat.step(1)
            self.exchange()

    def total_mass(self):
        import torch
        import torch.distributed as dist
        M, L = self.lat.total_mass()
        t = torch.tensor([M, L], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return float(t[0]), float(t[1])
