"""The allocation-free mass balance, fslbm_mass_balance_noalloc.

It serves callers that cannot allocate device memory once they are running:
applications whose framework has reserved the GPU's memory for its own pool,
and loops where the device-wide synchronisation of cudaMalloc/cudaFree would
stall other streams.  Its partial sums live in a fixed array inside the
library.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1409_5645_gb300 import cases, fslbm

pytestmark = pytest.mark.gpu

ERR_TOO_LARGE = -8
MAX_CELLS = 4096 * 65536
# rest-state values w_q of the links, in the library's population order
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _entry():
    L = fslbm.lib()
    fn = L.fslbm_mass_balance_noalloc
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_longlong, C.c_double, C.c_void_p,
                   C.c_void_p]
    fn.restype = C.c_int
    return fn


def _state():
    import torch
    dev = torch.device("cuda:0")
    c = cases.dam_break(nx=37, ny=13, nz=21, col_x=11, col_z=15, tau=0.56, g=3e-4)
    lat = fslbm.Lattice.from_case(c)
    lat.step(60)
    st = lat.get(fslbm.FIELD_FLAGS | fslbm.FIELD_F | fslbm.FIELD_MASS, device=dev)
    ref, lost = lat.total_mass()
    return c, dev, st, ref, lost


def test_noalloc_mass_balance_matches_total_mass_on_two_calls():
    import torch
    fn = _entry()
    c, dev, st, ref, lost = _state()
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    for _ in range(2):
        rc = fn(st["flags"].data_ptr(), st["f"].data_ptr(), fslbm.F64, st["m"].data_ptr(), c.N, lost,
                out.data_ptr(), None)
        torch.cuda.synchronize(dev)
        assert rc == 0
        assert out.item() == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("prec,dtype,rel", [("f32", "float32", 1e-7), ("f16", "float16", 1e-3)])
def test_noalloc_mass_balance_reduced_storage(prec, dtype, rel):
    """The reduced forms hand over f - w_q in float or half: the same state in
    that storage gives the FP64 mass to the storage's resolution, and a
    lattice run in that form gives its own fslbm_total_mass."""
    import torch
    fn = _entry()
    c, dev, st, ref, lost = _state()
    code = {"f32": fslbm.F32, "f16": fslbm.F16}[prec]
    shifted = (st["f"] - torch.as_tensor(W, device=dev)[:, None]).to(getattr(torch, dtype)).contiguous()
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    for _ in range(2):
        rc = fn(st["flags"].data_ptr(), shifted.data_ptr(), code, st["m"].data_ptr(), c.N, lost,
                out.data_ptr(), None)
        torch.cuda.synchronize(dev)
        assert rc == 0
        assert out.item() == pytest.approx(ref, rel=rel)
    # a lattice of this form: its stored populations through the entry point
    lat = fslbm.Lattice.from_case(c, precision=prec)
    lat.step(60)
    mine = lat.get(fslbm.FIELD_FLAGS | fslbm.FIELD_F | fslbm.FIELD_MASS, device=dev)
    M, L = lat.total_mass()
    raw = (mine["f"] - torch.as_tensor(W, device=dev)[:, None]).to(getattr(torch, dtype)).contiguous()
    for _ in range(2):
        rc = fn(mine["flags"].data_ptr(), raw.data_ptr(), code, mine["m"].data_ptr(), c.N, L, out.data_ptr(), None)
        torch.cuda.synchronize(dev)
        assert rc == 0
        assert out.item() == pytest.approx(M, rel=1e-12 if prec == "f32" else 1e-9)


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    fn = _entry()
    dev = torch.device("cuda:0")
    tiny = torch.zeros(8, dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    # rejected before any kernel runs, so the small buffers are never read
    rc = fn(tiny.data_ptr(), tiny.data_ptr(), fslbm.F64, tiny.data_ptr(), MAX_CELLS + 1, 0.0, out.data_ptr(), None)
    assert rc == ERR_TOO_LARGE
    assert fn(None, tiny.data_ptr(), fslbm.F64, tiny.data_ptr(), 8, 0.0, out.data_ptr(), None) == -1
