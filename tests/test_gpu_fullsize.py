"""The benchmark workload at full size (512 x 256 x 256 dam break), in the
launch configuration bench.py times: sampled windows against the oracle, and
properties that hold at any size."""
import numpy as np
import pytest

from oracle.oracle import F_POST, MASS, PHI, Oracle
from paper_1409_5645_gb300 import cases, fslbm

pytestmark = pytest.mark.gpu

DIMS = (512, 256, 256)
TAU, MAGIC = 0.53, 0.005  # the bench workload


def _dam(**kw):
    return cases.dam_break(nx=DIMS[0], ny=DIMS[1], nz=DIMS[2], col_x=128, col_z=192, tau=TAU, magic=MAGIC, **kw)


def _lattice(c, precision):
    import torch
    dev = torch.device("cuda:0")
    lat = fslbm.Lattice(c["dims"], c["params"], precision=precision)
    t = {k: torch.from_numpy(c[k]).to(dev) for k in ("flags", "rho", "u", "phi")}
    lat.init_equilibrium(t["flags"], t["rho"], t["u"], t["phi"])
    return lat, dev


def _window(field, centre, half, fill, per_link=False):
    """Cube of side 2*half around centre; cells beyond the lattice get `fill`
    (a face of the lattice is a wall, so flags are padded with WALL)."""
    import torch
    nx, ny, nz = DIMS
    cx_, cy_, cz_ = centre
    side = 2 * half
    shape = (19, side, side, side) if per_link else (side, side, side)
    out = torch.full(shape, fill, dtype=field.dtype, device=field.device)
    xs, ys, zs = (slice(max(c - half, 0), min(c + half, n)) for c, n in zip(centre, DIMS))
    ox, oy, oz = (s.start - (c - half) for s, c in zip((xs, ys, zs), centre))
    lx, ly, lz = (s.stop - s.start for s in (xs, ys, zs))
    if per_link:
        v = field.view(19, nz, ny, nx)[:, zs, ys, xs]
        out[:, oz:oz + lz, oy:oy + ly, ox:ox + lx] = v
    else:
        v = field.view(nz, ny, nx)[zs, ys, xs]
        out[oz:oz + lz, oy:oy + ly, ox:ox + lx] = v
    return out.cpu().numpy()


def test_full_size_windows_match_oracle_fp64():
    """After 300 steps of the full-size FP64 dam break (conversions under way),
    one more GPU step equals the oracle's step on windows of 24^3 around
    sampled interface cells: flags bit-exact, f~, m, phi within 1e-12 on the
    inner 14^3 of each window (its dependencies lie inside the window)."""
    c = _dam()
    lat, dev = _lattice(c, "f64")
    lat.step(300)
    mask = fslbm.FIELD_FLAGS | fslbm.FIELD_F | fslbm.FIELD_MASS | fslbm.FIELD_PHI
    s0 = lat.get(mask, device=dev)
    lat.step(1)
    s1 = lat.get(mask, device=dev)
    fl = s0["flags"].cpu().numpy()
    ifc = np.where(fl == cases.INTERFACE)[0]
    rng = np.random.default_rng(1409)
    half, margin = 12, 5
    nx, ny, nz = DIMS
    picks = rng.choice(ifc, size=6, replace=False)
    params = dict(c["params"])
    params["periodic"] = (0, 0, 0)
    checked = 0
    for i in picks:
        centre = (int(i % nx), int((i // nx) % ny), int(i // (nx * ny)))
        W = lambda st, name, fill, pl=False: _window(st[name], centre, half, fill, pl)
        o = Oracle((2 * half,) * 3, params)
        o.step_from_post(W(s0, "flags", cases.WALL).reshape(-1), W(s0, "f", 0.0, True).reshape(19, -1),
                         W(s0, "m", 0.0).reshape(-1), W(s0, "phi", 0.0).reshape(-1))
        side = 2 * half
        sl = slice(margin, side - margin)
        cube = lambda a: a.reshape(-1, side, side, side)[:, sl, sl, sl]
        fl_gpu = W(s1, "flags", cases.WALL).reshape(-1)
        fo = o.flags()
        assert np.array_equal(cube(fo), cube(fl_gpu)), f"flags differ near cell {i}"
        fluid = ((fo == 1) | (fo == 2)).astype(np.float64)
        ref = o.get(F_POST) * fluid[None, :]
        got = W(s1, "f", 0.0, True).reshape(19, -1) * fluid[None, :]
        err = np.abs(cube(got) - cube(ref)).max() / np.abs(ref).max()
        assert err < 1e-12, f"populations differ by {err:.2e} near cell {i}"
        for name, fid in (("m", MASS), ("phi", PHI)):
            g = W(s1, name, 0.0).reshape(-1)
            r = o.get(fid)
            e = np.abs(cube(g) - cube(r)).max() / max(np.abs(r).max(), 1e-300)
            assert e < 1e-12, f"{name} differs by {e:.2e} near cell {i}"
        checked += 1
    assert checked == len(picks)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-11), ("f32", 2e-3), ("f16", 2e-3)])
def test_full_size_invariants(precision, tol):
    """Mass ledger, no liquid cell next to gas, fills and empties happen, the
    run stays finite (1000 steps of the bench workload)."""
    import torch
    c = _dam()
    lat, dev = _lattice(c, precision)
    M0, _ = lat.total_mass()
    conv = np.zeros(4)
    for _ in range(10):
        lat.step(99)
        lat.step(1)
        conv += np.array(lat.counters()[:4])
    lat.sync()
    M1, lost = lat.total_mass()
    assert abs(M1 - M0) / M0 < tol
    st = lat.get(fslbm.FIELD_FLAGS, device=dev)
    fl = st["flags"].view(DIMS[2], DIMS[1], DIMS[0])
    liq = fl == cases.LIQUID
    gas = fl == cases.GAS
    for q in range(1, 19):
        c_ = cases.LINKS[q]
        sh = torch.roll(gas, shifts=(-int(c_[2]), -int(c_[1]), -int(c_[0])), dims=(0, 1, 2))
        # the roll wraps around the faces; faces are walls, so mask the wrapped layer
        valid = torch.ones_like(gas)
        for ax, cc in zip((2, 1, 0), c_):
            if cc == 1:
                valid.narrow(ax, valid.shape[ax] - 1, 1).zero_()
            elif cc == -1:
                valid.narrow(ax, 0, 1).zero_()
        assert not bool((liq & sh & valid).any()), f"liquid next to gas along link {q}"
    assert conv[0] > 0 and conv[2] > 0
