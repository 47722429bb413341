"""Helpers shared by the GPU tests: run the CUDA library and the oracle side
by side and compare them field by field."""
import numpy as np

from oracle.oracle import F_POST, MASS, PHI, Oracle
from paper_1409_5645_gb300 import fslbm

TOL = 1e-12  # FP64 parity bar: relative to the field's largest magnitude, and per interface cell


def compare(o: Oracle, g: "fslbm.Lattice", tol=TOL, where=""):
    got = g.get(fslbm.FIELD_FLAGS | fslbm.FIELD_F | fslbm.FIELD_MASS | fslbm.FIELD_PHI)
    fo = o.flags()
    bad = np.nonzero(got["flags"] != fo)[0]
    assert bad.size == 0, f"{where}: flags differ at {bad[:10]} gpu={got['flags'][bad[:10]]} oracle={fo[bad[:10]]}"
    fluid = (fo == 1) | (fo == 2)
    ref = o.get(F_POST)
    err = np.abs(got["f"][:, fluid] - ref[:, fluid]).max(initial=0.0) / max(np.abs(ref).max(), 1e-300)
    assert err <= tol, f"{where}: populations differ by {err:.3e}"
    ifc = fo == 2
    for name, fid in (("m", MASS), ("phi", PHI)):
        r = o.get(fid)
        e = np.abs(got[name] - r).max(initial=0.0) / max(np.abs(r).max(), 1e-300)
        assert e <= tol, f"{where}: {name} differs by {e:.3e}"
        # interface cells one by one, relative to each cell's own value, with
        # a floor of 0.1 (a tenth of the density) for cells that are nearly
        # empty: their mass is a sum of fluxes and excess shares, differences
        # of O(1) quantities, whose rounding is absolute, not relative
        d = np.abs(got[name][ifc] - r[ifc]) / np.maximum(np.abs(r[ifc]), 0.1)
        e1 = d.max(initial=0.0)
        assert e1 <= tol, f"{where}: interface {name} differs by {e1:.3e} (per cell)"
    return err


def run_parity(case, steps, every=1, precision="f64", tol=TOL, check_mass=True):
    o = Oracle.from_case(case)
    g = fslbm.Lattice.from_case(case, precision=precision)
    compare(o, g, tol, "t=0")
    conv = np.zeros(4, dtype=np.int64)
    for s in range(1, steps + 1):
        assert o.step(1) == 0
        g.step(1)
        if s % every == 0 or s == steps:
            compare(o, g, tol, f"t={s}")
            conv += np.array(g.counters()[:4])
    if check_mass:
        Mo, Lo = o.total_mass()
        Mg, Lg = g.total_mass()
        assert abs(Mg - Mo) <= 1e-12 * abs(Mo)
        assert abs(Lg - Lo) <= 1e-12 * max(abs(Mo), 1.0)
    g.sync()
    return o, g, conv
