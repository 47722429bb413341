"""Slab decomposition on one GPU: two or three library handles, each owning a
slab and holding ghost layers beside the cuts, refilled once per step by the
library's pack/unpack kernels through device buffers (slabs.LocalSlabs).
Against one handle stepping the whole lattice: flags, post-collision
populations, interface mass and fill levels of every owned cell equal bit
for bit, with cells filling, emptying and appearing on both sides of the
cuts; the sum of the owned masses and lost ledgers equals the whole's."""
import numpy as np
import pytest

from paper_1409_5645_gb300 import cases, fslbm, slabs

pytestmark = pytest.mark.gpu

MASK = fslbm.FIELD_FLAGS | fslbm.FIELD_F | fslbm.FIELD_MASS | fslbm.FIELD_PHI


def _check(c, parts, axis, steps, precision, every=10):
    whole = fslbm.Lattice.from_case(c, precision=precision)
    run = slabs.LocalSlabs(c, parts, axis=axis, precision=precision)
    conv = 0
    for t in range(1, steps + 1):
        whole.step(1)
        run.step(1)
        conv += sum(whole.counters()[:4])
        if t % every == 0 or t == steps:
            a = whole.get(MASK)
            b = run.owned_fields(MASK)
            for k in ("flags", "f", "m", "phi"):
                assert np.array_equal(a[k], b[k]), f"t={t}: {k} differs at {np.argwhere(a[k] != b[k])[:5]}"
    Mw, Lw = whole.total_mass()
    Ms, Ls = run.total_mass()
    assert Ms == pytest.approx(Mw, rel=1e-12)
    assert Ls == pytest.approx(Lw, rel=1e-9, abs=1e-13)
    return conv


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("rule", [0, 1])
def test_slabs_along_z_through_a_churning_surface(precision, rule):
    c = cases.churn(nx=24, ny=20, nz=48, base=24.0, plant=False, u_amp=0.05, rule=rule, tau=0.75)
    conv = _check(c, 2, 2, 200, precision)
    assert conv > 100


def test_three_slabs_along_x_through_a_dam_break_front():
    """The column's front runs through both cuts (x = 16 and x = 32)."""
    c = cases.dam_break(nx=48, ny=10, nz=24, col_x=14, col_z=20, tau=0.6, g=4e-4, rule=1)
    conv = _check(c, 3, 0, 400, "f64", every=20)
    assert conv > 50


def test_halo_arguments_are_checked():
    c = cases.churn(nx=8, ny=8, nz=20, base=10.0)
    lat = fslbm.Lattice.from_case(c)
    with pytest.raises(fslbm.FslbmError):
        lat.halo_bytes((0, 0, 0), (8, 8, 21))  # outside the lattice
    with pytest.raises(fslbm.FslbmError):
        lat.set_owned((0, 0, 5), (8, 8, 5))  # empty box
    n = lat.halo_bytes((0, 0, 0), (8, 8, 2))
    assert n % 16 == 0 and n >= 128 * (1 + 8 + 8 + 19 * 8)
