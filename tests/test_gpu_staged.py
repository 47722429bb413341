"""The other bulk kernels of FP32 and FP16 storage (cp.async copies and TMA
row copies into shared memory, two x-adjacent cells per lane): identical
results to the plain-load kernel, bit for bit, on lattices with a ragged last
x segment, walls, periodic wraps and conversions; the rule that selects
them."""
import numpy as np
import pytest

from paper_1409_5645_gb300 import cases, fslbm

pytestmark = pytest.mark.gpu

MASK = fslbm.FIELD_FLAGS | fslbm.FIELD_F | fslbm.FIELD_MASS | fslbm.FIELD_PHI


def _pair(c, precision, steps, every, loads):
    a = fslbm.Lattice.from_case(c, precision=precision, bulk_loads=loads)
    b = fslbm.Lattice.from_case(c, precision=precision, bulk_loads="plain")
    assert a.bulk_loads == loads and b.bulk_loads == "plain"
    conv = np.zeros(4)
    for s in range(0, steps, every):
        a.step(every)
        b.step(every)
        sa, sb = a.get(MASK), b.get(MASK)
        for k in ("flags", "f", "m", "phi"):
            assert np.array_equal(sa[k], sb[k]), f"{precision}: {k} differs after {s + every} steps"
        conv += np.array(a.counters()[:4])
    return conv


@pytest.mark.parametrize("loads", ["async", "tma", "pairs"])
@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_staged_equals_plain_dam_break(precision, loads):
    """72 x 40 x 48 dam break (last x segment 8 cells): walls on all faces,
    fills and empties."""
    c = cases.dam_break(nx=72, ny=40, nz=48, col_x=24, col_z=32, tau=0.6, g=2e-4, rule=1)
    conv = _pair(c, precision, 300, 50, loads)
    assert conv[0] > 0 and conv[2] > 0


@pytest.mark.parametrize("loads", ["async", "tma", "pairs"])
@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_staged_equals_plain_periodic_blob(precision, loads):
    """48^3 periodic box with a liquid blob in uniform flow: the wraps take the
    general path, the interior the staged rows."""
    n = 48
    N = n ** 3
    i = np.arange(N)
    x, y, z = i % n + 0.5, (i // n) % n + 0.5, i // (n * n) + 0.5
    r = np.sqrt((x - 24.2) ** 2 + (y - 23.7) ** 2 + ((z - 24.1) / 0.8) ** 2)
    phi = np.clip(14.3 - r + 0.5, 0.0, 1.0)
    params = cases.default_params(tau=0.7, rule=1, periodic=(1, 1, 1), g=(1e-4, 0.0, -5e-5))
    flags = cases.classify((n, n, n), params["periodic"], 0, phi)
    u = np.tile(np.array([0.02, -0.015, 0.01]), (N, 1))
    c = cases.Case(dims=(n, n, n), params=params, flags=flags, rho=np.ones(N), u=u,
                   phi=np.where(flags == 2, phi, 0.0), noise=cases.uniform(7, 19 * N, 1e-4), wall_delta=None)
    conv = _pair(c, precision, 200, 40, loads)
    assert conv[0] + conv[1] > 0


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_async_odd_sizes_equal_plain(precision):
    """cp.async staging on odd sizes (FP16 words straddling cells, the last
    word of the population array): 37 x 9 x 11 dam break."""
    c = cases.dam_break(nx=37, ny=9, nz=11, col_x=12, col_z=7, tau=0.6, g=2e-4, rule=1)
    _pair(c, precision, 120, 30, "async")


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_pairs_ragged_segment_all_faces(precision):
    """Two cells per lane on a 70 x 12 x 20 dam break: rows of 32 + 32 + 6
    cells, the column's front crossing segment ends, half-way bounce-back at
    all six faces (the x faces on the end lanes' extra words, the y and z
    faces on whole rows)."""
    c = cases.dam_break(nx=70, ny=12, nz=20, col_x=33, col_z=15, tau=0.6, g=3e-4, rule=1)
    conv = _pair(c, precision, 300, 60, "pairs")
    assert conv[0] > 0 and conv[2] > 0


@pytest.mark.parametrize("precision", ["f32", "f16"])
@pytest.mark.parametrize("make", [lambda: cases.inclined_film(), lambda: cases.plate_flow(),
                                  lambda: cases.standing_wave(n=64, depth=32.0)],
                         ids=["inclined_film_cli", "plate_flow_moving_wall", "standing_wave_sigma"])
def test_pairs_general_path_cases(precision, make):
    """Segments whose liquid cells need the general pull (CLI link fractions
    at WALL cells, the shifted x wrap, a moving wall, periodic faces) take
    it; the rest of the lattice the pairs."""
    _pair(make(), precision, 200, 50, "pairs")


@pytest.mark.parametrize("precision,loads", [("f32", "pairs"), ("f16", "pairs"), ("f64", "plain")])
@pytest.mark.parametrize("rule", [0, 1])
def test_overlap_equals_serial(precision, loads, rule):
    """The interface kernels on a second stream beside the bulk kernel give
    the step of every kernel in order, bit for bit, and the same mass (dam
    break with conversions, ragged rows)."""
    c = cases.dam_break(nx=70, ny=12, nz=20, col_x=33, col_z=15, tau=0.6, g=3e-4, rule=rule)
    a = fslbm.Lattice.from_case(c, precision=precision, bulk_loads=loads)
    b = fslbm.Lattice.from_case(c, precision=precision, bulk_loads=loads)
    b.set_overlap(False)
    conv = 0
    for s in range(5):
        a.step(60)
        b.step(60)
        sa, sb = a.get(MASK), b.get(MASK)
        for k in ("flags", "f", "m", "phi"):
            assert np.array_equal(sa[k], sb[k]), f"{precision}: {k} differs after {60 * (s + 1)} steps"
        (ma, la), (mb, lb) = a.total_mass(), b.total_mass()
        assert ma == mb
        assert la == pytest.approx(lb, rel=1e-12, abs=1e-15)  # (the ledger's atomics sum in any order)
        conv += sum(a.counters()[:4])
    assert conv > 0


def test_selection_rule():
    """Staged loads and pairs for FP32/FP16 storage only; TMA rows need nx a
    multiple of 16 bytes of elements and nx >= 32 cells + two 16-byte halos,
    pairs an even nx."""
    p = cases.default_params(tau=0.6)
    for dims, prec, loads, want in [
            ((72, 8, 8), "f32", "tma", "tma"), ((40, 8, 8), "f32", "tma", "tma"), ((36, 8, 8), "f32", "tma", "plain"),
            ((70, 8, 8), "f32", "tma", "plain"), ((72, 8, 8), "f16", "tma", "tma"), ((44, 8, 8), "f16", "tma", "plain"),
            ((68, 8, 8), "f16", "tma", "plain"), ((64, 8, 8), "f64", "tma", "plain"), ((64, 8, 8), "f64", "async", "plain"),
            ((37, 5, 3), "f32", "async", "async"), ((37, 5, 3), "f16", "async", "async"),
            ((72, 8, 8), "f16", "pairs", "pairs"), ((38, 5, 3), "f32", "pairs", "pairs"),
            ((37, 5, 3), "f16", "pairs", "plain"), ((64, 8, 8), "f64", "pairs", "plain")]:
        lat = fslbm.Lattice(dims, dict(p, bulk_loads=loads), precision=prec)
        assert lat.bulk_loads == want, (dims, prec, loads)
        lat.close()
