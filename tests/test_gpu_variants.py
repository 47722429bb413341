"""Interface-tracking variants of the works the paper's tracking follows
(Sec. 4.4, Sec. 6) on the CUDA path, against the oracle: the reconstruction of
the links along the surface normal (recon_nc) and the excess split along the
fill-level normal (excess_split); the grid barrier of the conversion kernel,
the step's mass reduction and launch count, and the extended interface kernel
in the reduced-precision forms."""
import numpy as np
import pytest

from gpu_util import run_parity
from paper_1409_5645_gb300 import cases

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rule", [0, 1])
def test_dam_break_parity_normal_links(rule):
    """Dam break with conversions, interior and edge interface cells."""
    c = cases.dam_break(nx=24, ny=12, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=rule, recon_nc=1)
    _, _, conv = run_parity(c, 120, every=1)
    assert conv[0] + conv[1] > 0 and conv[2] + conv[3] > 0


def test_inclined_film_parity_normal_links():
    """Tilted frozen surface (shifted wrap, CLI wall): the normal links are
    rebuilt on every interface cell."""
    run_parity(cases.inclined_film(h=8, rule=1, recon_nc=1), 300, every=30)


def test_wave_parity_normal_links_with_all_options():
    """Capillary wave with the shear term, the extrapolated u_b and the normal
    links together."""
    c = cases.standing_wave(n=24, depth=12.0, amp=1.5, tau=0.6, g=1e-4, sigma=5e-3, phi_noise=1e-4,
                            stress=1, ub_extrap=1, recon_nc=1)
    run_parity(c, 60, every=1)


@pytest.mark.parametrize("rule", [0, 1])
def test_dam_break_parity_weighted_split(rule):
    c = cases.dam_break(nx=24, ny=12, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=rule, excess_split=1)
    _, _, conv = run_parity(c, 150, every=1)
    assert conv[0] > 0 and conv[1] > 0


@pytest.mark.parametrize("phi_c", [1.05, -0.05])
def test_single_conversion_parity_weighted_split(phi_c):
    """One cell fills (or empties) under a flat surface: the weighted split
    sends its excess across the surface only."""
    c = cases.film(nx=4, ny=4, nz=16, h=8.5, gx=0.0, noise_amp=0.0, excess_split=1)
    c["phi"][1 + 4 * (2 + 4 * 8)] = phi_c
    _, _, conv = run_parity(c, 20, every=1)
    assert conv[0] + conv[1] >= 1


def test_dam_break_parity_all_tracking_variants():
    """Dam break of a ragged size with the normal links, the weighted split,
    the extrapolated u_b and the shear term together."""
    c = cases.dam_break(nx=21, ny=11, nz=17, col_x=7, col_z=12, tau=0.62, g=2e-4, rule=1,
                        recon_nc=1, excess_split=1, ub_extrap=1, stress=1)
    _, _, conv = run_parity(c, 150, every=1)
    assert conv[0] > 0 and conv[1] > 0


def test_grid_barrier_bounded_wait():
    """The grid barrier between the conversion stages completes, and when
    nothing completes it (it waits for one block more than exist) its bounded
    wait runs out with FSLBM_ERR_TIMEOUT instead of hanging; the context stays
    usable and a lattice steps normally afterwards."""
    import time
    from paper_1409_5645_gb300 import fslbm
    assert fslbm.check_grid_barrier(False) == "ok"
    t0 = time.time()
    assert fslbm.check_grid_barrier(True) == "timeout"
    assert time.time() - t0 < 10.0
    c = cases.dam_break(nx=24, ny=8, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=1)
    run_parity(c, 40, every=10)


@pytest.mark.parametrize("freeze", [0, 1])
def test_step_mass_equals_recount(freeze):
    """The mass reduced inside each step (by the cooperative conversion kernel,
    or by the stand-alone reduction with frozen flags) equals the full recount
    after the step, whose conversions conserve it (FP64, dam break with
    conversions; inclined film with a frozen interface)."""
    from paper_1409_5645_gb300 import fslbm
    if freeze:
        c = cases.inclined_film(h=8, rule=1)
    else:
        c = cases.dam_break(nx=24, ny=12, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=1)
    g = fslbm.Lattice.from_case(c, precision="f64")
    for _ in range(60):
        g.step(1)
        ms = g.step_mass()
        M, _ = g.total_mass()
        assert abs(ms - M) <= 1e-12 * M, (ms, M)
    g.close()


@pytest.mark.parametrize("precision,tol", [("f32", 2e-3), ("f16", 2e-2)])
def test_reduced_precision_with_all_options(precision, tol):
    """The extended interface kernel in the FP32 and FP16-storage forms (shear
    term, extrapolated u_b, normal links, weighted split): 300 steps of a dam
    break stay finite, keep the mass ledger, convert cells, and stay near the
    FP64 run (mean fill-level difference, share of cells of another kind)."""
    from paper_1409_5645_gb300 import fslbm
    c = cases.dam_break(nx=32, ny=12, nz=20, col_x=10, col_z=14, tau=0.6, g=2e-4, rule=1,
                        stress=1, ub_extrap=1, recon_nc=1, excess_split=1)
    out = {}
    for prec in ("f64", precision):
        g = fslbm.Lattice.from_case(c, precision=prec)
        M0, _ = g.total_mass()
        conv = np.zeros(4)
        for _ in range(30):
            g.step(10)
            conv += np.array(g.counters()[:4])
        M1, _ = g.total_mass()
        st = g.get(fslbm.FIELD_PHI | fslbm.FIELD_FLAGS)
        out[prec] = (M0, M1, conv, st["phi"], st["flags"])
        g.close()
    M0, M1, conv, phi, fl = out[precision]
    assert np.isfinite(phi).all() and conv[0] + conv[1] > 0
    assert abs(M1 - M0) / M0 < tol
    assert np.mean(np.abs(phi - out["f64"][3])) < 0.02
    assert np.mean(fl != out["f64"][4]) < 0.02


def test_launches_per_step():
    """The launch count a step reports: reset, segments, bulk, interface,
    the geometry kernel where the rule needs it, and the conversions with the
    mass reduction in one cooperative launch (two reduction launches and no
    conversions with frozen flags)."""
    from paper_1409_5645_gb300 import fslbm
    film = cases.film(nx=4, ny=4, nz=16, h=9.0)
    expect = {(1, 0): 6, (0, 0): 5, (1, 1): 7, (0, 1): 6}
    for (rule, freeze), n in expect.items():
        g = fslbm.Lattice(film["dims"], dict(film["params"], rule=rule, freeze=freeze))
        assert g.launches_per_step == n, (rule, freeze, g.launches_per_step)
        g.close()


def test_dam_break_parity_elvira():
    """The ELVIRA normal where the height columns are open (Sec. 5's
    higher-order reconstruction; walls and the column's corners leave many
    columns open): FSL dam break with conversions, every step against the
    oracle."""
    c = cases.dam_break(nx=24, ny=8, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=1, elvira=1)
    _, _, conv = run_parity(c, 150, every=1)
    assert conv[0] > 0


def test_plane_parity_elvira_open_columns():
    """A frozen plane 2.4 cells above a wall (every surface column open),
    FSL with ELVIRA: parity with the oracle, whose ELVIRA plane is exact
    there (the oracle pins)."""
    import sys
    sys.path.insert(0, __file__.rsplit("/", 1)[0])
    from test_oracle_pins import _plane_case
    case, _, _, _ = _plane_case(0.17, -0.11, 2.45, elvira=1)
    case["params"]["rule"] = 1
    run_parity(case, 60, every=5, check_mass=False)


def test_fp64_rate_is_measured():
    """The FP64 arithmetic ceiling the FP64 form is reported against: dependent
    FMA chains on every SM give a rate of the order of the device's nominal
    FP64 throughput (1.25 TFLOP/s for GB300)."""
    from paper_1409_5645_gb300 import fslbm
    r = fslbm.fp64_rate()
    print(f"FP64 FMA rate {r:.3f} TFLOP/s")
    assert 0.2 < r < 10.0
