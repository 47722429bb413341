"""The oracle's step against an exact-rational restatement (tests/rational_step.py).

The restatement is written independently from the paper (Eq. lbe1/lbe2,
Eq. eqEven/eqOdd, Eq. koerner, Eq. closure with Table 1, Sec. 2.3) and from
the readings of the interface tracking the paper takes from Koerner et al. and
Thuerey (Sec. 4.4): thresholds, isolated-cell rules, an emptied cell next to a
filled one staying interface, new cells from gas at the equilibrium of their
fluid neighbours' mean, new cells from liquid with m = rho, equal excess split
over the neighbours that are interface after the conversions and do not
convert themselves, the lost ledger.  Each step starts from the oracle's own
FP64 state (exact rationals), so the two differ only by the oracle's rounding
of one step: flags must agree bit for bit, populations, mass and fill levels
to a few ulp, and the rational step conserves mass exactly.
"""
import numpy as np
import pytest

import rational_step as rs
from oracle.oracle import F_PRE, MASS, PHI, Oracle
from paper_1409_5645_gb300 import cases

TOL = 2e-15  # one step's rounding in FP64, relative to the populations' scale


def _lattice(c):
    p = c["params"]
    return rs.Lattice(c["dims"], p["periodic"], p["tau"], p["magic"], p["g"], p["rho_G"], p["rule"],
                      p["eps"], p["cleanup"], p["linear_eq"], p["delta_min"])


def _state(o):
    """The oracle's state in rationals; m of a liquid cell is its exact
    density (the oracle reports it rounded)."""
    flags = [int(v) for v in o.flags()]
    f = [rs.from_float(row) for row in o.get(F_PRE)]
    m, phi = rs.from_float(o.get(MASS)), rs.from_float(o.get(PHI))
    for i, k in enumerate(flags):
        if k == rs.LIQ:
            m[i] = sum(f[q][i] for q in range(19))
    return flags, f, m, phi


def _compare(lat, o, state, variant=None, where=""):
    """One rational step from `state` against the oracle's next step; returns
    the events of the rational step.  Raises AssertionError on a mismatch."""
    flags, f, m, phi = state
    fl1, f1, m1, phi1, lost, ev = lat.step(flags, f, m, phi, variant=variant)
    # exact conservation of M = sum_liquid rho + sum_interface m + lost
    assert rs.total_mass(fl1, m1, lost) == rs.total_mass(flags, m, rs.Fr(0)), where
    L0 = o.total_mass()[1]
    assert o.step(1) == 0
    assert list(o.flags()) == fl1, f"{where}: flags differ"
    fo, mo, po = o.get(F_PRE), o.get(MASS), o.get(PHI)
    fe = np.array([[float(v) for v in row] for row in f1])
    assert np.abs(fo - fe).max() <= TOL, f"{where}: populations differ by {np.abs(fo - fe).max():.2e}"
    me = np.array([float(v) for v in m1])
    fluid = np.isin(np.array(fl1), (rs.LIQ, rs.IFC))
    assert np.abs(mo - me)[fluid].max(initial=0.0) <= TOL * 8, f"{where}: mass differs"
    ifc = np.array(fl1) == rs.IFC
    pe = np.array([float(v) for v in phi1])
    assert np.abs(po - pe)[ifc].max(initial=0.0) <= TOL * 8, f"{where}: fill levels differ"
    assert o.total_mass()[1] - L0 == pytest.approx(float(lost), abs=1e-15), f"{where}: lost ledger"
    return ev


def _run(c, steps, variant=None):
    o = Oracle.from_case(c)
    lat = _lattice(c)
    tot = {}
    for s in range(1, steps + 1):
        ev = _compare(lat, o, _state(o), variant, f"step {s}")
        for k, v in ev.items():
            tot[k] = tot.get(k, 0) + v
    return tot


@pytest.mark.parametrize("seed", [1409, 1415])
def test_oracle_step_equals_exact_step_fsk_with_conversions(seed):
    """FSK on the 3 x 3 x 6 churn lattice: 20 steps, each compared with the
    exact step, covering fills, empties, an empty cell kept next to a fill,
    new cells from gas and from liquid."""
    tot = _run(cases.churn(seed=seed), 20)
    print(seed, tot)
    for k in ("fill", "empty", "dropped", "new_gas", "new_liq"):
        assert tot[k] > 0, (k, tot)


def test_oracle_step_equals_exact_step_linear_equilibrium_srt():
    """The same with the linear equilibrium and a single relaxation rate."""
    tot = _run(cases.churn(seed=1411, linear_eq=1, magic=0.0), 12)
    assert tot["fill"] > 0 and tot["new_gas"] > 0


def _closed_surface_case(seed=1409):
    """4 x 4 x 14, x and y periodic: a surface near z = 6.4 with fill noise of
    amplitude 0.3, slow enough that every interface cell keeps closed height
    columns (rational link fractions) for the steps compared."""
    c = cases.film(nx=4, ny=4, nz=14, h=6.4, tau=0.8, gx=2e-4, rule=1, noise_amp=1e-4)
    ifc = c["flags"] == cases.INTERFACE
    c["phi"] = c["phi"].copy()
    c["phi"][ifc] = np.clip(c["phi"][ifc] + cases.uniform(seed, int(ifc.sum()), 0.3, offset=7), 0.02, 1.0)
    c["u"] = np.zeros((c.N, 3))
    fl = (c["flags"] == cases.LIQUID) | ifc
    c["u"][fl] = cases.uniform(seed, 3 * int(fl.sum()), 0.02, offset=99).reshape(-1, 3)
    return c


def test_oracle_step_equals_exact_step_fsl_closed_columns():
    """FSL where the link fraction is rational (closed height columns):
    10 steps, every gas link rebuilt with Table 1's FSL closure."""
    tot = _run(_closed_surface_case(), 10)
    assert tot["fsl_links"] > 100, tot


@pytest.mark.parametrize("variant", ["keep_empty", "new_avg_all", "new_avg_precollision", "recv_converting"])
def test_exact_comparison_detects_misread_conversion_rules(variant):
    """A plausible misreading of each conversion rule, planted in the
    rational restatement, makes the comparison fail on the churn lattice:
    the scenario exercises every rule, so the oracle is pinned on each."""
    with pytest.raises(AssertionError):
        _run(cases.churn(seed=1415), 20, variant=variant)


def test_plane_fit_regularisation_bound():
    """The plane fit keeps phi in [1e-9, 1 - 1e-9] before inverting the
    plane/cube volume (a corner cell's cube-root singularity).  Bound the
    plane shift this causes against the exact inverse: for phi below 1e-9 the
    true plane cuts off a corner tetrahedron, V = a^3 / (6 m1 m2 m3) with the
    L1-normalised normal m, so the offset along the unit normal moves by at
    most L1 * (6 m1 m2 m3 * 1e-9)^(1/3) <= sqrt(3) * (6/27 * 1e-9)^(1/3)."""
    from oracle.oracle import plic_offset
    rng = np.random.default_rng(11)
    bound = np.sqrt(3.0) * (6.0 / 27.0 * 1e-9) ** (1.0 / 3.0)
    worst = 0.0
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        a = np.sort(np.abs(n)) / np.abs(n).sum()
        L1 = np.abs(n).sum()
        for ph in (0.0, 1e-12, 5e-10):
            # exact corner-tetrahedron inverse, offset from the cell centre
            alpha = (6.0 * a[0] * a[1] * a[2] * ph) ** (1.0 / 3.0)
            exact = L1 * (alpha - 0.5)
            shift = abs(plic_offset(n, ph) - exact)
            worst = max(worst, shift)
            assert shift <= bound * (1 + 1e-9)
            # and the mirrored full corner
            shift_hi = abs(plic_offset(n, 1.0 - ph) + exact)
            assert shift_hi <= bound * (1 + 1e-6)
    print("largest plane shift from the fill clamp: %.3e cells (bound %.3e)" % (worst, bound))
    assert worst > 0.1 * bound  # the bound is reached in order of magnitude (the clamp is active)
