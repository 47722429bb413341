"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of these compares the oracle
with itself: they use closed forms (film profiles, plane geometry), the
paper's printed Table 1, invariants (equilibrium fixed point, mass ledger),
brute force (plane/cube volume) and the convergence orders the paper reports.
"""
import math
import os

import numpy as np
import pytest

from oracle.oracle import F_POST, F_PRE, PHI, RHO, VEL, Oracle, cube_volume, plic_offset
from paper_1409_5645_gb300 import cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
CQ = cases.LINKS.astype(np.float64)
OPP = np.array([0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17])


def load_table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_closure_coefficients.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, a0, ab0, a1, ap, C = line.split()
        rows[name] = (a0, ab0, a1, ap, C)
    return rows


def coeffs(rule, delta, lam):
    env = {"delta": delta, "lam": lam}
    return [eval(e, {}, env) for e in load_table1()[rule]]


# --------------------------------------------------------------------------
# Table 1 against the matching conditions of Sec. 3.3 (Eq. cl1 .. cl4)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("delta", [0.0, 0.17, 0.5, 0.83, 1.0])
def test_table1_matching_conditions(delta):
    rng = np.random.default_rng(5645)
    for _ in range(20):
        lp, lm = rng.uniform(-1.95, -0.05, 2)
        Lp = -(0.5 + 1 / lp)
        for rule in ("FSK", "FSL"):
            a0, ab0, a1, ap, C = coeffs(rule, delta, lp)
            alpha_p = 1 - a0 - ab0 - a1                       # Eq. cl1
            beta_p = 1 - (1 + lp) * (a0 + ab0) - a1 - C
            alpha_m = ab0 - a0 - a1 - 1
            beta_m = (1 + lm) * ab0 - (1 + lm) * a0 - a1 - 1
            assert alpha_p == pytest.approx(ap, abs=1e-14)
            assert alpha_m == pytest.approx(0.0, abs=1e-14)   # Eq. cl2
            cl3 = beta_m - ap * delta * lm                     # Eq. cl3
            cl4 = beta_p + ap * Lp * lp                        # Eq. cl4
            if rule == "FSL":
                assert cl3 == pytest.approx(0.0, abs=1e-13)
                assert cl4 == pytest.approx(0.0, abs=1e-13)
            elif delta == 0.5:  # FSK matches only at delta = 1/2 (Sec. 3.2)
                assert cl3 == pytest.approx(0.0, abs=1e-13)
            else:
                assert abs(cl3) > 1e-6


# --------------------------------------------------------------------------
# The oracle's free-surface closure against Table 1, link by link
# --------------------------------------------------------------------------
def _eplus(rho, u):
    cu = CQ @ u
    return W * (rho + 1.5 * (3 * cu * cu - u @ u))


@pytest.mark.parametrize("rule", ["FSK", "FSL"])
def test_oracle_closure_follows_table1(rule):
    h = 6.37
    c = cases.film(nx=4, ny=3, nz=12, h=h, rule=1 if rule == "FSL" else 0,
                   noise_amp=2e-3, freeze=1, g=(1e-4, -2e-5, 0.0))
    o = Oracle.from_case(c)
    N = c.N
    f0 = o.get(F_PRE)
    ft = o.get(F_POST)
    u0 = o.get(VEL)
    _, _, _, delta, _ = o.geometry()
    tau = c["params"]["tau"]
    lp = -1.0 / tau
    o.step(1)
    f1 = o.get(F_PRE)
    flags = c["flags"]
    nx, ny, nz = c["dims"]
    checked = 0
    for i in np.where(flags == cases.INTERFACE)[0]:
        x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
        rho = f0[:, i].sum()
        ep = _eplus(rho, u0[i])
        fp = 0.5 * (f0[:, i] + f0[OPP, i])
        nplus = fp - ep
        eb = _eplus(c["params"]["rho_G"], u0[i])
        for p in range(1, 19):
            cx, cy, cz = cases.LINKS[p]
            X, Y, Z = (x + cx) % nx, (y + cy) % ny, z + cz
            if not (0 <= Z < nz) or flags[X + nx * (Y + ny * Z)] != cases.GAS:
                continue
            q = OPP[p]
            Xu, Yu, Zu = (x - cx) % nx, (y - cy) % ny, z - cz
            up = Xu + nx * (Yu + ny * Zu)
            a0, ab0, a1, ap, C = coeffs(rule, delta[p, i], lp)
            expect = (a0 * ft[p, i] + ab0 * ft[q, i] + a1 * ft[p, up] + C * nplus[p]
                      + ap * eb[p])
            assert f1[q, i] == pytest.approx(expect, rel=0, abs=1e-14)
            checked += 1
    assert checked >= 4 * 3 * 5


# --------------------------------------------------------------------------
# Invariants: uniform equilibrium is a fixed point; mass is conserved
# --------------------------------------------------------------------------
def _blob_case(rule, u=(0.01, -0.02, 0.005)):
    n = 12
    dims = (n, n, n)
    N = n ** 3
    i = np.arange(N)
    x, y, z = i % n + 0.5, (i // n) % n + 0.5, i // (n * n) + 0.5
    r = np.sqrt((x - 6.2) ** 2 + (y - 5.7) ** 2 + ((z - 6.1) / 0.8) ** 2)
    phi = np.clip(4.3 - r + 0.5, 0.0, 1.0)
    params = cases.default_params(tau=0.7, rule=rule, periodic=(1, 1, 1))
    flags = cases.classify(dims, params["periodic"], 0, phi)
    return cases.Case(dims=dims, params=params, flags=flags, rho=np.ones(N),
                      u=np.tile(np.array(u), (N, 1)), phi=np.where(flags == 2, phi, 0.0),
                      noise=None, wall_delta=None)


@pytest.mark.parametrize("rule", [0, 1])
def test_uniform_equilibrium_is_fixed_point(rule):
    """A uniform equilibrium at (rho_G, u) is reproduced by both closures
    (alpha_+ = 1 - a0 - abar0 - a1 and a0 - abar0 + a1 = -1 in Table 1), so f
    stays uniform through streaming, closures and conversions."""
    c = _blob_case(rule)
    o = Oracle.from_case(c)
    M0, _ = o.total_mass()
    f0 = o.get(F_PRE)
    ref = f0[:, np.where(c["flags"] == 1)[0][0]]
    o.step(40)
    fl = o.flags()
    f1 = o.get(F_PRE)
    fluid = (fl == 1) | (fl == 2)
    assert np.abs(f1[:, fluid] - ref[:, None]).max() < 1e-15
    M1, lost = o.total_mass()
    assert abs(M1 - M0) / M0 < 1e-13
    conv, t = o.counters()
    assert t == 40


def _mini_dam(rule=1, **kw):
    return cases.dam_break(nx=24, ny=8, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4,
                           phi_noise=1e-3, rule=rule, **kw)


@pytest.mark.parametrize("rule", [0, 1])
def test_mass_ledger_conserved_through_conversions(rule):
    """Total mass sum_L rho + sum_I m + lost is invariant (exact in exact
    arithmetic: the mass exchange is pairwise antisymmetric and every
    conversion moves its excess to receivers or to the ledger)."""
    c = _mini_dam(rule)
    o = Oracle.from_case(c)
    M0, _ = o.total_mass()
    conv = np.zeros(4, dtype=np.int64)
    for _ in range(300):
        assert o.step(1) == 0
        conv += np.array(o.counters()[0])
    M1, lost = o.total_mass()
    assert abs(M1 - M0) / M0 < 2e-13
    assert conv[0] > 0 and conv[2] > 0  # cells filled, cells created from gas
    # every liquid cell keeps away from gas
    fl = o.flags()
    nx, ny, nz = c["dims"]
    i = np.arange(c.N)
    for q in range(1, 19):
        j = cases._neighbour_index(c["dims"], (0, 0, 0), 0, i, cases.LINKS[q])
        bad = (fl == 1) & (j >= 0) & (fl[np.maximum(j, 0)] == 4)
        assert not bad.any()


# --------------------------------------------------------------------------
# Film flows (Sec. 4.3): closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rule", [0, 1])
def test_film_transient_matches_series(rule):
    """4x4x32 film, h = 20, tau = 0.8, g = 1e-6, 5000 steps from rest: the
    velocity follows the separation-of-variables series of u_t = nu u_zz + g
    with u(0)=0, u_z(h)=0; mass is conserved."""
    c = cases.film(rule=rule)
    o = Oracle.from_case(c)
    M0, _ = o.total_mass()
    assert o.step(5000) == 0
    u = o.get(VEL)[:, 0].reshape(32, 4, 4)
    nu = (0.8 - 0.5) / 3
    z = np.arange(20) + 0.5
    ex = cases.film_transient(z, 5000, 20.0, 1e-6, nu)
    err = np.abs(u[:20] - ex[:, None, None]).max() / ex.max()
    assert err < 5e-5
    M1, _ = o.total_mass()
    assert abs(M1 - M0) / M0 < 1e-12


@pytest.mark.parametrize("h,rule,exact", [
    (8.0, 0, True), (8.0, 1, True),      # integer depth: delta = 1/2
    (8.33, 1, True), (8.6, 1, True),     # FSL exact for any depth (Sec. 4.3)
    (8.33, 0, False), (8.6, 0, False),   # FSK first order off delta = 1/2
])
def test_film_steady_state(h, rule, exact):
    freeze = int(h != int(h))
    c = cases.film(nz=16, h=h, rule=rule, noise_amp=0.0, freeze=freeze)
    o = Oracle.from_case(c)
    o.step(12000)
    fl = c["flags"].reshape(16, 4, 4)[:, 0, 0]
    n = int(np.sum((fl == 1) | (fl == 2)))
    u = o.get(VEL)[:, 0].reshape(16, 4, 4)[:n, 0, 0]
    ex = cases.film_profile(np.arange(n) + 0.5, h, 1e-6, 0.1)
    err = np.abs(u - ex).max() / ex.max()
    if exact:
        assert err < 1e-9
    else:
        assert err > 1e-2


@pytest.mark.parametrize("rule", [0, 1])
def test_hydrostatic_gravity_toward_wall(rule):
    """Gravity toward the wall adds a hydrostatic gradient that leaves the
    film profile unchanged with rho_0 = 1 (Sec. 4.3); u_z stays at round-off
    and the fill levels do not move."""
    h = 12.0
    c = cases.film(nz=16, h=h, rule=rule, noise_amp=0.0, g=(1e-6, 0.0, -1e-4))
    z = np.arange(c.N) // 16 + 0.5
    c["rho"] = 1.0 + 3 * 1e-4 * np.maximum(h - z, 0)
    o = Oracle.from_case(c)
    phi0 = o.get(PHI)
    o.step(20000)
    u = o.get(VEL).reshape(16, 16, 3)[:12, 0, :]
    ex = cases.film_profile(np.arange(12) + 0.5, h, 1e-6, 0.1)
    assert np.abs(u[:, 0] - ex).max() / ex.max() < 1e-9
    assert np.abs(u[:, 2]).max() < 1e-13
    assert np.abs(o.get(PHI) - phi0).max() < 1e-9


# --------------------------------------------------------------------------
# Inclined film (Sec. 4.3, rotated film): convergence orders
# --------------------------------------------------------------------------
def _inclined_error(h, rule):
    c = cases.inclined_film(h=h, rule=rule)
    o = Oracle.from_case(c)
    fl = c["flags"]
    fluid = (fl == 1) | (fl == 2)
    n = np.clip(c["ncoord"], 0, None)
    H, nu, g = c["H"], c["nu"], c["gmag"]
    ex = (g / (2 * nu) * (2 * H * n - n * n))[:, None] * c["t_hat"][None, :]
    prev = o.get(VEL)[fluid]
    for _ in range(2000):
        o.step(200)
        u = o.get(VEL)[fluid]
        ch = np.sqrt(((u - prev) ** 2).sum() / (u ** 2).sum())
        prev = u
        if ch < 1e-12:
            break
    e = u - ex[fluid]
    return np.sqrt((e ** 2).sum() / (ex[fluid] ** 2).sum())


def test_inclined_film_convergence_orders():
    """FSL second order, FSK first order on a film inclined to the lattice
    (slope 1/2, CLI wall, exact fill levels, fixed Reynolds number)."""
    e = {(r, h): _inclined_error(h, r) for r in (0, 1) for h in (8, 16)}
    fsk = math.log2(e[(0, 8)] / e[(0, 16)])
    fsl = math.log2(e[(1, 8)] / e[(1, 16)])
    assert 0.8 < fsk < 1.3
    assert fsl > 1.8
    assert e[(1, 16)] < e[(0, 16)] / 10


# --------------------------------------------------------------------------
# Geometry: plane/cube volume, PLIC inversion, height-function normals
# --------------------------------------------------------------------------
def _brute_volume(n, d, k=160):
    s = (np.arange(k) + 0.5) / k - 0.5
    X, Y, Z = np.meshgrid(s, s, s, indexing="ij")
    return np.mean(n[0] * X + n[1] * Y + n[2] * Z <= d)


def test_cube_volume_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(12):
        n = rng.normal(size=3)
        n[rng.integers(3)] *= rng.choice([0.0, 1e-9, 1.0])
        n /= np.linalg.norm(n)
        d = rng.uniform(-0.5, 0.5) * np.abs(n).sum()
        assert cube_volume(n, d) == pytest.approx(_brute_volume(n, d), abs=4e-3)
        assert cube_volume(n, d) + cube_volume(n, -d) == pytest.approx(1.0, abs=1e-14)


def test_plic_roundtrip_and_aligned_case():
    rng = np.random.default_rng(2)
    for _ in range(50):
        n = rng.normal(size=3)
        if rng.random() < 0.3:
            n[rng.integers(3)] = 0.0
        n /= np.linalg.norm(n)
        phi = 1e-6 + (1 - 2e-6) * rng.random()
        d = plic_offset(n, phi)
        assert cube_volume(n, d) == pytest.approx(phi, abs=1e-13)
    for phi in (0.0, 0.25, 0.5, 0.9, 1.0):
        # the fill is kept 1e-9 away from an empty / full cell
        assert plic_offset(np.array([0.0, 0.0, 1.0]), phi) == pytest.approx(phi - 0.5, abs=1.1e-9)
    for phi in (0.25, 0.5, 0.9):
        assert plic_offset(np.array([0.0, 0.0, 1.0]), phi) == pytest.approx(phi - 0.5, abs=1e-15)


def test_height_function_normal_exact_for_planes():
    """Height-function normals and plane offsets are exact for a plane, the
    accuracy Sec. 5 asks of the interface position."""
    rng = np.random.default_rng(3)
    n = 16
    for _ in range(4):
        a, b = rng.uniform(-0.7, 0.7, 2)
        c0 = 8.0 + rng.uniform(-0.5, 0.5)
        dims = (n, n, n)
        i = np.arange(n ** 3)
        x, y, z = i % n, (i // n) % n, i // (n * n)
        # exact cut volume of each cell below z = a x + b y + c0 (x,y cell-centred)
        qx, qw = np.polynomial.legendre.leggauss(6)
        qx = 0.5 * (qx + 1)
        qw = 0.5 * qw
        X = x[:, None, None] + qx[None, :, None]
        Y = y[:, None, None] + qx[None, None, :]
        s = a * (X - 8) + b * (Y - 8) + c0 - z[:, None, None]
        phi = np.einsum("iab,a,b->i", np.clip(s, 0, 1), qw, qw)
        params = cases.default_params(periodic=(0, 0, 0), freeze=1)
        flags = cases.classify(dims, params["periodic"], 0, phi, sharp=True)
        keep = (flags == 2) | (flags == 4)
        case = cases.Case(dims=dims, params=params, flags=flags, rho=np.ones(n ** 3),
                          u=np.zeros((n ** 3, 3)), phi=np.where(keep, phi, 0.0),
                          noise=None, wall_delta=None)
        o = Oracle.from_case(case)
        nn, d, _, _, ok = o.geometry()
        inner = ((flags == 2) & (x > 2) & (x < n - 3) & (y > 2) & (y < n - 3)
                 & (z > 2) & (z < n - 3))
        nex = np.array([-a, -b, 1.0]) / math.sqrt(1 + a * a + b * b)
        zc = a * (x + 0.5 - 8) + b * (y + 0.5 - 8) + c0
        dex = (zc - (z + 0.5)) * nex[2]
        assert inner.sum() > 40
        assert np.abs(nn[inner] - nex).max() < 1e-12
        assert np.abs(d[inner] - dex[inner]).max() < 1e-12


def test_height_function_curvature_of_cylinder():
    """Curvature of a liquid cylinder (axis y) from heights: about 1/R, positive
    for convex liquid (Sec. 2.3, Laplace pressure)."""
    n, R = 40, 12.0
    dims = (n, 4, n)
    N = n * 4 * n
    i = np.arange(N)
    x, y, z = i % n, (i // n) % 4, i // (n * 4)
    k = 8
    s = (np.arange(k) + 0.5) / k
    px = x[:, None, None] + s[None, :, None] - 20.0
    pz = z[:, None, None] + s[None, None, :] - 20.0
    phi = ((px ** 2 + pz ** 2) <= R * R).mean(axis=(1, 2))
    params = cases.default_params(periodic=(0, 1, 0), sigma=1e-3)
    flags = cases.classify(dims, params["periodic"], 0, phi)
    case = cases.Case(dims=dims, params=params, flags=flags, rho=np.ones(N),
                      u=np.zeros((N, 3)), phi=np.where(flags == 2, phi, 0.0), noise=None,
                      wall_delta=None)
    o = Oracle.from_case(case)
    _, _, kap, _, ok = o.geometry()
    sel = (flags == 2) & (kap != 0)
    assert sel.sum() > 20
    assert np.median(kap[sel]) == pytest.approx(1.0 / R, rel=0.1)
    assert (kap[sel] > 0).mean() > 0.9


def test_splitmix64_reference_value():
    """SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF (published
    reference sequence)."""
    assert int(cases.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_dam_break_fast_flags_match_generic_classifier():
    c = cases.dam_break(nx=20, ny=6, nz=14, col_x=7, col_z=9)
    phi = np.zeros(c.N)
    x = np.arange(c.N) % 20
    z = np.arange(c.N) // (20 * 6)
    phi[(x < 7) & (z < 9)] = 1.0
    assert np.array_equal(c["flags"], cases.classify(c["dims"], (0, 0, 0), 0, phi))


# --------------------------------------------------------------------------
# Tangent-linear (dual-number) mode of the oracle against central differences
# --------------------------------------------------------------------------
def _interface_mean_ux(o, tangent=False):
    fl = o.flags()
    return o.get(VEL, tangent=tangent)[fl == 2, 0].mean()


def test_tangent_linear_matches_central_differences():
    """J = mean u_x of interface cells after 300 steps of a film (depth 30):
    the dual-number tangent in tau, g_x and one interface fill level agrees
    with central finite differences of the FP64 oracle."""
    c = cases.adjoint_film(nz=48, h=30.0)
    steps = 300

    def J_fd(params=None, phi=None):
        cc = cases.Case(c)
        if params:
            p = dict(c["params"])
            p.update(params)
            cc["params"] = p
        if phi is not None:
            cc["phi"] = phi
        o = Oracle.from_case(cc)
        o.step(steps)
        return _interface_mean_ux(o)

    o = Oracle.from_case(c, dual=True)
    o.seed(dtau=1.0)
    o.step(steps)
    t_tau = _interface_mean_ux(o, True)
    h = 1e-6
    fd = (J_fd({"tau": 0.8 + h}) - J_fd({"tau": 0.8 - h})) / (2 * h)
    assert t_tau == pytest.approx(fd, rel=1e-5)

    o = Oracle.from_case(c, dual=True)
    o.seed(dg=[1.0, 0.0, 0.0])
    o.step(steps)
    t_g = _interface_mean_ux(o, True)
    h = 1e-9
    fd = (J_fd({"g": (1e-6 + h, 0.0, 0.0)}) - J_fd({"g": (1e-6 - h, 0.0, 0.0)})) / (2 * h)
    assert t_g == pytest.approx(fd, rel=1e-5)

    ifc = np.where(c["flags"] == cases.INTERFACE)[0]
    k = ifc[5]
    dphi = np.zeros(c.N)
    dphi[k] = 1.0
    o = Oracle.from_case(c, dual=True)
    o.seed(dphi=dphi)
    o.step(steps)
    t_phi = _interface_mean_ux(o, True)
    h = 1e-4  # dJ/dphi is ~1e-10: smaller steps drown in rounding of J
    pp, pm = c["phi"].copy(), c["phi"].copy()
    pp[k] += h
    pm[k] -= h
    fd = (J_fd(phi=pp) - J_fd(phi=pm)) / (2 * h)
    assert t_phi == pytest.approx(fd, rel=2e-3)


def _extensional_state(a=1e-3, dims=(12, 12, 10), h_if=5, fill=0.6, tau=0.8):
    """Steady linear extensional flow u = (a x', -a y', 0) under a flat free
    surface (interface layer z = h_if, normal along z, so the normal-tangential
    shear rates vanish and S = diag(a, -a, 0)).  With the linear equilibrium and
    no force the Chapman-Enskog solution (Eq. ce / Eq. nqp, Eq. nqm) terminates:
    f_q = w_q rho + 3 w_q c_q.u + (3 w_q / lambda_+) c_q.G.c_q, an exact fixed
    point of the bulk update."""
    nx, ny, nz = dims
    N = nx * ny * nz
    i = np.arange(N)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    flags = np.where(z < h_if, cases.LIQUID, np.where(z == h_if, cases.INTERFACE, cases.GAS)).astype(np.uint8)
    phi = np.where(z == h_if, fill, 0.0)
    xc, yc = (nx - 1) / 2, (ny - 1) / 2
    u = np.stack([a * (x - xc), -a * (y - yc), np.zeros(N)], axis=1)
    G = np.diag([a, -a, 0.0])
    lam_p = -1.0 / tau
    c = cases.LINKS.astype(np.float64)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    cu = u @ c.T                                       # (N, 19)
    cGc = np.einsum("qa,ab,qb->q", c, G, c)            # (19,)
    f = (w[None, :] * (1.0 + 3.0 * cu) + (3.0 * w * cGc / lam_p)[None, :]).T.copy()
    params = cases.default_params(tau=tau, rule=1, linear_eq=1, freeze=1, periodic=(0, 0, 0))
    return dims, params, flags, f, phi, (x, y, z)


@pytest.mark.parametrize("rule", [1, 0])
def test_stress_term_exact_for_linear_extensional_flow(rule):
    """With the boundary shear-rate term (Eq. bterm, D of Table 1, S^b from
    Eq. bstress) the free-surface closure reproduces the steady linear flow
    exactly; with D = 0 the tangential shear rates are forced to zero and the
    rebuilt populations are off by D c.S.c (checked against its value)."""
    dims, params, flags, f, phi, (x, y, z) = _extensional_state()
    params["rule"] = rule
    nx, ny, nz = dims
    inner = (flags == cases.INTERFACE) & (x >= 2) & (x < nx - 2) & (y >= 2) & (y < ny - 2)
    errs = {}
    for stress in (1, 0):
        o = Oracle(dims, dict(params, stress=stress))
        o.set_state(flags, f, phi)
        o.step(1)
        f1 = o.get(F_PRE)
        errs[stress] = np.abs(f1[:, inner] - f[:, inner]).max()
    assert errs[1] < 1e-14, errs
    # D = 0: the error on a gas link p is -D c_p.S.c_p = alpha_+ (tau - 1/2) 3 w_p a (c_px^2 - c_py^2);
    # the gas links of a surface with normal z are (+-1, 0, 1) and (0, +-1, 1), w_p = 1/36
    alpha = 1.0 if rule == 1 else 2.0
    expect = alpha * (0.8 - 0.5) * 3.0 / 36.0 * 1e-3
    assert errs[0] == pytest.approx(expect, rel=1e-6), (errs, expect)


def test_stress_term_projection_zeroes_normal_tangential_shear():
    """A shear u_x = b z' under the flat surface (S_xz = b/2) violates the
    tangential condition Eq. proj2; the boundary term keeps S^b_xz = 0 (Eq.
    bstress), so the rebuilt population on a gas link (c_x, 0, 1) differs from
    the steady field by D c.(S^b - S).c = 6 alpha_+ Lambda_+ w c_x S_xz."""
    b = 1e-3
    dims, params, flags, _, phi, (x, y, z) = _extensional_state()
    nx, ny, nz = dims
    N = nx * ny * nz
    u = np.stack([b * (z - 2.0), np.zeros(N), np.zeros(N)], axis=1)
    G = np.zeros((3, 3)); G[2, 0] = b                    # d_z u_x
    c = cases.LINKS.astype(np.float64)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    f = (w[None, :] * (1.0 + 3.0 * (u @ c.T)) + (3.0 * w * np.einsum("qa,ab,qb->q", c, G, c) / (-1.0 / 0.8))[None, :]).T.copy()
    o = Oracle(dims, dict(params, stress=1))
    o.set_state(flags, f, phi)
    o.step(1)
    f1 = o.get(F_PRE)
    inner = (flags == cases.INTERFACE) & (x >= 2) & (x < nx - 2) & (y >= 2) & (y < ny - 2)
    Lp = 0.8 - 0.5
    for q in range(1, 19):
        cq = cases.LINKS[q]
        if cq[2] != -1:          # populations arriving from the gas above: c_q = -c_p with c_p,z = +1
            continue
        cp = -cq
        d = f1[q, inner] - f[q, inner]
        expect = 6.0 * 1.0 * Lp * w[q] * cp[0] * (b / 2.0)
        assert np.allclose(d, expect, rtol=1e-9, atol=1e-15), (q, d[:3], expect)


def _plate_error(h, rule, T, tau=1.0):
    c = cases.plate_flow(h=h, tau=tau, rule=rule)
    nu = (tau - 0.5) / 3.0
    steps = int(round(T * h * h / nu))
    o = Oracle.from_case(c)
    o.step(steps)
    u = o.get(VEL)[:, 0]
    nx, ny = c["dims"][0], c["dims"][1]
    z = np.arange(c.N) // (nx * ny)
    fluid = (c["flags"] == cases.LIQUID) | (c["flags"] == cases.INTERFACE)
    col = fluid & (np.arange(c.N) % (nx * ny) == 0)
    ue = cases.plate_flow_exact(z[col] + 0.5, steps, h, nu, c["u_wall"])
    return np.sqrt(np.mean((u[col] - ue) ** 2)) / c["u_wall"]


@pytest.mark.parametrize("rule", [0, 1])
def test_plate_driven_transient_second_order(rule):
    """Plate-driven flow started from rest (Sec. 6): moving wall (half-way
    bounce-back with the wall velocity), free surface at integer height, mu =
    1/6, Lambda = 1/4: the profile follows the Fourier series and both rules
    converge at second order (T = 1/8 and 3/8; FSK 2.00 from h = 8, FSL
    1.7 -> 1.9 over h = 8 ... 64, smaller errors than FSK throughout)."""
    hs = (8, 16, 32) if rule == 0 else (8, 16, 32, 64)
    for T in (1 / 8, 3 / 8):
        e = np.array([_plate_error(h, rule, T) for h in hs])
        order = np.log2(e[:-1] / e[1:])
        assert e[0] < 2e-3, (T, e)
        if rule == 0:
            assert np.all(order > 1.95), (T, e, order)
        else:
            assert np.all(order > 1.65) and order[-1] > 1.85, (T, e, order)


def test_couette_prescribed_shear_exact():
    """Linear Couette flow driven by the prescribed shear rate S^b_xz at the
    free surface (Sec. 6, stress = 2, FSL): from rest the flow settles on
    u_x = 2 S_xz (z + 1/2) without numerical error, with the non-linear and
    with the linear equilibrium; with D = 0 nothing drives the flow."""
    for linear in (0, 1):
        c = cases.couette(h=8, linear_eq=linear)
        o = Oracle.from_case(c)
        o.step(8000)
        u = o.get(VEL)[:, 0]
        nx, ny = c["dims"][0], c["dims"][1]
        z = np.arange(c.N) // (nx * ny)
        fluid = (c["flags"] == cases.LIQUID) | (c["flags"] == cases.INTERFACE)
        ue = 2.0 * c["shear"] * (z + 0.5)
        err = np.abs(u[fluid] - ue[fluid]).max() / np.abs(ue[fluid]).max()
        assert err < 1e-10, (linear, err)
    c = cases.couette(h=8, stress=0)
    o = Oracle.from_case(c)
    o.step(2000)
    assert np.abs(o.get(VEL)).max() < 1e-15


def _skew_couette_error(h, shear, linear_eq, ub_extrap, tau=1.1, tol=1e-12, chunk=500, max_steps=200000):
    """Relative L2 error of the steady skew Couette flow (run from the exact
    velocity until the relative change per 500 steps is below tol)."""
    c = cases.skew_couette(h=h, shear=shear, tau=tau, linear_eq=linear_eq, ub_extrap=ub_extrap)
    o = Oracle.from_case(c)
    fl = c["flags"]
    fluid = (fl == cases.LIQUID) | (fl == cases.INTERFACE)
    prev = o.get(VEL)[fluid]
    for _ in range(max_steps // chunk):
        assert o.step(chunk) == 0
        u = o.get(VEL)[fluid]
        change = np.sqrt(((u - prev) ** 2).sum() / (u ** 2).sum())
        prev = u
        if change < tol:
            break
    ex = c["u_exact"][fluid]
    return np.sqrt(((u - ex) ** 2).sum() / (ex ** 2).sum())


def test_skew_couette_linear_equilibrium_exact():
    """Couette flow in a channel with slope 1/4 (Sec. 6, rotated linear
    flow): CLI wall below, free surface above with the surface shear rate
    prescribed through S^b = s/2 (t n^T + n t^T) (stress = 2, FSL); with the
    linear e^+ the steady profile u = s d t is recovered to round-off, whichever
    u_b the closure takes (u_b enters only the non-linear part of e^+)."""
    for h in (8, 16):
        for xu in (0, 1):
            e = _skew_couette_error(h, 1e-3, 1, xu)
            assert e < 1e-10, (h, xu, e)


def test_skew_couette_nonlinear_order_needs_extrapolated_ub():
    """The same flow with the non-linear e^+ at a fixed Reynolds number (shear
    rate ~ 1/h^2 at fixed tau, h = 8, 16, 32): with u_b extrapolated along the
    link to the surface point x_b + delta c_p the error falls at second order
    (Sec. 6); with the node's own velocity the surface shear rate is off by a
    fraction proportional to the surface velocity and the order drops to one."""
    hs = (8, 16, 32)
    ex = np.array([_skew_couette_error(h, 1e-3 * (8.0 / h) ** 2, 0, 1) for h in hs])
    node = np.array([_skew_couette_error(h, 1e-3 * (8.0 / h) ** 2, 0, 0) for h in hs])
    o_ex = np.log2(ex[:-1] / ex[1:])
    o_node = np.log2(node[:-1] / node[1:])
    assert np.all(o_ex > 1.9), (ex, o_ex)
    assert np.all((o_node > 0.9) & (o_node < 1.15)), (node, o_node)
    assert ex[0] < 2e-5 and node[0] > 5e-4


def test_aligned_couette_exact_with_extrapolated_ub():
    """The aligned Couette flow stays exact with u_b extrapolated along the
    link (non-linear and linear e^+)."""
    for linear in (0, 1):
        c = cases.couette(h=8, linear_eq=linear, ub_extrap=1)
        o = Oracle.from_case(c)
        o.step(8000)
        u = o.get(VEL)[:, 0]
        nx, ny = c["dims"][0], c["dims"][1]
        z = np.arange(c.N) // (nx * ny)
        fluid = (c["flags"] == cases.LIQUID) | (c["flags"] == cases.INTERFACE)
        ue = 2.0 * c["shear"] * (z + 0.5)
        err = np.abs(u[fluid] - ue[fluid]).max() / np.abs(ue[fluid]).max()
        assert err < 1e-10, (linear, err)


# --------------------------------------------------------------------------
# Koerner et al.'s reconstruction along the normal (recon_nc)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("rule", ["FSK", "FSL"])
def test_normal_links_rebuilt_exactly_where_the_plane_says(rule):
    """Inclined film (slope 1/2, frozen surface, exact plane with unit normal
    (-1, 0, 2)/sqrt5 into the gas): with recon_nc every interface cell
    rebuilds, besides its gas links, exactly the links p toward fluid nodes
    with n.c_p > 0 of the exact plane (links tangent to it, n.c_p = 0, stay
    streamed), each with the rule's closure of Table 1; all other links are
    streamed unchanged."""
    c = cases.inclined_film(h=8, rule=1 if rule == "FSL" else 0, recon_nc=1, init_exact=True)
    o = Oracle.from_case(c)
    dims, N = c["dims"], c.N
    per, zs = c["params"]["periodic"], c["params"]["zshift"]
    f0 = o.get(F_PRE)
    ft = o.get(F_POST)
    u0 = o.get(VEL)
    nrm, dpl, _, _, gok = o.geometry()
    lp = -1.0 / c["params"]["tau"]
    o.step(1)
    f1 = o.get(F_PRE)
    flags = c["flags"]
    n_exact = np.array([-1.0, 0.0, 2.0]) / math.sqrt(5.0)
    idx = np.arange(N)
    nb = {p: cases._neighbour_index(dims, per, zs, idx, cases.LINKS[p]) for p in range(1, 19)}
    rebuilt = streamed = 0
    for i in np.where(flags == cases.INTERFACE)[0]:
        assert gok[i] and np.allclose(nrm[i], n_exact, atol=1e-12)
        rho = f0[:, i].sum()
        nplus = 0.5 * (f0[:, i] + f0[OPP, i]) - _eplus(rho, u0[i])
        eb = _eplus(c["params"]["rho_G"], u0[i])
        for p in range(1, 19):
            q = OPP[p]
            j = nb[p][i]  # x + c_p, the source of f_q
            if j < 0 or flags[j] == cases.WALL:
                continue
            normal = flags[j] != cases.GAS and CQ[p] @ n_exact > 1e-9
            if flags[j] == cases.GAS or normal:
                cn = CQ[p] @ nrm[i]
                delta = min(max(dpl[i] / cn, 0.0), 1.0) if cn > 0 else 0.5
                up = nb[q][i]  # x - c_p
                r = rule if (up >= 0 and flags[up] in (cases.LIQUID, cases.INTERFACE)) else "FSK"
                a0, ab0, a1, ap, C = coeffs(r, delta, lp)
                expect = a0 * ft[p, i] + ab0 * ft[q, i] + ap * eb[p] + C * nplus[p]
                if a1 != 0.0:
                    expect += a1 * ft[p, up]
                assert f1[q, i] == pytest.approx(expect, rel=0, abs=1e-14), (i, p)
                rebuilt += normal
            else:
                assert f1[q, i] == ft[q, j], (i, p)
                streamed += 1
    assert rebuilt > 0 and streamed > 0


def test_normal_links_change_nothing_on_a_flat_surface():
    """On a lattice-aligned surface every link with n.c_p > 0 already points
    to a gas cell: recon_nc gives the same run bit for bit (film, 200 steps)."""
    runs = []
    for rn in (0, 1):
        c = cases.film(nx=4, ny=4, nz=16, h=9.0, recon_nc=rn, freeze=1)
        o = Oracle.from_case(c)
        o.step(200)
        runs.append(o.get(F_POST))
    assert np.array_equal(runs[0], runs[1])


# --------------------------------------------------------------------------
# Thuerey's excess split along the fill-level normal (excess_split)
# --------------------------------------------------------------------------
def _one_converting_cell(phi_c, split):
    """Film 4x4x16 at rest, surface at z = 8.5 (interface layer z = 8 with
    fill 1/2), no gravity, no noise; the interface cell (1, 2, 8) starts at
    fill phi_c so that it fills (phi_c > 1 + eps) or empties (phi_c < 0) in
    the first step.  Returns the state after one step, the cell index and
    the lattice dims."""
    c = cases.film(nx=4, ny=4, nz=16, h=8.5, gx=0.0, noise_amp=0.0, excess_split=split)
    nx, ny = 4, 4
    i = 1 + nx * (2 + ny * 8)
    assert c["flags"][i] == cases.INTERFACE
    c["phi"][i] = phi_c
    o = Oracle.from_case(c)
    M0, L0 = o.total_mass()
    assert o.step(1) == 0
    M1, L1 = o.total_mass()
    assert abs((M1 + L1) - (M0 + L0)) < 1e-12 * M0
    return o.get(2), i, c


@pytest.mark.parametrize("phi_c,side", [(1.05, +1), (-0.05, -1)])
def test_weighted_excess_goes_along_the_normal(phi_c, side):
    """A cell that fills under a flat surface (fill-level normal +z) gives
    its excess only to the five receivers above it, in equal parts; one that
    empties takes its deficit only from the five below.  Against the equal
    split over all 13 receivers (5 across, 8 in the layer), each cell in the
    layer receives -ex/13 less and each cell across ex/5 - ex/13 more, so the
    two changes stand in the ratio -8/5, and the changes sum to zero."""
    m_eq, i, c = _one_converting_cell(phi_c, 0)
    m_w, _, _ = _one_converting_cell(phi_c, 1)
    nx, ny, _ = c["dims"]
    diff = m_w - m_eq
    x0, y0, z0 = 1, 2, 8
    layer, across = [], []
    for p in range(1, 19):
        cx_, cy_, cz_ = cases.LINKS[p]
        j = (x0 + cx_) % nx + nx * ((y0 + cy_) % ny + ny * (z0 + cz_))
        if cz_ == 0:
            layer.append(diff[j])
        elif cz_ == side:
            across.append(diff[j])
    layer, across = np.array(layer), np.array(across)
    assert len(layer) == 8 and len(across) == 5
    assert np.ptp(layer) < 1e-15 and np.ptp(across) < 1e-15
    assert abs(layer[0]) > 1e-4
    assert across[0] / layer[0] == pytest.approx(-8.0 / 5.0, rel=1e-12)
    others = np.delete(diff, [i] + [
        (x0 + int(cq[0])) % nx + nx * ((y0 + int(cq[1])) % ny + ny * (z0 + int(cq[2]))) for cq in cases.LINKS[1:]])
    assert np.abs(others).max() < 1e-15
    assert abs(diff.sum()) < 1e-15


def test_mass_ledger_exact_with_weighted_split():
    """The mass ledger (total + lost) is exact through conversions with the
    weighted split (dam break with conversions, both rules)."""
    for rule in (0, 1):
        c = cases.dam_break(nx=24, ny=8, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=rule, excess_split=1)
        o = Oracle.from_case(c)
        M0, L0 = o.total_mass()
        conv = np.zeros(4)
        for _ in range(150):
            assert o.step(1) == 0
            conv += np.array(o.counters()[0])
        M1, L1 = o.total_mass()
        assert conv[0] > 0 and conv[1] > 0
        assert abs((M1 + L1) - (M0 + L0)) < 1e-12 * M0


def test_openmp_build_gives_the_same_bits():
    """The OpenMP build of the oracle (used only to time it on all cores)
    gives bit for bit the results of the plain build: dam break with
    conversions and a capillary wave with the shear term and all tracking
    variants."""
    from oracle import oracle as orc
    orc.threads(4)
    for c in (cases.dam_break(nx=24, ny=8, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=1),
              cases.standing_wave(n=16, depth=8.0, amp=1.0, tau=0.6, g=1e-4, sigma=5e-3, phi_noise=1e-4,
                                  stress=1, ub_extrap=1, recon_nc=1, excess_split=1)):
        a = Oracle.from_case(c)
        b = Oracle.from_case(c, omp=True)
        assert a.step(60) == 0 and b.step(60) == 0
        for fid in (F_POST, 2, PHI):
            assert np.array_equal(a.get(fid), b.get(fid))
        assert np.array_equal(a.flags(), b.flags())
        assert a.total_mass() == b.total_mass()


# --------------------------------------------------------------------------
# Static droplet: the Laplace jump (Sec. 2.3, Laplace pressure)
# --------------------------------------------------------------------------
def _droplet_jump(R, sigma=1e-3, steps=1500):
    c = cases.droplet(n=24, R=R, sigma=sigma)
    o = Oracle.from_case(c)
    assert o.step(steps) == 0
    rho = o.get(RHO)
    core = c["r"] < R / 2
    fl = c["flags"]
    umax = np.abs(o.get(VEL)[(fl == cases.LIQUID) | (fl == cases.INTERFACE)]).max()
    return (rho[core].mean() - 1.0) / (3.0 * sigma * 2.0 / R), umax


def test_static_droplet_laplace_jump():
    """A frozen spherical droplet (radius 6 and 8, off-centre in a periodic
    24^3 box, fill levels sampled on 16^3 points per cell) with surface
    tension settles on the Laplace density jump rho - rho_G = 3 sigma 2/R:
    within 6 % at R = 6 and 3 % at R = 8 (the error falls with R), with
    residual currents below 1e-3.  Where the height columns along the
    dominant axis are open, the curvature comes from the other axes' heights
    or the divergence of the normal; with kappa = 0 there the jump came out
    at half of the law."""
    r6, u6 = _droplet_jump(6.0)
    r8, u8 = _droplet_jump(8.0)
    assert abs(r6 - 1) < 0.06 and abs(r8 - 1) < 0.03 and abs(r8 - 1) < abs(r6 - 1)
    assert u6 < 1e-3 and u8 < 1e-3


def test_step_from_post_equals_the_step():
    """One step restarted from the post-collision populations (the entry the
    full-size window check uses: u and n^+ recovered from f~ by inverting the
    collision) equals the ordinary step: dam break with conversions, FSL, and
    a capillary wave with the shear term."""
    for c in (_mini_dam(1), cases.standing_wave(n=16, depth=8.0, amp=1.0, tau=0.6, g=1e-4, sigma=5e-3,
                                                  phi_noise=1e-4, stress=1)):
        a = Oracle.from_case(c)
        assert a.step(25) == 0
        # F_POST is the collision of the current state
        flags, m, phi, ft = a.flags().copy(), a.get(2), a.get(PHI), a.get(F_POST)
        assert a.step(1) == 0
        b = Oracle(c["dims"], c["params"])
        assert b.step_from_post(flags, ft, m, phi) == 0
        assert np.array_equal(a.flags(), b.flags())
        for fid in (F_PRE, 2, PHI):
            ra, rb = a.get(fid), b.get(fid)
            assert np.abs(ra - rb).max() <= 1e-13 * np.abs(ra).max(), fid


def test_tangent_linear_through_conversions_matches_central_differences():
    """The dual-number tangent through cell conversions (the new cells'
    equilibrium initialisation and the excess split are differentiated, the
    decisions held): dam-break miniature, 200 steps with conversions in most
    of them, tangent in tau and g_z against central differences of the FP64
    oracle (relative steps small enough that no decision flips)."""
    c = cases.dam_break(nx=24, ny=8, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=1)
    steps = 200

    def J(**params):
        cc = cases.Case(c)
        p = dict(c["params"])
        p.update(params)
        cc["params"] = p
        o = Oracle.from_case(cc)
        o.step(steps)
        return _interface_mean_ux(o)

    o = Oracle.from_case(c, dual=True)
    o.seed(dtau=1.0)
    conv = 0
    for _ in range(steps):
        o.step(1)
        conv += sum(o.counters()[0])
    assert conv > 20
    t_tau = _interface_mean_ux(o, True)
    h = 1e-7
    fd = (J(tau=0.6 + h) - J(tau=0.6 - h)) / (2 * h)
    assert t_tau == pytest.approx(fd, rel=1e-5)
    o = Oracle.from_case(c, dual=True)
    o.seed(dg=[0.0, 0.0, 1.0])
    o.step(steps)
    t_g = _interface_mean_ux(o, True)
    h = 2e-10
    fd = (J(g=(0.0, 0.0, -2e-4 + h)) - J(g=(0.0, 0.0, -2e-4 - h))) / (2 * h)
    assert t_g == pytest.approx(fd, rel=1e-5)


def _plane_case(a, b, c0, n=12, nz=8, elvira=1):
    """Fill levels of the plane z = a (x - 6) + b (y - 6) + c0 (liquid below)
    over a walled n x n x nz box, from the plane/cube volume (pinned by brute
    force above); frozen interface, so the geometry sees these fills."""
    from oracle.oracle import cube_volume as vol
    dims = (n, n, nz)
    N = n * n * nz
    i = np.arange(N)
    x, y, z = i % n, (i // n) % n, i // (n * n)
    nex = np.array([-a, -b, 1.0]) / math.sqrt(1 + a * a + b * b)
    X0 = np.array([6.0, 6.0, c0])
    dcell = ((X0[None, :] - np.stack([x + 0.5, y + 0.5, z + 0.5], 1)) @ nex)
    phi = np.array([vol(nex, dd) for dd in dcell])
    phi[phi < 1e-14] = 0.0
    phi[phi > 1 - 1e-14] = 1.0
    params = cases.default_params(periodic=(0, 0, 0), freeze=1, elvira=elvira)
    flags = cases.classify(dims, params["periodic"], 0, phi)
    flags[(flags == 1) & (phi < 1.0)] = 2  # every partly filled cell is an interface cell
    case = cases.Case(dims=dims, params=params, flags=flags, rho=np.ones(N), u=np.zeros((N, 3)),
                      phi=np.where(flags == 2, phi, 0.0), noise=None, wall_delta=None)
    return case, nex, dcell, (x, y, z)


def test_elvira_normal_exact_for_planes_at_open_columns():
    """Sec. 5 asks for an interface position of matching accuracy where the
    height columns are open too: a plane 2.4 cells above a wall leaves every
    7-cell column through the surface open, and there the ELVIRA normal and
    plane offset are exact (the Parker-Youngs normal is off by up to a few
    percent)."""
    rng = np.random.default_rng(17)
    for _ in range(4):
        a, b = rng.uniform(-0.3, 0.3, 2)
        c0 = 2.4 + rng.uniform(-0.2, 0.2)
        worst = {}
        for elv in (1, 0):
            case, nex, dcell, (x, y, z) = _plane_case(a, b, c0, elvira=elv)
            o = Oracle.from_case(case)
            nn, d, _, _, ok = o.geometry()
            # cells whose 3x3 columns of 3 cells (along z) all cross the
            # surface, the condition under which the ELVIRA heights are exact
            ph3 = np.where(case["flags"] == 1, 1.0, case["phi"]).reshape(8, 12, 12)
            full = np.zeros_like(ph3, dtype=bool)
            for zz in range(1, 7):
                col = ph3[zz - 1:zz + 2].sum(0)
                inside = (col > 1e-9) & (col < 3 - 1e-9)
                blk = np.ones((12, 12), dtype=bool)
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        blk[1:11, 1:11] &= inside[1 + dy:11 + dy, 1 + dx:11 + dx]
                blk[0, :] = blk[-1, :] = blk[:, 0] = blk[:, -1] = False
                full[zz] = blk
            sel = (case["flags"] == 2) & full.reshape(-1) & (z <= 2)
            assert sel.sum() > 20
            worst[elv] = (np.abs(nn[sel] - nex).max(), np.abs(d[sel] - dcell[sel]).max())
        assert worst[1][0] < 1e-10 and worst[1][1] < 1e-10, worst
        assert worst[0][0] > 1e-3, worst
