"""The hand-written adjoint against the oracle's tangent-linear model,
central finite differences of the CUDA forward path, the film series, and
through torch.autograd."""
import math

import numpy as np
import pytest

from oracle.oracle import VEL, Oracle
from paper_1409_5645_gb300 import cases, fslbm

pytestmark = pytest.mark.gpu


def _J_gpu(case, steps, precision="f64", **override):
    c = cases.Case(case)
    p = dict(case["params"])
    p.update(override)
    c["params"] = p
    g = fslbm.Lattice.from_case(c, precision=precision)
    return g.adjoint_forward(steps, K=max(1, steps // 4))


def _grad_gpu(case, steps, K, precision="f64", keep_f0=0, **kw):
    g = fslbm.Lattice.from_case(case, precision=precision, keep_f0=keep_f0, **kw)
    J = g.adjoint_forward(steps, K)
    dnu, dg, dphi = g.adjoint_backward()
    stats = g.adjoint_stats()
    return J, dnu, dg, dphi, stats


def _tlm(case, steps, dtau=0.0, dg=None, dphi=None):
    o = Oracle.from_case(case, dual=True)
    o.seed(dtau=dtau, dg=dg, dphi=dphi)
    o.step(steps)
    fl = o.flags()
    return o.get(VEL, tangent=True)[fl == 2, 0].mean()


def test_adjoint_matches_oracle_tangent_linear():
    """FP64 adjoint (several checkpoint segments) = FP64 tangent-linear model
    of the oracle, in nu, g_x and the interface fill levels."""
    c = cases.adjoint_film(nz=48, h=30.0)
    steps = 300
    J, dnu, dg, dphi, _ = _grad_gpu(c, steps, K=70)
    o = Oracle.from_case(c)
    o.step(steps)
    fl = o.flags()
    assert J == pytest.approx(o.get(VEL)[fl == 2, 0].mean(), rel=1e-11)
    t_tau = _tlm(c, steps, dtau=1.0)
    assert dnu == pytest.approx(3.0 * t_tau, rel=1e-7)  # tau = 3 nu + 1/2
    t_g = _tlm(c, steps, dg=[1.0, 0.0, 0.0])
    assert dg[0] == pytest.approx(t_g, rel=1e-7)
    ifc = np.where(c["flags"] == cases.INTERFACE)[0]
    scale = np.abs(dphi[ifc]).max()
    for k in ifc[[0, 5, 13, 31]]:
        e = np.zeros(c.N)
        e[k] = 1.0
        assert dphi[k] == pytest.approx(_tlm(c, steps, dphi=e), abs=1e-6 * scale)
    assert np.all(dphi[c["flags"] != cases.INTERFACE] == 0.0)


def test_adjoint_matches_central_differences_film_4000_steps():
    """Film 8x4x64, depth 40, 4000 steps, checkpoints every 200: the adjoint
    gradient against central differences of the CUDA forward path."""
    c = cases.adjoint_film()
    steps = 4000
    J, dnu, dg, dphi, stats = _grad_gpu(c, steps, K=200)
    nu = (c["params"]["tau"] - 0.5) / 3
    h = 1e-6 * nu
    fd = (_J_gpu(c, steps, tau=0.5 + 3 * (nu + h)) - _J_gpu(c, steps, tau=0.5 + 3 * (nu - h))) / (2 * h)
    assert dnu == pytest.approx(fd, rel=1e-4)
    gx = c["params"]["g"][0]
    h = 1e-6 * gx
    fd = (_J_gpu(c, steps, g=(gx + h, 0.0, 0.0)) - _J_gpu(c, steps, g=(gx - h, 0.0, 0.0))) / (2 * h)
    assert dg[0] == pytest.approx(fd, rel=1e-4)
    ifc = np.where(c["flags"] == cases.INTERFACE)[0]
    k = ifc[9]

    def cd(hp):
        cp, cm = cases.Case(c), cases.Case(c)
        cp["phi"] = c["phi"].copy()
        cm["phi"] = c["phi"].copy()
        cp["phi"][k] += hp
        cm["phi"][k] -= hp
        return (_J_gpu(cp, steps) - _J_gpu(cm, steps)) / (2 * hp)

    # dJ/dphi0 is ~1e-10 against J ~ 1e-3: a step of 1e-4 keeps the rounding
    # of J below 1e-5 of the difference, and Richardson extrapolation of the
    # steps 2e-4 and 1e-4 removes the O(h^2) truncation
    fd = (4.0 * cd(1e-4) - cd(2e-4)) / 3.0
    assert dphi[k] == pytest.approx(fd, rel=1e-4)
    fwd_ms, adj_ms, peak = stats
    assert fwd_ms > 0 and adj_ms > 0 and peak > 0


def test_adjoint_nu_derivative_against_film_series():
    """dJ/dnu against the nu-derivative of the transient film series at the
    interface nodes (z = h - 1/2) after 4000 steps (the closed-form steady
    limit is -u_s/nu)."""
    c = cases.adjoint_film()
    steps = 4000
    J, dnu, _, _, _ = _grad_gpu(c, steps, K=200)
    nu = (c["params"]["tau"] - 0.5) / 3
    z = 40.0 - 0.5
    series = lambda v: cases.film_transient(np.array([z]), steps, 40.0, 1e-6, v, terms=400)[0]
    assert J == pytest.approx(series(nu), rel=2e-3)
    h = 1e-6
    dser = (series(nu + h) - series(nu - h)) / (2 * h)
    assert dnu == pytest.approx(dser, rel=5e-3)
    us = cases.film_profile(np.array([z]), 40.0, 1e-6, nu)[0]
    # steady limit of the same derivative: d u_s / d nu = -u_s / nu
    assert dser > -us / nu


def test_adjoint_nu_derivative_steady_film_closed_form():
    """At steady state the film's surface velocity is u_s = g h^2 / (2 nu)
    (Sec. 4.3), so dJ/dnu = -J/nu exactly: a shallow film (depth 8, FSL, which
    is exact for the aligned film) run for 20 diffusion times h^2/nu."""
    c = cases.film(nx=4, ny=4, nz=12, h=8.0, gx=1e-6, rule=1, noise_amp=0.0)
    nu = (c["params"]["tau"] - 0.5) / 3
    steps = int(20 * 64 / nu)
    J, dnu, _, _, _ = _grad_gpu(c, steps, K=500)
    z = 8.0 - 0.5
    us = cases.film_profile(np.array([z]), 8.0, 1e-6, nu)[0]
    assert J == pytest.approx(us, rel=1e-6)
    assert dnu == pytest.approx(-J / nu, rel=1e-6)


def test_adjoint_keep_f0_equals_inversion_in_fp64():
    c = cases.adjoint_film(nz=48, h=30.0)
    _, a, ga, pa, _ = _grad_gpu(c, 200, K=100, precision="f64", keep_f0=0)
    _, b, gb, pb, _ = _grad_gpu(c, 200, K=100, precision="f64", keep_f0=1)
    assert a == pytest.approx(b, rel=1e-9)
    assert ga[0] == pytest.approx(gb[0], rel=1e-9)
    assert np.allclose(pa, pb, rtol=0, atol=1e-12 * np.abs(pb).max())


def test_adjoint_fp32_against_fp64():
    """FP32 populations carry the non-equilibrium parts to ~3e-9 absolute.
    On the slow film of the differentiation workload (u ~ 1e-4, gradients in
    phi0 ~ 1e-10) that rounding swamps dJ/dnu and dJ/dphi0, so the FP32 form is
    compared on a film driven 100x harder (g = 1e-4), where the signals stand
    well above the storage resolution.  The errors are stated by the test."""
    c = cases.adjoint_film(nz=48, h=30.0, gx=1e-4)
    _, d64, g64, p64, _ = _grad_gpu(c, 300, K=100, precision="f64", keep_f0=1)
    _, d32, g32, p32, _ = _grad_gpu(c, 300, K=100, precision="f32", keep_f0=1)
    ifc = c["flags"] == cases.INTERFACE
    e_nu = abs(d32 - d64) / abs(d64)
    e_g = abs(g32[0] - g64[0]) / abs(g64[0])
    e_phi = np.abs(p32[ifc] - p64[ifc]).max() / np.abs(p64[ifc]).max()
    print(f"FP32 adjoint vs FP64 (g = 1e-4 film): nu {e_nu:.2e}, g {e_g:.2e}, phi0 {e_phi:.2e}")
    assert e_g < 1e-6
    assert e_nu < 5e-3
    # the per-cell fill gradients rest on small differences of populations;
    # FP32 (storing f - w_q) carries them to a few percent of the largest
    assert e_phi < 0.1


def test_adjoint_fp32_arithmetic():
    """The reverse step in FP32 arithmetic (adjoint_fp32 = 1; it works in the
    deviations f - w_q as the forward step does) on the FP32 trajectory of
    the g = 1e-4 film: against the FP64 reverse step of the same trajectory
    (what the arithmetic alone changes) and against the FP64 lattice.
    dJ/dg and dJ/dphi0 keep 3e-6 and 2e-3; dJ/dnu loses about 1e-2 here: it
    is 3 (dJ/dlambda_+ dlambda_+/dtau + dJ/dlambda_- dlambda_-/dtau), two
    sums over every cell and step of non-equilibrium parts (differences of
    populations of order |u|) times adjoints, which cancel to a small
    remainder on this film, so their FP32 rounding shows in it (the default
    FP64 reverse arithmetic keeps it to 7e-4 against the FP64 lattice)."""
    c = cases.adjoint_film(nz=48, h=30.0, gx=1e-4)
    _, d64, g64, p64, _ = _grad_gpu(c, 300, K=100, precision="f64", keep_f0=1)
    _, d32, g32, p32, _ = _grad_gpu(c, 300, K=100, precision="f32", keep_f0=1)
    _, da, ga, pa, _ = _grad_gpu(c, 300, K=100, precision="f32", keep_f0=1, adjoint_fp32=1)
    ifc = c["flags"] == cases.INTERFACE
    a_nu, a_g = abs(da - d32) / abs(d32), abs(ga[0] - g32[0]) / abs(g32[0])
    a_phi = np.abs(pa[ifc] - p32[ifc]).max() / np.abs(p32[ifc]).max()
    e_nu, e_g = abs(da - d64) / abs(d64), abs(ga[0] - g64[0]) / abs(g64[0])
    e_phi = np.abs(pa[ifc] - p64[ifc]).max() / np.abs(p64[ifc]).max()
    print(f"FP32 reverse arithmetic vs FP64 reverse (same FP32 trajectory): nu {a_nu:.2e}, g {a_g:.2e}, "
          f"phi0 {a_phi:.2e}; vs the FP64 lattice: nu {e_nu:.2e}, g {e_g:.2e}, phi0 {e_phi:.2e}")
    assert a_g < 3e-5 and a_nu < 5e-2 and a_phi < 2e-2
    assert e_g < 3e-5 and e_nu < 5e-2 and e_phi < 0.1


@pytest.mark.parametrize("rule", [0, 1])
def test_adjoint_fp32_arithmetic_through_conversions(rule):
    """FP32 reverse arithmetic on the dam-break miniature with conversions
    (FP32 lattice, 200 steps, 800 conversions): against the FP64 reverse step
    of the same trajectory, about 1e-6 in nu, g_z and the fill levels (under
    FSK no population depends on a fill level, and both give dJ/dphi0 = 0)."""
    c = _dam(rule)
    _, d, g, ph, _ = _grad_gpu(c, 200, K=60, precision="f32")
    _, da, ga, pa, _ = _grad_gpu(c, 200, K=60, precision="f32", adjoint_fp32=1)
    ifc = c["flags"] == cases.INTERFACE
    e_nu, e_g = abs(da - d) / abs(d), abs(ga[2] - g[2]) / abs(g[2])
    scale = max(np.abs(ph[ifc]).max(), 1e-300)
    e_phi = np.abs(pa[ifc] - ph[ifc]).max() / scale
    print(f"rule {rule}: FP32 vs FP64 reverse arithmetic: nu {e_nu:.2e}, g_z {e_g:.2e}, phi0 {e_phi:.2e} "
          f"(max |dJ/dphi0| {np.abs(ph[ifc]).max():.2e})")
    assert e_nu < 1e-5 and e_g < 1e-5
    assert np.abs(pa[ifc] - ph[ifc]).max() <= 1e-4 * scale


def test_autograd_function_matches_c_interface():
    import torch
    from paper_1409_5645_gb300.autograd import run
    c = cases.adjoint_film(nz=48, h=30.0)
    dev = torch.device("cuda:0")
    nu = torch.tensor((c["params"]["tau"] - 0.5) / 3, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(c["params"]["g"], dtype=torch.float64, requires_grad=True)
    phi0 = torch.tensor(c["phi"], dtype=torch.float64, device=dev, requires_grad=True)
    J = run(nu, g, phi0, c, 200, K=50)
    J.backward()
    _, dnu, dg, dphi, _ = _grad_gpu(c, 200, K=50)
    assert float(nu.grad) == pytest.approx(dnu, rel=1e-12)
    assert np.allclose(g.grad.cpu().numpy(), dg, rtol=1e-12)
    assert np.allclose(phi0.grad.cpu().numpy(), dphi, rtol=1e-12, atol=0)


def test_adjoint_refuses_unsupported_settings():
    for kw in (dict(compressible=1), dict(excess_split=1), dict(sigma=1e-4)):
        c2 = cases.adjoint_film(nz=48, h=30.0, **kw)
        g2 = fslbm.Lattice.from_case(c2)
        with pytest.raises(fslbm.FslbmError) as e:
            g2.adjoint_forward(10, 5)
        assert e.value.code == -1


def _dam(rule=1):
    """Dam-break miniature whose cells fill, empty and appear every few
    steps inside the window (equal excess split)."""
    return cases.dam_break(nx=24, ny=8, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=rule)


def _tlm_dam(case, steps, **seed):
    o = Oracle.from_case(case, dual=True)
    o.seed(**seed)
    conv = 0
    for _ in range(steps):
        o.step(1)
        conv += sum(o.counters()[0])
    fl = o.flags()
    return o.get(VEL, tangent=True)[fl == 2, 0].mean(), conv


@pytest.mark.parametrize("rule", [0, 1])
def test_adjoint_through_conversions_matches_oracle_tangent_linear(rule):
    """Conversions replayed: on the dam-break miniature (200 steps, several
    checkpoint segments, conversions in every segment) the FP64 adjoint
    equals the oracle's FP64 tangent-linear model, which differentiates the
    conversion stage itself (new-cell equilibria, excess split), in nu, g and
    the initial fill levels."""
    c = _dam(rule)
    steps = 200
    J, dnu, dg, dphi, _ = _grad_gpu(c, steps, K=60)
    o = Oracle.from_case(c)
    o.step(steps)
    assert J == pytest.approx(o.get(VEL)[o.flags() == 2, 0].mean(), rel=1e-10)
    t_tau, conv = _tlm_dam(c, steps, dtau=1.0)
    print(f"rule {rule}: dJ/dnu adjoint {dnu:.10e} tangent {3.0 * t_tau:.10e}; conversions {conv}")
    assert conv > 20
    assert dnu == pytest.approx(3.0 * t_tau, rel=1e-7)
    for a in (0, 2):
        e = [0.0, 0.0, 0.0]
        e[a] = 1.0
        t_g, _ = _tlm_dam(c, steps, dg=e)
        assert dg[a] == pytest.approx(t_g, rel=1e-7, abs=1e-9 * abs(dg).max())
    ifc = np.where(c["flags"] == cases.INTERFACE)[0]
    scale = np.abs(dphi[ifc]).max()
    for k in ifc[[0, 7, 19, len(ifc) // 2, len(ifc) - 3]]:
        e = np.zeros(c.N)
        e[k] = 1.0
        t_phi, _ = _tlm_dam(c, steps, dphi=e)
        assert dphi[k] == pytest.approx(t_phi, rel=1e-6, abs=1e-8 * scale)


@pytest.mark.parametrize("rule", [0, 1])
def test_adjoint_through_conversions_central_differences(rule):
    """The same gradient against central differences of the CUDA forward
    path (relative steps 1e-6 in nu and g; the discrete decisions stay put
    within them): 1e-4 relative."""
    c = _dam(rule)
    steps = 200
    J, dnu, dg, dphi, _ = _grad_gpu(c, steps, K=60)
    nu = (c["params"]["tau"] - 0.5) / 3
    h = 1e-6 * nu
    fd = (_J_gpu(c, steps, tau=0.5 + 3 * (nu + h)) - _J_gpu(c, steps, tau=0.5 + 3 * (nu - h))) / (2 * h)
    print(f"rule {rule}: dJ/dnu adjoint {dnu:.10e} central difference {fd:.10e}")
    assert dnu == pytest.approx(fd, rel=1e-4)
    gz = c["params"]["g"][2]
    h = 1e-6 * abs(gz)
    fd = (_J_gpu(c, steps, g=(0.0, 0.0, gz + h)) - _J_gpu(c, steps, g=(0.0, 0.0, gz - h))) / (2 * h)
    assert dg[2] == pytest.approx(fd, rel=1e-4)
