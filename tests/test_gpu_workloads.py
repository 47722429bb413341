"""The prescribed-shear and moving-wall workloads of Sec. 6 on the CUDA path:
parity with the oracle, the plate-driven transient against its Fourier
series (second order), the linear Couette flow driven by a prescribed
surface shear rate (exact when aligned; in a channel with slope 1/4 exact
with the linear equilibrium and second order with the non-linear one and u_b
extrapolated along the link)."""
import numpy as np
import pytest

from gpu_util import run_parity
from paper_1409_5645_gb300 import cases, fslbm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rule,tau", [(0, 1.0), (1, 0.8)])
def test_plate_flow_parity(rule, tau):
    run_parity(cases.plate_flow(h=12, tau=tau, rule=rule), 600, every=50)


def test_couette_parity():
    run_parity(cases.couette(h=10), 600, every=50)


def _plate_error_gpu(h, rule, tau, T, precision="f64"):
    c = cases.plate_flow(h=h, tau=tau, rule=rule)
    nu = (tau - 0.5) / 3.0
    steps = int(round(T * h * h / nu))
    g = fslbm.Lattice.from_case(c, precision=precision)
    g.step(steps)
    u = g.get(fslbm.FIELD_U)["u"][:, 0]
    nx, ny = c["dims"][0], c["dims"][1]
    z = np.arange(c.N) // (nx * ny)
    fluid = (c["flags"] == cases.LIQUID) | (c["flags"] == cases.INTERFACE)
    col = fluid & (np.arange(c.N) % (nx * ny) == 0)
    ue = cases.plate_flow_exact(z[col] + 0.5, steps, h, nu, c["u_wall"])
    return np.sqrt(np.mean((u[col] - ue) ** 2)) / c["u_wall"]


@pytest.mark.parametrize("rule,tau", [(0, 1.0), (1, 0.8)])
def test_plate_flow_second_order(rule, tau):
    """h = 8 ... 64 at T = 3/8 (FSL at tau = 0.8: the library stores
    post-collision populations and needs tau != 1 for FSL)."""
    e = np.array([_plate_error_gpu(h, rule, tau, 3 / 8) for h in (8, 16, 32, 64)])
    order = np.log2(e[:-1] / e[1:])
    print("plate flow", "FSK" if rule == 0 else "FSL", "errors", e, "orders", order)
    assert order[-1] > 1.85 and np.all(order > 1.6)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_couette_prescribed_shear_exact(precision, tol):
    c = cases.couette(h=16)
    g = fslbm.Lattice.from_case(c, precision=precision)
    g.step(20000)
    u = g.get(fslbm.FIELD_U)["u"][:, 0]
    nx, ny = c["dims"][0], c["dims"][1]
    z = np.arange(c.N) // (nx * ny)
    fluid = (c["flags"] == cases.LIQUID) | (c["flags"] == cases.INTERFACE)
    ue = 2.0 * c["shear"] * (z + 0.5)
    err = np.abs(u[fluid] - ue[fluid]).max() / np.abs(ue[fluid]).max()
    print(f"Couette {precision}: max relative error {err:.2e}")
    assert err < tol


def test_skew_couette_parity():
    """Slope-1/4 channel (CLI wall, shifted wrap, prescribed S^b, u_b
    extrapolated along the link)."""
    run_parity(cases.skew_couette(h=8, ub_extrap=1), 400, every=50)


@pytest.mark.parametrize("stress", [0, 1])
def test_dam_break_parity_extrapolated_ub(stress):
    """Dam break with conversions (interior and edge interface cells) with u_b
    extrapolated along the link, with and without the boundary shear term."""
    c = cases.dam_break(nx=24, ny=12, nz=16, col_x=8, col_z=12, tau=0.6, g=2e-4, rule=1,
                        ub_extrap=1, stress=stress)
    _, _, conv = run_parity(c, 120, every=1)
    assert conv[0] + conv[1] > 0 and conv[2] + conv[3] > 0


def _skew_error_gpu(h, shear, linear_eq, precision="f64", tau=1.1, tol=1e-12, chunk=500, max_steps=400000):
    c = cases.skew_couette(h=h, shear=shear, tau=tau, linear_eq=linear_eq, ub_extrap=1)
    g = fslbm.Lattice.from_case(c, precision=precision)
    fl = c["flags"]
    fluid = (fl == cases.LIQUID) | (fl == cases.INTERFACE)
    prev = g.get(fslbm.FIELD_U)["u"][fluid]
    for _ in range(max_steps // chunk):
        g.step(chunk)
        u = g.get(fslbm.FIELD_U)["u"][fluid]
        change = np.sqrt(((u - prev) ** 2).sum() / (u ** 2).sum())
        prev = u
        if change < tol:
            break
    ex = c["u_exact"][fluid]
    return np.sqrt(((u - ex) ** 2).sum() / (ex ** 2).sum())


@pytest.mark.parametrize("precision,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_skew_couette_linear_equilibrium_exact(precision, tol):
    e = _skew_error_gpu(16, 1e-3, 1, precision, tol=1e-12 if precision == "f64" else 1e-7)
    print(f"skew Couette, linear e+, {precision}: L2 error {e:.2e}")
    assert e < tol


def test_skew_couette_second_order():
    """Non-linear e^+, fixed Reynolds number (shear ~ 1/h^2), h = 8 ... 64."""
    hs = (8, 16, 32, 64)
    e = np.array([_skew_error_gpu(h, 1e-3 * (8.0 / h) ** 2, 0) for h in hs])
    order = np.log2(e[:-1] / e[1:])
    print("skew Couette errors", e, "orders", order)
    assert np.all(order > 1.9)
