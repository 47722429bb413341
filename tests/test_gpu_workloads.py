"""The prescribed-shear and moving-wall workloads of Sec. 6 on the CUDA path:
parity with the oracle, the plate-driven transient against its Fourier
series (second order), and the linear Couette flow driven by a prescribed
surface shear rate (exact)."""
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
