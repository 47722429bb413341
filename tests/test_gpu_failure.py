"""Failure detection by host-side injection (no GPU fault, no device trap): a
state that breaks an invariant of the step, or the step's stability guard,
makes the library return its error code at the next synchronising call (the
step itself is asynchronous); setting a valid state afterwards clears the
error word and the same handle steps on."""
import numpy as np
import pytest

from paper_1409_5645_gb300 import cases, fslbm

pytestmark = pytest.mark.gpu

ERR_STATE, ERR_UNSTABLE = -4, -5


def _liquid_box(dims=(16, 8, 8)):
    """A periodic box full of liquid at rest."""
    N = int(np.prod(dims))
    params = cases.default_params(tau=0.8, periodic=(1, 1, 1))
    flags = np.full(N, cases.LIQUID, np.uint8)
    return dims, params, flags, np.ones(N), np.zeros((N, 3)), np.zeros(N)


@pytest.mark.parametrize("precision,loads", [("f64", "plain"), ("f32", "plain"), ("f32", "pairs"),
                                             ("f16", "pairs")])
def test_speed_guard(precision, loads):
    """Uniform flow at 0.35 lattice units steps; at 0.45 (above the guard's
    0.4) the step returns ERR_UNSTABLE; a state at rest set afterwards steps."""
    dims, params, flags, rho, u, phi = _liquid_box()
    lat = fslbm.Lattice(dims, dict(params, bulk_loads=loads), precision=precision)
    u[:, 0] = 0.35
    lat.init_equilibrium(flags, rho, u, phi)
    lat.step(3)
    lat.sync()
    u[:, 0] = 0.45
    lat.init_equilibrium(flags, rho, u, phi)
    with pytest.raises(fslbm.FslbmError) as e:
        lat.step(1)
        lat.sync()
    assert e.value.code == ERR_UNSTABLE and "velocity" in str(e.value)
    u[:] = 0.0
    lat.init_equilibrium(flags, rho, u, phi)
    lat.step(2)
    lat.sync()
    lat.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_non_finite_density(precision):
    """A NaN density in one liquid cell: the step reports a non-finite density."""
    dims, params, flags, rho, u, phi = _liquid_box()
    lat = fslbm.Lattice(dims, params, precision=precision)
    rho[123] = np.nan
    lat.init_equilibrium(flags, rho, u, phi)
    with pytest.raises(fslbm.FslbmError) as e:
        lat.step(1)
        lat.sync()
    assert e.value.code == ERR_UNSTABLE and "density" in str(e.value)
    rho[123] = 1.0
    lat.init_equilibrium(flags, rho, u, phi)
    lat.step(1)
    lat.sync()
    lat.close()


def test_liquid_next_to_gas_and_bad_flag():
    """Setting a state with a liquid cell next to a gas cell, or a flag that
    is no cell kind, returns ERR_STATE (checked when the state is set, before
    any step runs on it)."""
    dims, params, flags, rho, u, phi = _liquid_box()
    lat = fslbm.Lattice(dims, params)
    bad = flags.copy()
    bad[200] = cases.GAS
    with pytest.raises(fslbm.FslbmError) as e:
        lat.init_equilibrium(bad, rho, u, phi)
        lat.sync()
    assert e.value.code == ERR_STATE
    bad = flags.copy()
    bad[7] = 3  # two kinds at once
    with pytest.raises(fslbm.FslbmError) as e:
        lat.init_equilibrium(bad, rho, u, phi)
        lat.sync()
    assert e.value.code == ERR_STATE
    lat.init_equilibrium(flags, rho, u, phi)
    lat.step(1)
    lat.sync()
    lat.close()
