"""Linear stability of the scheme near tau = 1/2 (a property of the method,
recorded because the low-diffusivity workloads sit beyond it).

Small noise (1e-9) on a uniform state with |u| = |b| = 0.04 grows under the
oracle's step when the magnetic relaxation time is close to 1/2 (rates of 1e-3 to 1e-2 per
step) and decays when both relaxation times are away from it.  With the
fluid alone at tau_f -> 1/2 any growth is an order of magnitude slower.
The magnetic BGK collision (Eq. collide_g) leaves its non-hydrodynamic
moments undamped as omega_m -> 2.  Regularising the magnetic collision onto
the first Hermite moment (the extension the Conclusions name) does not
remove the instability, and with tau_f near 1/2 and an oblique field it
grows faster (6e-3 per step at tau_m = 0.51, where the BGK form decays).
"""
import numpy as np
import pytest


def _growth(orc, tau_f, tau_m, U, B, n=16, steps=300, mag=0):
    p = orc.Params(n, n, tau_f, tau_m, mag_collision=mag)
    one = np.ones((n, n))
    f0, g0 = orc.init(p, U[0] * one, U[1] * one, B[0] * one, B[1] * one)
    rng = np.random.default_rng(0)
    f = f0 + 1e-9 * rng.normal(size=f0.shape)
    g = g0 + 1e-9 * rng.normal(size=g0.shape)
    d0 = max(np.abs(f - f0).max(), np.abs(g - g0).max())
    f, g = orc.run(p, f, g, steps)
    d1 = max(np.abs(f - f0).max(), np.abs(g - g0).max())
    return np.log(d1 / d0) / steps


@pytest.mark.parametrize("U,B", [((0.04, 0.0), (0.04, 0.0)), ((0.0, 0.0), (0.04, 0.04))])
def test_unstable_when_magnetic_tau_near_half(orc, U, B):
    assert _growth(orc, 0.50006, 0.50006, U, B) > 1e-3
    assert _growth(orc, 0.53, 0.50006, U, B) > 1e-3     # magnetic part alone suffices


@pytest.mark.parametrize("U,B", [((0.04, 0.0), (0.04, 0.0)), ((0.0, 0.0), (0.04, 0.04))])
def test_stable_when_relaxation_times_away_from_half(orc, U, B):
    assert _growth(orc, 0.53, 0.53, U, B) < 0


@pytest.mark.parametrize("U,B", [((0.04, 0.0), (0.04, 0.0)), ((0.0, 0.0), (0.04, 0.04))])
def test_fluid_near_half_alone_grows_much_slower(orc, U, B):
    assert _growth(orc, 0.50006, 0.53, U, B) < 0.1 * _growth(orc, 0.50006, 0.50006, U, B)


@pytest.mark.parametrize("U,B", [((0.04, 0.0), (0.04, 0.0)), ((0.0, 0.0), (0.04, 0.04))])
def test_regularised_magnetic_collision_does_not_remove_it(orc, U, B):
    assert _growth(orc, 0.50006, 0.50006, U, B, mag=1) > 1e-3
    assert _growth(orc, 0.53, 0.53, U, B, mag=1) < 0


def test_regularised_magnetic_collision_less_stable_with_oblique_field(orc):
    U, B = (0.0, 0.0), (0.04, 0.04)
    assert _growth(orc, 0.50006, 0.51, U, B, mag=0) < 1e-3
    assert _growth(orc, 0.50006, 0.51, U, B, mag=1) > 3e-3
