"""Closed-form decay of small-amplitude modes through the FP64 oracle.

In the incompressible limit a shear wave u_x = A sin(k y) decays as
exp(-nu k^2 t) and a magnetic wave b_x = B sin(k y) (u = 0) as
exp(-eta k^2 t) (the induction and momentum equations of the paper's
introduction).  With nu = cs^2 (tau_f - 1/2) and eta = cs^2 (tau_m - 1/2) the
fitted rates must agree within 0.5 %; the paper's printed transport relation
without cs^2 would be off by a factor of 3.  Wall cases use the half-way
bounce-back modes sin / cos(pi (y + 1/2) / ny).  The current of Eq. current is
checked against -d_y b_x of the decaying magnetic wave.
"""
import math

import numpy as np
import pytest

CS2 = 1.0 / 3.0


def _tau(nu):
    return 0.5 + nu / CS2


def _amplitude(field, shape):
    prof = field.mean(axis=1)
    return float((prof * shape).sum() / (shape * shape).sum())


def _decay_rate(orc, p, init_fields, comp, shape, steps):
    f, g = orc.init(p, *init_fields)
    t1 = steps // 4
    f, g = orc.run(p, f, g, t1)
    a1 = _amplitude(orc.fields(p, f, g)[comp], shape)
    f, g = orc.run(p, f, g, steps - t1)
    a2 = _amplitude(orc.fields(p, f, g)[comp], shape)
    return math.log(a1 / a2) / (steps - t1)


@pytest.mark.parametrize("nu", [0.01, 0.05, 0.1])
def test_periodic_shear_wave(orc, nu):
    nx, ny = 4, 64
    k = 2 * math.pi / ny
    y = np.arange(ny)
    shape = np.sin(k * y)
    p = orc.Params(nx, ny, tau_f=_tau(nu), tau_m=0.8)
    ux = 1e-4 * np.tile(shape[:, None], (1, nx))
    z = np.zeros((ny, nx))
    rate = _decay_rate(orc, p, (ux, z, z, z), 1, shape, int(0.5 / (nu * k * k)))
    assert abs(rate / (nu * k * k) - 1) < 5e-3


@pytest.mark.parametrize("mag_collision", [0, 1])
@pytest.mark.parametrize("eta", [0.01, 0.05, 0.1])
def test_periodic_magnetic_wave(orc, eta, mag_collision):
    """Also with the regularised magnetic collision: it keeps the first
    moment of g - g_eq, which alone carries the diffusive flux, so eta is
    unchanged."""
    nx, ny = 4, 64
    k = 2 * math.pi / ny
    y = np.arange(ny)
    shape = np.sin(k * y)
    p = orc.Params(nx, ny, tau_f=0.8, tau_m=_tau(eta), mag_collision=mag_collision)
    bx = 1e-4 * np.tile(shape[:, None], (1, nx))
    z = np.zeros((ny, nx))
    rate = _decay_rate(orc, p, (z, z, bx, z), 3, shape, int(0.5 / (eta * k * k)))
    assert abs(rate / (eta * k * k) - 1) < 5e-3


@pytest.mark.parametrize("nu", [0.01, 0.05])
def test_wall_shear_mode(orc, nu):
    nx, ny = 4, 32
    q = math.pi / ny
    y = np.arange(ny)
    shape = np.sin(q * (y + 0.5))
    p = orc.Params(nx, ny, tau_f=_tau(nu), tau_m=0.8, wall_y=True)
    ux = 1e-4 * np.tile(shape[:, None], (1, nx))
    z = np.zeros((ny, nx))
    rate = _decay_rate(orc, p, (ux, z, z, z), 1, shape, int(0.5 / (nu * q * q)))
    assert abs(rate / (nu * q * q) - 1) < 1e-2


@pytest.mark.parametrize("eta", [0.01, 0.05])
def test_wall_magnetic_mode(orc, eta):
    nx, ny = 4, 32
    q = math.pi / ny
    y = np.arange(ny)
    shape = np.cos(q * (y + 0.5))
    p = orc.Params(nx, ny, tau_f=0.8, tau_m=_tau(eta), wall_y=True)
    bx = 1e-4 * np.tile(shape[:, None], (1, nx))
    z = np.zeros((ny, nx))
    rate = _decay_rate(orc, p, (z, z, bx, z), 3, shape, int(0.5 / (eta * q * q)))
    assert abs(rate / (eta * q * q) - 1) < 1e-2


@pytest.mark.parametrize("tau_m", [0.53, 0.8])
def test_current_density_of_magnetic_wave(orc, tau_m):
    """Eq. current: j_z = -d_y b_x for b = (B sin ky, 0), sign and scale."""
    nx, ny = 4, 64
    k = 2 * math.pi / ny
    y = np.arange(ny)
    p = orc.Params(nx, ny, tau_f=0.8, tau_m=tau_m)
    bx = 1e-4 * np.tile(np.sin(k * y)[:, None], (1, nx))
    z = np.zeros((ny, nx))
    f, g = orc.init(p, z, z, bx, z)
    f, g = orc.run(p, f, g, 60)
    amp = _amplitude(orc.fields(p, f, g)[3], np.sin(k * y))
    jz = orc.current(p, f, g).mean(axis=1)
    expect = -amp * k * np.cos(k * y)
    assert np.abs(jz - expect).max() < 1e-2 * amp * k
