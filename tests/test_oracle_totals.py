"""Pins of the oracle's global diagnostics against closed forms.

The totals are sums over nodes of the moments (mass, momentum, sum of b),
the mean energies of the Orszag-Tang section (E_k = mean |u|^2 / 2 and
E_m = mean |b|^2 / 2, i.e. 1/(2 L^2) times the integral), the mean cross
helicity u.b, and the extrema of the current density (Eq. current), of the
vorticity and of div b taken with the isotropic lattice gradient.  On
equilibrium states built from sinusoidal fields each of them has a closed
form; the fields are chosen so that a plausible slip (a density weight
dropped or added, a swapped component in u.b, a missing 1/2, a sum taken
where a mean is meant, a wrong sign in the vorticity) changes a value by
far more than rounding.
"""
import math

import numpy as np
import pytest


def _state(orc, n, fields, rho=None, tau=(0.6, 0.7)):
    p = orc.Params(n, n, *tau)
    f, g = orc.init(p, *fields, rho=rho)
    return p, f, g


@pytest.mark.parametrize("m", [1, 3])
def test_totals_of_shear_and_magnetic_waves(orc, m):
    """u = A (sin K y, 0), b = B (0, sin K x), rho = 1: mass = N^2, no net
    momentum or b, E_k = A^2/4, E_m = B^2/4, u.b = 0 pointwise, div b = 0,
    omega = -d_y u_x = -A sin K cos K y (isotropic stencil), and j_z = 0
    because the magnetic populations are at equilibrium."""
    n, A, B = 32, 0.03, 0.05
    K = 2 * math.pi * m / n
    X, Y = np.meshgrid(np.arange(n), np.arange(n))
    z = np.zeros((n, n))
    p, f, g = _state(orc, n, (A * np.sin(K * Y), z, z, B * np.sin(K * X)))
    t = orc.totals(p, f, g)
    assert abs(t["mass"] - n * n) < 1e-12 * n * n
    for k in ("mom_x", "mom_y", "bsum_x", "bsum_y", "cross_hel"):
        assert abs(t[k]) < 1e-14 * n * n, (k, t[k])
    assert abs(t["e_kin"] - A * A / 4) < 1e-15
    assert abs(t["e_mag"] - B * B / 4) < 1e-15
    assert t["divb_max"] < 1e-15 and t["divb_rms"] < 1e-15
    assert abs(t["omega_max"] - A * math.sin(K)) < 1e-15
    assert t["jz_max"] < 1e-15


def test_totals_with_density_weighting_and_aligned_fields(orc):
    """rho = 1 + e cos K x, u = (U0 + A cos K x, V0), b = beta u.
    Sum rho = N^2; sum rho u_x = N^2 (U0 + e A / 2) (the density weight
    matters); sum rho u_y = N^2 V0 (1 + 0); E_k = (U0^2 + A^2/2 + V0^2)/2
    (not density weighted); E_m = beta^2 E_k; mean u.b = 2 beta E_k;
    sum b = N^2 beta (U0, V0); div b = d_x b_x = -beta A sin K sin K x, so
    max |div b| = beta A sin K and its rms beta A sin K / sqrt 2; the
    vorticity is zero (u_y uniform, u_x independent of y)."""
    n, e, U0, A, V0, beta = 32, 0.2, 0.02, 0.03, -0.015, 1.7
    K = 2 * math.pi * 2 / n
    X, _ = np.meshgrid(np.arange(n), np.arange(n))
    rho = 1 + e * np.cos(K * X)
    ux = U0 + A * np.cos(K * X)
    uy = np.full((n, n), V0)
    p, f, g = _state(orc, n, (ux, uy, beta * ux, beta * uy), rho=rho)
    t = orc.totals(p, f, g)
    N2 = n * n
    ek = 0.5 * (U0 * U0 + A * A / 2 + V0 * V0)
    assert abs(t["mass"] - N2) < 1e-12 * N2
    assert abs(t["mom_x"] - N2 * (U0 + e * A / 2)) < 1e-13 * N2
    assert abs(t["mom_y"] - N2 * V0) < 1e-13 * N2
    assert abs(t["e_kin"] - ek) < 1e-15
    assert abs(t["e_mag"] - beta * beta * ek) < 1e-15
    assert abs(t["cross_hel"] - 2 * beta * ek) < 1e-15
    assert abs(t["bsum_x"] - N2 * beta * U0) < 1e-13 * N2
    assert abs(t["bsum_y"] - N2 * beta * V0) < 1e-13 * N2
    amp = beta * A * math.sin(K)
    assert abs(t["divb_max"] - amp) < 1e-14
    assert abs(t["divb_rms"] - amp / math.sqrt(2)) < 1e-14
    assert t["omega_max"] < 1e-15
    assert t["jz_max"] < 1e-15


def test_cross_helicity_pairs_like_components(orc):
    """u = (a, c), b = (d, h) uniform: mean u.b = a d + c h, which differs
    from the transposed pairing a h + c d."""
    n = 8
    a, c, d, h = 0.01, -0.03, 0.07, 0.02
    one = np.ones((n, n))
    p, f, g = _state(orc, n, (a * one, c * one, d * one, h * one))
    t = orc.totals(p, f, g)
    assert abs(t["cross_hel"] - (a * d + c * h)) < 1e-16
    assert abs(t["e_kin"] - 0.5 * (a * a + c * c)) < 1e-16
    assert abs(t["e_mag"] - 0.5 * (d * d + h * h)) < 1e-16


def test_current_maximum_of_a_decaying_magnetic_wave(orc):
    """b = (B sin K y, 0), u = 0: Eq. current gives j_z = -d_y b_x =
    -B(t) K cos K y, so the largest |j_z| is B(t) K with B(t) the measured
    amplitude, up to the O(K^2) lattice error of the first-order moment."""
    nx, ny, B = 4, 64, 1e-4
    K = 2 * math.pi / ny
    y = np.arange(ny)
    p = orc.Params(nx, ny, 0.8, 0.62)
    bx = B * np.tile(np.sin(K * y)[:, None], (1, nx))
    z = np.zeros((ny, nx))
    f, g = orc.run(p, *orc.init(p, z, z, bx, z), 50)
    b_now = orc.fields(p, f, g)[3][:, 0]
    amp = float(np.dot(b_now, np.sin(K * y)) / np.dot(np.sin(K * y), np.sin(K * y)))
    t = orc.totals(p, f, g)
    assert amp > 0.5 * B
    assert abs(t["jz_max"] / (amp * K) - 1) < 1e-2


@pytest.mark.parametrize("flip", [False, True])
def test_vorticity_and_divergence_of_diagonal_waves(orc, flip):
    """Fields along the diagonal, s(x, y) = sin K (x + y).  The isotropic
    stencil gives d_x s = d_y s = G cos K (x + y), G = sin K (2 + cos K)/3.
    u = A (1, 1) s is irrotational and b = B (1, -1) s solenoidal, so
    omega = d_x u_y - d_y u_x and div b vanish; swapping the two directions
    (flip) gives |omega| = 2 A G |cos|, |div b| = 2 B G |cos|.  A sign slip
    in either combination turns a zero into the maximum or back."""
    n, A, B = 32, 0.02, 0.03
    K = 2 * math.pi * 2 / n
    X, Y = np.meshgrid(np.arange(n), np.arange(n))
    s = np.sin(K * (X + Y))
    G = math.sin(K) * (2 + math.cos(K)) / 3
    su, sb = (-1.0, 1.0) if flip else (1.0, -1.0)
    p, f, g = _state(orc, n, (A * s, su * A * s, B * s, sb * B * s))
    t = orc.totals(p, f, g)
    if flip:
        assert abs(t["omega_max"] - 2 * A * G) < 1e-15
        assert abs(t["divb_max"] - 2 * B * G) < 1e-15
        assert abs(t["divb_rms"] - 2 * B * G / math.sqrt(2)) < 1e-15
    else:
        assert t["omega_max"] < 1e-15
        assert t["divb_max"] < 1e-15 and t["divb_rms"] < 1e-15
