"""The FP64 oracle against an exact rational brute force on tiny lattices.

``oracle/exact.py`` restates the step with the printed closed forms (Eq.
feq_4th, the per-component recursion, Eq. fineq_reg with folded permutation
counts) and pull streaming; the C oracle uses Hermite tensor loops and push
streaming.  Agreement to FP64 rounding on random non-equilibrium states pins
both.  Exact conservation of mass, momentum and b is checked in rationals.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import exact


def _rand_frac(rng, lo, hi, den=1000):
    return Fr(int(rng.integers(int(lo * den), int(hi * den) + 1)), den)


def _state(rng, nx, ny, variant):
    f = [[[None] * nx for _ in range(ny)] for _ in range(9)]
    g = [[[None] * nx for _ in range(ny)] for _ in range(5)]
    for y in range(ny):
        for x in range(nx):
            rho = _rand_frac(rng, 0.9, 1.1)
            ux, uy, bx, by = (_rand_frac(rng, -0.08, 0.08) for _ in range(4))
            fe = exact.feq(rho, ux, uy, bx, by, variant)
            ge = exact.geq(ux, uy, bx, by)
            for i in range(9):
                f[i][y][x] = fe[i] + _rand_frac(rng, -0.002, 0.002, 100000) * exact.W[i]
            for j in range(5):
                g[j][y][x] = (ge[j][0] + _rand_frac(rng, -0.002, 0.002, 100000),
                              ge[j][1] + _rand_frac(rng, -0.002, 0.002, 100000))
    return f, g


def _to_np(f, g, nx, ny):
    fa = np.array([[[float(f[i][y][x]) for x in range(nx)] for y in range(ny)] for i in range(9)])
    ga = np.array([[[[float(g[j][y][x][a]) for x in range(nx)] for y in range(ny)]
                    for a in range(2)] for j in range(5)])
    return fa, ga


CASES = [
    # nx, ny, tau_f, tau_m, wall_x, wall_y, variant, collision, mag_collision, steps
    (4, 4, Fr(3, 5), Fr(7, 10), False, False, 0, 0, 0, 3),
    (4, 6, Fr(11, 20), Fr(9, 10), False, True, 1, 0, 0, 2),
    (5, 4, Fr(13, 10), Fr(3, 5), True, True, 0, 1, 0, 2),
    (3, 5, Fr(51, 100), Fr(51, 100), True, False, 1, 0, 0, 2),
    (4, 4, Fr(3, 5), Fr(13, 20), False, False, 0, 0, 1, 3),
    (5, 4, Fr(11, 20), Fr(3, 2), True, True, 1, 1, 1, 2),
]


@pytest.mark.parametrize("case", CASES,
                         ids=lambda c: f"{c[0]}x{c[1]}_w{int(c[4])}{int(c[5])}_v{c[6]}_c{c[7]}_m{c[8]}")
def test_oracle_matches_exact_brute_force(orc, case):
    nx, ny, tf, tm, wx, wy, variant, collision, mag, steps = case
    rng = np.random.default_rng(nx * 100 + ny + 7 * mag)
    f, g = _state(rng, nx, ny, variant)
    f0, g0 = _to_np(f, g, nx, ny)
    for _ in range(steps):
        f, g = exact.step(f, g, nx, ny, tf, tm, wx, wy, variant, collision, mag)
    fe, ge = _to_np(f, g, nx, ny)
    p = orc.Params(nx, ny, float(tf), float(tm), wall_x=wx, wall_y=wy, eq_variant=variant,
                   collision=collision, mag_collision=mag)
    fo, go = orc.run(p, f0, g0, steps)
    np.testing.assert_allclose(fo, fe, rtol=0, atol=1e-14 * np.abs(fe).max())
    np.testing.assert_allclose(go, ge, rtol=0, atol=1e-14 * np.abs(ge).max())


@pytest.mark.parametrize("walls", [(False, False), (False, True), (True, True)])
def test_exact_conservation(walls):
    nx, ny = 4, 4
    rng = np.random.default_rng(99)
    f, g = _state(rng, nx, ny, 0)

    def totals(f, g):
        mass = sum(f[i][y][x] for i in range(9) for y in range(ny) for x in range(nx))
        bx = sum(g[j][y][x][0] for j in range(5) for y in range(ny) for x in range(nx))
        by = sum(g[j][y][x][1] for j in range(5) for y in range(ny) for x in range(nx))
        mx = sum(f[i][y][x] * exact.CX[i] for i in range(9) for y in range(ny) for x in range(nx))
        my = sum(f[i][y][x] * exact.CY[i] for i in range(9) for y in range(ny) for x in range(nx))
        return mass, bx, by, mx, my

    t0 = totals(f, g)
    f1, g1 = exact.step(f, g, nx, ny, Fr(3, 5), Fr(4, 5), walls[0], walls[1])
    t1 = totals(f1, g1)
    assert t1[:3] == t0[:3]          # mass and sum b: exact, with or without walls
    if not any(walls):
        assert t1[3:] == t0[3:]      # momentum: exact on a periodic lattice
