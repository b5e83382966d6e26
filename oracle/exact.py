"""Exact rational brute force of the RR-MHD step for tiny lattices.

TEST INFRASTRUCTURE ONLY (a pin for ``mhd_oracle.c``; the CUDA library never
imports it).  Every quantity is a ``fractions.Fraction``; the method needs only
+, -, x and division (u = m / rho, omega = 1 / tau), so one step is exact.

It restates the step differently from the C oracle, so that an index, sign or
permutation slip in either shows up as a mismatch:
  * f_eq is Eq. feq_4th written out as printed (with 1/(4 cs^8) on the H_xxyy
    term), plus the u (x) M cross terms of Eq. a0_4 for equilibrium variant B;
  * a1^(2) is the projection of Task 3 with H2 written per component;
  * the third- and fourth-order coefficients are the recursion of Task 3
    contracted by hand to the xxy, xyy and xxyy components;
  * f_neq,reg is Eq. fineq_reg with the permutation counts folded in
    (3 for xxy / xyy, 6 for xxyy);
  * streaming is in pull form, f_i(x) = f*_i(x - c_i), where the C oracle
    pushes.
"""
from __future__ import annotations

from fractions import Fraction as Fr

CX = (0, -1, -1, -1, 0, 1, 1, 1, 0)
CY = (0, 1, 0, -1, -1, -1, 0, 1, 1)
W = (Fr(4, 9), Fr(1, 36), Fr(1, 9), Fr(1, 36), Fr(1, 9), Fr(1, 36), Fr(1, 9), Fr(1, 36), Fr(1, 9))
EX = (0, -1, 0, 1, 0)
EY = (0, 0, -1, 0, 1)
PSI = (Fr(1, 3), Fr(1, 6), Fr(1, 6), Fr(1, 6), Fr(1, 6))
CS2 = Fr(1, 3)
OPP_F = (0, 5, 6, 7, 8, 1, 2, 3, 4)
OPP_G = (0, 3, 4, 1, 2)


def _herm(i):
    cx, cy = CX[i], CY[i]
    return dict(xx=cx * cx - CS2, yy=cy * cy - CS2, xy=Fr(cx * cy),
                xxy=(cx * cx - CS2) * cy, xyy=cx * (cy * cy - CS2),
                xxyy=(cx * cx - CS2) * (cy * cy - CS2))


def feq(rho, ux, uy, bx, by, variant=0):
    mxx = (bx * bx + by * by) / 2 - bx * bx
    myy = (bx * bx + by * by) / 2 - by * by
    mxy = -bx * by
    out = []
    for i in range(9):
        h = _herm(i)
        cx, cy = CX[i], CY[i]
        cu = cx * ux + cy * uy
        h2uu = h["xx"] * ux * ux + 2 * h["xy"] * ux * uy + h["yy"] * uy * uy
        t3 = h["xxy"] * ux * ux * uy + h["xyy"] * ux * uy * uy
        t4 = h["xxyy"] * ux * ux * uy * uy
        v = W[i] * rho * (1 + cu / CS2 + h2uu / (2 * CS2 ** 2) + t3 / (2 * CS2 ** 3)
                          + t4 / (4 * CS2 ** 4))
        c2 = cx * cx + cy * cy
        cb = cx * bx + cy * by
        v += W[i] / (2 * CS2 ** 2) * ((bx * bx + by * by) * c2 / 2 - cb * cb)
        if variant == 1:
            m3xxy = 2 * ux * mxy + uy * mxx
            m3xyy = ux * myy + 2 * uy * mxy
            m4 = ux * ux * myy + 4 * ux * uy * mxy + uy * uy * mxx
            v += W[i] * ((h["xxy"] * m3xxy + h["xyy"] * m3xyy) / (2 * CS2 ** 3)
                         + h["xxyy"] * m4 / (4 * CS2 ** 4))
        out.append(v)
    return out


def geq(ux, uy, bx, by):
    out = []
    for j in range(5):
        ex, ey = EX[j], EY[j]
        gx = PSI[j] * (bx + ey * (uy * bx - ux * by) / CS2)
        gy = PSI[j] * (by + ex * (ux * by - uy * bx) / CS2)
        out.append((gx, gy))
    return out


def collide_node(f, g, tau_f, tau_m, variant=0, collision=0, mag_collision=0):
    """f: 9 Fractions, g: 5 pairs.  Returns (f*, g*).  mag_collision = 1:
    only the first Hermite moment of g - g_eq relaxes; on D2Q5 that keeps
    the antisymmetric half of each opposite pair's non-equilibrium,
    (n_3 - n_1)/2 and (n_4 - n_2)/2 with opposite signs, and sets the rest
    population's to zero."""
    rho = sum(f)
    ux = sum(f[i] * CX[i] for i in range(9)) / rho
    uy = sum(f[i] * CY[i] for i in range(9)) / rho
    bx = sum(g[j][0] for j in range(5))
    by = sum(g[j][1] for j in range(5))
    fe = feq(rho, ux, uy, bx, by, variant)
    ge = geq(ux, uy, bx, by)
    omega = 1 / Fr(tau_f)
    omega_m = 1 / Fr(tau_m)
    a2xx = sum(_herm(i)["xx"] * (f[i] - fe[i]) for i in range(9))
    a2xy = sum(_herm(i)["xy"] * (f[i] - fe[i]) for i in range(9))
    a2yy = sum(_herm(i)["yy"] * (f[i] - fe[i]) for i in range(9))
    a3xxy = 2 * ux * a2xy + uy * a2xx
    a3xyy = 2 * uy * a2xy + ux * a2yy
    a4 = 2 * ux * a3xyy + 2 * uy * a3xxy - ux * ux * a2yy - 4 * ux * uy * a2xy - uy * uy * a2xx
    fs = []
    for i in range(9):
        h = _herm(i)
        fneq = W[i] * ((h["xx"] * a2xx + 2 * h["xy"] * a2xy + h["yy"] * a2yy) / (2 * CS2 ** 2)
                       + 3 * (h["xxy"] * a3xxy + h["xyy"] * a3xyy) / (6 * CS2 ** 3)
                       + 6 * h["xxyy"] * a4 / (24 * CS2 ** 4))
        if collision == 1:
            fneq = f[i] - fe[i]
        fs.append(fe[i] + (1 - omega) * fneq)
    if mag_collision == 1:
        n = [(g[j][0] - ge[j][0], g[j][1] - ge[j][1]) for j in range(5)]
        h13 = [(n[3][a] - n[1][a]) / 2 for a in range(2)]
        h24 = [(n[4][a] - n[2][a]) / 2 for a in range(2)]
        reg = [(0, 0), (-h13[0], -h13[1]), (-h24[0], -h24[1]), (h13[0], h13[1]), (h24[0], h24[1])]
        gs = [(ge[j][0] + (1 - omega_m) * reg[j][0], ge[j][1] + (1 - omega_m) * reg[j][1])
              for j in range(5)]
    else:
        gs = [(ge[j][0] + (1 - omega_m) * (g[j][0] - ge[j][0]),
               ge[j][1] + (1 - omega_m) * (g[j][1] - ge[j][1])) for j in range(5)]
    return fs, gs


def step(f, g, nx, ny, tau_f, tau_m, wall_x=False, wall_y=False, variant=0, collision=0,
         mag_collision=0):
    """One collide-then-stream step.  f[i][y][x], g[j][y][x] = (gx, gy)."""
    fs = [[[None] * nx for _ in range(ny)] for _ in range(9)]
    gs = [[[None] * nx for _ in range(ny)] for _ in range(5)]
    for y in range(ny):
        for x in range(nx):
            fl, gl = collide_node([f[i][y][x] for i in range(9)], [g[j][y][x] for j in range(5)],
                                  tau_f, tau_m, variant, collision, mag_collision)
            for i in range(9):
                fs[i][y][x] = fl[i]
            for j in range(5):
                gs[j][y][x] = gl[j]

    def outside(sx, sy):
        return (wall_x and not 0 <= sx < nx) or (wall_y and not 0 <= sy < ny)

    fn = [[[None] * nx for _ in range(ny)] for _ in range(9)]
    gn = [[[None] * nx for _ in range(ny)] for _ in range(5)]
    for y in range(ny):
        for x in range(nx):
            for i in range(9):
                sx, sy = x - CX[i], y - CY[i]
                fn[i][y][x] = fs[OPP_F[i]][y][x] if outside(sx, sy) else fs[i][sy % ny][sx % nx]
            for j in range(5):
                sx, sy = x - EX[j], y - EY[j]
                gn[j][y][x] = gs[OPP_G[j]][y][x] if outside(sx, sy) else gs[j][sy % ny][sx % nx]
    return fn, gn
