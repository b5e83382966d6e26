"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks a property that a plausible slip in the oracle (a dropped
term, a wrong sign, a swapped index, a wrong permutation count) would break:
moment identities of the equilibria (Eq. feq_4th, Eq. a0_4, the magnetic
equilibrium), moments of the regularised non-equilibrium (Eq. fineq_reg),
exact conservation, the special cases, the lattice symmetry group, and the
closed form of the isotropic gradient (Orszag-Tang section).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_sets():
    out = {}
    with open(os.path.join(HERE, "golden", "lattice_sets.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [float(Fraction(v)) for v in vals]
    return out


G = _golden_sets()
CX = np.array(G["cx"]); CY = np.array(G["cy"]); W = np.array(G["w"])
EX = np.array(G["ex"]); EY = np.array(G["ey"]); PSI = np.array(G["psi"])
CS2 = 1.0 / 3.0

# Hermite polynomials on the nine velocities, written per component.
HXX = CX * CX - CS2
HYY = CY * CY - CS2
HXY = CX * CY
HXXY = (CX * CX - CS2) * CY
HXYY = CX * (CY * CY - CS2)
HXXYY = (CX * CX - CS2) * (CY * CY - CS2)


def _maxwell(bx, by):
    b2 = bx * bx + by * by
    return 0.5 * b2 - bx * bx, -bx * by, 0.5 * b2 - by * by  # M_xx, M_xy, M_yy


def _rand_state(rng, amp_u=0.1, amp_b=0.1):
    rho = rng.uniform(0.8, 1.2)
    ux, uy, bx, by = rng.uniform(-amp_u, amp_u, 2).tolist() + rng.uniform(-amp_b, amp_b, 2).tolist()
    return rho, ux, uy, bx, by


def test_lattice_matches_paper(orc):
    cx, cy, w, ex, ey, psi = orc.lattice()
    np.testing.assert_array_equal(cx, CX)
    np.testing.assert_array_equal(cy, CY)
    np.testing.assert_allclose(w, W, rtol=0, atol=1e-17)
    np.testing.assert_array_equal(ex, EX)
    np.testing.assert_array_equal(ey, EY)
    np.testing.assert_allclose(psi, PSI, rtol=0, atol=1e-17)
    # weights are normalised and isotropic to the order the expansion needs
    assert abs(W.sum() - 1) < 1e-15 and abs(PSI.sum() - 1) < 1e-15
    assert abs((W * CX * CX).sum() - CS2) < 1e-15 and abs((PSI * EX * EX).sum() - CS2) < 1e-15


def test_hermite_tensors_match_definition(orc):
    # spot values of the definition on D2Q9: H_xx, H_xxy, H_xxyy, and the
    # vanishing / aliased classes that the truncation handles
    for i in range(9):
        assert abs(orc.hermite(2, [0, 0], i) - HXX[i]) < 1e-15
        assert abs(orc.hermite(2, [0, 1], i) - HXY[i]) < 1e-15
        assert abs(orc.hermite(3, [0, 0, 1], i) - HXXY[i]) < 1e-15
        assert abs(orc.hermite(3, [1, 0, 1], i) - HXYY[i]) < 1e-15
        assert abs(orc.hermite(4, [0, 1, 0, 1], i) - HXXYY[i]) < 1e-15
        assert abs(orc.hermite(3, [0, 0, 0], i)) < 1e-15            # H_xxx = 0 on D2Q9
        assert abs(orc.hermite(4, [0, 0, 0, 1], i)) < 1e-15         # H_xxxy = 0 on D2Q9
        assert abs(orc.hermite(4, [0, 0, 0, 0], i) + HXX[i]) < 1e-15  # H_xxxx = -H_xx


@pytest.mark.parametrize("variant", [0, 1])
def test_equilibrium_moments(orc, variant):
    rng = np.random.default_rng(11 + variant)
    for _ in range(20):
        rho, ux, uy, bx, by = _rand_state(rng)
        f = orc.feq(rho, ux, uy, bx, by, variant)
        mxx, mxy, myy = _maxwell(bx, by)
        assert abs(f.sum() - rho) < 1e-14
        assert abs((f * CX).sum() - rho * ux) < 1e-15
        assert abs((f * CY).sum() - rho * uy) < 1e-15
        # sum f c c = rho u u + cs^2 rho I + |b|^2 I / 2 - b b
        assert abs((f * CX * CX).sum() - (rho * ux * ux + CS2 * rho + mxx)) < 1e-15
        assert abs((f * CX * CY).sum() - (rho * ux * uy + mxy)) < 1e-15
        assert abs((f * CY * CY).sum() - (rho * uy * uy + CS2 * rho + myy)) < 1e-15
        extra3x = 2 * ux * mxy + uy * mxx if variant else 0.0
        extra3y = ux * myy + 2 * uy * mxy if variant else 0.0
        extra4 = ux * ux * myy + 4 * ux * uy * mxy + uy * uy * mxx if variant else 0.0
        assert abs((f * HXXY).sum() - (rho * ux * ux * uy + extra3x)) < 1e-15
        assert abs((f * HXYY).sum() - (rho * ux * uy * uy + extra3y)) < 1e-15
        assert abs((f * HXXYY).sum() - (rho * ux * ux * uy * uy + extra4)) < 1e-15


def test_variants_agree_to_second_order(orc):
    rng = np.random.default_rng(5)
    rho, ux, uy, bx, by = _rand_state(rng)
    fa = orc.feq(rho, ux, uy, bx, by, 0)
    fb = orc.feq(rho, ux, uy, bx, by, 1)
    d = fb - fa
    for h in (np.ones(9), CX, CY, CX * CX, CX * CY, CY * CY):
        assert abs((d * h).sum()) < 1e-16
    # ... and differ at O(u b^2) above it
    assert np.abs(d).max() > 1e-6
    # without a magnetic field the two are the same
    np.testing.assert_array_equal(orc.feq(rho, ux, uy, 0, 0, 0), orc.feq(rho, ux, uy, 0, 0, 1))


def test_magnetic_equilibrium_moments(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        _, ux, uy, bx, by = _rand_state(rng)
        g = orc.geq(ux, uy, bx, by)  # (5, 2)
        assert abs(g[:, 0].sum() - bx) < 1e-16 and abs(g[:, 1].sum() - by) < 1e-16
        # first moment = induction flux u_a b_b - u_b b_a (antisymmetric)
        lam = np.array([[(EX * g[:, 0]).sum(), (EX * g[:, 1]).sum()],
                        [(EY * g[:, 0]).sum(), (EY * g[:, 1]).sum()]])
        u = np.array([ux, uy]); b = np.array([bx, by])
        expect = np.outer(u, b) - np.outer(b, u)
        np.testing.assert_allclose(lam, expect, rtol=0, atol=1e-16)
        # second moment = cs^2 delta b
        for a, ea in enumerate((EX, EY)):
            for c, ec in enumerate((EX, EY)):
                m2 = np.array([(ea * ec * g[:, k]).sum() for k in range(2)])
                np.testing.assert_allclose(m2, CS2 * (a == c) * b, rtol=0, atol=1e-16)


def _noneq_node(orc, rng, variant=0):
    rho, ux, uy, bx, by = _rand_state(rng)
    f = orc.feq(rho, ux, uy, bx, by, variant) + rng.normal(0, 2e-3, 9) * W
    g = orc.geq(ux, uy, bx, by) + rng.normal(0, 2e-3, (5, 2))
    return f, g


@pytest.mark.parametrize("variant", [0, 1])
def test_regularised_moments_and_recursion(orc, variant):
    rng = np.random.default_rng(21 + variant)
    p = orc.Params(4, 4, tau_f=0.61, tau_m=0.77, eq_variant=variant)
    for _ in range(20):
        f, g = _noneq_node(orc, rng, variant)
        _, _, info = orc.collide_node(p, f, g)
        rho, ux, uy, bx, by = info[:5]
        a2xx, a2xy, a2yy, a3xxy, a3xyy, a4 = info[5:11]
        fneq = info[11:]
        # moments of the input
        assert abs(rho - f.sum()) < 1e-15
        assert abs(ux - (f * CX).sum() / rho) < 1e-15
        assert abs(bx - g[:, 0].sum()) < 1e-15 and abs(by - g[:, 1].sum()) < 1e-15
        # projection = sum c c f - cs^2 rho I - rho u u - M (Hermite orthogonality)
        mxx, mxy, myy = _maxwell(bx, by)
        assert abs(a2xx - ((f * CX * CX).sum() - CS2 * rho - rho * ux * ux - mxx)) < 1e-15
        assert abs(a2xy - ((f * CX * CY).sum() - rho * ux * uy - mxy)) < 1e-15
        assert abs(a2yy - ((f * CY * CY).sum() - CS2 * rho - rho * uy * uy - myy)) < 1e-15
        # recursion contracted to the supported components
        assert abs(a3xxy - (2 * ux * a2xy + uy * a2xx)) < 1e-17
        assert abs(a3xyy - (2 * uy * a2xy + ux * a2yy)) < 1e-17
        a4_expect = (2 * ux * a3xyy + 2 * uy * a3xxy - ux * ux * a2yy - 4 * ux * uy * a2xy
                     - uy * uy * a2xx)
        assert abs(a4 - a4_expect) < 1e-18
        # f_neq,reg carries no mass or momentum and reproduces its coefficients
        assert abs(fneq.sum()) < 1e-17
        assert abs((fneq * CX).sum()) < 1e-17 and abs((fneq * CY).sum()) < 1e-17
        assert abs((fneq * HXX).sum() - a2xx) < 1e-17
        assert abs((fneq * HXY).sum() - a2xy) < 1e-17
        assert abs((fneq * HYY).sum() - a2yy) < 1e-17
        assert abs((fneq * HXXY).sum() - a3xxy) < 1e-17
        assert abs((fneq * HXYY).sum() - a3xyy) < 1e-17
        assert abs((fneq * HXXYY).sum() - a4) < 1e-18


@pytest.mark.parametrize("collision", [0, 1])
def test_collision_conserves_mass_momentum_and_b(orc, collision):
    rng = np.random.default_rng(7)
    p = orc.Params(4, 4, tau_f=0.5 + 3e-4, tau_m=0.9, collision=collision)
    for _ in range(20):
        f, g = _noneq_node(orc, rng)
        fs, gs, _ = orc.collide_node(p, f, g)
        assert abs(fs.sum() - f.sum()) < 1e-15
        assert abs((fs * CX).sum() - (f * CX).sum()) < 1e-15
        assert abs((fs * CY).sum() - (f * CY).sum()) < 1e-15
        np.testing.assert_allclose(gs.sum(axis=0), g.sum(axis=0), rtol=0, atol=2e-17)


def test_unit_relaxation_gives_equilibrium(orc):
    rng = np.random.default_rng(8)
    f, g = _noneq_node(orc, rng)
    fs, gs, info = orc.collide_node(orc.Params(4, 4, tau_f=1.0, tau_m=1.0), f, g)
    rho, ux, uy, bx, by = info[:5]
    np.testing.assert_allclose(fs, orc.feq(rho, ux, uy, bx, by), rtol=0, atol=1e-17)
    np.testing.assert_allclose(gs, orc.geq(ux, uy, bx, by), rtol=0, atol=1e-17)


def test_equilibrium_is_a_collision_fixed_point(orc):
    rng = np.random.default_rng(9)
    for tau in (0.5003, 0.8, 1.7):
        rho, ux, uy, bx, by = _rand_state(rng)
        f = orc.feq(rho, ux, uy, bx, by); g = orc.geq(ux, uy, bx, by)
        fs, gs, info = orc.collide_node(orc.Params(4, 4, tau_f=tau, tau_m=tau), f, g)
        assert np.abs(info[5:]).max() < 1e-16
        np.testing.assert_allclose(fs, f, rtol=0, atol=1e-16)
        np.testing.assert_allclose(gs, g, rtol=0, atol=1e-16)


def test_rest_state_and_uniform_flow_are_fixed_points(orc):
    p = orc.Params(6, 5, tau_f=0.56, tau_m=0.6)
    zero = np.zeros((5, 6))
    f, g = orc.init(p, zero, zero, zero, zero)
    np.testing.assert_allclose(f, W[:, None, None] * np.ones((9, 5, 6)), rtol=0, atol=1e-15)
    f1, g1 = orc.run(p, f, g, 5)
    np.testing.assert_allclose(f1, f, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(g1, 0)
    one = np.ones((5, 6))
    f, g = orc.init(p, 0.03 * one, -0.02 * one, 0.05 * one, 0.01 * one, rho=1.1 * one)
    f1, g1 = orc.run(p, f, g, 5)
    np.testing.assert_allclose(f1, f, rtol=0, atol=1e-15)
    np.testing.assert_allclose(g1, g, rtol=0, atol=1e-16)


def test_no_field_is_hydrodynamic(orc):
    """b = 0: the fluid update does not see g and keeps g at zero."""
    rng = np.random.default_rng(12)
    p = orc.Params(4, 4, tau_f=0.55, tau_m=0.7)
    rho, ux, uy, _, _ = _rand_state(rng)
    f = orc.feq(rho, ux, uy, 0, 0) + rng.normal(0, 1e-3, 9) * W
    fs0, gs0, _ = orc.collide_node(p, f, np.zeros((5, 2)))
    np.testing.assert_array_equal(gs0, 0)
    # hydrodynamic pressure tensor: sum c c f_eq = rho u u + cs^2 rho I
    fe = orc.feq(rho, ux, uy, 0, 0)
    assert abs((fe * CX * CY).sum() - rho * ux * uy) < 1e-16


# ---- lattice symmetry group --------------------------------------------------

def _perm(cx, cy, tx, ty):
    """index map k(i) with (cx_k, cy_k) = T(cx_i, cy_i)."""
    out = []
    for i in range(len(cx)):
        vx, vy = tx(cx[i], cy[i]), ty(cx[i], cy[i])
        out.append([k for k in range(len(cx)) if cx[k] == vx and cy[k] == vy][0])
    return out


SYMMETRIES = {
    "rot90": (lambda x, y: -y, lambda x, y: x),
    "mirror_x": (lambda x, y: -x, lambda x, y: y),
    "transpose": (lambda x, y: y, lambda x, y: x),
}


def _transform(name, f, g, n):
    tx, ty = SYMMETRIES[name]
    pf = _perm(CX, CY, tx, ty)
    pg = _perm(EX, EY, tx, ty)
    f2 = np.zeros_like(f); g2 = np.zeros_like(g)
    for y in range(n):
        for x in range(n):
            X, Y = tx(x, y) % n, ty(x, y) % n
            for i in range(9):
                f2[pf[i], Y, X] = f[i, y, x]
            for j in range(5):
                vx, vy = g[j, 0, y, x], g[j, 1, y, x]
                g2[pg[j], 0, Y, X] = tx(vx, vy)
                g2[pg[j], 1, Y, X] = ty(vx, vy)
    return f2, g2


@pytest.mark.parametrize("name", sorted(SYMMETRIES))
@pytest.mark.parametrize("variant,mag", [(0, 0), (1, 0), (0, 1)])
def test_step_commutes_with_lattice_symmetries(orc, name, variant, mag):
    n = 6
    rng = np.random.default_rng(31)
    p = orc.Params(n, n, tau_f=0.57, tau_m=0.83, eq_variant=variant, mag_collision=mag)
    ux, uy, bx, by = (rng.uniform(-0.08, 0.08, (n, n)) for _ in range(4))
    f, g = orc.init(p, ux, uy, bx, by, rho=rng.uniform(0.9, 1.1, (n, n)))
    f = f + rng.normal(0, 1e-3, f.shape) * W[:, None, None]
    g = g + rng.normal(0, 1e-3, g.shape)
    fa, ga = orc.run(p, *_transform(name, f, g, n), 2)
    fb, gb = _transform(name, *orc.run(p, f, g, 2), n)
    np.testing.assert_allclose(fa, fb, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ga, gb, rtol=0, atol=1e-15)


def test_isotropic_gradient_closed_form(orc):
    """The stencil applied to sin(k x + q y) gives sin(k) (2 + cos q)/3 cos(k x + q y)."""
    nx, ny = 16, 12
    p = orc.Params(nx, ny, 0.6, 0.6)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    k, q = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    th = k * X + q * Y
    dx, dy, valid = orc.gradient(p, np.sin(th))
    assert valid.all()
    np.testing.assert_allclose(dx, np.sin(k) * (2 + np.cos(q)) / 3 * np.cos(th), rtol=0, atol=1e-14)
    np.testing.assert_allclose(dy, np.sin(q) * (2 + np.cos(k)) / 3 * np.cos(th), rtol=0, atol=1e-14)
    # on a wall axis the rows whose stencil leaves the lattice are excluded
    pw = orc.Params(nx, ny, 0.6, 0.6, wall_y=True)
    _, _, valid = orc.gradient(pw, np.sin(th))
    assert not valid[0].any() and not valid[-1].any() and valid[1:-1].all()


def test_stream_is_a_permutation(orc):
    rng = np.random.default_rng(4)
    for wx, wy in ((False, False), (False, True), (True, True)):
        p = orc.Params(5, 4, 0.6, 0.6, wall_x=wx, wall_y=wy)
        fs = rng.normal(size=(9, 4, 5)); gs = rng.normal(size=(5, 2, 4, 5))
        f, g = orc.stream(p, fs, gs)
        np.testing.assert_allclose(np.sort(f.ravel()), np.sort(fs.ravel()))
        np.testing.assert_allclose(np.sort(g.ravel()), np.sort(gs.ravel()))
        # rest populations do not move
        np.testing.assert_array_equal(f[0], fs[0]); np.testing.assert_array_equal(g[0], gs[0])


# ---- regularised magnetic collision ------------------------------------------

def test_regularised_magnetic_collision_moments(orc):
    """g* - g_eq keeps sum = 0 (b conserved) and the first moment
    (1 - omega_m) Lambda, and has no second-order content: sum_j e_jx^2 and
    sum_j e_jy^2 of it vanish.  A non-equilibrium that is already first
    order is left as BGK leaves it; omega_m = 1 gives g_eq."""
    rng = np.random.default_rng(41)
    tau_m = 0.74
    om1 = 1 - 1 / tau_m
    ex, ey = np.array(EX, float), np.array(EY, float)
    for _ in range(20):
        ux, uy, bx, by = rng.uniform(-0.1, 0.1, 4)
        f = orc.feq(1.0 + rng.uniform(-0.05, 0.05), ux, uy, bx, by, 0)
        f = f + rng.normal(0, 1e-3, 9) * W
        rho = f.sum()
        u = (f * CX).sum() / rho, (f * CY).sum() / rho
        geq0 = orc.geq(u[0], u[1], bx, by).reshape(5, 2)
        neq = rng.normal(0, 1e-3, (5, 2))
        neq -= neq.mean(axis=0)                       # zero sum: the node's b is (bx, by)
        g = geq0 + neq
        fs, gs, _ = orc.collide_node(orc.Params(1, 1, 0.6, tau_m, mag_collision=1), f, g)
        d = gs - geq0
        np.testing.assert_allclose(d.sum(axis=0), 0, atol=1e-16)
        lam = np.array([[(e * neq[:, c]).sum() for c in range(2)] for e in (ex, ey)])
        got = np.array([[(e * d[:, c]).sum() for c in range(2)] for e in (ex, ey)])
        np.testing.assert_allclose(got, om1 * lam, rtol=0, atol=1e-16)
        for e in (ex, ey):
            np.testing.assert_allclose(((e * e)[:, None] * d).sum(axis=0), 0, atol=1e-16)
        # first-order non-equilibrium: regularised == BGK
        first = np.array([[PSI[j] * (ex[j] * lam[0, c] + ey[j] * lam[1, c]) * 3 for c in range(2)]
                          for j in range(5)])
        g1 = geq0 + first
        _, gr, _ = orc.collide_node(orc.Params(1, 1, 0.6, tau_m, mag_collision=1), f, g1)
        _, gb, _ = orc.collide_node(orc.Params(1, 1, 0.6, tau_m, mag_collision=0), f, g1)
        np.testing.assert_allclose(gr, gb, rtol=0, atol=1e-16)
        _, g_one, _ = orc.collide_node(orc.Params(1, 1, 0.6, 1.0, mag_collision=1), f, g)
        np.testing.assert_allclose(g_one, geq0, rtol=0, atol=1e-16)
