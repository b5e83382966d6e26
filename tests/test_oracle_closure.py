"""Pins of the closure oracle (oracle/closure.py) against the mathematics:
finite-difference gradients of the MLP, Adam's first step, the filter's
conservation, closed forms of the stencils, and the target formula (zero
on a plain coarse trajectory, and exactly the applied correction when the
next state was produced by a corrected collision)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def clo(orc):
    from oracle import closure
    return closure


def test_mlp_gradients_match_finite_differences(clo):
    rng = np.random.default_rng(0)
    X = rng.normal(size=(40, clo.N_IN))
    T = rng.normal(size=(40, clo.N_OUT))
    net = clo.MLP(seed=3)
    net.p["mean"] = rng.normal(size=clo.N_IN) * 0.1
    net.p["scale"] = rng.uniform(0.5, 2.0, clo.N_IN)
    net.p["out_scale"] = rng.uniform(0.5, 2.0, clo.N_OUT)
    net.p["b1"] = rng.normal(size=clo.N_HID) * 0.1
    loss, grads = net.loss_and_grads(X, T)
    h = 1e-6
    for name in clo.TRAINABLE:
        flat = net.p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = net.loss_and_grads(X, T)
            flat[idx] = old - h
            lm, _ = net.loss_and_grads(X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[name].reshape(-1)[idx]) < 1e-6 * max(1.0, abs(fd)), (name, idx)


def test_adam_first_step_is_lr_times_sign(clo):
    params = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -1e-3, 4.0])}
    Adam = clo.Adam(lr=0.01, eps=1e-12)
    Adam.step(params, g)
    np.testing.assert_allclose(params["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], rtol=0, atol=1e-9)


def test_bf16_rounding(clo):
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -3.14159265, 1e-3])
    r = clo.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0            # tie to even
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == 1.0 + 2 ** -6                  # tie to even (upwards)
    assert abs(r[4] / x[4] - 1) < 2 ** -8 and abs(r[5] / x[5] - 1) < 2 ** -8


def test_filter_conserves_and_averages(orc, clo):
    rng = np.random.default_rng(1)
    f = rng.normal(size=(9, 16, 24))
    g = rng.normal(size=(5, 2, 16, 24))
    fc, gc = clo.box_filter(f, g, 4)
    assert fc.shape == (9, 4, 6) and gc.shape == (5, 2, 4, 6)
    np.testing.assert_allclose(fc.sum(axis=(1, 2)) * 16, f.sum(axis=(1, 2)), rtol=1e-13)
    np.testing.assert_allclose(gc.sum(axis=(2, 3)) * 16, g.sum(axis=(2, 3)), rtol=1e-13)
    assert abs(fc[3, 1, 2] - f[3, 4:8, 8:12].mean()) < 1e-15


def test_stencil_closed_forms(clo):
    nx, ny = 16, 12
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    k, q = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    th = k * X + q * Y
    s = np.sin(th)
    lap = (8 * (np.cos(k) + np.cos(q)) + 4 * np.cos(k) * np.cos(q) - 20) / 6 * s
    np.testing.assert_allclose(clo.lap9(s), lap, rtol=0, atol=1e-14)
    np.testing.assert_allclose(clo.dxy(s), -np.sin(k) * np.sin(q) * s, rtol=0, atol=1e-14)


def test_feature_columns(orc, clo):
    import mhd_inputs
    n = 16
    p = orc.Params(n, n, 0.6, 0.7)
    ux, uy, bx, by = mhd_inputs.orszag_tang(n, 0.05, 0.03)
    f, g = orc.init(p, ux, uy, bx, by)
    X, a2 = clo.features(p, f, g)
    assert X.shape == (n * n, 24)
    np.testing.assert_allclose(X[:, 1], ux.reshape(-1), atol=1e-15)
    np.testing.assert_allclose(X[:, 4], by.reshape(-1), atol=1e-15)
    np.testing.assert_allclose(X[:, 5:8], 0, atol=1e-16)        # equilibrium: no non-equilibrium
    dx, dy, _ = orc.gradient(p, uy)
    np.testing.assert_allclose(X[:, 12], dx.reshape(-1), atol=1e-16)  # d_x u_y
    np.testing.assert_allclose(X[:, 14], clo.lap9(uy).reshape(-1), atol=1e-16)


def _state(orc, n, seed):
    import mhd_inputs
    p = orc.Params(n, n, 0.53, 0.56)
    f, g = orc.init(p, *mhd_inputs.random_spectrum(n, n, seed, 0.03, 0.03, kmax=3))
    return p, *orc.run(p, f, g, 7)


def test_target_is_zero_on_a_plain_coarse_step(orc, clo):
    p, f, g = _state(orc, 16, 5)
    f1, g1 = clo.closure_step(p, f, g, None)
    assert np.abs(clo.targets(p, f, g, f1, g1)).max() < 1e-14


def test_target_recovers_an_applied_correction(orc, clo):
    p, f, g = _state(orc, 16, 6)
    rng = np.random.default_rng(2)
    da = rng.normal(0, 1e-4, (16, 16, 3))
    fs, gs = orc.collide_da(p, f, g, da)
    f1, g1 = orc.stream(p, fs, gs)
    np.testing.assert_allclose(clo.targets(p, f, g, f1, g1), da.reshape(-1, 3), rtol=0, atol=1e-13)


def test_closure_keeps_mass_and_momentum_and_zero_net_is_plain(orc, clo):
    p, f, g = _state(orc, 16, 7)
    net = clo.MLP(seed=1)
    net.p["out_scale"][:] = 1e-4
    f1, g1 = clo.closure_step(p, f, g, net)
    cx, cy, *_ = orc.lattice()
    assert abs(f1.sum() - f.sum()) < 1e-12
    assert abs((f1 * cx[:, None, None]).sum() - (f * cx[:, None, None]).sum()) < 1e-13
    zero = clo.MLP(seed=1)
    for k in clo.TRAINABLE:
        zero.p[k][:] = 0
    fz, gz = clo.closure_step(p, f, g, zero)
    fp, gp = clo.closure_step(p, f, g, None)
    np.testing.assert_array_equal(fz, fp)
    assert np.abs(f1 - fp).max() > 1e-8


def test_sgs_target_vanishes_for_block_constant_fields(orc, clo):
    n, r = 16, 4
    p = orc.Params(n, n, 0.6, 0.6)
    rng = np.random.default_rng(8)
    blocks = [np.kron(rng.uniform(-0.05, 0.05, (n // r, n // r)), np.ones((r, r))) for _ in range(4)]
    f, g = orc.init(p, *blocks, rho=np.kron(rng.uniform(0.95, 1.05, (n // r, n // r)), np.ones((r, r))))
    assert np.abs(clo.sgs_targets(p, f, g, r, 0.51)).max() < 1e-15


def test_sgs_target_trace_is_the_weighted_velocity_variance(orc, clo):
    """tr(tau_sgs) = <rho |u|^2> - <rho u>^2 / <rho> >= 0 (the Maxwell part
    is traceless in 2-D)."""
    n, r, tau_c = 16, 4, 0.52
    p = orc.Params(n, n, 0.6, 0.6)
    rng = np.random.default_rng(9)
    ux, uy, bx, by = (rng.uniform(-0.05, 0.05, (n, n)) for _ in range(4))
    rho = rng.uniform(0.95, 1.05, (n, n))
    f, g = orc.init(p, ux, uy, bx, by, rho=rho)
    t = clo.sgs_targets(p, f, g, r, tau_c) * (1 - 1 / tau_c)
    def avg(a):
        return a.reshape(n // r, r, n // r, r).mean(axis=(1, 3)).reshape(-1)
    var = avg(rho * (ux ** 2 + uy ** 2)) - (avg(rho * ux) ** 2 + avg(rho * uy) ** 2) / avg(rho)
    np.testing.assert_allclose(t[:, 0] + t[:, 2], var, rtol=1e-9, atol=1e-15)
    assert (var > 0).all()


def test_sgs_target_of_fields_linear_inside_each_block(orc, clo):
    """Inside each r x r block let the fields be linear in the in-block
    offsets (i, j), with rho = 1:  u = (alpha j, delta j) + U_B and
    b = (beta i, gamma i) + B_B, where U_B, B_B are random per-block
    constants.  Over a block i and j are independent and uniform on
    {0, ..., r-1} with variance V = (r^2 - 1)/12, so the filtered fluxes
    minus the fluxes of the filtered fields are the covariances:
      <uu> - u_bar u_bar = V [[a^2, a d], [a d, d^2]],
      <M> - M(b_bar) = (1/2) tr(C) I - C,  C = V [[b^2, b g], [b g, g^2]],
    so tau_xx = V (a^2 + (g^2 - b^2)/2), tau_xy = V (a d - b g),
    tau_yy = V (d^2 + (b^2 - g^2)/2), and the target is tau / (1 - 1/tau_c).
    The off-diagonal Maxwell term enters with the sign opposite to the
    Reynolds term, and the Maxwell diagonal is traceless: a sign or a
    transposition in either part fails here."""
    n, r, tau_c = 16, 4, 0.515
    al, de, be, ga = 0.011, -0.007, 0.013, 0.005
    p = orc.Params(n, n, 0.6, 0.6)
    rng = np.random.default_rng(10)
    X, Y = np.meshgrid(np.arange(n), np.arange(n))
    i, j = X % r, Y % r
    const = [np.kron(rng.uniform(-0.02, 0.02, (n // r, n // r)), np.ones((r, r))) for _ in range(4)]
    f, g = orc.init(p, al * j + const[0], de * j + const[1], be * i + const[2], ga * i + const[3])
    got = clo.sgs_targets(p, f, g, r, tau_c)
    V = (r * r - 1) / 12.0
    want = np.array([V * (al * al + (ga * ga - be * be) / 2), V * (al * de - be * ga),
                     V * (de * de + (be * be - ga * ga) / 2)]) / (1 - 1 / tau_c)
    assert abs(want[1]) > 0.5 * np.abs(want).max()
    np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), rtol=1e-9, atol=1e-16)


def test_gradient_scales_bound_the_gradients_and_the_bf16_backward_rounding(clo):
    """The scales of loss_and_grads are sums of absolute values of the terms
    each gradient element sums, so |grad| <= scale, with equality when every
    term has one sign (nonnegative weights and activations and a target
    below every output make all of them nonnegative).  Rounding the
    back-propagated operands to bfloat16 (at most 2^-9 relative each, and a
    weight gradient meets at most three such roundings along its chain)
    moves every element by less than 3 * 2^-9 of its scale."""
    rng = np.random.default_rng(12)
    X = rng.normal(size=(300, clo.N_IN))
    net = clo.MLP(seed=5)
    for k in ("W1", "W2", "W3"):
        net.p[k] = np.abs(net.p[k])
    net.p["b1"][:] = 0.1
    net.p["b2"][:] = 0.1
    Xp = np.abs(X)
    T = np.full((300, clo.N_OUT), -50.0)
    _, g, s = net.loss_and_grads(Xp, T, bf16_like_gpu=True, scales=True)
    for k in clo.TRAINABLE:
        np.testing.assert_allclose(np.abs(g[k]), s[k], rtol=1e-12, atol=0)
    net2 = clo.MLP(seed=6)
    T2 = rng.normal(size=(300, clo.N_OUT))
    _, g0, s0 = net2.loss_and_grads(X, T2, bf16_like_gpu=True, scales=True)
    _, gb = net2.loss_and_grads(X, T2, bf16_like_gpu=True, bf16_backward=True)
    moved = False
    for k in clo.TRAINABLE:
        assert (np.abs(g0[k]) <= s0[k] * (1 + 1e-12)).all(), k
        assert (np.abs(gb[k] - g0[k]) <= 3 * 2.0 ** -9 * s0[k]).all(), k
        moved |= bool(np.any(gb[k] != g0[k]))
    assert moved


def test_closure_interval_with_a_constant_correction_changes_nothing(orc, clo):
    """A network whose output does not depend on its input (zero weights, a
    bias on the last layer) gives the same correction on every step, so
    evaluating it every k-th step and reusing it in between must give the
    same run for every k; with a state-dependent network the runs differ."""
    import mhd_inputs
    n = 16
    p = orc.Params(n, n, 0.56, 0.6)
    f, g = orc.init(p, *mhd_inputs.random_spectrum(n, n, 3, 0.03, 0.03, kmax=3))
    const = clo.MLP(seed=2)
    for k in ("W1", "W2", "W3"):
        const.p[k][:] = 0.0
    const.p["b3"] = np.array([0.3, -0.2, 0.1])
    const.p["out_scale"][:] = 1e-4
    ref = clo.closure_run(p, f, g, 9, const, interval=1)
    for k in (2, 4, 9):
        got = clo.closure_run(p, f, g, 9, const, interval=k)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), k
    net = clo.MLP(seed=2)
    net.p["out_scale"][:] = 1e-4
    a = clo.closure_run(p, f, g, 9, net, interval=1)
    b = clo.closure_run(p, f, g, 9, net, interval=4)
    assert np.abs(a[0] - b[0]).max() > 1e-10
