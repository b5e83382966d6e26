"""The equilibrium variant B and the regularised magnetic collision on the
CUDA path: parity with the FP64 oracle, and their effect on the paper's
low-Reynolds Orszag-Tang results (Tables 1-2) and on the 64^2 vortex.

Regularised magnetic collision (MHD_MAG_REGULARISED): only the first
Hermite moment of g - g_eq relaxes -- the extension of the regularisation to
the magnetic populations that the Conclusions name as the next step.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pert_state(orc, p, seed):
    rng = np.random.default_rng(seed)
    ux, uy, bx, by = (rng.uniform(-0.06, 0.06, (p.ny, p.nx)) for _ in range(4))
    f, g = orc.init(p, ux, uy, bx, by, rho=rng.uniform(0.95, 1.05, (p.ny, p.nx)))
    f = f + rng.normal(0, 3e-4, f.shape) * np.array([4 / 9] + [1 / 36, 1 / 9] * 4)[:, None, None]
    g = g + rng.normal(0, 3e-4, g.shape)
    return f, g


@pytest.mark.parametrize("nx,ny,wx,wy,variant", [
    (48, 40, False, False, 0),
    (37, 29, False, False, 1),
    (30, 34, True, True, 0),
    (96, 24, False, True, 1),
])
def test_fp64_regularised_magnetic_collision_elementwise(orc, nx, ny, wx, wy, variant):
    import mhd_inputs
    from paper_2602_14667_gb300 import MHD_MAG_REGULARISED, Lattice
    steps = 50
    p = orc.Params(nx, ny, 0.56, 0.71, wall_x=wx, wall_y=wy, eq_variant=variant, mag_collision=1)
    fields = mhd_inputs.orszag_tang(nx, 0.05, 0.05, ny)
    f, g = orc.run(p, *orc.init(p, *fields), steps)
    fo, go = orc.collide(p, f, g)
    with Lattice(nx, ny, 0.56, 0.71, precision="fp64", wall_x=wx, wall_y=wy, eq_variant=variant,
                 mag_collision=MHD_MAG_REGULARISED) as lat:
        lat.set_fields(*fields)
        lat.advance(steps)
        fg, gg = lat.get_populations()
        tot = lat.get_totals()
    np.testing.assert_allclose(fg, fo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(gg, go, rtol=0, atol=1e-14)
    ref = orc.totals(p, f, g)
    assert abs(tot["jz_max"] - ref["jz_max"]) <= 1e-11 * ref["jz_max"]


@pytest.mark.parametrize("prec,shape,tol", [("fp32", (2, 8), 2e-6), ("fp32", (1, 1), 2e-6),
                                            ("fp32", (4, 2), 2e-6), ("fp16s", (4, 2), None)])
def test_one_step_regularised_magnetic_collision(orc, prec, shape, tol):
    from paper_2602_14667_gb300 import MHD_MAG_REGULARISED, Lattice
    nx, ny = 256, 24
    p = orc.Params(nx, ny, 0.5 + 3e-4, 0.51, mag_collision=1)
    f_pre, g_pre = _pert_state(orc, p, 17)
    fs, gs = orc.collide(p, f_pre, g_pre)
    with Lattice(nx, ny, p.tau_f, p.tau_m, precision=prec, mag_collision=MHD_MAG_REGULARISED) as lat:
        lat.kernel_config = shape
        lat.set_populations(fs, gs)
        fs_in, gs_in = lat.get_populations()       # the stored (rounded) state
        lat.advance(1)
        fg, gg = lat.get_populations()
    fo, go = orc.collide(p, *orc.stream(p, fs_in, gs_in))
    if tol is None:   # FP16S: half rounding of the output (see the FP16S parity test)
        w = np.array([4 / 9] + [1 / 36, 1 / 9] * 4)[:, None, None]
        tol = 4 * 2.0 ** -11 * max(np.abs(fo - w).max(), np.abs(go).max())
    assert np.abs(fg - fo).max() < tol and np.abs(gg - go).max() < tol


def test_batch_regularised_magnetic_collision(orc):
    import mhd_inputs
    from paper_2602_14667_gb300 import MHD_MAG_REGULARISED, Batch
    sizes, taus = [(64, 64), (96, 32)], [(0.55, 0.6), (0.6, 0.53)]
    with Batch(sizes, taus, mag_collision=MHD_MAG_REGULARISED) as b:
        for i, (nx, ny) in enumerate(sizes):
            b.set_fields(i, *mhd_inputs.random_spectrum(nx, ny, 50 + i, 0.02, 0.02))
        b.advance(100)
        for i, (nx, ny) in enumerate(sizes):
            p = orc.Params(nx, ny, *taus[i], mag_collision=1)
            f, g = orc.run(p, *orc.init(p, *mhd_inputs.random_spectrum(nx, ny, 50 + i, 0.02, 0.02)), 100)
            ref = orc.fields(p, f, g)
            got = b.get_fields(i)
            for k, r in zip(("ux", "uy", "bx", "by"), ref[1:]):
                assert np.linalg.norm(got[k] - r) / np.linalg.norm(r) < 1e-5, (i, k)


def test_variant_and_magnetic_collision_effect_on_the_64_vortex(orc):
    """64^2 Orszag-Tang, u0 = b0 = 0.05, nu = eta = 0.01, 1000 steps (FP64):
    each option's GPU run equals its oracle run to 1e-12, and its fields
    differ from the default scheme's by O(1e-3) (variant B: O(u b^2) terms;
    regularised g: the dropped second-order non-equilibrium of g)."""
    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice
    n = 64
    fields = mhd_inputs.orszag_tang(n, 0.05, 0.05)
    out = {}
    for variant, mag in ((0, 0), (1, 0), (0, 1), (1, 1)):
        with Lattice(n, n, 0.53, 0.53, precision="fp64", eq_variant=variant, mag_collision=mag) as lat:
            lat.set_fields(*fields)
            lat.advance(1000)
            got = lat.get_fields()
        p = orc.Params(n, n, 0.53, 0.53, eq_variant=variant, mag_collision=mag)
        ref = orc.fields(p, *orc.run(p, *orc.init(p, *fields), 1000))
        for k, r in zip(("ux", "uy", "bx", "by"), ref[1:]):
            assert np.linalg.norm(got[k] - r) / np.linalg.norm(r) < 1e-12, (variant, mag, k)
        out[(variant, mag)] = got
    base = out[(0, 0)]
    for key in ((1, 0), (0, 1), (1, 1)):
        d = {k: float(np.linalg.norm(out[key][k] - base[k]) / np.linalg.norm(base[k]))
             for k in ("ux", "uy", "bx", "by")}
        print(f"variant {'AB'[key[0]]}, magnetic {'BGK reg'.split()[key[1]]}: rel L2 vs default {d}")
        assert 1e-5 < max(d.values()) < 1e-2


@pytest.mark.parametrize("variant,mag", [(1, 0), (0, 1), (1, 1)])
def test_options_keep_the_paper_tables(variant, mag):
    """Tables 1-2 (Re = 200 pi) at N = 128 and 256: each option moves j_max
    by under 2 % and omega_max by under 1 % from the default scheme, and
    stays within 4 % / 2 % of the printed RR values (the default meets 3 % /
    2 %; the regularised magnetic collision raises j_max at N = 128, t = 1
    by 0.8 %, to 3.4 % above the printed value)."""
    import os
    from paper_2602_14667_gb300 import orszag_tang
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "ot_tables_rr.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                t, n, j, w, d = line.split()
                rows[(float(t), int(n))] = (float(j), float(w))
    for n in (128, 256):
        base = orszag_tang.run(n, (0.5, 1.0))
        opt = orszag_tang.run(n, (0.5, 1.0), eq_variant=variant, mag_collision=mag)
        for (t, j0, w0, _, _), (_, j, w, _, _) in zip(base, opt):
            jr, wr = rows[(t, n)]
            print(f"N={n} t={t}: j_max {j:.3f} (default {j0:.3f}, paper {jr}); "
                  f"omega_max {w:.4f} (default {w0:.4f}, paper {wr})")
            assert abs(j / j0 - 1) < 0.02 and abs(w / w0 - 1) < 0.01
            assert abs(j / jr - 1) < 0.04 and abs(w / wr - 1) < 0.02
