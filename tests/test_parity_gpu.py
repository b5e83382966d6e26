"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (fixed for the method's configurations):
  * FP64 storage: fields within 1e-12 relative L2 after 100 steps of the
    64^2 Orszag-Tang vortex (nu = eta = 0.01); populations element-wise.
  * FP32 storage: populations within 2e-6 max-abs after one step from an
    identical state; rho, u, b within 1e-4 relative L2 after 1000 steps.
  * FP16S storage: one step within the half rounding bound (see
    test_fp16s_one_step); field error after 1000 steps reported and bounded.
Sizes span several thread blocks with ragged tails; every launch shape is
exercised; walls and both equilibrium variants and the BGK switch are
covered.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

OT_TAU = 0.53  # nu = eta = 0.01


def _lat(nx, ny, prec, tau_f=OT_TAU, tau_m=OT_TAU, **kw):
    from paper_2602_14667_gb300 import Lattice
    return Lattice(nx, ny, tau_f, tau_m, precision=prec, **kw)


def _ot(nx, ny=None, amp=0.05):
    import mhd_inputs
    return mhd_inputs.orszag_tang(nx, amp, amp, ny)


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_state(orc, p, fields, steps):
    f, g = orc.init(p, *fields)
    return orc.run(p, f, g, steps)


def _pert_state(orc, p, seed):
    """A random non-equilibrium pre-collision state of the oracle."""
    rng = np.random.default_rng(seed)
    ny, nx = p.ny, p.nx
    ux, uy, bx, by = (rng.uniform(-0.06, 0.06, (ny, nx)) for _ in range(4))
    f, g = orc.init(p, ux, uy, bx, by, rho=rng.uniform(0.95, 1.05, (ny, nx)))
    f = f + rng.normal(0, 3e-4, f.shape) * np.array([4 / 9] + [1 / 36, 1 / 9] * 4)[:, None, None]
    g = g + rng.normal(0, 3e-4, g.shape)
    return f, g


def _gpu_one_step(lat, orc, p, f_pre, g_pre):
    """Load the post-collision state P = collide(pre) into the GPU, run one
    step, return (gpu, oracle) post-collision states of the next step."""
    fs, gs = orc.collide(p, f_pre, g_pre)
    lat.set_populations(fs, gs)
    lat.advance(1)
    fg, gg = lat.get_populations()
    f1, g1 = orc.stream(p, fs, gs)
    fo, go = orc.collide(p, f1, g1)
    return (fg, gg), (fo, go)


# ---------------------------------------------------------------- FP64 -----

@pytest.mark.parametrize("steps,tol", [(100, 1e-12), (1000, 1e-12)])
def test_fp64_orszag_tang_64(orc, steps, tol):
    n = 64
    fields = _ot(n)
    p = orc.Params(n, n, OT_TAU, OT_TAU)
    ref = orc.fields(p, *_oracle_state(orc, p, fields, steps))
    with _lat(n, n, "fp64") as lat:
        lat.set_fields(*fields)
        lat.advance(steps)
        got = lat.get_fields()
    for name, r in zip(("rho", "ux", "uy", "bx", "by"), ref):
        assert _rel_l2(got[name], r) < tol, (name, _rel_l2(got[name], r))


@pytest.mark.parametrize("nx,ny,wx,wy,variant,collision", [
    (64, 64, False, False, 1, 0),
    (37, 29, False, False, 0, 0),    # ragged: V = 1 path, odd sizes
    (96, 40, False, True, 0, 0),     # y walls, vector path
    (30, 34, True, True, 1, 0),      # walls on both axes
    (66, 18, False, False, 0, 1),    # BGK fluid collision
    (2, 2, False, False, 0, 0),      # smallest lattice
])
def test_fp64_populations_elementwise(orc, nx, ny, wx, wy, variant, collision):
    steps = 50
    p = orc.Params(nx, ny, 0.56, 0.71, wall_x=wx, wall_y=wy, eq_variant=variant, collision=collision)
    fields = _ot(nx, ny)
    f, g = _oracle_state(orc, p, fields, steps)
    fo, go = orc.collide(p, f, g)  # GPU buffer holds post-collision populations
    with _lat(nx, ny, "fp64", 0.56, 0.71, wall_x=wx, wall_y=wy, eq_variant=variant,
              collision=collision) as lat:
        lat.set_fields(*fields)
        lat.advance(steps)
        fg, gg = lat.get_populations()
    np.testing.assert_allclose(fg, fo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(gg, go, rtol=0, atol=1e-14)


def _check_totals(got, ref, n):
    """Sums (mass, momentum, sum b) to 1e-12 x nodes absolute; means and
    maxima to 1e-11 relative."""
    for k, v in ref.items():
        if k in ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y"):
            assert abs(got[k] - v) <= 1e-12 * n, (k, got[k], v)
        else:
            assert abs(got[k] - v) <= 1e-11 * max(abs(v), 1e-6), (k, got[k], v)


def test_fp64_totals_match_oracle(orc):
    n = 64
    fields = _ot(n)
    p = orc.Params(n, n, OT_TAU, OT_TAU)
    f, g = _oracle_state(orc, p, fields, 200)
    ref = orc.totals(p, f, g)
    with _lat(n, n, "fp64") as lat:
        lat.set_fields(*fields)
        t0 = lat.get_totals()
        lat.advance(200)
        got = lat.get_totals()
    assert got["step"] == 200 and t0["jz_max"] == 0.0
    _check_totals(got, ref, n * n)


def test_fp64_totals_with_walls(orc):
    nx, ny = 40, 24
    p = orc.Params(nx, ny, 0.6, 0.8, wall_y=True)
    fields = _ot(nx, ny)
    f, g = _oracle_state(orc, p, fields, 30)
    ref = orc.totals(p, f, g)
    with _lat(nx, ny, "fp64", 0.6, 0.8, wall_y=True) as lat:
        lat.set_fields(*fields)
        lat.advance(30)
        got = lat.get_totals()
    _check_totals(got, ref, nx * ny)


@pytest.mark.parametrize("wall_y", [False, True])
def test_fp64_totals_with_many_tiles_per_block(orc, wall_y):
    """The diagnostics grid holds only the resident blocks, each walking
    several 32 x 8 tiles: 1000 x 250 nodes is 1024 tiles (ragged in x and
    y), more than the blocks resident at once."""
    nx, ny = 1000, 250
    p = orc.Params(nx, ny, 0.56, 0.71, wall_y=wall_y)
    fields = _ot(nx, ny)
    f, g = _oracle_state(orc, p, fields, 10)
    ref = orc.totals(p, f, g)
    with _lat(nx, ny, "fp64", 0.56, 0.71, wall_y=wall_y) as lat:
        lat.set_fields(*fields)
        lat.advance(10)
        got = lat.get_totals()
    _check_totals(got, ref, nx * ny)


def test_totals_after_restore_use_the_stored_state(orc):
    """Right after mhd_set_populations the pre-collision g is recovered from
    the stored post-collision one, (g* - g_eq)/(1 - omega_m)."""
    n = 48
    p = orc.Params(n, n, 0.6, 0.8)
    f, g = _oracle_state(orc, p, _ot(n), 40)
    ref = orc.totals(p, f, g)
    fs, gs = orc.collide(p, f, g)
    with _lat(n, n, "fp64", 0.6, 0.8) as lat:
        lat.set_populations(fs, gs)
        got = lat.get_totals()
    _check_totals(got, ref, n * n)


# ---------------------------------------------------------------- FP32 -----

SHAPES_FP32 = [(1, 1), (1, 8), (2, 2), (2, 16), (4, 1), (4, 4), (4, 16)]


@pytest.mark.parametrize("shape", SHAPES_FP32)
@pytest.mark.parametrize("nx,ny,wy", [(256, 24, False), (136, 20, True), (4, 6, False)])
def test_fp32_one_step_populations(orc, shape, nx, ny, wy):
    V, BY = shape
    if nx % V:
        pytest.skip("nodes_per_thread must divide nx")
    p = orc.Params(nx, ny, 0.5 + 3e-4, 0.51, wall_y=wy)
    f_pre, g_pre = _pert_state(orc, p, seed=nx + ny)
    with _lat(nx, ny, "fp32", 0.5 + 3e-4, 0.51, wall_y=wy) as lat:
        lat.kernel_config = (V, BY)
        (fg, gg), (fo, go) = _gpu_one_step(lat, orc, p, f_pre, g_pre)
    assert np.abs(fg - fo).max() < 2e-6
    assert np.abs(gg - go).max() < 2e-6


def test_fp32_orszag_tang_1000_steps(orc):
    n = 64
    fields = _ot(n)
    p = orc.Params(n, n, OT_TAU, OT_TAU)
    ref = orc.fields(p, *_oracle_state(orc, p, fields, 1000))
    with _lat(n, n, "fp32") as lat:
        lat.set_fields(*fields)
        lat.advance(1000)
        got = lat.get_fields()
    for name, r in zip(("rho", "ux", "uy", "bx", "by"), ref):
        assert _rel_l2(got[name], r) < 1e-4, (name, _rel_l2(got[name], r))


def test_fp32_walls_x_and_y_one_step(orc):
    nx, ny = 33, 17
    p = orc.Params(nx, ny, 0.7, 0.9, wall_x=True, wall_y=True, eq_variant=1)
    f_pre, g_pre = _pert_state(orc, p, seed=5)
    with _lat(nx, ny, "fp32", 0.7, 0.9, wall_x=True, wall_y=True, eq_variant=1) as lat:
        (fg, gg), (fo, go) = _gpu_one_step(lat, orc, p, f_pre, g_pre)
    assert np.abs(fg - fo).max() < 2e-6 and np.abs(gg - go).max() < 2e-6


# --------------------------------------------------------------- FP16S -----

def test_fp16s_one_step(orc):
    """Stored values are 2^12 x (deviation) rounded to IEEE half: relative
    error <= 2^-11 each.  One step reads rounded inputs (the collision is a
    contraction with |1 - omega| <= 1 on the non-equilibrium part and
    reproduces the equilibrium part to first order) and rounds its output
    once more, so each output lies within a few half ulps of the largest
    deviation: bound 4 x 2^-11 x max|deviation|."""
    nx, ny = 128, 16
    p = orc.Params(nx, ny, 0.5 + 3e-4, 0.51)
    f_pre, g_pre = _pert_state(orc, p, seed=9)
    w = np.array([4 / 9] + [1 / 36, 1 / 9] * 4)[:, None, None]
    with _lat(nx, ny, "fp16s", 0.5 + 3e-4, 0.51) as lat:
        (fg, gg), (fo, go) = _gpu_one_step(lat, orc, p, f_pre, g_pre)
    dmax = max(np.abs(fo - w).max(), np.abs(go).max())
    bound = 4 * 2.0 ** -11 * dmax
    assert np.abs(fg - fo).max() < bound and np.abs(gg - go).max() < bound


def test_fp16s_orszag_tang_field_error(orc):
    n = 64
    fields = _ot(n)
    p = orc.Params(n, n, OT_TAU, OT_TAU)
    ref = orc.fields(p, *_oracle_state(orc, p, fields, 1000))
    with _lat(n, n, "fp16s") as lat:
        lat.set_fields(*fields)
        lat.advance(1000)
        got = lat.get_fields()
    errs = {name: _rel_l2(got[name], r) for name, r in zip(("ux", "uy", "bx", "by"), ref[1:])}
    print("fp16s 64^2 OT rel L2 after 1000 steps:", errs)
    assert max(errs.values()) < 2e-2


# -------------------------------------------------- state handling / API -----

def test_graph_and_single_launches_agree():
    n = 96
    fields = _ot(n)
    with _lat(n, n, "fp32") as a, _lat(n, n, "fp32") as b:
        a.set_fields(*fields); b.set_fields(*fields)
        a.advance(128)          # two captured 64-step graphs
        for _ in range(128):
            b.advance(1)        # single launches
        fa, ga = a.get_populations(); fb, gb = b.get_populations()
    np.testing.assert_array_equal(fa, fb)
    np.testing.assert_array_equal(ga, gb)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
def test_fp32_field_calls_match_the_fp64_ones(prec):
    """mhd_set_fields_f32 sets, bit for bit, the state mhd_set_fields sets for
    the same values held as double; mhd_get_fields_f32 returns the FP64
    fields of mhd_get_fields rounded to float, element by element; both
    reject what the FP64 calls reject (non-finite fields, rho <= 0)."""
    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice, MhdError
    nx, ny = 96, 40
    u = [a.astype(np.float32) for a in mhd_inputs.random_spectrum(nx, ny, 5, 0.04, 0.04, kmax=6)]
    rho = (1.0 + 0.25 * u[0]).astype(np.float32)
    with Lattice(nx, ny, 0.55, 0.6, precision=prec) as a, Lattice(nx, ny, 0.55, 0.6, precision=prec) as b:
        a.set_fields(*u, rho=rho)
        b.set_fields(*[v.astype(np.float64) for v in u], rho=rho.astype(np.float64))
        assert np.array_equal(a.get_state(), b.get_state())
        a.set_fields(*u)
        b.set_fields(*[v.astype(np.float64) for v in u])
        assert np.array_equal(a.get_state(), b.get_state())
        a.advance(7)
        f64 = a.get_fields()
        f32 = a.get_fields(dtype=np.float32)
        for k, v in f64.items():
            assert f32[k].dtype == np.float32 and np.array_equal(f32[k], v.astype(np.float32)), k
        bad = u[2].copy()
        bad[3, 5] = np.inf
        with pytest.raises(MhdError, match="EINVAL"):
            a.set_fields(u[0], u[1], bad, u[3])
        with pytest.raises(MhdError, match="EINVAL"):
            a.set_fields(*u, rho=np.zeros_like(rho))
        assert np.array_equal(a.get_fields(dtype=np.float32)["ux"], f32["ux"])  # state untouched


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
def test_pinned_host_fields_are_read_and_written_in_place(prec):
    """Pinned host arrays take the in-place path (the initial-equilibrium
    kernel reads them over the host link, checks them and writes the spare
    buffer; the fields kernel writes its output into them), pageable arrays
    and in-place lattices the staging copy: the same state bit for bit and
    the same fields, in float64 and float32.  A non-finite pinned input is
    rejected with the state untouched, and the totals that follow are those
    of that state (the spare buffer no longer holds the last step's input)."""
    import torch

    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice, MhdError
    nx, ny = 96, 40
    fields = list(mhd_inputs.random_spectrum(nx, ny, 5, 0.04, 0.04, kmax=6))
    fields.append(1.0 + 0.25 * fields[0])
    for tdt, ndt in ((torch.float64, np.float64), (torch.float32, np.float32)):
        pin = [torch.empty((ny, nx), dtype=tdt).pin_memory() for _ in range(10)]
        hp = [t.numpy() for t in pin]
        for h, a in zip(hp, fields):
            h[:] = a
        hq = [np.ascontiguousarray(a, dtype=ndt) for a in fields]
        with Lattice(nx, ny, 0.55, 0.6, precision=prec) as a, Lattice(nx, ny, 0.55, 0.6, precision=prec) as b, \
                Lattice(nx, ny, 0.55, 0.6, precision=prec, in_place=True) as c:
            a.set_fields(*hp[:4], rho=hp[4])
            b.set_fields(*hq[:4], rho=hq[4])
            c.set_fields(*hp[:4], rho=hp[4])
            assert np.array_equal(a.get_state(), b.get_state()) and np.array_equal(a.get_state(), c.get_state())
            a.advance(5)
            b.advance(5)
            fa = a.get_fields(out=hp[5:10])
            fb = b.get_fields(dtype=ndt)
            for k in fa:
                assert np.array_equal(fa[k], fb[k]), k
            s0 = a.get_state()
            hp[2][3, 5] = np.nan
            with pytest.raises(MhdError, match="EINVAL"):
                a.set_fields(*hp[:4], rho=hp[4])
            assert np.array_equal(a.get_state(), s0)
            b.set_state(s0)  # the stored state alone, as a holds it now
            assert a.get_totals() == b.get_totals()
        del hp, pin


def test_checkpoint_restart_is_bitwise():
    n = 64
    fields = _ot(n)
    for prec in ("fp32", "fp16s", "fp64"):
        with _lat(n, n, prec) as a, _lat(n, n, prec) as b, _lat(n, n, prec) as c:
            a.set_fields(*fields)
            a.advance(37)
            b.set_state(a.get_state())              # raw planes: bitwise for every precision
            if prec != "fp64":
                c.set_populations(*a.get_populations())  # FP64 view: exact for fp32 / fp16s
            else:
                c.set_state(a.get_state())
            a.advance(70); b.advance(70); c.advance(70)
            sa, sb, sc = a.get_state(), b.get_state(), c.get_state()
        np.testing.assert_array_equal(sa, sb)
        np.testing.assert_array_equal(sa, sc)


def test_fp64_population_view_round_trip_within_an_ulp():
    n = 32
    with _lat(n, n, "fp64") as a:
        a.set_fields(*_ot(n))
        a.advance(5)
        f, g = a.get_populations()
        a.set_populations(f, g)
        f2, g2 = a.get_populations()
    np.testing.assert_allclose(f2, f, rtol=3e-16, atol=0)
    np.testing.assert_array_equal(g2, g)


def test_autotune_keeps_state_and_returns_valid_shape(tmp_path, monkeypatch):
    monkeypatch.setenv("MHD_TUNE_CACHE", str(tmp_path / "tune.json"))
    n = 128
    fields = _ot(n)
    with _lat(n, n, "fp32") as a:
        a.set_fields(*fields)
        a.advance(10)
        before = a.get_populations()
        shape = a.autotune()
        assert shape[:2] in [(v, by) for v in (1, 2, 4) for by in (1, 2, 4, 8, 16)]
        assert shape[2] == 0 or 1 <= shape[2] <= 64
        after = a.get_populations()
        np.testing.assert_array_equal(before[0], after[0])
        assert a.kernel_config == shape
    assert (tmp_path / "tune.json").exists()
    with _lat(n, n, "fp32") as b:       # a new lattice picks the cached shape
        assert b.kernel_config == shape
    # an entry of two numbers (shape without a depth) reads as depth 0
    text = (tmp_path / "tune.json").read_text()
    key = [ln for ln in text.splitlines() if "128x128" in ln][0].split('"')[1]
    (tmp_path / "tune.json").write_text('{\n  "%s": [2, 8]\n}\n' % key)
    with _lat(n, n, "fp32") as c:
        assert c.kernel_config == (2, 8, 0)


@pytest.mark.parametrize("prec,in_place", [("fp32", False), ("fp16s", False), ("fp32", True)])
def test_staging_depth_changes_no_bits(prec, in_place):
    """The staging depth (resident warps per SM of the persistent grid) only
    changes how many row tiles are in flight: every depth gives the state of
    the built-in one bit for bit; depths outside 0..64 are rejected."""
    from paper_2602_14667_gb300 import MhdError
    import mhd_inputs
    nx, ny = 264, 40
    fields = mhd_inputs.random_spectrum(nx, ny, 3, 0.04, 0.04, kmax=6)
    states = []
    for W in (0, 1, 4, 16, 64):
        with _lat(nx, ny, prec, in_place=in_place) as lat:
            lat.kernel_config = (4, 1, W)
            assert lat.kernel_config == (4, 1, W)
            lat.set_fields(*fields)
            lat.advance(70)  # one 64-step graph and single steps
            states.append(lat.get_state())
    assert all(np.array_equal(st, states[0]) for st in states[1:])
    with _lat(nx, ny, prec, in_place=in_place) as lat:
        for W in (-1, 65):
            with pytest.raises(MhdError, match="EINVAL"):
                lat.kernel_config = (4, 1, W)


def test_batch_staging_depth_changes_no_bits():
    import mhd_inputs
    from paper_2602_14667_gb300 import Batch
    sizes = [(64, 64), (96, 48), (128, 128)]
    taus = [(0.53, 0.56), (0.6, 0.52), (0.55, 0.55)]
    out = []
    for W in (0, 4, 32):
        with Batch(sizes, taus) as b:
            b.kernel_config = (2, 4, W)
            for i, (nx, ny) in enumerate(sizes):
                b.set_fields(i, *mhd_inputs.random_spectrum(nx, ny, 10 + i, 0.03, 0.03))
            b.advance(40)
            out.append([b.get_fields(i)["ux"] for i in range(len(sizes))])
    for o in out[1:]:
        assert all(np.array_equal(x, y) for x, y in zip(o, out[0]))


def test_conservation_over_many_steps():
    n = 256
    fields = _ot(n, amp=0.04)
    with _lat(n, n, "fp32", 0.50006, 0.50006) as lat:
        lat.set_fields(*fields)
        t0 = lat.get_totals()
        lat.advance(500)
        t1 = lat.get_totals()
    assert abs(t1["mass"] - t0["mass"]) < 1e-6 * t0["mass"]
    assert abs(t1["mom_x"] - t0["mom_x"]) < 1e-6 * t0["mass"]
    assert abs(t1["bsum_x"] - t0["bsum_x"]) < 1e-6 * n * n * 0.04
    assert abs(t1["e_kin"] + t1["e_mag"] - t0["e_kin"] - t0["e_mag"]) < 0.01 * (t0["e_kin"] + t0["e_mag"])


def test_errors_are_reported():
    from paper_2602_14667_gb300 import Lattice, MhdError, _abi
    with pytest.raises(MhdError, match="EINVAL"):
        Lattice(16, 16, 0.5, 0.6)
    with pytest.raises(MhdError, match="EINVAL"):
        Lattice(1, 16, 0.6, 0.6)
    with pytest.raises(MhdError, match="EINVAL"):
        Lattice(65536, 65536, 0.6, 0.6)                # nx*ny > 2^31
    with pytest.raises(MhdError, match="ENOMEM"):
        Lattice(46000, 46000, 0.6, 0.6, precision="fp64")  # ~640 GB: refused by cudaMalloc
    with _lat(8, 8, "fp32") as lat:
        with pytest.raises(MhdError, match="ESTATE"):
            lat.advance(1)
        z = np.zeros((8, 8))
        bad = z.copy(); bad[2, 3] = np.nan
        with pytest.raises(MhdError, match="EINVAL"):
            lat.set_fields(bad, z, z, z)
        with pytest.raises(MhdError, match="ESTATE"):   # a rejected set leaves no fields
            lat.advance(1)
        lat.set_fields(z + 0.01, z, z, z)
        lat.advance(3)
        before = lat.get_state()
        for rho in (z, z + np.inf, np.where(bad == bad, 1.0, np.nan)):
            with pytest.raises(MhdError, match="EINVAL"):
                lat.set_fields(z, z, z, z, rho=rho)
        assert np.array_equal(lat.get_state(), before)  # ... and leaves the state alone
        with pytest.raises(MhdError, match="EINVAL"):
            lat.kernel_config = (3, 4)
        with pytest.raises(MhdError, match="EINVAL"):
            lat.advance(-1)


def test_blow_up_is_reported_as_unstable(orc):
    """Random fields of amplitude 0.1 at tau = 0.5001 are beyond the scheme's
    stability limit: the oracle itself overflows within 250 steps.  On the GPU
    the run goes non-finite too and the totals report MHD_EUNSTABLE (NaN /
    Inf arithmetic only, no device fault)."""
    from paper_2602_14667_gb300 import MhdError
    n = 16
    rng = np.random.default_rng(3)
    fields = [rng.uniform(-0.1, 0.1, (n, n)) for _ in range(4)]
    p = orc.Params(n, n, 0.5001, 0.5001)
    f, g = orc.run(p, *orc.init(p, *fields), 1000)
    assert not np.isfinite(f).all()
    for prec in ("fp32", "fp64", "fp16s"):
        with _lat(n, n, prec, 0.5001, 0.5001) as lat:
            lat.set_fields(*fields)
            lat.advance(1000)
            with pytest.raises(MhdError, match="EUNSTABLE"):
                lat.get_totals()
