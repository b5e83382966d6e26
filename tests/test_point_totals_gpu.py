"""The fused sample step (mhd_advance_totals) against the plain step, the
diagnostics pass and the oracle.

The step that reduces the point totals writes the populations of the plain
step bit for bit; its totals (mass, momentum, energies, cross helicity,
sum b, max |j_z|) are those of the diagnostics pass on the same gathered
state up to the summation order (the per-node quantities are the same
arithmetic: the sums and the maximum of |j_z| agree to the rounding of
the reduction), and the oracle's within the bounds of
the diagnostics tests.  Lattices the fused step does not cover (x walls, in
place, ghost rows) take the diagnostics pass and fill every field.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

POINT = ("mass", "mom_x", "mom_y", "e_kin", "e_mag", "cross_hel", "bsum_x", "bsum_y", "jz_max")
GRAD = ("divb_max", "divb_rms", "omega_max")


def _fields(nx, ny, seed):
    import mhd_inputs
    return mhd_inputs.random_spectrum(nx, ny, seed, 0.03, 0.03)


def _same_order_bounds(a, b, n, fp64):
    """Totals of one state reduced in two orders."""
    for k in POINT:
        if k in ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y"):
            tol = (1e-12 if fp64 else 5e-9) * n
            assert abs(a[k] - b[k]) <= tol, (k, a[k], b[k])
        else:
            tol = (1e-12 if fp64 else 1e-6) * abs(b[k])
            assert abs(a[k] - b[k]) <= tol, (k, a[k], b[k])


@pytest.mark.parametrize("wall_y", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
def test_fused_step_writes_the_plain_steps_populations(prec, wall_y):
    """264 x 40 (a ragged last warp of the vector rows), 37 steps one way or
    the other, then 5 plain steps on both: the states are bitwise equal."""
    from paper_2602_14667_gb300 import Lattice
    nx, ny = 264, 40
    f0 = _fields(nx, ny, 3)
    states = []
    for fused in (False, True):
        with Lattice(nx, ny, 0.53, 0.56, precision=prec, wall_y=wall_y) as lat:
            lat.set_fields(*f0)
            if fused:
                t = lat.advance_totals(37)
                assert t["step"] == 37 and all(math.isnan(t[k]) for k in GRAD)
            else:
                lat.advance(37)
            a = lat.get_state()
            lat.advance(5)
            states.append((a, lat.get_state()))
    assert np.array_equal(states[0][0], states[1][0]) and np.array_equal(states[0][1], states[1][1])


@pytest.mark.parametrize("shape", [None, (1, 4), (2, 16), (4, 1)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
def test_point_totals_match_the_diagnostics_pass(prec, shape):
    """The fused step's totals against mhd_get_totals of the state it
    gathered (read right after it), for the launch shapes the step takes
    (rows per block above 8 are split into blocks of 8)."""
    from paper_2602_14667_gb300 import Lattice
    nx, ny = 200, 136
    if prec == "fp64" and shape is not None:  # FP64: at most 2 nodes per lane, 8 rows per block
        shape = (min(shape[0], 2), min(shape[1], 8))
    with Lattice(nx, ny, 0.58, 0.62, precision=prec) as lat:
        if shape is not None:
            lat.kernel_config = shape
        lat.set_fields(*_fields(nx, ny, 5))
        lat.advance(20)
        fused = lat.advance_totals(3)
        ref = lat.get_totals()
    assert fused["step"] == ref["step"] == 23
    _same_order_bounds(fused, ref, nx * ny, prec == "fp64")


@pytest.mark.parametrize("wall_y", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
def test_point_totals_against_oracle(orc, prec, wall_y):
    """A rough non-equilibrium state set as populations, one fused step: its
    totals against the oracle's totals of the stream of the state it read
    (the bounds of the diagnostics tests)."""
    from test_diag_gpu import _check, _rough_state
    from paper_2602_14667_gb300 import Lattice
    nx, ny, tau = 200, 136, (0.58, 0.62)
    p = orc.Params(nx, ny, *tau, wall_y=wall_y)
    f, g = _rough_state(orc, p, 7)
    fs, gs = orc.collide(p, f, g)
    with Lattice(nx, ny, *tau, precision=prec, wall_y=wall_y) as lat:
        lat.set_populations(fs, gs)
        P_f, P_g = lat.get_populations()  # what the device holds
        got = lat.advance_totals(1)
    ref = orc.totals(p, *orc.stream(p, P_f, P_g))
    _check({k: got[k] for k in POINT}, {k: ref[k] for k in POINT}, nx * ny, prec == "fp64")


@pytest.mark.parametrize("kind", ["wall_x", "in_place"])
def test_lattices_without_the_fused_step_get_every_total(kind):
    """x walls and in-place streaming: the call is mhd_advance followed by
    mhd_get_totals (every field, div b and vorticity included)."""
    from paper_2602_14667_gb300 import Lattice
    nx, ny = 96, 64
    kw = {"wall_x": True} if kind == "wall_x" else {"in_place": True}
    f0 = _fields(nx, ny, 9)
    with Lattice(nx, ny, 0.55, 0.6, precision="fp32", **kw) as a, \
            Lattice(nx, ny, 0.55, 0.6, precision="fp32", **kw) as b:
        a.set_fields(*f0)
        b.set_fields(*f0)
        ta = a.advance_totals(11)
        b.advance(11)
        tb = b.get_totals()
    for k in POINT + GRAD:
        assert math.isfinite(ta[k]) and ta[k] == tb[k], (k, ta[k], tb[k])


def test_fused_step_rejects_what_it_cannot_run():
    from paper_2602_14667_gb300 import Lattice
    with Lattice(64, 32, 0.6, 0.6, precision="fp32") as lat:
        with pytest.raises(Exception):
            lat.advance_totals(1)  # no fields yet
        lat.set_fields(*_fields(64, 32, 1))
        with pytest.raises(Exception):
            lat.advance_totals(0)
        assert lat.advance_totals(1)["step"] == 1


@pytest.mark.parametrize("prec,code", [("fp32", 1), ("fp16s", 2)])
def test_point_totals_at_the_bench_shape_4096(prec, code):
    """The timed 4096^2 workload in its benchmark launch shape: the fused
    sample step writes the plain step's populations and its totals are the
    diagnostics pass's."""
    import mhd_inputs
    from test_fullsize_gpu import _bench_shape
    from paper_2602_14667_gb300 import Lattice
    n, tau = 4096, 0.50006
    f0 = mhd_inputs.orszag_tang(n, 0.04, 0.04)
    out = []
    for fused in (False, True):
        with Lattice(n, n, tau, tau, precision=prec) as lat:
            lat.kernel_config = _bench_shape(code, n)
            lat.set_fields(*f0)
            lat.advance(20)
            t = lat.advance_totals(4) if fused else (lat.advance(4), None)[1]
            out.append((lat.get_state(), t, lat.get_totals()))
    assert np.array_equal(out[0][0], out[1][0])
    _same_order_bounds(out[1][1], out[1][2], n * n, False)
