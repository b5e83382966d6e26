"""GPU parity of the global diagnostics (mhd_get_totals) against the oracle.

The diagnostics kernel forms every per-node quantity in the compute type of
the storage (FP64 for FP64 storage, FP32 for FP32 and FP16S) and reduces in
FP64.  The oracle evaluates the same definitions in FP64 on the very values
the GPU holds (read back from the device), so for FP64 storage the totals
agree to rounding (1e-12 of the node count for the sums, 1e-11 relative for
the rest).  For FP32 arithmetic the bounds follow from single rounding of
the per-node quantities (relative 2^-24 per operation, a handful of
operations): sums of deviations to a few 1e-9 per node, means of squares
to 1e-6 relative, gradient extrema (where b varies by O(0.05) between
nodes) to 1e-5 relative, and the current density, a non-equilibrium
quantity 20-100 times smaller than the populations it is taken from, to
1e-4 relative; the last two also carry an absolute floor of 2e-8, the
FP32 rounding of the moments (|u|, |b| <= 0.07) carried through the
stencil.  Lattices cover ragged strips and tiles, the per-node
(x-wall) path, widths that are not a multiple of the vector width, y walls,
and both ways of obtaining the pre-collision state: gathered from the
buffer the last step read, or recovered from the stored post-collision
state.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 36, 1 / 9] * 4)
SUMS = ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y")


def _rough_state(orc, p, seed):
    """A non-smooth, non-equilibrium pre-collision state (div b, vorticity
    and the current density all O(1) in lattice units of the gradient)."""
    rng = np.random.default_rng(seed)
    ny, nx = p.ny, p.nx
    ux, uy, bx, by = (rng.uniform(-0.06, 0.06, (ny, nx)) for _ in range(4))
    f, g = orc.init(p, ux, uy, bx, by, rho=rng.uniform(0.95, 1.05, (ny, nx)))
    f = f + rng.normal(0, 3e-4, f.shape) * W9[:, None, None]
    g = g + rng.normal(0, 3e-4, g.shape)
    return f, g


def _check(got, ref, n, fp64):
    for k, v in ref.items():
        if fp64:
            if k in SUMS:
                assert abs(got[k] - v) <= 1e-12 * n, (k, got[k], v)
            else:
                assert abs(got[k] - v) <= 1e-11 * max(abs(v), 1e-6), (k, got[k], v)
            continue
        if k in ("mass", "mom_x", "mom_y"):
            tol = 5e-9 * n
        elif k in ("bsum_x", "bsum_y"):
            tol = 2e-8 * n
        elif k in ("e_kin", "e_mag"):
            tol = 1e-6 * abs(v)
        elif k == "cross_hel":
            tol = 2e-6 * np.sqrt(ref["e_kin"] * ref["e_mag"])
        elif k == "jz_max":
            tol = 1e-4 * abs(v) + 2e-8
        else:  # divb_max, divb_rms, omega_max
            tol = 1e-5 * abs(v) + 2e-8
        assert abs(got[k] - v) <= tol, (k, got[k], v, tol)


def _gather_case(orc, prec, nx, ny, tau=(0.58, 0.62), wall_x=False, wall_y=False, seed=0):
    """Totals of the pre-collision state the last step gathered, against
    the oracle's totals of the stream of the state that step read."""
    from paper_2602_14667_gb300 import Lattice
    p = orc.Params(nx, ny, *tau, wall_x=wall_x, wall_y=wall_y)
    f, g = _rough_state(orc, p, seed)
    fs, gs = orc.collide(p, f, g)
    with Lattice(nx, ny, *tau, precision=prec, wall_x=wall_x, wall_y=wall_y) as lat:
        lat.set_populations(fs, gs)
        P_f, P_g = lat.get_populations()      # what the device holds
        lat.advance(1)
        got = lat.get_totals()
    ref = orc.totals(p, *orc.stream(p, P_f, P_g))
    return got, ref


@pytest.mark.parametrize("wall_y", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "fp16s", "fp64"])
def test_totals_of_the_gathered_state(orc, prec, wall_y):
    """200 x 136: two strips of 128 columns, the second ragged (72), and
    three tiles of up to 62 rows, the last ragged (12)."""
    got, ref = _gather_case(orc, prec, 200, 136, wall_y=wall_y, seed=1)
    _check(got, ref, 200 * 136, prec == "fp64")


@pytest.mark.parametrize("prec", ["fp32", "fp16s", "fp64"])
def test_totals_of_the_stored_state(orc, prec):
    """Right after a restore the pre-collision moments are those of the
    stored post-collision state (collision invariants) and the magnetic
    non-equilibrium is (g* - g_eq) / (1 - omega_m).  The stored state is
    the rounded collision of the oracle's state, so the current density
    carries the storage rounding divided by |1 - omega_m| (0.61 here)."""
    from paper_2602_14667_gb300 import Lattice
    nx, ny, tau = 200, 136, (0.58, 0.62)
    p = orc.Params(nx, ny, *tau)
    f, g = _rough_state(orc, p, 2)
    fs, gs = orc.collide(p, f, g)
    with Lattice(nx, ny, *tau, precision=prec) as lat:
        lat.set_populations(fs, gs)
        got = lat.get_totals()
    ref = orc.totals(p, f, g)
    if prec == "fp16s":
        # half storage: the moments carry 2^-11 of the deviations they are
        # summed from; compare what half rounding leaves
        for k in ("mass", "mom_x", "mom_y"):
            assert abs(got[k] - ref[k]) <= 2e-6 * nx * ny, k
        for k in ("e_kin", "e_mag", "divb_max", "divb_rms", "omega_max"):
            assert abs(got[k] - ref[k]) <= 2e-3 * abs(ref[k]), k
        return
    _check(got, ref, nx * ny, prec == "fp64")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("nx,ny,wall_x,wall_y", [
    (101, 70, False, False),   # width not a multiple of the vector width: one node per lane
    (40, 24, True, False),     # x walls: the per-node path
    (66, 130, True, True),     # walls on both axes, three tiles
    (5, 3, False, False),      # a lattice far smaller than one strip
    (2, 2, False, False),
])
def test_totals_on_narrow_and_walled_lattices(orc, prec, nx, ny, wall_x, wall_y):
    got, ref = _gather_case(orc, prec, nx, ny, wall_x=wall_x, wall_y=wall_y, seed=3)
    _check(got, ref, nx * ny, prec == "fp64")
