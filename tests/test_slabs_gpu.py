"""Row slabs of one lattice on the GPU (bc_y = MHD_HALO, mhd_slab_exchange).

The slabs of a periodic lattice, each advanced by the fused step and
exchanging the crossing populations of their edge rows after every step,
must hold bit for bit the state of the same lattice advanced whole (same
kernel and launch shape: the update of a node does not depend on which
slab holds it).  The totals of the slabs, combined, must match the whole
lattice's (the gradient stencil at a slab's edge rows reads the ghost
rows' moments): the whole lattice gathers the pre-collision state, the
slabs recover it from the stored post-collision one, so they differ by the
storage rounding of the stored populations (FP64 to rounding; the current
density, a non-equilibrium quantity, by that rounding over |1 - omega_m|).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _fields(nx, ny, seed=4):
    import mhd_inputs
    return mhd_inputs.random_spectrum(nx, ny, seed, 0.04, 0.04, kmax=6)


@pytest.mark.parametrize("prec,rows,shape,wall_x", [
    ("fp64", None, (2, 8), False),                      # two equal slabs
    ("fp32", [(0, 40), (40, 64)], (4, 4), False),       # uneven
    ("fp16s", [(0, 2), (2, 33), (33, 64)], (4, 16), False),  # a two-row slab
    ("fp32", [(0, 30), (30, 64)], (1, 8), True),        # x walls (the per-node step)
])
def test_slabs_reproduce_the_whole_lattice_bitwise(prec, rows, shape, wall_x):
    from paper_2602_14667_gb300 import Lattice
    from paper_2602_14667_gb300.slabs import SlabGroup
    nx, ny, steps = 96, 64, 100
    fields = _fields(nx, ny)
    with Lattice(nx, ny, 0.55, 0.6, precision=prec, wall_x=wall_x) as whole, \
            SlabGroup(nx, ny, 2, 0.55, 0.6, precision=prec, rows=rows, wall_x=wall_x) as sg:
        whole.kernel_config = shape
        sg.kernel_config = shape
        whole.set_fields(*fields)
        sg.set_fields(*fields)
        whole.advance(steps)
        sg.advance(steps)
        fw, gw = whole.get_populations()
        fs, gs = sg.get_populations()
        assert np.array_equal(fw, fs) and np.array_equal(gw, gs)
        tw, ts = whole.get_totals(), sg.get_totals()
    n = nx * ny
    # (sums, current density, everything else): storage rounding of the
    # post-collision state the slabs reduce (half storage: 2^-11 of each
    # deviation, which the gradients of the smooth b amplify)
    tol = {"fp64": (1e-12, 1e-10, 1e-11), "fp32": (1e-7, 2e-3, 1e-5), "fp16s": (1e-5, 2e-2, 1e-2)}[prec]
    for k, v in tw.items():
        if k == "step":
            assert ts[k] == v == steps
        elif k in ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y"):
            assert abs(ts[k] - v) <= tol[0] * n, (k, ts[k], v)
        elif k == "jz_max":
            assert abs(ts[k] - v) <= tol[1] * abs(v) + 1e-12, (k, ts[k], v)
        else:
            assert abs(ts[k] - v) <= tol[2] * abs(v) + 1e-15, (k, ts[k], v)


def test_one_slab_is_its_own_neighbour():
    """A single slab exchanging with itself is the periodic lattice."""
    from paper_2602_14667_gb300 import Lattice
    from paper_2602_14667_gb300.slabs import SlabGroup
    nx, ny = 64, 40
    fields = _fields(nx, ny, 9)
    with Lattice(nx, ny, 0.53, 0.57, precision="fp32") as whole, SlabGroup(nx, ny, 1, 0.53, 0.57) as sg:
        whole.kernel_config = (2, 8)
        sg.kernel_config = (2, 8)
        whole.set_fields(*fields)
        sg.set_fields(*fields)
        whole.advance(60)
        sg.advance(60)
        assert all(np.array_equal(a, b) for a, b in zip(whole.get_populations(), sg.get_populations()))


def test_exchange_rejects_mismatched_lattices():
    from paper_2602_14667_gb300 import Lattice, MhdError, _abi
    with Lattice(32, 8, 0.6, 0.6, halo_y=True) as a, Lattice(48, 8, 0.6, 0.6, halo_y=True) as b, \
            Lattice(32, 8, 0.6, 0.6) as c:
        with pytest.raises(MhdError, match="EINVAL"):
            _abi.slab_exchange(a, b)
        with pytest.raises(MhdError, match="EINVAL"):
            _abi.slab_exchange(a, c)
    with pytest.raises(MhdError, match="EINVAL"):
        Lattice(32, 8, 0.6, 0.6, halo_y=True, in_place=True)
