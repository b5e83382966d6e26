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


@pytest.mark.parametrize("prec,nslabs", [("fp32", 2), ("fp16s", 3), ("fp64", 2), ("fp32", 1), ("fp32", 4)])
def test_slab_group_matches_stepwise_slabs_and_the_whole_lattice(prec, nslabs):
    """mhd_slab_group_advance (every round's exchanges in one kernel, runs of
    64 rounds in a CUDA graph) gives the bits of the slabs stepped one by one
    with one exchange call per boundary, and of the whole lattice: over 130
    steps (two graphs and two single rounds), again after a change of launch
    shape (the group's graphs are captured anew), and the step counters
    advance as for single slabs."""
    from paper_2602_14667_gb300 import Lattice
    from paper_2602_14667_gb300.slabs import SlabGroup
    nx, ny = 96, 64
    fields = _fields(nx, ny, 6)
    with Lattice(nx, ny, 0.55, 0.6, precision=prec) as whole, \
            SlabGroup(nx, ny, nslabs, 0.55, 0.6, precision=prec) as a, \
            SlabGroup(nx, ny, nslabs, 0.55, 0.6, precision=prec) as b:
        for lat in (whole, a, b):
            lat.kernel_config = (2, 4)
            lat.set_fields(*fields)
        whole.advance(130)
        a.advance(130)
        b.advance(130, stepwise=True)
        pw, pa, pb = whole.get_populations(), a.get_populations(), b.get_populations()
        assert all(np.array_equal(x, y) for x, y in zip(pa, pb)) and all(np.array_equal(x, y) for x, y in zip(pa, pw))
        for lat in (whole, a):
            lat.kernel_config = (1, 8)
        whole.advance(65)
        a.advance(65)
        assert all(np.array_equal(x, y) for x, y in zip(a.get_populations(), whole.get_populations()))
        assert all(s.get_totals()["step"] == 195 for s in a.slabs)


def test_slab_group_rejects_what_it_cannot_step():
    import torch

    from paper_2602_14667_gb300 import Lattice, MhdError, _abi
    nx = 32
    s1 = torch.cuda.Stream()
    with Lattice(nx, 8, 0.6, 0.6, halo_y=True) as a, Lattice(nx, 8, 0.6, 0.6, halo_y=True) as b, \
            Lattice(nx, 8, 0.6, 0.6) as c, Lattice(48, 8, 0.6, 0.6, halo_y=True) as d, \
            Lattice(nx, 8, 0.6, 0.6, halo_y=True, stream=s1.cuda_stream) as e:
        for bad in ([a, c], [a, d], [a, e]):
            with pytest.raises(MhdError, match="EINVAL"):
                _abi.SlabSteps(bad)
        g = _abi.SlabSteps([a, b])
        try:
            with pytest.raises(MhdError, match="ESTATE"):  # no fields yet
                g.advance(1)
            f = _fields(nx, 16, 2)
            a.set_fields(*(np.ascontiguousarray(x[:8]) for x in f))
            b.set_fields(*(np.ascontiguousarray(x[8:]) for x in f))
            a.advance(1)  # one slab a step ahead
            with pytest.raises(MhdError, match="ESTATE"):
                g.advance(1)
            b.advance(1)
            g.advance(3)
            assert a.get_totals()["step"] == b.get_totals()["step"] == 4
        finally:
            g.close()
