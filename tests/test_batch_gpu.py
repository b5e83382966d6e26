"""GPU parity of the batched persistent ensemble kernel.

Each lattice of a batch must be bitwise identical to the same lattice
advanced alone through the single-lattice path with the same launch shape
(the per-node arithmetic is shared), and within the FP32 tolerance of the
FP64 oracle.  Sizes are uneven (several tiles, partial warps for widths
below 32 x nodes_per_thread) and each lattice has its own nu and eta.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIZES = [(64, 64), (96, 32), (32, 40), (128, 96), (64, 128)]
TAUS = [(0.53, 0.56), (0.6, 0.52), (0.51, 0.7), (0.55, 0.55), (0.8, 0.9)]


def _fields(i, nx, ny):
    import mhd_inputs
    return mhd_inputs.random_spectrum(nx, ny, seed=1000 + i, rms_u=0.02, rms_b=0.02)


@pytest.mark.parametrize("shape", [(1, 4), (2, 8), (4, 2), (4, 16)])
def test_batch_equals_single_lattices_bitwise(shape):
    from paper_2602_14667_gb300 import Batch, Lattice
    steps = 150
    with Batch(SIZES, TAUS) as b:
        b.kernel_config = shape
        for i, (nx, ny) in enumerate(SIZES):
            b.set_fields(i, *_fields(i, nx, ny))
        b.advance(steps)
        got = [b.get_fields(i) for i in range(len(SIZES))]
    for i, (nx, ny) in enumerate(SIZES):
        with Lattice(nx, ny, *TAUS[i], precision="fp32") as lat:
            lat.kernel_config = shape
            lat.set_fields(*_fields(i, nx, ny))
            lat.advance(steps)
            ref = lat.get_fields()
        for k in ("rho", "ux", "uy", "bx", "by"):
            np.testing.assert_array_equal(got[i][k], ref[k], err_msg=f"lattice {i} {k}")


def test_batch_matches_oracle(orc):
    from paper_2602_14667_gb300 import Batch
    steps = 200
    with Batch(SIZES, TAUS) as b:
        for i, (nx, ny) in enumerate(SIZES):
            b.set_fields(i, *_fields(i, nx, ny))
        b.advance(steps)
        for i, (nx, ny) in enumerate(SIZES):
            p = orc.Params(nx, ny, *TAUS[i])
            f, g = orc.run(p, *orc.init(p, *_fields(i, nx, ny)), steps)
            ref = orc.fields(p, f, g)
            got = b.get_fields(i)
            for k, r in zip(("ux", "uy", "bx", "by"), ref[1:]):
                err = np.linalg.norm(got[k] - r) / np.linalg.norm(r)
                assert err < 1e-4, (i, k, err)
            tot = b.get_totals(i)
            otot = orc.totals(p, f, g)
            assert abs(tot["mass"] - otot["mass"]) < 1e-5 * nx * ny
            assert abs(tot["e_kin"] - otot["e_kin"]) < 1e-4 * otot["e_kin"]
            assert abs(tot["jz_max"] - otot["jz_max"]) < 1e-3 * otot["jz_max"]


def test_batch_autotune_keeps_state():
    from paper_2602_14667_gb300 import Batch
    with Batch(SIZES, TAUS) as b:
        for i, (nx, ny) in enumerate(SIZES):
            b.set_fields(i, *_fields(i, nx, ny))
        b.advance(10)
        before = [b.get_fields(i)["ux"] for i in range(len(SIZES))]
        shape = b.autotune()
        assert shape == b.kernel_config
        after = [b.get_fields(i)["ux"] for i in range(len(SIZES))]
        for x, y in zip(before, after):
            np.testing.assert_array_equal(x, y)
        assert b.nodes == sum(nx * ny for nx, ny in SIZES)


def test_batch_errors():
    from paper_2602_14667_gb300 import Batch, MhdError
    with pytest.raises(MhdError, match="EINVAL"):
        Batch([(64, 64)], [(0.5, 0.6)])
    with Batch([(64, 64), (32, 32)], [(0.6, 0.6), (0.6, 0.6)]) as b:
        z = np.zeros((64, 64))
        b.set_fields(0, z, z, z, z)
        with pytest.raises(MhdError, match="ESTATE"):
            b.advance(1)            # lattice 1 has no fields yet
        from paper_2602_14667_gb300 import _abi
        assert _abi.lib().mhd_batch_get_fields(b.handle, 2, None, None, None, None, None) == _abi.MHD_EINVAL
        with pytest.raises(MhdError, match="EINVAL"):
            b.kernel_config = (3, 4)


def test_all_totals_equal_the_per_lattice_totals():
    """mhd_batch_get_all_totals (one launch over every lattice's tiles)
    against mhd_batch_get_totals of each index: the per-node quantities are
    the same arithmetic, so the maxima and the gradient-node count agree
    exactly and the sums to their summation order; after 30 steps (the
    gathered state) and right after the fields are set (the stored
    equilibrium); unset lattices are refused."""
    from paper_2602_14667_gb300 import Batch, MhdError
    with Batch(SIZES, TAUS) as b:
        with pytest.raises(MhdError, match="ESTATE"):
            b.get_all_totals()
        for i, (nx, ny) in enumerate(SIZES):
            b.set_fields(i, *_fields(i, nx, ny))
        for steps in (0, 30):
            b.advance(steps)
            every = b.get_all_totals()
            assert len(every) == len(SIZES)
            arrays = b.get_all_totals(as_arrays=True)
            for k, col in arrays.items():
                assert [e[k] for e in every] == list(col), k
            for i, (nx, ny) in enumerate(SIZES):
                one = b.get_totals(i)
                assert every[i]["step"] == one["step"]
                for k in ("divb_max", "jz_max", "omega_max"):
                    assert every[i][k] == one[k], (i, k)
                for k in ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y"):
                    assert abs(every[i][k] - one[k]) <= 1e-12 * nx * ny, (i, k)
                for k in ("e_kin", "e_mag", "cross_hel", "divb_rms"):
                    assert abs(every[i][k] - one[k]) <= 1e-12 * abs(one[k]) + 1e-300, (i, k)


@pytest.mark.parametrize("shape", [(1, 4), (2, 2), (4, 16)])
def test_sample_step_of_the_ensemble(shape):
    """mhd_batch_advance_totals: the fields after it (and after 5 more plain
    steps) equal the plain batch's bit for bit, and its point totals are
    those of mhd_batch_get_all_totals of the same gathered state up to the
    order of the sums (the maximum of |j_z| to the same bound)."""
    import math
    from paper_2602_14667_gb300 import Batch
    runs = []
    for fused in (False, True):
        with Batch(SIZES, TAUS) as b:
            b.kernel_config = shape
            for i, (nx, ny) in enumerate(SIZES):
                b.set_fields(i, *_fields(i, nx, ny))
            if fused:
                pt = b.advance_totals(13)
            else:
                b.advance(13)
                pt = None
            ref = b.get_all_totals()
            f13 = [b.get_fields(i) for i in range(len(SIZES))]
            b.advance(5)
            f18 = [b.get_fields(i) for i in range(len(SIZES))]
            runs.append((pt, ref, f13, f18))
    for i in range(len(SIZES)):
        for k in ("rho", "ux", "uy", "bx", "by"):
            assert np.array_equal(runs[0][2][i][k], runs[1][2][i][k]), (i, k)
            assert np.array_equal(runs[0][3][i][k], runs[1][3][i][k]), (i, k)
    pt, ref = runs[1][0], runs[1][1]
    for i, (nx, ny) in enumerate(SIZES):
        assert pt[i]["step"] == ref[i]["step"] == 13
        assert all(math.isnan(pt[i][k]) for k in ("divb_max", "divb_rms", "omega_max"))
        for k in ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y"):
            assert abs(pt[i][k] - ref[i][k]) <= 5e-9 * nx * ny, (i, k)
        for k in ("e_kin", "e_mag", "cross_hel", "jz_max"):
            assert abs(pt[i][k] - ref[i][k]) <= 1e-6 * abs(ref[i][k]), (i, k)
