"""A lattice whose state has more than 2^31 elements.

12000 x 12000 nodes: 19 planes of 12000 x 12032 (padded pitch) elements is
2.7e9 elements per buffer, so every plane offset past the first few planes
needs 64-bit index arithmetic in the step, the initialisation, the state
image and the diagnostics.  One step is checked on sampled nodes against
the oracle's node collision (the pre-step state is read back and pulled on
the host), for FP16S with two buffers and for FP32 in place; the nodes
include the last, ragged warp of every sampled row and the first and last
rows.  The totals must be finite and conserve mass.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = 12000
CX = np.array([0, -1, -1, -1, 0, 1, 1, 1, 0])
CY = np.array([0, 1, 0, -1, -1, -1, 0, 1, 1])
EX = np.array([0, -1, 0, 1, 0])
EY = np.array([0, 0, -1, 0, 1])
W9 = np.array([4 / 9] + [1 / 36, 1 / 9] * 4)


def _planes(img, prec):
    """The state image (plane after plane, packed) as FP64 populations:
    f (9, ny, nx) with the w_i rho0 shift put back, g (10, ny, nx)."""
    dt = np.float16 if prec == "fp16s" else np.float32
    a = img.view(dt).reshape(19, N, N)
    scale = 1.0 / 4096.0 if prec == "fp16s" else 1.0
    return a, scale


def _node_pre(a, scale, x, y):
    f = np.array([float(a[i, (y - CY[i]) % N, (x - CX[i]) % N]) * scale + W9[i] for i in range(9)])
    g = np.array([[float(a[9 + 2 * j + c, (y - EY[j]) % N, (x - EX[j]) % N]) * scale for c in range(2)]
                  for j in range(5)])
    return f, g


def _node_post(a, scale, x, y):
    f = np.array([float(a[i, y, x]) * scale + W9[i] for i in range(9)])
    g = np.array([[float(a[9 + 2 * j + c, y, x]) * scale for c in range(2)] for j in range(5)])
    return f, g


@pytest.mark.parametrize("prec,in_place", [("fp16s", False), ("fp32", True)])
def test_state_beyond_2_31_elements(orc, prec, in_place):
    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice
    tau = 0.51
    p = orc.Params(N, N, tau, tau)
    with Lattice(N, N, tau, tau, precision=prec, in_place=in_place) as lat:
        lat.set_fields(*mhd_inputs.orszag_tang(N, 0.04, 0.04))
        t0 = lat.get_totals()
        lat.advance(2)
        before = lat.get_state()
        lat.advance(1)
        after = lat.get_state()
        t1 = lat.get_totals()
    assert abs(t1["mass"] / t0["mass"] - 1) < 1e-6 and np.isfinite(t1["e_kin"])
    a0, scale = _planes(before, prec)
    a1, _ = _planes(after, prec)
    rng = np.random.default_rng(12000)
    xs = list(rng.integers(0, N, 600)) + [N - 1, N - 2, N - 3, N - 65, N - 128, 0, 1, 127, 128] * 8
    ys = list(rng.integers(0, N, 600)) + [int(v) for v in rng.integers(0, N, 72)]
    ys[600:609] = [0] * 9
    ys[609:618] = [N - 1] * 9
    worst = dmax = 0.0
    for x, y in zip(xs, ys):
        fs, gs, _ = orc.collide_node(p, *_node_pre(a0, scale, int(x), int(y)))
        fg, gg = _node_post(a1, scale, int(x), int(y))
        worst = max(worst, np.abs(fs - fg).max(), np.abs(gs - gg).max())
        dmax = max(dmax, np.abs(fs - W9).max(), np.abs(gs).max())
    # FP16S: half rounding of input and output (see the one-step FP16S test)
    tol = 4 * 2.0 ** -11 * dmax if prec == "fp16s" else 2e-6
    print(f"{prec} {'in place' if in_place else 'two buffers'} {N}^2: {len(xs)} nodes, worst {worst:.2e} (tol {tol:.1e})")
    assert worst < tol
