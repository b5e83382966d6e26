"""Parity at the benchmark's full sizes, in the launch shapes bench.py times.

The 4096^2 Orszag-Tang lattice (FP32 and FP16S) and the 512-lattice ensemble
are too large for the oracle to step whole, so sampled nodes are checked one
by one: the post-collision state before the last step is read back, each
sampled node's pre-collision populations are pulled from it (periodic), the
oracle collides that node, and the GPU's post-step populations at the node
must agree (FP32: 2e-6; FP16S: the half-rounding bound of the one-step
test).  Samples cover random interior nodes plus every warp / vector-lane /
tile edge column and the first and last rows.  Conservation over the bench's
600 steps, and the global diagnostics against the oracle's, are checked on
the whole lattice.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CX = np.array([0, -1, -1, -1, 0, 1, 1, 1, 0])
CY = np.array([0, 1, 0, -1, -1, -1, 0, 1, 1])
EX = np.array([0, -1, 0, 1, 0])
EY = np.array([0, 0, -1, 0, 1])
W9 = np.array([4 / 9] + [1 / 36, 1 / 9] * 4)


def _bench_shape(prec_code, n):
    with open(os.path.join(ROOT, "paper_2602_14667_gb300", "tune_cache.json")) as fh:
        cache = json.load(fh)
    return tuple(cache[f"NVIDIA GB300|p{prec_code}|{n}x{n}|bc00"])


def _samples(nx, ny, rng, count=3000):
    xs = list(rng.integers(0, nx, count))
    ys = list(rng.integers(0, ny, count))
    edge_cols = sorted({c for k in range(0, nx, 32) for c in (k - 1, k, k + 1) if 0 <= c < nx} | {nx - 1})
    for c in edge_cols[:400]:
        for r in (0, ny - 1, int(rng.integers(0, ny))):
            xs.append(c)
            ys.append(r)
    return np.array(xs), np.array(ys)


def _check_nodes(orc, p, Pf, Pg, Qf, Qg, xs, ys, tol):
    ny, nx = Pf.shape[1:]
    worst = 0.0
    for x, y in zip(xs, ys):
        f = np.array([Pf[i, (y - CY[i]) % ny, (x - CX[i]) % nx] for i in range(9)])
        g = np.array([[Pg[j, a, (y - EY[j]) % ny, (x - EX[j]) % nx] for a in range(2)] for j in range(5)])
        fs, gs, _ = orc.collide_node(p, f, g)
        worst = max(worst, np.abs(fs - Qf[:, y, x]).max(), np.abs(gs - Qg[:, :, y, x]).max())
    assert worst < tol, worst
    return worst


@pytest.mark.parametrize("prec,code", [("fp32", 1), ("fp16s", 2)])
def test_orszag_tang_4096_sampled_nodes(orc, prec, code):
    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice
    n, tau = 4096, 0.50006
    p = orc.Params(n, n, tau, tau)
    with Lattice(n, n, tau, tau, precision=prec) as lat:
        lat.kernel_config = _bench_shape(code, n)
        lat.set_fields(*mhd_inputs.orszag_tang(n, 0.04, 0.04))
        lat.advance(23)
        Pf, Pg = lat.get_populations()
        lat.advance(1)
        Qf, Qg = lat.get_populations()
    if prec == "fp32":
        tol = 2e-6
    else:
        dmax = max(np.abs(Qf - W9[:, None, None]).max(), np.abs(Qg).max())
        tol = 4 * 2.0 ** -11 * dmax
    rng = np.random.default_rng(4096 + code)
    xs, ys = _samples(n, n, rng)
    worst = _check_nodes(orc, p, Pf, Pg, Qf, Qg, xs, ys, tol)
    print(f"{prec} 4096^2: {len(xs)} nodes, worst |GPU - oracle| = {worst:.2e} (tol {tol:.1e})")


@pytest.mark.parametrize("prec,code", [("fp32", 1), ("fp16s", 2)])
def test_orszag_tang_4096_totals_against_oracle(orc, prec, code):
    """The diagnostics of the timed 4096^2 workload, whole: the totals of the
    pre-collision state the last step gathered against the oracle's totals
    of the stream of the state that step read (the bounds of the
    diagnostics tests; the fields are smooth, so div b stays at the FP32
    rounding floor of the moments)."""
    import mhd_inputs
    from test_diag_gpu import _check
    from paper_2602_14667_gb300 import Lattice
    n, tau = 4096, 0.50006
    p = orc.Params(n, n, tau, tau)
    with Lattice(n, n, tau, tau, precision=prec) as lat:
        lat.kernel_config = _bench_shape(code, n)
        lat.set_fields(*mhd_inputs.orszag_tang(n, 0.04, 0.04))
        lat.advance(23)
        Pf, Pg = lat.get_populations()
        lat.advance(1)
        got = lat.get_totals()
    ref = orc.totals(p, *orc.stream(p, Pf, Pg))
    _check(got, ref, n * n, False)


def test_orszag_tang_4096_conservation_over_bench_steps():
    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice
    n, tau = 4096, 0.50006
    with Lattice(n, n, tau, tau, precision="fp32") as lat:
        lat.kernel_config = _bench_shape(1, n)
        lat.set_fields(*mhd_inputs.orszag_tang(n, 0.04, 0.04))
        t0 = lat.get_totals()
        lat.advance(600)
        t1 = lat.get_totals()
    assert abs(t1["mass"] - t0["mass"]) < 1e-7 * t0["mass"]
    assert abs(t1["mom_x"]) < 1e-6 * t0["mass"] and abs(t1["mom_y"]) < 1e-6 * t0["mass"]
    assert abs(t1["bsum_x"]) < 1e-6 * n * n * 0.04 and abs(t1["bsum_y"]) < 1e-6 * n * n * 0.04


def test_ensemble_full_batch_against_oracle(orc):
    """The whole 512-lattice ensemble in the shape its autotuner picks (the
    bench's launch), 20 steps; every 32nd lattice against the oracle."""
    import mhd_inputs
    from paper_2602_14667_gb300 import Batch
    draws = mhd_inputs.ensemble(512)
    sizes = [(d["n"], d["n"]) for d in draws]
    taus = [(0.5 + 3 * d["nu"], 0.5 + 3 * d["eta"]) for d in draws]
    steps = 20
    with Batch(sizes, taus) as b:
        for i, d in enumerate(draws):
            b.set_fields(i, *mhd_inputs.random_spectrum(d["n"], d["n"], d["seed"], 0.02, 0.02))
        b.autotune()
        b.advance(steps)
        for i in range(0, 512, 32):
            d, n = draws[i], sizes[i][0]
            p = orc.Params(n, n, *taus[i])
            f, g = orc.run(p, *orc.init(p, *mhd_inputs.random_spectrum(n, n, d["seed"], 0.02, 0.02)), steps)
            ref = orc.fields(p, f, g)
            got = b.get_fields(i)
            for k, r in zip(("ux", "uy", "bx", "by"), ref[1:]):
                err = np.linalg.norm(got[k] - r) / np.linalg.norm(r)
                assert err < 1e-5, (i, k, err)
            assert abs(b.get_totals(i)["mass"] - n * n) < 1e-5 * n * n
