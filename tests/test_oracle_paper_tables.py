"""End-to-end pin of the oracle against the values the paper prints for its
Orszag-Tang runs (Tables 1-3, RR column, Re = 200 pi).

Physical-to-lattice mapping (the paper's text on it is garbled; this is the
reading taken): the Orszag-Tang amplitude is u0 = b0 = 2 (the rms of the
fields), its lattice value is 0.2/pi, the domain [0, 2 pi) has N nodes, so
dx = 2 pi / N, dt = (0.2/pi) dx / u0 (t = 1 is 5 N steps), Re = u0 L / nu
with L = 2 pi, nu_lattice = nu dt / dx^2, tau = 1/2 + 3 nu_lattice (both
populations, magnetic Prandtl number 1).  Quantities are converted back by
1 / (lattice velocity per unit speed x dx).  j_z comes from the populations
(Eq. current), omega_z and div b from the isotropic lattice gradient.
j_max and omega_max are pinned; max|div b|, a small lattice-error quantity,
is pinned at t = 1 only (at t = 0.5 it differs by about 30 % and is printed).
"""
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load_table():
    rows = []
    with open(os.path.join(HERE, "golden", "ot_tables_rr.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                t, n, j, w, d = line.split()
                rows.append((float(t), int(n), float(j), float(w), float(d)))
    return rows


def lattice_setup(n, re=200 * math.pi, u0=2.0):
    ut = 0.2 / math.pi / u0          # lattice velocity per unit physical speed
    dx = 2 * math.pi / n
    dt = ut * dx
    nu = u0 * 2 * math.pi / re
    tau = 0.5 + 3 * nu * dt / dx ** 2
    return ut, dx, dt, tau


def test_orszag_tang_n128_matches_tables(orc):
    import mhd_inputs
    n = 128
    ut, dx, dt, tau = lattice_setup(n)
    p = orc.Params(n, n, tau, tau)
    f, g = orc.init(p, *mhd_inputs.orszag_tang(n, 2.0 * ut, 2.0 * ut))
    table = {(t, nn): (j, w, d) for t, nn, j, w, d in load_table()}
    done = 0
    for t in (0.5, 1.0):
        steps = int(round(t / dt))
        f, g = orc.run(p, f, g, steps - done)
        done = steps
        tot = orc.totals(p, f, g)
        s = 1.0 / (ut * dx)
        j, w, d = tot["jz_max"] * s, tot["omega_max"] * s, tot["divb_max"] * s
        jr, wr, dr = table[(t, n)]
        print(f"t={t} N={n}: j_max {j:.3f} ({jr}), omega_max {w:.4f} ({wr}), divb {d:.4f} ({dr})")
        assert abs(j / jr - 1) < (0.015 if t == 0.5 else 0.03)
        assert abs(w / wr - 1) < 0.01
        if t == 1.0:
            assert abs(d / dr - 1) < 0.02
