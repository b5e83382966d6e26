"""Orszag-Tang vortex runs in the paper's physical units (Section
"Orszag-Tang vortex", Eq. OT_initial, Tables 1-3 at Re = 200 pi and Tables
4, 5, 7, 8 at Re = 2500 and 5000).

Physical-to-lattice mapping (the paper's wording of it is garbled; this is
the reading taken): the field amplitude u0 = b0 = 2 is the rms of the
initial fields and has the lattice value 0.2/pi; the domain [0, 2 pi)^2 has
N x N nodes (dx = 2 pi / N), so one lattice step is dt = (0.2/pi) dx / u0
of physical time (t = 1 is 5 N steps); Re = u0 L / nu with L = 2 pi gives
nu in lattice units as nu dt / dx^2 and tau = 1/2 + 3 nu_lattice for both
populations (magnetic Prandtl number 1).  Current density (Eq. current),
vorticity and div b are converted back by 1 / (lattice speed per unit
physical speed x dx).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

from ._abi import Lattice


@dataclass
class OTSetup:
    n: int
    tau: float
    u_lattice: float   # lattice velocity of one physical speed unit
    dx: float
    dt: float

    def steps(self, t: float) -> int:
        return int(round(t / self.dt))

    @property
    def scale(self) -> float:
        """Factor from lattice j_z, omega_z, div b to physical units."""
        return 1.0 / (self.u_lattice * self.dx)


def setup(n: int, reynolds: float = 200 * math.pi, u0: float = 2.0,
          u0_lattice: float = 0.2 / math.pi) -> OTSetup:
    ut = u0_lattice / u0
    dx = 2 * math.pi / n
    dt = ut * dx
    nu = u0 * 2 * math.pi / reynolds
    return OTSetup(n=n, tau=0.5 + 3 * nu * dt / dx ** 2, u_lattice=ut, dx=dx, dt=dt)


def run(n: int, times, precision: str = "fp64", reynolds: float = 200 * math.pi,
        collision: int = 0, stream=None, stop_on_failure: bool = False, eq_variant: int = 0,
        mag_collision: int = 0):
    """Advance the OT vortex on the GPU and return, for each physical time,
    (t, j_max, omega_max, divb_max, step) in physical units.

    A run that goes non-finite raises MhdError (MHD_EUNSTABLE), unless
    stop_on_failure: then the first non-finite checkpoint is returned as
    (t, None, None, None, step) and the run ends there (the paper's "Fail")."""
    import mhd_inputs
    s = setup(n, reynolds)
    out = []
    with Lattice(n, n, s.tau, s.tau, precision=precision, collision=collision, stream=stream,
                 eq_variant=eq_variant, mag_collision=mag_collision) as lat:
        lat.set_fields(*mhd_inputs.orszag_tang(n, 2.0 * s.u_lattice, 2.0 * s.u_lattice))
        done = 0
        for t in times:
            k = s.steps(t)
            lat.advance(k - done)
            done = k
            tot = lat.get_totals(check_stable=not stop_on_failure)
            if not all(math.isfinite(tot[q]) for q in ("mass", "e_kin", "e_mag", "jz_max", "omega_max")):
                out.append((t, None, None, None, k))
                break
            out.append((t, tot["jz_max"] * s.scale, tot["omega_max"] * s.scale,
                        tot["divb_max"] * s.scale, k))
    return out
