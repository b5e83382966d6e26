"""Storage precision over long Orszag-Tang runs: FP32 and FP16S against FP64.

Two workloads, each run in FP64, FP32 and FP16S storage side by side on the
GPU from the same initial fields (Section "Orszag-Tang vortex", Eq.
OT_initial, lattice amplitudes u0 = b0):

- 1024^2, u0 = b0 = 0.05, tau = 0.5003 (nu = eta = 1e-4), checkpoints up
  to 20,000 steps (among them 1,000, 5,000, 10,000);
- 4096^2, u0 = b0 = 0.04, tau = 0.50006 (nu = eta = 2e-5), checkpoints up
  to 5,000 steps (among them 600, the benchmark's step count).

Both lie beyond the scheme's stability at these grid Reynolds numbers
(u0 N / nu of 5e5 and 8e6): the runs go non-finite, FP16S first, then
FP32, then FP64, and the checkpoints bracket where.

At each checkpoint: the relative L2 error of u_x, u_y, b_x, b_y against the
FP64 run, and for every precision the drift of E_k + E_m (relative to t = 0)
and of the cross helicity H_c (absolute).  A run whose totals go non-finite
is reported as unstable from that checkpoint on and is not advanced further.

Usage: python -m paper_2602_14667_gb300.precision_study [--quick]
(one JSON line per checkpoint; --quick: the first two checkpoints only;
the run stops once every precision is non-finite).
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from ._abi import Lattice

WORKLOADS = (
    {"n": 1024, "amp": 0.05, "tau": 0.5003,
     "checkpoints": (100, 200, 300, 400, 500, 600, 800, 1000, 1500, 2000, 3000, 4000, 5000, 10000, 20000)},
    {"n": 4096, "amp": 0.04, "tau": 0.50006,
     "checkpoints": (300, 600, 700, 800, 900, 1000, 1200, 1400, 1600, 1800, 2000, 3000, 4000, 5000)},
)
PRECISIONS = ("fp64", "fp32", "fp16s")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _finite(tot):
    return all(math.isfinite(tot[k]) for k in ("mass", "e_kin", "e_mag", "cross_hel"))


def run(n: int, amp: float, tau: float, checkpoints, stream=None):
    """Yield one record per checkpoint (see the module docstring)."""
    import mhd_inputs
    fields0 = mhd_inputs.orszag_tang(n, amp, amp)
    lats, t0, alive = {}, {}, {}
    try:
        for p in PRECISIONS:
            lats[p] = Lattice(n, n, tau, tau, precision=p, stream=stream)
            lats[p].set_fields(*fields0)
            t0[p] = lats[p].get_totals()
            alive[p] = True
        done = 0
        for k in checkpoints:
            rec = {"n": n, "tau": tau, "amp": amp, "step": k, "precisions": {}}
            fields = {}
            for p in PRECISIONS:
                if not alive[p]:
                    rec["precisions"][p] = {"stable": False}
                    continue
                lats[p].advance(k - done)
                tot = lats[p].get_totals(check_stable=False)
                if not _finite(tot):
                    alive[p] = False
                    rec["precisions"][p] = {"stable": False}
                    continue
                e0 = t0[p]["e_kin"] + t0[p]["e_mag"]
                rec["precisions"][p] = {
                    "stable": True,
                    "energy_drift": (tot["e_kin"] + tot["e_mag"]) / e0 - 1.0,
                    "cross_helicity_drift": tot["cross_hel"] - t0[p]["cross_hel"],
                    "divb_max": tot["divb_max"],
                }
                fields[p] = lats[p].get_fields()
            done = k
            if "fp64" in fields:
                ref = fields["fp64"]
                for p in ("fp32", "fp16s"):
                    if p in fields:
                        rec["precisions"][p]["rel_l2_vs_fp64"] = {
                            q: _rel(fields[p][q], ref[q]) for q in ("ux", "uy", "bx", "by")}
            yield rec
            if not any(alive.values()):
                break
    finally:
        for lat in lats.values():
            lat.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--quick", action="store_true", help="the first two checkpoints of each workload")
    args = ap.parse_args()
    for w in WORKLOADS:
        cps = w["checkpoints"][:2] if args.quick else w["checkpoints"]
        for rec in run(w["n"], w["amp"], w["tau"], cps):
            print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
