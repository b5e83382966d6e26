#!/usr/bin/env python3
"""Throughput of the fused RR-MHD lattice Boltzmann step on GB300.

Workload (default): the Orszag-Tang vortex on a 4096 x 4096 periodic lattice,
u0 = b0 = 0.04, nu = eta = 2e-5 (tau = 0.50006), FP32 storage of the
populations as deviations f_i - w_i rho0.  One bench step = one time step =
one launch of the fused stream-and-collide kernel over all 16.8 M nodes
(queued through mhd_advance, 64-step CUDA graphs).

Prints ONE JSON line (rank 0):
  value     MLUPS over all ranks (nodes x steps / max-over-ranks device time),
            inputs resident in HBM, timed with CUDA events on the lattice stream;
  e2e       the same metric through the C ABI with pinned HOST buffers:
            mhd_set_fields (H2D) + mhd_advance + mhd_get_fields (D2H) +
            mhd_get_totals inside the timed region, the host fields in the
            path's compute type (float32 for FP32 / FP16S storage; the
            float64 figure beside it);
  roofline  achieved HBM GB/s of the step kernel (152 algorithmic bytes per
            node for FP32: 19 values read + 19 written) vs the measured copy
            bandwidth in MEASURED_PEAKS.json;
  cpu_baseline  the FP64 oracle on the host cores, bounded sample.
--impl reference times the oracle itself (the only reference this method
has) on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank advances its own replica (weak scaling, no
data-path collective).

Other rows of the path have their own line (--workload): ensemble (512
lattices in one persistent launch per step), closure (the learned-closure
study), closure_step (the closure step's cost), diagnostics (the global
totals) and training (the closure MLP's training).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_NODE = {"fp64": 304, "fp32": 152, "fp16s": 76}
ESIZE = {"fp64": 8, "fp32": 4, "fp16s": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16s": "f32 (f16 storage)"}
METRIC = "MLUPS & % HBM roofline (4096² RR-MHD step); coarse+closure vs plain error"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16s"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="ot4096", choices=["ot4096", "ensemble", "closure", "closure_step", "diagnostics", "training", "slabs"],
                    help="ot4096: the headline single lattice; ensemble: 512 random-spectrum "
                         "lattices in one persistent launch per step; closure: the learned-closure "
                         "study; closure_step: the closure step's cost; diagnostics: the global "
                         "totals; training: the closure MLP's training")
    ap.add_argument("--retune", action="store_true",
                    help="time every launch shape instead of using the autotuner's cache")
    ap.add_argument("--shape", default=None,
                    help="fixed launch shape 'V,BY' or 'V,BY,W' (W: resident warps per SM, the staging "
                         "depth; skips the autotuner; for profiling)")
    ap.add_argument("--in-place", action="store_true",
                    help="ot4096 on one state buffer (in-place streaming) instead of two")
    ap.add_argument("--lattices", type=int, default=512,
                    help="ensemble: the first K of the 512 drawn lattices (a smaller case for profiling)")
    ap.add_argument("--no-extra", action="store_true",
                    help="ot4096 at N=1: leave out the extra rows (FP16S line and field error, ensemble)")
    return ap.parse_args()


def workload(n, prec):
    return {"workload": f"orszag_tang_{n}x{n}_{prec}", "nx": n, "ny": n, "u0": 0.04, "b0": 0.04,
            "nu": 2e-5, "eta": 2e-5, "tau_f": 0.50006, "tau_m": 0.50006, "precision": prec,
            "collision": "recursive_regularised", "eq_variant": "A"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# The device code of the step kernels: step.cu and the device headers it
# includes (internal.h holds only host declarations).
STEP_KERNEL_SOURCES = ("f32x2.cuh", "lbm_device.cuh", "step.cu", "step_row.cuh")
DIAG_KERNEL_SOURCES = ("diag.cu", "diag_device.cuh", "f32x2.cuh", "lbm_device.cuh", "step_row.cuh")


def kernel_source_hash(sources=STEP_KERNEL_SOURCES):
    """Hash of a kernel's sources: a profile summary taken from other
    sources no longer describes the timed kernel."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2602_14667_gb300", "csrc")
    for name in sources:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled(prec, shape, key, name=None, sources=STEP_KERNEL_SOURCES):
    """A per-node figure from a committed ncu summary, if it was taken from
    the current kernel sources with the same launch shape (else None)."""
    path = os.path.join(ROOT, "profiles", name or f"rr_step_{prec}_ncu.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha") != kernel_source_hash(sources):
        return None
    if shape is not None:
        # (nodes_per_thread, rows_per_block[, warps_per_sm]); a summary
        # without a depth key was taken at the built-in depth (0)
        depth = shape[2] if len(shape) > 2 else 0
        if vals.get("shape") != f"{shape[0]},{shape[1]}" or vals.get("warps_per_sm", "0") != str(depth):
            return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def profiled_traffic(prec, n, shape):
    """DRAM bytes per launch (see profiled)."""
    per_node = profiled(prec, shape, "dram_bytes_per_node")
    return None if per_node is None else per_node * n * n


# FP64 units of a GB300: 2 DFMA per clock per SM (ncu peak_sustained: 304 per
# cycle on 152 SMs) at the 2070 MHz maximum SM clock
FP64_INSTR_PEAK = 304 * 2.07e9


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for name, v in zip(names, r[4:8]):
                    if v.lower() in ("active", "1"):
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n_sample=512, budget_s=12.0):
    """The FP64 oracle, as it stands, on all host cores: an OT lattice of
    n_sample^2 with the bench's physical parameters, as many steps as fit in
    about budget_s seconds."""
    import mhd_inputs
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    p = oracle.Params(n_sample, n_sample, 0.50006, 0.50006)
    f, g = oracle.init(p, *mhd_inputs.orszag_tang(n_sample, 0.04, 0.04))
    t0 = time.perf_counter()
    f, g = oracle.run(p, f, g, 1)
    t1 = time.perf_counter() - t0
    steps = max(1, min(200, int(budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(p, f, g, steps)
    dt = time.perf_counter() - t0
    return {"value": n_sample * n_sample * steps / dt / 1e6, "unit": "MLUPS",
            "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{n_sample}x{n_sample} Orszag-Tang, {steps} steps, FP64 oracle "
                      f"(same u0, nu as the workload), {dt:.1f} s"}


def partition(items, rank, world):
    """The share of an ensemble that one rank advances (replicas: no data
    exchange between ranks)."""
    return items[rank::world]


def reduce_max(value, dist, device="cpu"):
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle (the method's only reference implementation) timed on the
    host cores on a bounded sample of the workload: each step is one oracle
    step of an n_s x n_s Orszag-Tang lattice with the workload's physics,
    n_s chosen so that warmup + steps end in about two minutes."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import mhd_inputs
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    total = args.warmup + args.steps
    ns = 512
    while True:
        p = oracle.Params(ns, ns, 0.50006, 0.50006)
        f, g = oracle.init(p, *mhd_inputs.orszag_tang(ns, 0.04, 0.04))
        t0 = time.perf_counter()
        f, g = oracle.run(p, f, g, 1)
        t1 = time.perf_counter() - t0
        if t1 * total <= 120.0 or ns <= 16:
            break
        ns //= 2
    f, g = oracle.run(p, f, g, args.warmup)
    t0 = time.perf_counter()
    oracle.run(p, f, g, args.steps)
    dt = time.perf_counter() - t0
    v = ns * ns * args.steps / dt / 1e6
    sample = f"{ns}x{ns} Orszag-Tang sub-lattice per step (u0=b0=0.04, nu=eta=2e-5), FP64 oracle"
    out = {"metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": dict(workload(args.n, args.precision),
                          workload=f"orszag_tang_{ns}x{ns}_fp64_oracle_sample_of_{args.n}x{args.n}",
                          nx=ns, ny=ns, sample_of=workload(args.n, args.precision)["workload"]),
           "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


TUNE_CACHE = os.path.join(ROOT, "paper_2602_14667_gb300", "tune_cache.json")


def extra_rows(fp32_mlups, peak):
    """The other throughput targets of the path, measured in the same run
    (each timed region well under a second):
      fp16s     the 4096^2 workload with FP16 storage shifted by w_i rho0
                (200 steps), its MLUPS, ratio to FP32 and HBM fraction, and
                the FP16S field error where FP16S is usable: the 1024^2
                Orszag-Tang vortex at tau = 0.51 after 1000 steps against
                an FP64 run of the same lattice (relative L2 of u and b);
      ensemble  the 512-lattice random-spectrum ensemble (39 M nodes) in one
                persistent launch per step (100 steps);
      cost_scaling  time per step of the RR and BGK collisions at 1024^2,
                2048^2 and 4096^2 (the paper's runtime-scaling figure);
      diagnostics, closure_step, closure
                the --workload lines of the global totals (4096^2 FP32,
                100 calls), of the closure step's cost (512^2, 512 steps) and
                of the learned-closure study (2048^2 -> 512^2, the closure
                against plain 512^2, the untrained control and the plain
                grid of equal GPU time, the MLP on every 1st / 2nd / 4th / 8th
                step), the last in compact form."""
    import numpy as np
    import torch

    import mhd_inputs
    from paper_2602_14667_gb300 import Batch, Lattice, MhdError
    out = {}
    stream = torch.cuda.Stream()

    def timed(obj, steps):
        obj.advance(10)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obj.advance(steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    n = 4096
    with Lattice(n, n, 0.50006, 0.50006, precision="fp16s", stream=stream.cuda_stream) as lat:
        lat.set_fields(*mhd_inputs.orszag_tang(n, 0.04, 0.04))
        shape = lat.autotune()
        ms16 = timed(lat, 200)
    v16 = n * n / (ms16 * 1e-3) / 1e6
    gbs16 = BYTES_PER_NODE["fp16s"] * n * n / (ms16 * 1e-3) / 1e9
    m, tau, steps = 1024, 0.51, 1000
    fields = mhd_inputs.orszag_tang(m, 0.04, 0.04)
    got = {}
    for prec in ("fp64", "fp16s"):
        with Lattice(m, m, tau, tau, precision=prec, stream=stream.cuda_stream) as lat:
            lat.set_fields(*fields)
            lat.advance(steps)
            got[prec] = lat.get_fields()
    err = {k: float(np.linalg.norm(got["fp16s"][k] - got["fp64"][k]) / np.linalg.norm(got["fp64"][k]))
           for k in ("ux", "uy", "bx", "by")}
    out["fp16s"] = {"value": v16, "unit": "MLUPS", "ms_per_step": ms16, "steps": 200,
                    "ratio_to_fp32": v16 / fp32_mlups, "kernel_config": list(shape),
                    "roofline": {"bound": "hbm", "achieved": gbs16, "peak": peak, "unit": "GB/s",
                                 "frac": gbs16 / peak, "bytes_per_node": BYTES_PER_NODE["fp16s"]},
                    "field_error": {"workload": f"orszag_tang_{m}x{m}_tau_{tau}", "steps": steps,
                                    "reference": "fp64 run of the same lattice",
                                    "rel_l2": err, "max_rel_l2": max(err.values())}}
    draws = mhd_inputs.ensemble(512)
    sizes = [(d["n"], d["n"]) for d in draws]
    taus = [(0.5 + 3 * d["nu"], 0.5 + 3 * d["eta"]) for d in draws]
    with Batch(sizes, taus, stream=stream.cuda_stream) as b:
        for i, d in enumerate(draws):
            b.set_fields(i, *mhd_inputs.random_spectrum(d["n"], d["n"], d["seed"], 0.02, 0.02))
        bshape = b.autotune()
        msb = timed(b, 100)
        nodes = b.nodes
        # the totals of all 512 lattices: one call per lattice, and one call
        # (not timed if a lattice has gone non-finite)
        loop_ms = all_ms = None
        try:
            b.get_all_totals()
            t0 = time.perf_counter()
            for i in range(len(draws)):
                b.get_totals(i)
            loop_ms = (time.perf_counter() - t0) * 1e3
            t0 = time.perf_counter()
            b.get_all_totals(as_arrays=True)
            all_ms = (time.perf_counter() - t0) * 1e3
        except MhdError:
            pass
        # a sample step of the ensemble three ways, one step per call
        sample = None
        try:
            def per_call(fn, reps=20):
                fn()
                stream.synchronize()
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                for _ in range(reps):
                    fn()
                a1.record(stream)
                a1.synchronize()
                return a0.elapsed_time(a1) / reps
            # (the totals as one array per field: building 512 dicts in Python
            # would take ~0.7 ms per call, during which the GPU idles)
            sample = {"ms_plain_step": per_call(lambda: b.advance(1)),
                      "ms_step_then_all_totals": per_call(lambda: (b.advance(1), b.get_all_totals(as_arrays=True))),
                      "ms_fused_step": per_call(lambda: b.advance_totals(1, as_arrays=True))}
        except MhdError:
            pass
    gbsb = 152 * nodes / (msb * 1e-3) / 1e9
    out["ensemble"] = {"value": nodes / (msb * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": msb, "steps": 100,
                       "workload": "ensemble_512_random_spectrum_fp32", "lattices": len(draws), "nodes": nodes,
                       "kernel_config": list(bshape),
                       "roofline": {"bound": "hbm", "achieved": gbsb, "peak": peak, "unit": "GB/s",
                                    "frac": gbsb / peak, "bytes_per_node": 152},
                       "totals_ms": {"per_lattice_calls": loop_ms, "all_lattices_call": all_ms},
                       "sample_step": sample}
    # The paper's only cost result (Fig. runtime_scaling): runtime linear in
    # N^2 with the RR collision above BGK.  Here: FP32, tau 0.51 (where BGK
    # is stable too), 200 graph-launched steps per lattice.
    from paper_2602_14667_gb300 import MHD_BGK, MHD_RR
    cost = {}
    for name, coll in (("rr", MHD_RR), ("bgk", MHD_BGK)):
        cost[name] = {}
        for m in (1024, 2048, 4096):
            with Lattice(m, m, 0.51, 0.51, precision="fp32", collision=coll, stream=stream.cuda_stream) as lat:
                lat.set_fields(*mhd_inputs.orszag_tang(m, 0.04, 0.04))
                ms = timed(lat, 200)
            cost[name][str(m)] = {"ms_per_step": ms, "ns_per_node": ms * 1e6 / (m * m)}
    out["cost_scaling"] = {"collisions": cost, "rr_over_bgk_time_4096": cost["rr"]["4096"]["ms_per_step"]
                           / cost["bgk"]["4096"]["ms_per_step"],
                           "note": "the paper's Fig. runtime_scaling: runtime linear in N^2, RR slower than BGK "
                                   "(C++/Kokkos, hardware unstated, no absolute values)"}
    d = diagnostics_line(4096, "fp32", 100, 3)
    out["diagnostics"] = {k: d[k] for k in ("metric", "value", "unit", "ms_per_call", "config", "roofline",
                                            "sample_step")}
    c = closure_step_line(512, 512, 64)
    out["closure_step"] = {k: c[k] for k in ("metric", "value", "unit", "ms_per_step", "config", "roofline")}
    cl = closure_line()
    et = cl["equal_gpu_time"]
    grid = et["plain_grid"]
    out["closure"] = {
        "metric": cl["metric"], "workload": cl["config"]["workload"], "checkpoints": cl["config"]["checkpoints"],
        "closure_arm": cl["closure_arm"], "amplitude": cl["config"]["amplitude"],
        "errors": "per checkpoint: [energy-spectrum error, current-density error]",
        "closure_512": et["errors"]["closure_512"], "plain_512": et["errors"]["plain_512"],
        "untrained_control_512": et["errors"]["untrained_512"],
        "equal_gpu_time": {"plain_grid": grid, "errors": et["errors"]["plain_grid"], "gpu_s": et["gpu_s"],
                           "plain_grid_gpu_s": et["plain_grid_gpu_s"]},
        "closure_interval": {k: {"cost_vs_plain_512": v["cost_vs_plain_512"], "amplitude": v["amplitude"],
                                 "errors": v["errors"], "equal_time_plain_grid": v["equal_time_plain_grid"],
                                 "equal_time_plain_errors": v["equal_time_plain_errors"]}
                             for k, v in cl["closure_interval"].items()},
        "training": cl["training"], "wall_s": cl["wall_s"]}
    return out


def run_gb300(args):
    import numpy as np
    import torch

    if not args.retune and "MHD_TUNE_CACHE" not in os.environ:
        # the autotuner's results for this GPU (measured with --retune); a
        # lattice without an entry is timed on the spot
        os.environ["MHD_TUNE_CACHE"] = TUNE_CACHE

    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice, MhdError

    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, prec = args.n, args.precision
    tau = 0.50006
    stream = torch.cuda.Stream(device=dev)
    ux, uy, bx, by = mhd_inputs.orszag_tang(n, 0.04, 0.04)

    lat = Lattice(n, n, tau, tau, precision=prec, stream=stream.cuda_stream, in_place=args.in_place)
    lat.set_fields(ux, uy, bx, by)
    if args.shape:
        lat.kernel_config = tuple(int(v) for v in args.shape.split(","))
        shape = lat.kernel_config
    else:
        shape = lat.autotune()
    lat.advance(args.warmup)
    stream.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        lat.advance(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max = reduce_max(ms, dist, dev)
    try:
        tot = lat.get_totals()
        stable = True
    except MhdError:
        tot, stable = None, False

    nodes = n * n
    value = world * nodes * args.steps / (ms_max * 1e-3) / 1e6
    per_launch_s = ms * 1e-3 / args.steps
    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_NODE[prec] * nodes / per_launch_s / 1e9
    # the committed ncu summary describes the two-buffer step kernel
    traffic = None if args.in_place else profiled_traffic(prec, n, shape)

    e2e = None
    if not args.no_e2e:
        def e2e_run(io_dtype):
            pin = [torch.empty((n, n), dtype=io_dtype).pin_memory() for _ in range(9)]
            for t_, a in zip(pin[:4], (ux, uy, bx, by)):
                t_.numpy()[:] = a
            h = [t_.numpy() for t_ in pin]
            lat2 = Lattice(n, n, tau, tau, precision=prec, stream=stream.cuda_stream, in_place=args.in_place)
            lat2.kernel_config = shape
            # an untimed pass of the same calls first: every kernel of the
            # path loaded, the step graph captured
            lat2.set_fields(*h[:4])
            lat2.advance(max(args.warmup, args.steps))
            lat2.get_fields(out=h[4:9])
            lat2.get_totals(check_stable=False)
            stream.synchronize()
            barrier()
            t0 = time.perf_counter()
            lat2.set_fields(*h[:4])                 # H2D of the initial fields
            lat2.advance(args.steps)
            lat2.get_fields(out=h[4:9])            # D2H of rho, u, b
            lat2.get_totals(check_stable=False)    # D2H of the totals
            t_e2e = reduce_max(time.perf_counter() - t0, dist, dev)
            lat2.close()
            esz = pin[0].element_size()
            return (world * nodes * args.steps / t_e2e / 1e6, 4 * esz * nodes / args.steps,
                    (5 * esz * nodes + 13 * 8) / args.steps)

        # host fields in the path's compute type (FP32 for FP32 and FP16S
        # storage: mhd_set_fields_f32 / mhd_get_fields_f32), and in FP64
        io32 = prec in ("fp32", "fp16s")
        v, h2d, d2h = e2e_run(torch.float32 if io32 else torch.float64)
        e2e = {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "host_fields": "float32" if io32 else "float64",
               "note": "mhd_set_fields + mhd_advance(steps) + mhd_get_fields + mhd_get_totals "
                       "from/to pinned host memory; bytes amortised over the steps"}
        if io32:
            v64, h2d64, d2h64 = e2e_run(torch.float64)
            e2e["float64_host_fields"] = {"value": v64, "h2d_bytes_per_step": h2d64, "d2h_bytes_per_step": d2h64}
    lat.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline()
    extra = None
    if not args.no_extra and world == 1 and prec == "fp32" and n == 4096 and not args.in_place:
        extra = extra_rows(value, peak)
    cfg = workload(n, prec)
    nbuf = 1 if args.in_place else 2
    cfg.update({"kernel_config": list(shape), "graph_steps": 64,
                "streaming": "in_place" if args.in_place else "two_buffers",
                "l2": (f"no flush: the {nbuf} x 19-plane state ({nbuf * 19 * n * n * ESIZE[prec] / 1e9:.2f} GB "
                       f"{prec.upper()}) is far above the 129 MB L2"),
                "stable": stable, "replicas": world})
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "frac_of_nominal_8tbs": achieved / 8000.0,
                "bytes_per_node": BYTES_PER_NODE[prec],
                "traffic": traffic}
    fl = profiled(prec, shape, "fp64_flops_per_node") if prec == "fp64" else None
    ins = profiled(prec, shape, "fp64_instructions_per_node") if prec == "fp64" else None
    if fl is not None and ins is not None:
        # FP64 on GB300 is bound by the FP64 units, not by HBM
        rate = nodes / per_launch_s
        roofline = {"bound": "alu", "achieved": fl * rate / 1e12, "peak": 2 * FP64_INSTR_PEAK / 1e12,
                    "unit": "TFLOP/s", "frac": fl * rate / (2 * FP64_INSTR_PEAK),
                    "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2 flop",
                    "fp64_flops_per_node": fl, "fp64_instructions_per_node": ins,
                    "fp64_pipe_frac": ins * rate / FP64_INSTR_PEAK,
                    "hbm_frac": achieved / peak, "traffic": traffic}
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
           "config": cfg,
           "roofline": roofline,
           "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
           "clocks": clk.summary()}
    if tot is not None:
        out["totals"] = {k: tot[k] for k in ("mass", "e_kin", "e_mag", "jz_max", "divb_max")}
    if extra is not None:
        out.update(extra)
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_ensemble(args):
    """The batched ensemble: 512 periodic lattices, sizes in {64..512}^2,
    log-uniform nu, eta in [1e-4, 1e-2], random-spectrum fields (|k| <= 8,
    rms 0.02), one persistent launch per step, 64-step graphs."""
    import numpy as np
    import torch

    import mhd_inputs
    from paper_2602_14667_gb300 import Batch, MhdError

    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    draws = mhd_inputs.ensemble(512)[:max(1, min(512, args.lattices))]
    mine = partition(draws, rank, world)           # replicas: lattices split over ranks
    stream = torch.cuda.Stream()
    sizes = [(d["n"], d["n"]) for d in mine]
    taus = [(0.5 + 3 * d["nu"], 0.5 + 3 * d["eta"]) for d in mine]
    b = Batch(sizes, taus, stream=stream.cuda_stream)
    for i, d in enumerate(mine):
        b.set_fields(i, *mhd_inputs.random_spectrum(d["n"], d["n"], d["seed"], 0.02, 0.02))
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else b.autotune()
    if args.shape:
        b.kernel_config = shape
    b.advance(args.warmup)
    stream.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        b.advance(args.steps)
        ev1.record(stream)
        ev1.synchronize()
    if dist is not None:
        dist.barrier()
    ms = reduce_max(ev0.elapsed_time(ev1), dist, torch.device("cuda", local))
    # the totals of every lattice: one call per lattice, and one call for all
    finite = 0
    t0 = time.perf_counter()
    for i in range(len(mine)):
        try:
            b.get_totals(i)
            finite += 1
        except MhdError:
            pass
    loop_ms = (time.perf_counter() - t0) * 1e3
    all_ms = None
    if finite == len(mine):
        b.get_all_totals(as_arrays=True)
        t0 = time.perf_counter()
        b.get_all_totals(as_arrays=True)
        all_ms = (time.perf_counter() - t0) * 1e3
    nodes = b.nodes
    if dist is not None:
        t = torch.tensor([nodes], dtype=torch.float64, device=torch.device("cuda", local))
        dist.all_reduce(t)
        nodes = int(t.item())
    b.close()
    peak, peak_kind = measured_peaks()
    achieved = 152 * nodes / (ms * 1e-3 / args.steps) / 1e9
    out = {"metric": "MLUPS (batched ensemble, one persistent launch per step)",
           "value": nodes * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": f"ensemble_{len(draws)}_random_spectrum_fp32", "lattices": len(mine),
                      "nodes": nodes, "kernel_config": list(shape), "finite_after_run": finite},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "peak_source": peak_kind, "traffic": None},
           "gpu_launches": args.steps, "clocks": clk.summary(),
           "totals": {"per_lattice_calls_ms": loop_ms, "all_lattices_call_ms": all_ms,
                      "note": "host wall time for the totals of every lattice: mhd_batch_get_totals per "
                              "index, and one mhd_batch_get_all_totals"}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def training_rate(res):
    """Throughput of the GPU training (fit_normalisation excluded): samples
    per second over all epochs, and the MLP's algorithmic tensor work --
    forward 11,648 flop per sample, backward twice that (input and weight
    gradients) -- against the measured dense BF16 peak."""
    per_sample = 3 * 2 * (24 * 64 + 64 * 64 + 64 * 3)
    rate = res["samples"] * res["epochs"] / res["train_s"]
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        peak = float(json.load(fh)["bf16_tflops"])
    tflops = rate * per_sample / 1e12
    return {"samples_per_s": rate, "seconds": res["train_s"], "epochs": res["epochs"],
            "flop_per_sample": per_sample, "tflops": tflops, "frac_of_bf16_peak": tflops / peak}


def run_closure(args):
    print(json.dumps(closure_line()), flush=True)


def closure_line():
    """The learned-closure workload: 2048^2 fine runs (random-spectrum fields,
    rms 0.03) filtered 4x onto 512^2; MLP trained on the GPU on ~2 M samples
    from two seeds, amplitude calibrated on one of them, coarse closure and
    plain runs judged on a held-out seed against the filtered fine run.  The
    fine relaxation time is 0.54 (coarse 0.51): the workload's nu = eta =
    5e-5 lies beyond the scheme's stability limit near tau = 1/2, and a
    coarse 0.505 already lets some seeds go non-finite.
    Two more arms: the untrained network of the same seed put through the
    same calibration (what it gains is not due to training), and the plain
    scheme on the finest grid whose run is predicted to take no more GPU
    time than the closure run (equal GPU time; its fields box-filtered onto
    the 512^2 grid like the fine run's).  And the closure with its MLP
    evaluated on every 2nd, 4th and 8th step only (the stored correction
    reused between), each calibrated, judged, timed and compared with its
    own equal-time plain grid."""
    import torch

    from paper_2602_14667_gb300 import closure_study as cs
    torch.cuda.set_device(0)
    cfg = cs.StudyConfig(n_fine=2048, factor=4, tau_fine=0.54, rms=0.03, sample_start=2000,
                         sample_stride=1500, samples_per_seed=4,
                         eval_coarse_steps=(500, 1000, 1500, 2000), epochs=20, batch=8192)
    t0 = time.perf_counter()
    res = cs.run(cfg, control=True, equal_time=True, intervals=(2, 4, 8))
    wall = time.perf_counter() - t0
    steps = cfg.eval_coarse_steps
    last = steps[-1]
    has_closure = "closure" in res
    sp, jp = res["plain"][last]
    sc, jc = res["closure"][last] if has_closure else (None, None)
    cost_p = res["plain"]["s_per_step"]
    cost_c = res["closure"]["s_per_step"] if has_closure else None
    unt = res["untrained"]
    et = res["equal_time"]
    fine = et["plain_fine"]

    def arm(r):
        return None if r is None else {str(k): r[k] for k in steps}

    out = {"metric": "coarse+closure vs plain error (energy spectrum, current density) against the "
                     "filtered 2048^2 run",
           "value": sc, "unit": "relative spectrum error (closure, last checkpoint)",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "f32 (bf16 MLP)",
           "config": {"workload": "closure_2048_to_512", "tau_fine": cfg.tau_fine,
                      "tau_coarse": cs.coarse_tau(cfg.tau_fine, cfg.factor), "rms": cfg.rms,
                      "samples": res["samples"], "train_loss": res["train_loss"],
                      "amplitude": res["amplitude"], "checkpoints": list(steps),
                      "calibration_scores": {str(k): v for k, v in res["calibration_scores"].items()}},
           "closure_arm": "present" if has_closure else "absent (calibration chose amplitude 0)",
           "plain": arm(res["plain"]), "closure": arm(res.get("closure")),
           "spectrum_error": {"plain": sp, "closure": sc}, "current_error": {"plain": jp, "closure": jc},
           "s_per_coarse_step": {"plain": cost_p, "closure": cost_c},
           "untrained_control": {"amplitude": unt["amplitude"],
                                 "calibration_scores": {str(k): v for k, v in unt["calibration_scores"].items()},
                                 "errors": arm(unt["run"])},
           "equal_gpu_time": {"gpu_s": et["gpu_s"],
                              "plain_grid": None if fine is None else fine["n"],
                              "plain_grid_tau": None if fine is None else fine["tau"],
                              "plain_grid_gpu_s": None if fine is None else fine["gpu_s"],
                              "errors": {"closure_512": arm(res.get("closure")), "plain_512": arm(res["plain"]),
                                         "plain_grid": arm(fine), "untrained_512": arm(unt["run"])}},
           "closure_interval": {str(k): {"amplitude": v["amplitude"], "gpu_s": v["gpu_s"],
                                         "cost_vs_plain_512": v["gpu_s"] / et["gpu_s"]["plain_coarse"],
                                         "errors": arm(v["run"]),
                                         "equal_time_plain_grid": None if v["plain_fine"] is None
                                         else v["plain_fine"]["n"],
                                         "equal_time_plain_errors": arm(v["plain_fine"])}
                                 for k, v in res["intervals"].items()},
           "training": training_rate(res),
           "wall_s": wall}
    return out


def run_closure_step(args):
    print(json.dumps(closure_step_line(args.n if args.n != 4096 else 512, args.steps, args.warmup)), flush=True)


def closure_step_line(n, steps, warmup):
    """Cost of the closure step alone: an n^2 FP32 lattice (512^2 unless --n
    names another size; random-spectrum fields, tau 0.505) advanced with the plain step and with the closure step
    (an untrained network: the MLP cost does not depend on the weights),
    CUDA events around `steps` graph-launched steps each."""
    import torch

    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice, _abi
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    fields = mhd_inputs.random_spectrum(n, n, 7, 0.03, 0.03)
    out = {}
    mlp = _abi.MLP(seed=3, max_batch=64)
    prm = mlp.get_params()
    prm[48:51] = 1e-7                       # small output scale: a stable, non-trivial correction
    mlp.set_params(prm)
    for name in ("plain", "closure", "closure_tcgen05"):
        with Lattice(n, n, 0.505, 0.505, precision="fp32", stream=stream.cuda_stream) as lat:
            if name != "plain":
                _abi.set_closure(lat, mlp)
                _abi.set_closure_kernel(lat, _abi.MHD_CLOSURE_TCGEN05 if name == "closure_tcgen05"
                                        else _abi.MHD_CLOSURE_WARP_MMA)
            lat.set_fields(*fields)
            lat.advance(warmup)
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.advance(steps)
            e1.record(stream)
            e1.synchronize()
            out[name] = e0.elapsed_time(e1) / steps
    mlp.close()
    # Dominant kernel: step_closure.  Its algorithmic work is the MLP,
    # 24x64 + 64x64 + 64x3 multiply-adds = 11,648 flop per node (BF16 tensor
    # cores, FP32 accumulation); its state (2 x 19 planes FP32: 40 MB at
    # 512^2, 160 MB at 1024^2) stays mostly in L2 across steps.  Peak: the measured dense BF16 burst.
    flops = 2 * (24 * 64 + 64 * 64 + 64 * 3) * n * n
    # the closure kernel autotune would keep: the faster of the two
    best_kind = "closure" if out["closure"] <= out["closure_tcgen05"] else "closure_tcgen05"
    achieved = flops / (out[best_kind] * 1e-3) / 1e12
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        peak = float(json.load(fh)["bf16_tflops"])
    res = {"metric": f"closure step cost ({n}^2 coarse lattice)", "value": out[best_kind] / out["plain"],
           "unit": "closure / plain time per step", "higher_is_better": False, "n_gpus": 1,
           "ms_per_step": out, "mlups": {k: n * n / (v * 1e-3) / 1e6 for k, v in out.items()},
           "config": {"workload": f"closure_step_{n}x{n}_fp32", "tau": 0.505,
                      "closure_kernel": "warp_mma" if best_kind == "closure" else "tcgen05"},
           "data": "synthetic",
           "steps": steps, "warmup": warmup,
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "peak_source": "measured bf16 dense (burst)",
                        "flops_per_node": flops // (n * n), "traffic": None}}
    return res


def run_training(args):
    """Throughput of the closure MLP's training alone: 2,097,152 synthetic
    samples (24 normal features with a smooth 3-output teacher: the size of
    the closure study's training set), 8,192-row batches, Adam; one warm-up
    epoch, then CUDA events around `steps` Adam steps (whole epochs).  Algorithmic work: forward 11,648 flop per sample and the
    backward pass twice that, against the measured dense BF16 peak.  Each
    train call records its epoch graph once, so at least 8 epochs are
    timed."""
    import torch

    from paper_2602_14667_gb300 import _abi
    torch.cuda.set_device(0)
    n, batch = 2097152, 8192
    per_epoch = (n + batch - 1) // batch
    epochs = max(8, round(args.steps / per_epoch))  # the per-call set-up is amortised over 8+ epochs
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn((n, 24), device="cuda", generator=g)
    T = torch.tanh(X @ torch.randn((24, 3), device="cuda", generator=g) * 0.3).contiguous()
    stream = torch.cuda.current_stream()
    with _abi.MLP(seed=0, max_batch=batch) as m:
        m.fit_normalisation(X, T)
        m.train(X, T, epochs=1, batch=batch, lr=1e-3, seed=1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(0) as clk:
            e0.record(stream)
            loss = m.train(X, T, epochs=epochs, batch=batch, lr=1e-3, seed=2)
            e1.record(stream)
            e1.synchronize()
        s = e0.elapsed_time(e1) * 1e-3
    rate = n * epochs / s
    per_sample = 3 * 2 * (24 * 64 + 64 * 64 + 64 * 3)
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        peak = float(json.load(fh)["bf16_tflops"])
    tflops = rate * per_sample / 1e12
    out = {"metric": "closure MLP training throughput", "value": rate / 1e6, "unit": "M samples/s",
           "higher_is_better": True, "n_gpus": 1, "steps": epochs * per_epoch, "warmup": per_epoch,
           "us_per_adam_step": s / (epochs * per_epoch) * 1e6, "dtype": "bf16 (f32 accumulate, f32 Adam)",
           "data": "synthetic",
           "config": {"workload": "closure_mlp_training_24_64_64_3", "samples": n, "batch": batch,
                      "epochs": epochs, "final_epoch_loss": loss},
           "clocks": clk.summary(), "gpu_launches": epochs * (1 + 2 * per_epoch),
           "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                        "frac": tflops / peak, "peak_source": "measured bf16 dense (burst)",
                        "flops_per_sample": per_sample, "traffic": None}}
    print(json.dumps(out), flush=True)


def run_diagnostics(args):
    print(json.dumps(diagnostics_line(args.n, args.precision, args.steps, args.warmup)), flush=True)


def diagnostics_line(n, prec, steps, warmup):
    """Cost of the global diagnostics (mass, momentum, energies, cross
    helicity, sum b, div b rms / max, current-density and vorticity maxima):
    the Orszag-Tang lattice (4096^2 FP32 by default) after `warmup` steps,
    CUDA events on the lattice's stream around `steps` calls of the totals
    (each: one persistent kernel over the lattice, the fixed-order final
    reduction, the copy of the 13 values to the host and the host's wait).
    The kernel reads each of the 19 planes once (the pre-collision state is
    gathered from the buffer the last step read), so its roofline is HBM
    bandwidth at 19 x element-size bytes per node; the per-call time
    includes the host's round trip, so the fraction is a lower bound."""
    import torch

    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    nodes = n * n
    with Lattice(n, n, 0.50006, 0.50006, precision=prec, stream=stream.cuda_stream) as lat:
        lat.set_fields(*mhd_inputs.orszag_tang(n, 0.04, 0.04))
        lat.advance(max(warmup, 1))
        for _ in range(3):
            lat.get_totals()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            e0.record(stream)
            for _ in range(steps):
                tot = lat.get_totals()
            e1.record(stream)
            e1.synchronize()
        ms = e0.elapsed_time(e1) / steps

        # A sample step three ways, one step per call: the plain step alone;
        # the step then the diagnostics pass (mhd_advance + mhd_get_totals);
        # the fused step that reduces the point totals (mhd_advance_totals).
        def per_call(fn):
            for _ in range(3):
                fn()
            stream.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(steps):
                fn()
            a1.record(stream)
            a1.synchronize()
            return a0.elapsed_time(a1) / steps

        ms_plain = per_call(lambda: lat.advance(1))
        ms_pass = per_call(lambda: (lat.advance(1), lat.get_totals()))
        ms_fused = per_call(lambda: lat.advance_totals(1))
        sample = {"ms_plain_step": ms_plain, "ms_step_then_totals_pass": ms_pass, "ms_fused_step": ms_fused,
                  "extra_ms_totals_pass": ms_pass - ms_plain, "extra_ms_fused": ms_fused - ms_plain,
                  "note": "one step per call; the pass and the fused step include the copy of the totals "
                          "to the host and the host's wait; the fused step gives the point totals (mass, "
                          "momentum, energies, cross helicity, sum b, max |j_z|), the pass every total"}
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        peak = float(json.load(fh)["hbm_gbs"])
    per_node = 19 * ESIZE[prec]
    gbs = per_node * nodes / (ms * 1e-3) / 1e9
    dram = profiled(prec, None, "dram_bytes_per_node", name=f"diag_kernel_{prec}_ncu.md",
                    sources=DIAG_KERNEL_SOURCES)
    roofline = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "peak_source": "measured", "bytes_per_node": per_node,
                "traffic": None if dram is None else dram * nodes,
                "note": "per call, including the final reduction, the D2H copy and the host wait"}
    out = {"metric": "global diagnostics rate", "value": nodes / (ms * 1e-3) / 1e6, "unit": "Mnodes/s",
           "ms_per_call": ms, "higher_is_better": True, "n_gpus": 1, "steps": steps,
           "warmup": warmup, "dtype": DTYPE[prec] + " (f64 sums)", "data": "synthetic",
           "config": {"workload": f"diagnostics_orszag_tang_{n}x{n}_{prec}", "nx": n, "ny": n,
                      "calls": steps, "l2": "no flush: the state is far above the 129 MB L2"},
           "totals_sample": {"mass": tot["mass"], "divb_max": tot["divb_max"], "jz_max": tot["jz_max"]},
           "clocks": clk.summary(), "gpu_launches": 2 * steps, "roofline": roofline,
           "sample_step": sample}
    return out


def run_slabs(args):
    """Cost of the row-slab decomposition of one lattice on one GPU: the
    Orszag-Tang lattice (4096^2 FP32 by default) advanced whole and as S = 2
    and 4 slabs of equal rows (bc_y = MHD_HALO), every slab on the same
    stream.  Each step is the fused step of every slab, then the exchange of
    the boundary-crossing rows of every boundary: through the slab group
    (mhd_slab_group_advance: one exchange kernel per step, 64-step CUDA
    graphs; the whole lattice also runs its 64-step graphs), and stepwise
    (one mhd_advance per slab and one mhd_slab_exchange per boundary and
    step, two copy kernels each).  CUDA events around `steps` steps.  The
    slabs' populations equal the whole lattice's bit for bit
    (tests/test_slabs_gpu.py)."""
    import torch

    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice
    from paper_2602_14667_gb300.slabs import SlabGroup
    torch.cuda.set_device(0)
    n, prec, tau = args.n, args.precision, 0.50006
    stream = torch.cuda.Stream()
    fields = mhd_inputs.orszag_tang(n, 0.04, 0.04)

    def timed(fn, reps, steps):
        fn()  # untimed: graphs captured, kernels loaded
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps

    out = {}
    with Lattice(n, n, tau, tau, precision=prec, stream=stream.cuda_stream) as lat:
        lat.set_fields(*fields)
        shape = lat.kernel_config
        out["whole"] = {"ms_per_step": timed(lambda: lat.advance(args.steps), 1, args.steps)}
    with ClockSampler(0) as clk:
        for S in (2, 4):
            with SlabGroup(n, n, S, tau, tau, precision=prec, stream=stream.cuda_stream) as sg:
                sg.kernel_config = shape
                sg.set_fields(*fields)
                ms = timed(lambda: sg.advance(args.steps), 1, args.steps)
                msw = timed(lambda: sg.advance(1, stepwise=True), args.steps, args.steps)
                ex = timed(sg.exchange, args.steps, args.steps)
            w = out["whole"]["ms_per_step"]
            out[f"slabs_{S}"] = {"ms_per_step": ms, "overhead_vs_whole": ms / w - 1,
                                 "stepwise_ms_per_step": msw, "stepwise_overhead_vs_whole": msw / w - 1,
                                 "exchange_call_us": ex * 1e3}
    for v in out.values():
        v["mlups"] = n * n / (v["ms_per_step"] * 1e-3) / 1e6
    res = {"metric": f"row-slab decomposition on one GPU ({n}^2 {prec})", "value": out["slabs_2"]["mlups"],
           "unit": "MLUPS (2 slabs)", "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "dtype": DTYPE[prec], "data": "synthetic",
           "config": {"workload": f"slabs_orszag_tang_{n}x{n}_{prec}", "kernel_config": list(shape),
                      "stream": "all slabs on one stream"},
           "runs": out, "clocks": clk.summary()}
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "closure":
        run_closure(args)
    elif args.workload == "closure_step":
        run_closure_step(args)
    elif args.workload == "diagnostics":
        run_diagnostics(args)
    elif args.workload == "training":
        run_training(args)
    elif args.workload == "slabs":
        run_slabs(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
