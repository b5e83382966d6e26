"""Learned closure study: fine-grid data, GPU training, coarse rollouts.

Setting (acoustic scaling by `factor`): a fine periodic lattice of n_fine^2
nodes at relaxation times tau_f_fine is the reference; its pre-collision
populations are box-filtered factor x factor onto a coarse lattice, where one
coarse step is `factor` fine steps, the lattice velocity unit is shared and
the lattice viscosity is divided by `factor`:
    tau_coarse = 1/2 + (tau_fine - 1/2) / factor.
Training pairs are (features of the filtered state F(T), the filtered
sub-grid stress of the fine state at T as an a1^(2) correction); the
non-equilibrium feature columns (5..7) are masked (scale 0): the filtered
fine populations carry the fine lattice's non-equilibrium, about
factor * tau_coarse / tau_fine times smaller than what the coarse lattice
develops, so their values would not transfer.  The coarse runs start, like
the fine run, from the t = 0 fields (block-averaged, equilibrium populations)
and are judged against the filtered fine run at the same time by the
rms log10 deviation of the energy spectrum (kinetic + magnetic, shells
1 <= k <= n_coarse / 4) and the relative L2 error of the current density.
The plain coarse RR run is over-dissipative at high k against the filtered
fine run, while the filtered sub-grid stress is mostly dissipative; the
amplitude of the learned stress is therefore calibrated a posteriori on a
training seed (calibrate()), and the held-out seed judges the result.
All arithmetic runs in the library's kernels; numpy only scores outputs.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import _abi
from ._abi import Lattice


def coarse_tau(tau_fine: float, factor: int) -> float:
    return 0.5 + (tau_fine - 0.5) / factor


@dataclass
class StudyConfig:
    n_fine: int = 512
    factor: int = 4
    tau_fine: float = 0.54
    rms: float = 0.03
    train_seeds: tuple = (101, 102)
    eval_seed: int = 203
    sample_start: int = 800          # fine steps before the first training snapshot
    sample_stride: int = 200         # fine steps between training snapshots
    samples_per_seed: int = 12
    eval_coarse_steps: tuple = (200, 400, 600)
    epochs: int = 40
    batch: int = 4096
    lr: float = 1e-3
    train_seed: int = 7
    mlp_seed: int = 11

    @property
    def n_coarse(self) -> int:
        return self.n_fine // self.factor


def _fine_lattice(cfg: StudyConfig, seed: int, stream=None) -> Lattice:
    import mhd_inputs
    lat = Lattice(cfg.n_fine, cfg.n_fine, cfg.tau_fine, cfg.tau_fine, precision="fp32", stream=stream)
    lat.set_fields(*mhd_inputs.random_spectrum(cfg.n_fine, cfg.n_fine, seed, cfg.rms, cfg.rms))
    return lat


def _state_tensor(cfg: StudyConfig):
    import torch
    return torch.empty((19, cfg.n_coarse * cfg.n_coarse), dtype=torch.float32, device="cuda")


def generate_data(cfg: StudyConfig, seeds=None):
    """Features X (n x 24) and sub-grid stress targets T (n x 3), CUDA tensors."""
    import torch
    seeds = cfg.train_seeds if seeds is None else seeds
    nc = cfg.n_coarse
    tau_c = coarse_tau(cfg.tau_fine, cfg.factor)
    xs, ts = [], []
    for seed in seeds:
        with _fine_lattice(cfg, seed) as lat:
            lat.advance(cfg.sample_start)
            for _ in range(cfg.samples_per_seed):
                s0 = _state_tensor(cfg)
                _abi.closure_filter(lat, cfg.factor, s0)
                X = torch.empty((nc * nc, 24), dtype=torch.float32, device="cuda")
                T = torch.empty((nc * nc, 3), dtype=torch.float32, device="cuda")
                _abi.closure_features(s0, nc, nc, 1.0, X)
                _abi.closure_sgs_targets(lat, cfg.factor, tau_c, T)
                xs.append(X)
                ts.append(T)
                lat.advance(cfg.sample_stride)
    return torch.cat(xs), torch.cat(ts)


MASKED_FEATURES = (5, 6, 7)   # the a1^(2) columns


def train(cfg: StudyConfig, X, T):
    """A trained closure network (its final epoch loss in .last_loss)."""
    mlp = _abi.MLP(seed=cfg.mlp_seed, max_batch=cfg.batch)
    mlp.fit_normalisation(X, T)
    prm = mlp.get_params()
    for c in MASKED_FEATURES:
        prm[24 + c] = 0.0          # scale of the masked columns
    mlp.set_params(prm)
    mlp.last_loss = mlp.train(X, T, epochs=cfg.epochs, batch=cfg.batch, lr=cfg.lr, seed=cfg.train_seed)
    return mlp


def untrained(cfg: StudyConfig, X, T):
    """The control: the network of the same seed with the same input and
    output normalisation and masked columns, not trained."""
    mlp = _abi.MLP(seed=cfg.mlp_seed, max_batch=cfg.batch)
    mlp.fit_normalisation(X, T)
    prm = mlp.get_params()
    for c in MASKED_FEATURES:
        prm[24 + c] = 0.0
    mlp.set_params(prm)
    return mlp


def _coarse_fields_from_state(state, n):
    """rho, ux, uy, bx, by of a packed FP32 coarse pre-collision state (host)."""
    w = np.array([4 / 9] + [1 / 36, 1 / 9] * 4)
    a = state.detach().cpu().numpy().astype(np.float64).reshape(19, n, n)
    f = a[:9] + w[:, None, None]
    cx = np.array([0, -1, -1, -1, 0, 1, 1, 1, 0])
    cy = np.array([0, 1, 0, -1, -1, -1, 0, 1, 1])
    rho = f.sum(axis=0)
    ux = (f * cx[:, None, None]).sum(axis=0) / rho
    uy = (f * cy[:, None, None]).sum(axis=0) / rho
    g = a[9:].reshape(5, 2, n, n)
    return rho, ux, uy, g[:, 0].sum(axis=0), g[:, 1].sum(axis=0)


def energy_spectrum(ux, uy, bx, by, kmax):
    """Shell-summed kinetic + magnetic energy spectrum E(k), k = 1..kmax."""
    n = ux.shape[0]
    e = sum(np.abs(np.fft.fft2(q)) ** 2 for q in (ux, uy, bx, by)) / (2.0 * n ** 4)
    k = np.fft.fftfreq(n, 1.0 / n)
    kk = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    shells = np.rint(kk).astype(int)
    return np.array([e[shells == s].sum() for s in range(1, kmax + 1)])


def current_density(bx, by):
    """j_z = d_x b_y - d_y b_x by the isotropic lattice gradient (periodic)."""
    def dx(q):
        e = np.roll(q, -1, 1) - np.roll(q, 1, 1)
        d = (np.roll(np.roll(q, -1, 1), -1, 0) - np.roll(np.roll(q, 1, 1), -1, 0)
             + np.roll(np.roll(q, -1, 1), 1, 0) - np.roll(np.roll(q, 1, 1), 1, 0))
        return e / 3.0 + d / 12.0
    def dy(q):
        return dx(q.T).T
    return dx(by) - dy(bx)


def errors(model, ref, kmax):
    """(spectrum error, current-density error) of model fields against ref.
    The spectrum error is the rms over shells 1..kmax of log10(E / E_ref),
    over the shells holding at least 1e-12 of the reference's largest shell
    energy (the deviation on a log-log spectrum plot)."""
    em = energy_spectrum(*model[1:], kmax)
    er = energy_spectrum(*ref[1:], kmax)
    keep = er > 1e-12 * er.max()
    spec = float(np.sqrt(np.mean(np.log10(np.maximum(em[keep], 1e-300) / er[keep]) ** 2)))
    jm, jr = current_density(model[3], model[4]), current_density(ref[3], ref[4])
    return spec, float(np.linalg.norm(jm - jr) / np.linalg.norm(jr))


def _block_mean(a, r):
    n0, n1 = a.shape
    return a.reshape(n0 // r, r, n1 // r, r).mean(axis=(1, 3))


def filtered_onto_coarse(fields, n_fine: int, factor: int, n_coarse: int):
    """(rho, ux, uy, bx, by) of a periodic run on an n x n grid (any n),
    box-filtered and sampled like the fine reference: coarse node X holds the
    average over the fine nodes factor X .. factor X + factor - 1 (fine
    spacing 2 pi / n_fine) of the run's trigonometric interpolant.  Linear
    in rho, rho u and b, so u follows from the filtered momentum."""
    rho, ux, uy, bx, by = fields
    n = rho.shape[0]
    k = np.fft.fftfreq(n, 1.0 / n)                       # signed integer wave numbers
    h = 2.0 * np.pi / n_fine
    D = np.mean([np.exp(1j * k * j * h) for j in range(factor)], axis=0)
    K = np.rint(k).astype(int) % n_coarse
    out = []
    for q in (rho, rho * ux, rho * uy, bx, by):
        c = np.fft.fft2(q) / (n * n) * D[:, None] * D[None, :]
        acc = np.zeros((n_coarse, n_coarse), dtype=complex)
        np.add.at(acc, (K[:, None], K[None, :]), c)
        out.append(np.real(np.fft.ifft2(acc)) * n_coarse * n_coarse)
    r, mx, my, b_x, b_y = out
    return r, mx / r, my / r, b_x, b_y


def reference(cfg: StudyConfig, seed: int):
    """Filtered fine fields at each of eval_coarse_steps, and the t = 0 fields
    block-averaged onto the coarse grid."""
    import mhd_inputs
    nc = cfg.n_coarse
    refs = {}
    with _fine_lattice(cfg, seed) as lat:
        done = 0
        for k in cfg.eval_coarse_steps:
            lat.advance(cfg.factor * (k - done))
            done = k
            st = _state_tensor(cfg)
            _abi.closure_filter(lat, cfg.factor, st)
            refs[k] = _coarse_fields_from_state(st, nc)
    fields0 = [_block_mean(q, cfg.factor)
               for q in mhd_inputs.random_spectrum(cfg.n_fine, cfg.n_fine, seed, cfg.rms, cfg.rms)]
    return refs, fields0


def coarse_run(cfg: StudyConfig, fields0, refs, mlp=None, timing=False, interval=1):
    """Coarse run (closure if mlp, its MLP evaluated on every interval-th
    step) started, like the fine run, from the t = 0 fields with equilibrium
    populations; (spectrum, current) errors at each checkpoint, and the GPU
    time per coarse step if timing."""
    import torch
    nc = cfg.n_coarse
    tau_c = coarse_tau(cfg.tau_fine, cfg.factor)
    res = {}
    with Lattice(nc, nc, tau_c, tau_c, precision="fp32") as c:
        if mlp is not None:
            _abi.set_closure(c, mlp)
            _abi.set_closure_interval(c, interval)
        c.set_fields(*fields0)
        done = 0
        for k in cfg.eval_coarse_steps:
            c.advance(k - done)
            done = k
            f = c.get_fields()
            res[k] = errors((f["rho"], f["ux"], f["uy"], f["bx"], f["by"]), refs[k], nc // 4)
        if timing:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c.advance(256)
            c.get_totals(check_stable=False)
            res["s_per_step"] = (time.perf_counter() - t0) / 256
    return res


def plain_run_at(cfg: StudyConfig, n: int, seed: int, refs, stream=None):
    """Plain RR run of the same flow on an n x n lattice (acoustic scaling:
    n / n_coarse steps per coarse step, tau = 1/2 + (tau_fine - 1/2) n / n_fine),
    started from the t = 0 fields sampled at its nodes; its fields are
    box-filtered onto the coarse grid and judged like the coarse runs.  A
    checkpoint falls on the nearest whole step (at most half a step of the
    n-grid off).  Returns the errors per checkpoint and the GPU seconds of
    its steps."""
    import torch

    import mhd_inputs
    nc = cfg.n_coarse
    tau = 0.5 + (cfg.tau_fine - 0.5) * n / cfg.n_fine
    res, gpu_s = {}, 0.0
    with Lattice(n, n, tau, tau, precision="fp32", stream=None if stream is None else stream.cuda_stream) as lat:
        lat.set_fields(*mhd_inputs.random_spectrum(n, n, seed, cfg.rms, cfg.rms))
        done = 0
        for k in cfg.eval_coarse_steps:
            steps = (2 * k * n + nc) // (2 * nc) - done   # round(k n / nc)
            done += steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.advance(steps)
            e1.record(stream)
            e1.synchronize()
            gpu_s += e0.elapsed_time(e1) * 1e-3
            f = lat.get_fields()
            model = filtered_onto_coarse((f["rho"], f["ux"], f["uy"], f["bx"], f["by"]), cfg.n_fine,
                                         cfg.factor, nc)
            res[k] = errors(model, refs[k], nc // 4)
    res["gpu_s"] = gpu_s
    res["n"] = n
    res["tau"] = tau
    return res


def coarse_gpu_seconds(cfg: StudyConfig, fields0, mlp=None, stream=None, interval=1):
    """GPU seconds of the coarse run's steps up to the last checkpoint."""
    import torch
    nc = cfg.n_coarse
    tau_c = coarse_tau(cfg.tau_fine, cfg.factor)
    with Lattice(nc, nc, tau_c, tau_c, precision="fp32", stream=None if stream is None else stream.cuda_stream) as c:
        c.set_fields(*fields0)
        if mlp is not None:
            _abi.set_closure(c, mlp)
            c.autotune()          # the faster closure kernel; the state is kept
            _abi.set_closure_interval(c, interval)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.advance(cfg.eval_coarse_steps[-1])
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3


def equal_time_grid(cfg: StudyConfig, t_closure: float, t_plain: float, step: int = 32) -> int:
    """The finest n (a multiple of `step`) at which a plain run to the last
    checkpoint is predicted to take at most the closure run's GPU time:
    acoustic scaling makes the cost grow as n^3 (n^2 nodes, n steps per unit
    time)."""
    n = cfg.n_coarse
    while (n + step) ** 3 / cfg.n_coarse ** 3 * t_plain <= t_closure:
        n += step
    return n


def _score(res, cfg):
    """Calibration objective: spectrum plus current-density errors, summed
    over the checkpoints (+inf for a run that went non-finite)."""
    s = sum(res[k][0] + res[k][1] for k in cfg.eval_coarse_steps)
    return s if math.isfinite(s) else math.inf


CALIBRATION_GRID = (-4.0, -3.0, -2.0, -1.5, -1.0, -0.5, 0.0, 0.5, 1.0)


def calibrate(cfg: StudyConfig, mlp, seed=None, interval=1):
    """A posteriori amplitude of the learned stress: scale out_scale by each c
    of CALIBRATION_GRID, run the coarse closure on a TRAINING seed and keep
    the c with the smallest summed spectrum + current errors (c = 0 is the
    plain scheme).  Returns (c, scores)."""
    seed = cfg.train_seeds[0] if seed is None else seed
    refs, fields0 = reference(cfg, seed)
    base = mlp.get_params()
    scores = {}
    for c in CALIBRATION_GRID:
        p = base.copy()
        p[48:51] *= c
        mlp.set_params(p)
        scores[c] = _score(coarse_run(cfg, fields0, refs, None if c == 0.0 else mlp, interval=interval), cfg)
    best = min(scores, key=scores.get)
    p = base.copy()
    p[48:51] *= best
    mlp.set_params(p)
    return best, scores


def evaluate(cfg: StudyConfig, mlp=None, seed=None):
    """Plain and (if mlp) closure coarse runs on `seed` (default: the held-out
    evaluation seed) against the filtered fine run."""
    seed = cfg.eval_seed if seed is None else seed
    refs, fields0 = reference(cfg, seed)
    out = {"plain": coarse_run(cfg, fields0, refs, None, timing=True)}
    if mlp is not None:
        out["closure"] = coarse_run(cfg, fields0, refs, mlp, timing=True)
    return out


def run(cfg: StudyConfig | None = None, control: bool = False, equal_time: bool = False,
        intervals=()) -> dict:
    """Data from the training seeds, GPU training, a posteriori calibration
    on the first training seed, evaluation on the held-out seed.

    control: also calibrate and evaluate the untrained network of the same
    seed and normalisation (res["untrained"]): whatever it gains is not due
    to training.  equal_time: also time the coarse closure and plain runs on
    the GPU and run the plain scheme on the finest grid that is predicted to
    cost no more than the closure run (res["equal_time"]).  intervals: for
    each k, the closure with its MLP evaluated on every k-th step, its
    amplitude calibrated anew, judged and timed the same way, with its own
    equal-time plain grid (res["intervals"][k])."""
    import torch
    cfg = cfg or StudyConfig()
    X, T = generate_data(cfg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mlp = train(cfg, X, T)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    raw = mlp.get_params()        # before calibration scales the output
    c, scores = calibrate(cfg, mlp)
    res = evaluate(cfg, mlp if c != 0.0 else None)
    res.update(samples=int(X.shape[0]), train_loss=mlp.last_loss, amplitude=c,
               calibration_scores=scores, train_s=train_s, epochs=cfg.epochs)
    if control:
        ctl = untrained(cfg, X, T)
        cu, su = calibrate(cfg, ctl)
        refs, fields0 = reference(cfg, cfg.eval_seed)
        res["untrained"] = {"amplitude": cu, "calibration_scores": su,
                            "run": coarse_run(cfg, fields0, refs, ctl if cu != 0.0 else None)}
        ctl.close()
    if equal_time or intervals:
        refs, fields0 = reference(cfg, cfg.eval_seed)
        stream = torch.cuda.Stream()
        t_plain = coarse_gpu_seconds(cfg, fields0, None, stream)
        plain_at = {}

        def equal_time_arm(t_closure):
            n = equal_time_grid(cfg, t_closure, t_plain)
            if n > cfg.n_coarse and n not in plain_at:
                plain_at[n] = plain_run_at(cfg, n, cfg.eval_seed, refs, stream)
            return plain_at.get(n)

        if equal_time:
            t_closure = coarse_gpu_seconds(cfg, fields0, mlp if c != 0.0 else None, stream)
            res["equal_time"] = {"gpu_s": {"plain_coarse": t_plain, "closure_coarse": t_closure},
                                 "plain_fine": equal_time_arm(t_closure)}
        res["intervals"] = {}
        for k in intervals:
            mlp.set_params(raw)
            ck, sk = calibrate(cfg, mlp, interval=k)
            net = mlp if ck != 0.0 else None
            t_k = coarse_gpu_seconds(cfg, fields0, net, stream, interval=k)
            res["intervals"][k] = {"amplitude": ck, "calibration_scores": sk,
                                   "run": coarse_run(cfg, fields0, refs, net, interval=k),
                                   "gpu_s": t_k, "plain_fine": equal_time_arm(t_k)}
    mlp.close()
    return res
