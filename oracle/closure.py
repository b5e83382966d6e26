"""FP64 oracle of the learned sub-grid closure (TEST INFRASTRUCTURE ONLY).

The closure is not in the paper: a per-node MLP predicts a correction dA of
the projected second-order non-equilibrium coefficient a1^(2) (task 3 of the
paper's "Algorithm of computation") on a coarse lattice; dA is added before
the recursion, so only non-conserved moments change.  This module is the
plain reference for the GPU kernels (no shared code with them):

* box_filter   -- r x r block average of fine populations (linear, so the
                  coarse moments are the block averages of the fine ones);
* features     -- 24 per-node inputs: rho - rho0, u, b, a1^(2) (xx, xy, yy),
                  and for each of u_x, u_y, b_x, b_y the isotropic gradient
                  (d_x, d_y), the 9-point lattice Laplacian and d_xy;
* targets      -- the correction that makes one coarse step reproduce the
                  filtered fine state one coarse step later (see targets());
* sgs_targets  -- the filtered sub-grid momentum flux of the fine state,
                  as a correction of a1^(2) (see sgs_targets());
* MLP          -- 24 -> 64 -> 64 -> 3, ReLU, with input / output scaling,
                  forward and backward in FP64, optional BF16 rounding of the
                  weights and of each layer's input (as the tensor-core
                  kernels do), Adam;
* closure_run  -- coarse steps with the correction applied (evaluated on
                  every step, or on every k-th step and reused between).
Arrays: f (9, ny, nx), g (5, 2, ny, nx) as in oracle/__init__.py.
"""
from __future__ import annotations

import numpy as np

from . import Params, collide_da, gradient, lattice, node_info, stream

N_IN, N_HID, N_OUT = 24, 64, 3
CS2 = 1.0 / 3.0


def box_filter(f: np.ndarray, g: np.ndarray, r: int):
    """Average over r x r blocks: coarse[Y, X] = mean of fine[rY + dy, rX + dx]."""
    def blk(a):
        *lead, ny, nx = a.shape
        return a.reshape(*lead, ny // r, r, nx // r, r).mean(axis=(-3, -1))
    return blk(f), blk(g)


def _at(a: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """Periodic a(x + dx, y + dy) for arrays indexed [..., y, x]."""
    return np.roll(np.roll(a, -dy, axis=-2), -dx, axis=-1)


def lap9(phi: np.ndarray) -> np.ndarray:
    """Isotropic lattice Laplacian 6 sum_i w_i (phi(x + c_i) - phi(x))."""
    axes = _at(phi, 1, 0) + _at(phi, -1, 0) + _at(phi, 0, 1) + _at(phi, 0, -1)
    diag = _at(phi, 1, 1) + _at(phi, -1, 1) + _at(phi, 1, -1) + _at(phi, -1, -1)
    return (4.0 * axes + diag - 20.0 * phi) / 6.0


def dxy(phi: np.ndarray) -> np.ndarray:
    """Mixed derivative (phi_NE - phi_NW - phi_SE + phi_SW) / 4."""
    return (_at(phi, 1, 1) - _at(phi, -1, 1) - _at(phi, 1, -1) + _at(phi, -1, -1)) / 4.0


def features(p: Params, f: np.ndarray, g: np.ndarray):
    """(X, a2): X of shape (n, 24) in the documented column order, and the
    projected a1^(2) (n, 3) of the pre-collision state (f, g)."""
    info = node_info(p, f, g)
    rho, ux, uy, bx, by = (info[..., k] for k in range(5))
    a2 = info[..., 5:8]
    cols = [rho - p.rho0, ux, uy, bx, by, a2[..., 0], a2[..., 1], a2[..., 2]]
    for phi in (ux, uy, bx, by):
        dx, dy, _ = gradient(p, phi)
        cols += [dx, dy, lap9(phi), dxy(phi)]
    X = np.stack(cols, axis=-1).reshape(-1, N_IN)
    return X, a2.reshape(-1, 3)


def targets(p: Params, fT, gT, fT1, gT1) -> np.ndarray:
    """dA* per coarse node (n, 3).

    One coarse step maps the pre-collision state F(T) to F(T+1) by
    collide-then-stream.  The post-collision populations that would stream
    into the given F(T+1) are F*_i(x) = F_i(x + c_i, T+1).  The collision
    gives sum_i H2_i F*_i = a0^(2) + (1 - omega) a1^(2) (Hermite
    orthogonality), so the a1^(2) that reproduces them is
    (sum_i H2_i F*_i - a0^(2)) / (1 - omega); dA* is that minus the
    projection of F(T).  Periodic lattices only."""
    cx, cy, _, _, _, _ = lattice()
    info = node_info(p, fT, gT)
    rho, ux, uy, bx, by = (info[..., k] for k in range(5))
    a2 = info[..., 5:8]
    fstar = np.stack([_at(fT1[i], int(cx[i]), int(cy[i])) for i in range(9)])
    sxx = sum(fstar[i] * (cx[i] * cx[i] - CS2) for i in range(9))
    sxy = sum(fstar[i] * (cx[i] * cy[i]) for i in range(9))
    syy = sum(fstar[i] * (cy[i] * cy[i] - CS2) for i in range(9))
    b2 = bx * bx + by * by
    a0xx = rho * ux * ux + 0.5 * b2 - bx * bx
    a0xy = rho * ux * uy - bx * by
    a0yy = rho * uy * uy + 0.5 * b2 - by * by
    om1 = 1.0 - 1.0 / p.tau_f
    tgt = np.stack([(sxx - a0xx) / om1, (sxy - a0xy) / om1, (syy - a0yy) / om1], axis=-1)
    return (tgt - a2).reshape(-1, 3)


def sgs_targets(p_fine: Params, f, g, r: int, tau_coarse: float) -> np.ndarray:
    """Sub-grid stress target per coarse node (n_coarse, 3).

    From the fine pre-collision state: block averages over r x r of rho,
    rho u, b and of the momentum flux rho u u + M(b); the resolved flux of the
    averaged fields is rho_bar u_t u_t + M(b_bar) with u_t = (rho u)_bar /
    rho_bar; tau_sgs = flux_bar - resolved flux (xx, xy, yy).  Adding
    dA = tau_sgs / (1 - omega_coarse) to a1^(2) adds tau_sgs to the
    post-collision momentum flux that streaming carries."""
    info = node_info(p_fine, f, g)
    rho, ux, uy, bx, by = (info[..., k] for k in range(5))

    def avg(a):
        ny, nx = a.shape
        return a.reshape(ny // r, r, nx // r, r).mean(axis=(1, 3))

    b2 = bx * bx + by * by
    fxx = avg(rho * ux * ux + 0.5 * b2 - bx * bx)
    fxy = avg(rho * ux * uy - bx * by)
    fyy = avg(rho * uy * uy + 0.5 * b2 - by * by)
    R, MX, MY, BX, BY = avg(rho), avg(rho * ux), avg(rho * uy), avg(bx), avg(by)
    UX, UY = MX / R, MY / R
    B2 = BX * BX + BY * BY
    txx = fxx - (R * UX * UX + 0.5 * B2 - BX * BX)
    txy = fxy - (R * UX * UY - BX * BY)
    tyy = fyy - (R * UY * UY + 0.5 * B2 - BY * BY)
    om1 = 1.0 - 1.0 / tau_coarse
    return (np.stack([txx, txy, tyy], axis=-1) / om1).reshape(-1, 3)


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


PARAM_NAMES = ("mean", "scale", "out_scale", "W1", "b1", "W2", "b2", "W3", "b3")
PARAM_SHAPES = {"mean": (N_IN,), "scale": (N_IN,), "out_scale": (N_OUT,), "W1": (N_IN, N_HID),
                "b1": (N_HID,), "W2": (N_HID, N_HID), "b2": (N_HID,), "W3": (N_HID, N_OUT),
                "b3": (N_OUT,)}
TRAINABLE = ("W1", "b1", "W2", "b2", "W3", "b3")


class MLP:
    """y = out_scale * (W3^T relu(W2^T relu(W1^T ((x - mean) * scale) + b1) + b2) + b3).
    Weights W[in, out].  The flat parameter vector concatenates PARAM_NAMES in
    order (6006 values)."""

    def __init__(self, params: dict | None = None, seed: int = 0):
        if params is None:
            rng = np.random.default_rng(seed)
            params = {"mean": np.zeros(N_IN), "scale": np.ones(N_IN), "out_scale": np.ones(N_OUT)}
            for w, b, fan_in in (("W1", "b1", N_IN), ("W2", "b2", N_HID), ("W3", "b3", N_HID)):
                n_out = PARAM_SHAPES[w][1]
                params[w] = rng.normal(0, np.sqrt(2.0 / fan_in), (fan_in, n_out))
                params[b] = np.zeros(n_out)
        self.p = {k: np.array(v, dtype=np.float64).reshape(PARAM_SHAPES[k]) for k, v in params.items()}

    @classmethod
    def from_flat(cls, flat):
        flat = np.asarray(flat, dtype=np.float64)
        out, o = {}, 0
        for k in PARAM_NAMES:
            size = int(np.prod(PARAM_SHAPES[k]))
            out[k] = flat[o:o + size].reshape(PARAM_SHAPES[k])
            o += size
        assert o == flat.size
        return cls(out)

    def flat(self) -> np.ndarray:
        return np.concatenate([self.p[k].reshape(-1) for k in PARAM_NAMES])

    def forward(self, X, bf16_like_gpu: bool = False):
        """Returns (y_raw (n,3), cache).  With bf16_like_gpu the weights and
        the input of every layer are rounded to bfloat16 (FP64 sums)."""
        q = bf16 if bf16_like_gpu else (lambda a: a)
        P = self.p
        xn = (np.asarray(X, dtype=np.float64) - P["mean"]) * P["scale"]
        a0 = q(xn)
        z1 = a0 @ q(P["W1"]) + P["b1"]
        h1 = q(np.maximum(z1, 0.0))
        z2 = h1 @ q(P["W2"]) + P["b2"]
        h2 = q(np.maximum(z2, 0.0))
        yn = h2 @ q(P["W3"]) + P["b3"]
        return yn * P["out_scale"], (a0, z1, h1, z2, h2, yn)

    def loss_and_grads(self, X, T, bf16_like_gpu: bool = False, bf16_backward: bool = False,
                       scales: bool = False):
        """MSE over all n*3 entries in scaled output units,
        L = mean((yn - T / out_scale)^2), and its gradients w.r.t. TRAINABLE.

        bf16_backward (with bf16_like_gpu) also rounds the back-propagated
        gradients dY, dH2, dH1 to bfloat16 where they enter a product (the
        weight gradients Act^T dZ and the next layer's dZ W^T), as the
        tensor-core kernels do; the bias gradients sum the unrounded values.
        With scales=True a third dict holds, per parameter, the magnitude
        every element is a sum of: sum_n |Act_ni| D_nj for a weight and
        sum_n D_nj for a bias, where D is the gradient propagated with
        absolute values (|dY|, then (D |W|^T) under the ReLU mask).  A
        relative rounding of eps in any operand moves an element by at most
        eps times that magnitude."""
        P = self.p
        _, (a0, z1, h1, z2, h2, yn) = self.forward(X, bf16_like_gpu)
        tn = np.asarray(T, dtype=np.float64) / P["out_scale"]
        n = yn.shape[0]
        d = yn - tn
        loss = float(np.mean(d * d))
        dy = 2.0 * d / (n * N_OUT)
        q = bf16 if bf16_like_gpu else (lambda a: a)
        qb = bf16 if (bf16_like_gpu and bf16_backward) else (lambda a: a)
        dyq = qb(dy)
        g = {"W3": h2.T @ dyq, "b3": dy.sum(axis=0)}
        dh2 = (dyq @ q(P["W3"]).T) * (z2 > 0)
        dh2q = qb(dh2)
        g["W2"] = h1.T @ dh2q
        g["b2"] = dh2.sum(axis=0)
        dh1 = (dh2q @ q(P["W2"]).T) * (z1 > 0)
        g["W1"] = a0.T @ qb(dh1)
        g["b1"] = dh1.sum(axis=0)
        if not scales:
            return loss, g
        D3 = np.abs(dy)
        D2 = (D3 @ np.abs(q(P["W3"])).T) * (z2 > 0)
        D1 = (D2 @ np.abs(q(P["W2"])).T) * (z1 > 0)
        s = {"W3": np.abs(h2).T @ D3, "b3": D3.sum(axis=0), "W2": np.abs(h1).T @ D2,
             "b2": D2.sum(axis=0), "W1": np.abs(a0).T @ D1, "b1": D1.sum(axis=0)}
        return loss, g, s


class Adam:
    """theta -= lr * m_hat / (sqrt(v_hat) + eps) with the usual bias-corrected
    first / second moment estimates (Kingma and Ba)."""

    def __init__(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m, self.v, self.t = {}, {}, 0

    def step(self, params: dict, grads: dict):
        self.t += 1
        for k, gk in grads.items():
            m = self.m.setdefault(k, np.zeros_like(gk))
            v = self.v.setdefault(k, np.zeros_like(gk))
            m *= self.b1
            m += (1 - self.b1) * gk
            v *= self.b2
            v += (1 - self.b2) * gk * gk
            mh = m / (1 - self.b1 ** self.t)
            vh = v / (1 - self.b2 ** self.t)
            params[k] -= self.lr * mh / (np.sqrt(vh) + self.eps)


def closure_step(p: Params, f, g, mlp: MLP | None, bf16_like_gpu: bool = False):
    """One coarse step with the correction dA = mlp(features) (None: plain)."""
    da = None
    if mlp is not None:
        X, _ = features(p, f, g)
        da, _ = mlp.forward(X, bf16_like_gpu)
        da = da.reshape(p.ny, p.nx, 3)
    fs, gs = collide_da(p, f, g, da)
    return stream(p, fs, gs)


def closure_run(p: Params, f, g, steps: int, mlp: MLP | None, bf16_like_gpu: bool = False,
                interval: int = 1):
    """steps coarse steps with the correction.  interval k > 1: the
    correction is evaluated from the state on steps 0, k, 2k, ... and the
    same per-node values are applied on the k - 1 steps after each."""
    da = None
    for s in range(steps):
        if mlp is not None and s % interval == 0:
            X, _ = features(p, f, g)
            da, _ = mlp.forward(X, bf16_like_gpu)
            da = da.reshape(p.ny, p.nx, 3)
        fs, gs = collide_da(p, f, g, da)
        f, g = stream(p, fs, gs)
    return f, g
