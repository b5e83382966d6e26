"""Seeded synthetic inputs for the RR-MHD lattice Boltzmann step.

This module is shared by the CUDA-side callers (benchmark, tests, closure
data generation) and the oracle-side tests.  It holds none of the method's
arithmetic: it only produces initial velocity / magnetic fields and random
draws, in lattice units, as FP64 numpy arrays of shape (ny, nx) with x
fastest.

* ``orszag_tang`` -- the Orszag-Tang vortex of the paper (Eq. OT_initial),
  u = u0 (-sin y, sin x), b = b0 (-sin y, sin 2x) on [0, 2 pi)^2 sampled at
  x_i = 2 pi i / N (periodic, no duplicated end point).
* ``random_spectrum`` -- a divergence-free random-phase field with an
  E(k) ~ k^(-5/3) spectrum for 1 <= |k| <= kmax, built from a stream function
  psi = sum_k A(|k|) cos(k.x + phi_k) with A ~ |k|^(-7/3), u = (d_y psi, -d_x psi)
  evaluated analytically, rescaled to a target rms.
* ``SplitMix64`` -- the SplitMix64 generator (Steele, Lea and Flood 2014, as
  published by Vigna) for per-lattice seeded draws.
* ``ensemble`` -- the per-lattice sizes and (nu, eta) draws of the batched
  ensemble workload.
"""
from __future__ import annotations

import math

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += golden gamma; mix with two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def grid(nx: int, ny: int):
    """Node coordinates on [0, 2 pi)^2: X[y, x] = 2 pi x / nx, Y[y, x] = 2 pi y / ny."""
    x = 2.0 * math.pi * np.arange(nx) / nx
    y = 2.0 * math.pi * np.arange(ny) / ny
    return np.meshgrid(x, y)


def orszag_tang(n: int, u0: float, b0: float, ny: int | None = None):
    """Orszag-Tang initial fields (ux, uy, bx, by) on an n x ny lattice."""
    ny = n if ny is None else ny
    X, Y = grid(n, ny)
    ux = -u0 * np.sin(Y)
    uy = u0 * np.sin(X)
    bx = -b0 * np.sin(Y)
    by = b0 * np.sin(2.0 * X)
    return ux, uy, bx, by


def _spectral_modes(kmax: int):
    """Integer wave vectors with 1 <= |k| <= kmax on the half plane (no +-k duplicates)."""
    modes = []
    for kx in range(0, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            if kx == 0 and ky <= 0:
                continue
            k2 = kx * kx + ky * ky
            if 1 <= k2 <= kmax * kmax:
                modes.append((kx, ky))
    return modes


def _solenoidal(nx: int, ny: int, rng: SplitMix64, kmax: int, rms: float):
    """u = (d_y psi, -d_x psi) for psi = sum_k A(|k|) cos(k.x + phi_k), evaluated
    on the grid as the inverse DFT of its sparse spectrum (the same values as
    the direct sum of cosines, up to rounding)."""
    cx = np.zeros((ny, nx), dtype=np.complex128)
    cy = np.zeros((ny, nx), dtype=np.complex128)
    for kx, ky in _spectral_modes(kmax):
        kk = math.hypot(kx, ky)
        amp = kk ** (-7.0 / 3.0)
        phase = 2.0 * math.pi * rng.uniform()
        c = amp * complex(math.cos(phase), math.sin(phase))
        # d_y cos(k.x + phi) = Re(i ky e^{i(k.x + phi)}); -d_x likewise with -i kx
        cx[ky % ny, kx % nx] += 1j * ky * c
        cy[ky % ny, kx % nx] += -1j * kx * c
    vx = np.real(np.fft.ifft2(cx)) * (nx * ny)
    vy = np.real(np.fft.ifft2(cy)) * (nx * ny)
    cur = math.sqrt(float(np.mean(vx * vx + vy * vy)))
    scale = rms / cur if cur > 0 else 0.0
    return vx * scale, vy * scale


def random_spectrum(nx: int, ny: int, seed: int, rms_u: float, rms_b: float, kmax: int = 8):
    """Independent divergence-free random-phase u and b (rms of |u|, |b| given)."""
    rng = SplitMix64(seed)
    ux, uy = _solenoidal(nx, ny, rng, kmax, rms_u)
    bx, by = _solenoidal(nx, ny, rng, kmax, rms_b)
    return ux, uy, bx, by


ENSEMBLE_SIZES = (64, 96, 128, 192, 256, 384, 512)
ENSEMBLE_SEED0 = 260214667


def ensemble(count: int = 512, seed0: int = ENSEMBLE_SEED0):
    """Per-lattice draws of the batched ensemble: a list of dicts with
    n (side), nu, eta, seed.  Each lattice l uses SplitMix64(seed0 + l): the
    size index uniform over ENSEMBLE_SIZES, then log10 nu and log10 eta
    uniform in [-4, -2], then one 64-bit draw that seeds the lattice's field
    phases (``random_spectrum``)."""
    out = []
    for l in range(count):
        rng = SplitMix64(seed0 + l)
        n = ENSEMBLE_SIZES[min(int(rng.uniform() * len(ENSEMBLE_SIZES)), len(ENSEMBLE_SIZES) - 1)]
        nu = 10.0 ** (-4.0 + 2.0 * rng.uniform())
        eta = 10.0 ** (-4.0 + 2.0 * rng.uniform())
        out.append(dict(n=n, nu=nu, eta=eta, seed=rng.next_u64()))
    return out

