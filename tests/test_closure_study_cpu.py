"""Host-side scoring of the closure study (no GPU): the box-filtered
resampling that lets a plain run on another grid be judged against the
filtered fine run.  A field band-limited below every grid's Nyquist
wave number has one trigonometric interpolant, so resampling it from any
grid must give the direct block average of its values on the fine grid."""
import numpy as np
import pytest


def _field(n, seed, kmax=5):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    out = np.zeros((n, n))
    for kx in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            a, ph = rng.normal(), rng.uniform(0, 2 * np.pi)
            out += a * np.cos(kx * X + ky * Y + ph)
    return out / (4 * kmax * kmax)


def _fields(n):
    rho = 1.0 + 0.05 * _field(n, 1)
    return rho, 0.03 * _field(n, 2), 0.03 * _field(n, 3), 0.02 * _field(n, 4), 0.02 * _field(n, 5)


def _block(a, r):
    n = a.shape[0]
    return a.reshape(n // r, r, n // r, r).mean(axis=(1, 3))


@pytest.mark.parametrize("n", [64, 48, 40, 96])
def test_filtered_resampling_equals_the_fine_block_average(n):
    from paper_2602_14667_gb300.closure_study import filtered_onto_coarse
    n_fine, factor = 64, 4
    fine = _fields(n_fine)
    rho, ux, uy, bx, by = fine
    want_rho = _block(rho, factor)
    want = (want_rho, _block(rho * ux, factor) / want_rho, _block(rho * uy, factor) / want_rho,
            _block(bx, factor), _block(by, factor))
    # the same continuous fields, sampled on an n x n grid
    got = filtered_onto_coarse(_fields(n), n_fine, factor, n_fine // factor)
    for g, w in zip(got, want):
        np.testing.assert_allclose(g, w, rtol=0, atol=1e-13)
