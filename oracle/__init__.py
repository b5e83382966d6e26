"""FP64 CPU oracle of the recursive regularised MHD lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the library under
``paper_2602_14667_gb300`` never imports it.  It shares no code with the CUDA
path.

``mhd_oracle.c`` follows the six tasks of the paper's "Algorithm of
computation" literally (Hermite series, projection, recursion as full
tensors, push streaming); ``exact.py`` restates the same step with the printed
closed forms in exact rational arithmetic for tiny lattices.

Parity status: every exported function is pinned by ``tests/test_oracle_*.py``
(moment identities, conservation, special cases, closed-form decay, lattice
symmetry, exact brute force); none is "parity unpinned".

Array layout (shared with nothing): ``f`` has shape (9, ny, nx) and ``g`` has
shape (5, 2, ny, nx), FP64, C order, x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile mhd_oracle.c into liboracle.so (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("rho0", ctypes.c_double), ("tau_f", ctypes.c_double), ("tau_m", ctypes.c_double),
        ("wall_x", ctypes.c_int), ("wall_y", ctypes.c_int),
        ("eq_variant", ctypes.c_int), ("collision", ctypes.c_int),
        ("mag_collision", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        for name in ("orc_collide", "orc_stream"):
            getattr(_lib, name).restype = None
        _lib.orc_run.restype = ctypes.c_int
        _lib.orc_totals.restype = ctypes.c_int
        _lib.orc_hermite.restype = ctypes.c_double
        _lib.orc_hermite.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        _lib.orc_supported.restype = ctypes.c_int
        _lib.orc_feq.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, d]
        _lib.orc_geq.argtypes = [ctypes.c_double] * 4 + [d]
        _lib.orc_threads.restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """Lattice size and relaxation times.  nu = (tau_f - 1/2)/3, eta = (tau_m - 1/2)/3."""
    nx: int
    ny: int
    tau_f: float
    tau_m: float
    rho0: float = 1.0
    wall_x: bool = False
    wall_y: bool = False
    eq_variant: int = 0
    collision: int = 0  # 0 recursive regularised, 1 BGK
    mag_collision: int = 0  # 0 BGK, 1 regularised onto the first Hermite moment

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, self.rho0, self.tau_f, self.tau_m, int(self.wall_x),
                       int(self.wall_y), self.eq_variant, self.collision, self.mag_collision)


def lattice():
    """The velocity sets and weights the oracle uses: (cx, cy, w, ex, ey, psi)."""
    cx = (ctypes.c_int * 9)(); cy = (ctypes.c_int * 9)(); w = (ctypes.c_double * 9)()
    ex = (ctypes.c_int * 5)(); ey = (ctypes.c_int * 5)(); psi = (ctypes.c_double * 5)()
    lib().orc_lattice(cx, cy, w, ex, ey, psi)
    return (np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(ex[:]), np.array(ey[:]),
            np.array(psi[:]))


def hermite(n: int, idx, i: int) -> float:
    arr = (ctypes.c_int * max(n, 1))(*idx)
    return lib().orc_hermite(n, arr, i)


def feq(rho, ux, uy, bx, by, variant=0) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, bx, by, variant, _p(out))
    return out


def geq(ux, uy, bx, by) -> np.ndarray:
    """Magnetic equilibrium, shape (5, 2)."""
    out = np.zeros(10)
    lib().orc_geq(ux, uy, bx, by, _p(out))
    return out.reshape(5, 2)


def collide_node(p: Params, f: np.ndarray, g: np.ndarray):
    """One node through tasks 1-5.  Returns (f*, g*, info) where info holds
    rho, ux, uy, bx, by, a2_xx, a2_xy, a2_yy, a3_xxy, a3_xyy, a4_xxyy, fneq_reg[9]."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(10))
    fs = np.zeros(9); gs = np.zeros(10); info = np.zeros(20)
    pc = p.c()
    lib().orc_collide_node(ctypes.byref(pc), _p(f), _p(g), _p(fs), _p(gs), _p(info))
    return fs, gs.reshape(5, 2), info


def init(p: Params, ux, uy, bx, by, rho=None):
    """Equilibrium populations for given fields (arrays of shape (ny, nx))."""
    n = p.nx * p.ny
    f = np.zeros((9, p.ny, p.nx)); g = np.zeros((5, 2, p.ny, p.nx))
    arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(n) for a in (ux, uy, bx, by)]
    r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).reshape(n)
    pc = p.c()
    lib().orc_init(ctypes.byref(pc), _p(r) if r is not None else None, *[_p(a) for a in arrs],
                   _p(f), _p(g))
    return f, g


def collide(p: Params, f: np.ndarray, g: np.ndarray):
    fs = np.zeros_like(f); gs = np.zeros_like(g)
    pc = p.c()
    lib().orc_collide(ctypes.byref(pc), _p(f), _p(g), _p(fs), _p(gs))
    return fs, gs


def collide_da(p: Params, f: np.ndarray, g: np.ndarray, da):
    """Collision with a per-node correction da (shape (ny, nx, 3): xx, xy, yy)
    added to a1^(2) before the recursion; da=None is the plain collision."""
    fs = np.zeros_like(f); gs = np.zeros_like(g)
    pc = p.c()
    d = None if da is None else np.ascontiguousarray(da, dtype=np.float64).reshape(-1)
    lib().orc_collide_da(ctypes.byref(pc), _p(f), _p(g), _p(d) if d is not None else None,
                         _p(fs), _p(gs))
    return fs, gs


def node_info(p: Params, f: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Per-node (ny, nx, 20): rho, ux, uy, bx, by, a2 (xx, xy, yy), a3 (xxy, xyy),
    a4_xxyy, fneq_reg[9] of the pre-collision state (f, g)."""
    out = np.zeros((p.ny, p.nx, 20))
    pc = p.c()
    lib().orc_node_info(ctypes.byref(pc), _p(f), _p(g), _p(out))
    return out


def stream(p: Params, fs: np.ndarray, gs: np.ndarray):
    f = np.zeros_like(fs); g = np.zeros_like(gs)
    pc = p.c()
    lib().orc_stream(ctypes.byref(pc), _p(fs), _p(gs), _p(f), _p(g))
    return f, g


def run(p: Params, f: np.ndarray, g: np.ndarray, nsteps: int):
    """nsteps of collide-then-stream; returns new (f, g) (pre-collision state)."""
    f = np.array(f, dtype=np.float64, order="C"); g = np.array(g, dtype=np.float64, order="C")
    pc = p.c()
    if lib().orc_run(ctypes.byref(pc), _p(f), _p(g), ctypes.c_long(nsteps)) != 0:
        raise MemoryError("oracle scratch allocation failed")
    return f, g


def fields(p: Params, f: np.ndarray, g: np.ndarray):
    """(rho, ux, uy, bx, by), each of shape (ny, nx)."""
    out = [np.zeros((p.ny, p.nx)) for _ in range(5)]
    pc = p.c()
    lib().orc_fields(ctypes.byref(pc), _p(f), _p(g), *[_p(a) for a in out])
    return tuple(out)


def current(p: Params, f: np.ndarray, g: np.ndarray) -> np.ndarray:
    jz = np.zeros((p.ny, p.nx))
    pc = p.c()
    lib().orc_current(ctypes.byref(pc), _p(f), _p(g), _p(jz))
    return jz


def gradient(p: Params, phi: np.ndarray):
    """Isotropic lattice gradient: (d_x phi, d_y phi, valid mask)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    dx = np.zeros_like(phi); dy = np.zeros_like(phi)
    valid = np.zeros(phi.shape, dtype=np.uint8)
    pc = p.c()
    lib().orc_gradient(ctypes.byref(pc), _p(phi), _p(dx), _p(dy),
                       valid.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return dx, dy, valid.astype(bool)


TOTAL_NAMES = ("mass", "mom_x", "mom_y", "e_kin", "e_mag", "cross_hel", "bsum_x", "bsum_y",
               "divb_max", "divb_rms", "jz_max", "omega_max")


def totals(p: Params, f: np.ndarray, g: np.ndarray) -> dict:
    out = np.zeros(12)
    pc = p.c()
    if lib().orc_totals(ctypes.byref(pc), _p(f), _p(g), _p(out)) != 0:
        raise MemoryError("oracle scratch allocation failed")
    return dict(zip(TOTAL_NAMES, out.tolist()))


def threads() -> int:
    return lib().orc_threads()


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))
