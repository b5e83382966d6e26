"""ctypes binding of ``libmhdlbm.so`` (the C ABI in ``include/mhd.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built --
there is no CPU fallback.  Functions keep the C names (``mhd_create``, ...);
``Lattice`` is a small owner object over them that converts numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmhdlbm.so")

MHD_OK, MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA, MHD_EUNSTABLE, MHD_ESTATE = range(6)
MHD_FP64, MHD_FP32, MHD_FP16S = range(3)
MHD_PERIODIC, MHD_WALL, MHD_HALO = range(3)
MHD_RR, MHD_BGK = range(2)
MHD_MAG_BGK, MHD_MAG_REGULARISED = range(2)
MHD_TWO_BUFFERS, MHD_IN_PLACE = range(2)
STATUS_NAMES = {0: "MHD_OK", 1: "MHD_EINVAL", 2: "MHD_ENOMEM", 3: "MHD_ECUDA", 4: "MHD_EUNSTABLE",
                5: "MHD_ESTATE"}
PRECISIONS = {"fp64": MHD_FP64, "fp32": MHD_FP32, "fp16s": MHD_FP16S}


class mhd_params(ctypes.Structure):
    _fields_ = [("rho0", ctypes.c_double), ("tau_f", ctypes.c_double), ("tau_m", ctypes.c_double),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int), ("precision", ctypes.c_int),
                ("eq_variant", ctypes.c_int), ("collision", ctypes.c_int),
                ("mag_collision", ctypes.c_int), ("streaming", ctypes.c_int)]


TOTAL_FIELDS = ("mass", "mom_x", "mom_y", "e_kin", "e_mag", "cross_hel", "bsum_x", "bsum_y",
                "divb_max", "divb_rms", "jz_max", "omega_max")


class mhd_totals(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in TOTAL_FIELDS] + [("step", ctypes.c_longlong)]


class mhd_kernel_config(ctypes.Structure):
    _fields_ = [("nodes_per_thread", ctypes.c_int), ("rows_per_block", ctypes.c_int),
                ("warps_per_sm", ctypes.c_int)]


def _shape_in(v) -> "mhd_kernel_config":
    """(nodes_per_thread, rows_per_block[, warps_per_sm]) -> the C struct;
    a two-number shape keeps the built-in staging depth (warps_per_sm 0)."""
    v = tuple(int(x) for x in v)
    if len(v) not in (2, 3):
        raise ValueError("a launch shape is (nodes_per_thread, rows_per_block[, warps_per_sm])")
    return mhd_kernel_config(v[0], v[1], v[2] if len(v) == 3 else 0)


def _shape_out(c: "mhd_kernel_config"):
    return c.nodes_per_thread, c.rows_per_block, c.warps_per_sm


class MhdError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)

_SIGNATURES = {
    "mhd_create": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(mhd_params), _P, ctypes.POINTER(_P)],
    "mhd_set_fields": [_P, _D, _D, _D, _D, _D],
    "mhd_advance": [_P, ctypes.c_longlong],
    "mhd_get_fields": [_P, _D, _D, _D, _D, _D],
    "mhd_set_fields_f32": [_P, _F, _F, _F, _F, _F],
    "mhd_get_fields_f32": [_P, _F, _F, _F, _F, _F],
    "mhd_get_totals": [_P, ctypes.POINTER(mhd_totals)],
    "mhd_advance_totals": [_P, ctypes.c_longlong, ctypes.POINTER(mhd_totals)],
    "mhd_get_populations": [_P, _D, _D],
    "mhd_set_populations": [_P, _D, _D],
    "mhd_get_kernel_config": [_P, ctypes.POINTER(mhd_kernel_config)],
    "mhd_set_kernel_config": [_P, ctypes.POINTER(mhd_kernel_config)],
    "mhd_autotune": [_P, ctypes.POINTER(mhd_kernel_config)],
    "mhd_destroy": [_P],
    "mhd_state_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "mhd_slab_exchange": [_P, _P, ctypes.c_int],
    "mhd_slab_group_create": [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)],
    "mhd_slab_group_advance": [_P, ctypes.c_longlong],
    "mhd_slab_group_destroy": [_P],
    "mhd_totals_noalloc": [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(mhd_params), _P,
                           ctypes.POINTER(mhd_totals)],
    "mhd_batch_create": [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(mhd_params), _P, ctypes.POINTER(_P)],
    "mhd_batch_set_fields": [_P, ctypes.c_int, _D, _D, _D, _D, _D],
    "mhd_batch_advance": [_P, ctypes.c_longlong],
    "mhd_batch_get_fields": [_P, ctypes.c_int, _D, _D, _D, _D, _D],
    "mhd_batch_get_totals": [_P, ctypes.c_int, ctypes.POINTER(mhd_totals)],
    "mhd_batch_get_all_totals": [_P, ctypes.POINTER(mhd_totals)],
    "mhd_batch_advance_totals": [_P, ctypes.c_longlong, ctypes.POINTER(mhd_totals)],
    "mhd_batch_nodes": [_P, ctypes.POINTER(ctypes.c_longlong)],
    "mhd_batch_get_kernel_config": [_P, ctypes.POINTER(mhd_kernel_config)],
    "mhd_batch_set_kernel_config": [_P, ctypes.POINTER(mhd_kernel_config)],
    "mhd_batch_autotune": [_P, ctypes.POINTER(mhd_kernel_config)],
    "mhd_batch_destroy": [_P],
    "mhd_mlp_create": [ctypes.c_ulonglong, ctypes.c_int, _P, ctypes.POINTER(_P)],
    "mhd_mlp_destroy": [_P],
    "mhd_mlp_get_params": [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t],
    "mhd_mlp_set_params": [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t],
    "mhd_mlp_fit_normalisation": [_P, _P, _P, ctypes.c_longlong],
    "mhd_mlp_gradients": [_P, _P, _P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_float),
                          ctypes.POINTER(ctypes.c_double)],
    "mhd_mlp_train": [_P, _P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                      ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double)],
    "mhd_mlp_predict": [_P, _P, ctypes.c_longlong, _P],
    "mhd_closure_filter": [_P, ctypes.c_int, _P],
    "mhd_closure_features": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P],
    "mhd_closure_targets": [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _P, _P],
    "mhd_set_precollision_state": [_P, _P],
    "mhd_set_closure_kernel": [_P, ctypes.c_int],
    "mhd_get_closure_kernel": [_P, ctypes.POINTER(ctypes.c_int)],
    "mhd_set_closure_interval": [_P, ctypes.c_int],
    "mhd_get_closure_interval": [_P, ctypes.POINTER(ctypes.c_int)],
    "mhd_closure_sgs_targets": [_P, ctypes.c_int, ctypes.c_double, _P],
    "mhd_set_closure": [_P, _P],
    "mhd_get_state": [_P, _P, ctypes.c_size_t],
    "mhd_set_state": [_P, _P, ctypes.c_size_t],
}


def lib() -> ctypes.CDLL:
    """Load the library (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        l = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(l, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        l.mhd_last_error.argtypes = []
        l.mhd_last_error.restype = ctypes.c_char_p
        _lib = l
    return _lib


def check(status: int, where: str) -> None:
    if status != MHD_OK:
        raise MhdError(status, where, lib().mhd_last_error().decode())


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _fptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_F)


def _in(a, n):
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr


class Lattice:
    """One nx x ny lattice on the current CUDA device (owner of the C handle)."""

    def __init__(self, nx: int, ny: int, tau_f: float, tau_m: float, precision="fp32",
                 rho0: float = 1.0, wall_x: bool = False, wall_y: bool = False, eq_variant: int = 0,
                 collision: int = MHD_RR, stream=None, mag_collision: int = MHD_MAG_BGK,
                 in_place: bool = False, halo_y: bool = False):
        self.nx, self.ny = int(nx), int(ny)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        bc_y = MHD_HALO if halo_y else int(wall_y)
        self.params = mhd_params(rho0, tau_f, tau_m, int(wall_x), bc_y, prec, eq_variant,
                                 collision, mag_collision, MHD_IN_PLACE if in_place else MHD_TWO_BUFFERS)
        self._h = _P()
        s = None if stream is None else _P(int(stream))
        check(lib().mhd_create(self.nx, self.ny, ctypes.byref(self.params), s, ctypes.byref(self._h)),
              "mhd_create")

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            check(lib().mhd_destroy(self._h), "mhd_destroy")
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_fields(self, ux, uy, bx, by, rho=None):
        """Initial equilibrium from u, b (and rho); float32 arrays (all of
        them C-contiguous float32) go through mhd_set_fields_f32, anything
        else is converted to float64 for mhd_set_fields."""
        given = [a for a in (ux, uy, bx, by, rho) if a is not None]
        if all(isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"] for a in given):
            for a in given:
                if a.size != self.n:
                    raise ValueError(f"expected {self.n} values, got {a.size}")
            check(lib().mhd_set_fields_f32(self._h, *[_fptr(a) for a in (ux, uy, bx, by, rho)]),
                  "mhd_set_fields_f32")
            return
        arrs = [_in(a, self.n) for a in (ux, uy, bx, by)]
        r = None if rho is None else _in(rho, self.n)
        check(lib().mhd_set_fields(self._h, *[_dptr(a) for a in arrs], _dptr(r)), "mhd_set_fields")

    def advance(self, nsteps: int):
        check(lib().mhd_advance(self._h, int(nsteps)), "mhd_advance")

    def get_fields(self, out=None, dtype=np.float64):
        """rho, ux, uy, bx, by as a dict of float64 (or float32: dtype, or
        float32 `out` arrays, read through mhd_get_fields_f32); `out` may give
        five C-contiguous arrays of nx*ny, all of one of the two types, to
        fill instead (e.g. pinned host memory)."""
        if out is None:
            out = [np.empty((self.ny, self.nx), dtype=dtype) for _ in range(5)]
        dt = out[0].dtype
        if dt not in (np.float64, np.float32):
            raise ValueError("out arrays must be float64 or float32")
        for a in out:
            if a.dtype != dt or not a.flags["C_CONTIGUOUS"] or a.size != self.n:
                raise ValueError("out arrays must be C-contiguous, of one type, with nx*ny values")
        if dt == np.float32:
            check(lib().mhd_get_fields_f32(self._h, *[_fptr(a) for a in out]), "mhd_get_fields_f32")
        else:
            check(lib().mhd_get_fields(self._h, *[_dptr(a) for a in out]), "mhd_get_fields")
        return dict(zip(("rho", "ux", "uy", "bx", "by"), out))

    def get_totals(self, check_stable: bool = True) -> dict:
        t = mhd_totals()
        st = lib().mhd_get_totals(self._h, ctypes.byref(t))
        if st != MHD_EUNSTABLE or check_stable:
            check(st, "mhd_get_totals")
        d = {n: getattr(t, n) for n in TOTAL_FIELDS}
        d["step"] = t.step
        return d

    def advance_totals(self, nsteps: int, check_stable: bool = True) -> dict:
        """mhd_advance_totals: advance, the last step reducing the point
        totals (divb_max, divb_rms, omega_max are NaN on the fused path)."""
        t = mhd_totals()
        st = lib().mhd_advance_totals(self._h, int(nsteps), ctypes.byref(t))
        if st != MHD_EUNSTABLE or check_stable:
            check(st, "mhd_advance_totals")
        d = {n: getattr(t, n) for n in TOTAL_FIELDS}
        d["step"] = t.step
        return d

    def get_populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((5, 2, self.ny, self.nx))
        check(lib().mhd_get_populations(self._h, _dptr(f), _dptr(g)), "mhd_get_populations")
        return f, g

    def set_populations(self, f, g):
        fa = _in(f, 9 * self.n)
        ga = _in(g, 10 * self.n)
        check(lib().mhd_set_populations(self._h, _dptr(fa), _dptr(ga)), "mhd_set_populations")

    def get_state(self) -> np.ndarray:
        """Bitwise checkpoint of the stored planes (raw bytes, uint8)."""
        nb = ctypes.c_size_t()
        check(lib().mhd_state_bytes(self._h, ctypes.byref(nb)), "mhd_state_bytes")
        buf = np.empty(nb.value, dtype=np.uint8)
        check(lib().mhd_get_state(self._h, buf.ctypes.data_as(_P), nb.value), "mhd_get_state")
        return buf

    def set_state(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(lib().mhd_set_state(self._h, buf.ctypes.data_as(_P), buf.size), "mhd_set_state")

    @property
    def kernel_config(self):
        c = mhd_kernel_config()
        check(lib().mhd_get_kernel_config(self._h, ctypes.byref(c)), "mhd_get_kernel_config")
        return _shape_out(c)

    @kernel_config.setter
    def kernel_config(self, v):
        c = _shape_in(v)
        check(lib().mhd_set_kernel_config(self._h, ctypes.byref(c)), "mhd_set_kernel_config")

    def autotune(self):
        c = mhd_kernel_config()
        check(lib().mhd_autotune(self._h, ctypes.byref(c)), "mhd_autotune")
        return _shape_out(c)


def slab_exchange(lower: "Lattice", upper: "Lattice", all_planes: bool = False) -> None:
    """mhd_slab_exchange: fill the ghost rows across the boundary between two
    neighbouring slabs (lower: the rows just below upper)."""
    check(lib().mhd_slab_exchange(lower.handle, upper.handle, int(all_planes)), "mhd_slab_exchange")


class SlabSteps:
    """mhd_slab_group_*: the slabs of one lattice (in order along y, on one
    device and one stream) stepped together, every round's exchanges in one
    kernel and runs of 64 rounds in one CUDA graph.  Borrows the lattices."""

    def __init__(self, lattices):
        self.lattices = list(lattices)
        arr = (_P * len(self.lattices))(*[l.handle for l in self.lattices])
        self._h = _P()
        check(lib().mhd_slab_group_create(arr, len(self.lattices), ctypes.byref(self._h)), "mhd_slab_group_create")

    def advance(self, nsteps: int):
        check(lib().mhd_slab_group_advance(self._h, int(nsteps)), "mhd_slab_group_advance")

    def close(self):
        if self._h:
            check(lib().mhd_slab_group_destroy(self._h), "mhd_slab_group_destroy")
            self._h = _P()


def totals_noalloc(state_ptr: int, nx: int, ny: int, params: "mhd_params", prev_ptr=None,
                   stream=None) -> dict:
    """mhd_totals_noalloc on caller-owned device memory (integer device
    pointers, e.g. ``tensor.data_ptr()``); allocates nothing."""
    t = mhd_totals()
    check(lib().mhd_totals_noalloc(_P(int(state_ptr)), None if prev_ptr is None else _P(int(prev_ptr)),
                                   int(nx), int(ny), ctypes.byref(params),
                                   None if stream is None else _P(int(stream)), ctypes.byref(t)),
          "mhd_totals_noalloc")
    return _totals_dict(t)


def _totals_arrays(ts) -> dict:
    """A ctypes array of mhd_totals as one numpy array per field."""
    dt = np.dtype([(n, np.float64 if t is ctypes.c_double else np.int64) for n, t in mhd_totals._fields_])
    assert dt.itemsize == ctypes.sizeof(mhd_totals)
    a = np.frombuffer(ts, dtype=dt)
    return {n: a[n].copy() for n in TOTAL_FIELDS + ("step",)}


def _totals_dict(t: "mhd_totals") -> dict:
    d = {n: getattr(t, n) for n in TOTAL_FIELDS}
    d["step"] = t.step
    return d


class Batch:
    """Ensemble of independent periodic FP32 lattices advanced by one
    persistent kernel launch per step (owner of the C handle).
    sizes: list of (nx, ny); taus: list of (tau_f, tau_m)."""

    def __init__(self, sizes, taus, rho0: float = 1.0, eq_variant: int = 0, collision: int = MHD_RR,
                 stream=None, mag_collision: int = MHD_MAG_BGK):
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        n = len(self.sizes)
        if len(taus) != n:
            raise ValueError("one (tau_f, tau_m) per lattice")
        nx = (ctypes.c_int * n)(*[s[0] for s in self.sizes])
        ny = (ctypes.c_int * n)(*[s[1] for s in self.sizes])
        ps = (mhd_params * n)(*[mhd_params(rho0, tf, tm, MHD_PERIODIC, MHD_PERIODIC, MHD_FP32, eq_variant,
                                           collision, mag_collision, MHD_TWO_BUFFERS) for tf, tm in taus])
        self._h = _P()
        s = None if stream is None else _P(int(stream))
        check(lib().mhd_batch_create(n, nx, ny, ps, s, ctypes.byref(self._h)), "mhd_batch_create")

    def __len__(self):
        return len(self.sizes)

    @property
    def handle(self):
        return self._h

    @property
    def nodes(self) -> int:
        v = ctypes.c_longlong()
        check(lib().mhd_batch_nodes(self._h, ctypes.byref(v)), "mhd_batch_nodes")
        return v.value

    def close(self):
        if self._h:
            check(lib().mhd_batch_destroy(self._h), "mhd_batch_destroy")
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_fields(self, i, ux, uy, bx, by, rho=None):
        nx, ny = self.sizes[i]
        arrs = [_in(a, nx * ny) for a in (ux, uy, bx, by)]
        r = None if rho is None else _in(rho, nx * ny)
        check(lib().mhd_batch_set_fields(self._h, int(i), *[_dptr(a) for a in arrs], _dptr(r)),
              "mhd_batch_set_fields")

    def advance(self, nsteps: int):
        check(lib().mhd_batch_advance(self._h, int(nsteps)), "mhd_batch_advance")

    def get_fields(self, i):
        nx, ny = self.sizes[i]
        out = [np.empty((ny, nx)) for _ in range(5)]
        check(lib().mhd_batch_get_fields(self._h, int(i), *[_dptr(a) for a in out]), "mhd_batch_get_fields")
        return dict(zip(("rho", "ux", "uy", "bx", "by"), out))

    def get_totals(self, i) -> dict:
        t = mhd_totals()
        check(lib().mhd_batch_get_totals(self._h, int(i), ctypes.byref(t)), "mhd_batch_get_totals")
        return _totals_dict(t)

    def advance_totals(self, nsteps: int, as_arrays: bool = False):
        """mhd_batch_advance_totals: advance, the last step reducing every
        lattice's point totals (divb_max, divb_rms, omega_max are NaN): a
        list of dicts, or with as_arrays one array per field."""
        ts = (mhd_totals * len(self.sizes))()
        check(lib().mhd_batch_advance_totals(self._h, int(nsteps), ts), "mhd_batch_advance_totals")
        return _totals_arrays(ts) if as_arrays else [_totals_dict(t) for t in ts]

    def get_all_totals(self, as_arrays: bool = False):
        """mhd_batch_get_all_totals: the totals of every lattice, one wait;
        a list of dicts, or with as_arrays one array per field."""
        ts = (mhd_totals * len(self.sizes))()
        check(lib().mhd_batch_get_all_totals(self._h, ts), "mhd_batch_get_all_totals")
        return _totals_arrays(ts) if as_arrays else [_totals_dict(t) for t in ts]

    @property
    def kernel_config(self):
        c = mhd_kernel_config()
        check(lib().mhd_batch_get_kernel_config(self._h, ctypes.byref(c)), "mhd_batch_get_kernel_config")
        return _shape_out(c)

    @kernel_config.setter
    def kernel_config(self, v):
        c = _shape_in(v)
        check(lib().mhd_batch_set_kernel_config(self._h, ctypes.byref(c)), "mhd_batch_set_kernel_config")

    def autotune(self):
        c = mhd_kernel_config()
        check(lib().mhd_batch_autotune(self._h, ctypes.byref(c)), "mhd_batch_autotune")
        return _shape_out(c)


MLP_PARAMS = 6006


def _ptr(t) -> "_P":
    """Device pointer of a torch tensor (or an int address)."""
    return _P(int(t) if isinstance(t, int) else t.data_ptr())


class MLP:
    """The closure network (owner of the C handle); tensors are torch CUDA tensors."""

    def __init__(self, seed: int = 0, max_batch: int = 16384, stream=None):
        self._h = _P()
        self.stream = stream
        check(lib().mhd_mlp_create(int(seed), int(max_batch), None if stream is None else _P(int(stream)),
                                   ctypes.byref(self._h)), "mhd_mlp_create")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            check(lib().mhd_mlp_destroy(self._h), "mhd_mlp_destroy")
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def get_params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        check(lib().mhd_mlp_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size),
              "mhd_mlp_get_params")
        return out

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        check(lib().mhd_mlp_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
              "mhd_mlp_set_params")

    def fit_normalisation(self, X, T):
        check(lib().mhd_mlp_fit_normalisation(self._h, _ptr(X), _ptr(T), X.shape[0]), "mhd_mlp_fit_normalisation")

    def gradients(self, X, T):
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        check(lib().mhd_mlp_gradients(self._h, _ptr(X), _ptr(T), X.shape[0],
                                      g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)),
              "mhd_mlp_gradients")
        return loss.value, g

    def train(self, X, T, epochs=10, batch=8192, lr=1e-3, seed=0) -> float:
        loss = ctypes.c_double()
        check(lib().mhd_mlp_train(self._h, _ptr(X), _ptr(T), X.shape[0], int(epochs), int(batch), float(lr),
                                  int(seed), ctypes.byref(loss)), "mhd_mlp_train")
        return loss.value

    def predict(self, X, Y):
        check(lib().mhd_mlp_predict(self._h, _ptr(X), X.shape[0], _ptr(Y)), "mhd_mlp_predict")


def closure_filter(lattice: "Lattice", factor: int, out):
    check(lib().mhd_closure_filter(lattice.handle, int(factor), _ptr(out)), "mhd_closure_filter")


def closure_features(state, nx, ny, rho0, X, stream=None):
    check(lib().mhd_closure_features(_ptr(state), int(nx), int(ny), float(rho0), _ptr(X),
                                     None if stream is None else _P(int(stream))), "mhd_closure_features")


def closure_targets(state_t, state_t1, nx, ny, rho0, tau_f, T, stream=None):
    check(lib().mhd_closure_targets(_ptr(state_t), _ptr(state_t1), int(nx), int(ny), float(rho0),
                                    float(tau_f), _ptr(T), None if stream is None else _P(int(stream))),
          "mhd_closure_targets")


def closure_sgs_targets(lattice: "Lattice", factor: int, tau_coarse: float, out):
    check(lib().mhd_closure_sgs_targets(lattice.handle, int(factor), float(tau_coarse), _ptr(out)),
          "mhd_closure_sgs_targets")


def set_precollision_state(lattice: "Lattice", state):
    check(lib().mhd_set_precollision_state(lattice.handle, _ptr(state)), "mhd_set_precollision_state")


MHD_CLOSURE_WARP_MMA, MHD_CLOSURE_TCGEN05 = range(2)


def set_closure_kernel(lattice: "Lattice", kind: int):
    """MLP kernel of the closure step: MHD_CLOSURE_WARP_MMA or MHD_CLOSURE_TCGEN05."""
    check(lib().mhd_set_closure_kernel(lattice.handle, int(kind)), "mhd_set_closure_kernel")


def get_closure_kernel(lattice: "Lattice") -> int:
    k = ctypes.c_int()
    check(lib().mhd_get_closure_kernel(lattice.handle, ctypes.byref(k)), "mhd_get_closure_kernel")
    return k.value


def set_closure_interval(lattice: "Lattice", k: int):
    """Evaluate the closure MLP on every k-th step and reuse its stored
    correction on the steps between (mhd_set_closure_interval)."""
    check(lib().mhd_set_closure_interval(lattice.handle, int(k)), "mhd_set_closure_interval")


def get_closure_interval(lattice: "Lattice") -> int:
    k = ctypes.c_int()
    check(lib().mhd_get_closure_interval(lattice.handle, ctypes.byref(k)), "mhd_get_closure_interval")
    return k.value


def set_closure(lattice: "Lattice", mlp):
    check(lib().mhd_set_closure(lattice.handle, None if mlp is None else mlp.handle), "mhd_set_closure")
