"""CPU-only checks of the boundary and the input generators (no GPU calls).

The C-ABI library must load and export every function ``include/*.h``
declares, and the Python binding must bind each of them; the seeded input
generators must produce what their documentation states.
"""
import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(mhd_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2602_14667_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(built_lib):
    declared = _declared()
    assert "mhd_create" in declared and "mhd_advance" in declared
    missing = [n for n in sorted(declared) if not hasattr(built_lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    from paper_2602_14667_gb300 import _abi
    bound = set(_abi._SIGNATURES) | {"mhd_last_error"}
    bound |= set(getattr(_abi, "_EXTRA_SYMBOLS", ()))
    assert _declared() <= bound, sorted(_declared() - bound)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2602_14667_gb300 import _abi
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _abi.lib()


def test_library_does_not_link_the_oracle(built_lib):
    # the product library and the oracle share no code: no orc_ symbol leaks in
    from paper_2602_14667_gb300 import build
    data = open(build.LIB, "rb").read()
    assert b"orc_collide" not in data and b"orc_feq" not in data


def test_splitmix64_reference_value():
    import mhd_inputs
    # first two outputs of SplitMix64 seeded with 0 (published reference stream)
    r = mhd_inputs.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4
    u = mhd_inputs.SplitMix64(7)
    vals = [u.uniform() for _ in range(1000)]
    assert 0.0 <= min(vals) and max(vals) < 1.0 and abs(np.mean(vals) - 0.5) < 0.05


def test_orszag_tang_fields():
    import mhd_inputs
    n = 16
    ux, uy, bx, by = mhd_inputs.orszag_tang(n, 0.05, 0.04)
    x = 2 * math.pi * np.arange(n) / n
    np.testing.assert_allclose(ux[:, 0], -0.05 * np.sin(x))
    np.testing.assert_allclose(uy[0, :], 0.05 * np.sin(x))
    np.testing.assert_allclose(bx[:, 3], -0.04 * np.sin(x))
    np.testing.assert_allclose(by[5, :], 0.04 * np.sin(2 * x))


def test_random_spectrum_is_solenoidal_band_limited_and_scaled():
    import mhd_inputs
    nx, ny = 64, 48
    ux, uy, bx, by = mhd_inputs.random_spectrum(nx, ny, seed=123, rms_u=0.02, rms_b=0.03)
    for vx, vy, rms in ((ux, uy, 0.02), (bx, by, 0.03)):
        assert abs(math.sqrt(np.mean(vx ** 2 + vy ** 2)) - rms) < 1e-12
        fx, fy = np.fft.fft2(vx), np.fft.fft2(vy)
        kx = np.fft.fftfreq(nx, 1.0 / nx)[None, :]
        ky = np.fft.fftfreq(ny, 1.0 / ny)[:, None]
        div = kx * fx + ky * fy
        assert np.abs(div).max() < 1e-9 * np.abs(fx).max()
        kk = np.sqrt(kx ** 2 + ky ** 2)
        power = np.abs(fx) ** 2 + np.abs(fy) ** 2
        assert power[(kk > 8.0 + 1e-9) | (kk < 1.0 - 1e-9)].max() < 1e-20 * power.max()
    # reproducible per seed, different across seeds
    again = mhd_inputs.random_spectrum(nx, ny, seed=123, rms_u=0.02, rms_b=0.03)
    np.testing.assert_array_equal(again[0], ux)
    other = mhd_inputs.random_spectrum(nx, ny, seed=124, rms_u=0.02, rms_b=0.03)
    assert np.abs(other[0] - ux).max() > 1e-3


def test_random_spectrum_equals_direct_sum_of_modes():
    import mhd_inputs
    nx, ny, kmax = 24, 20, 5
    ux, uy, bx, by = mhd_inputs.random_spectrum(nx, ny, seed=77, rms_u=1.0, rms_b=1.0, kmax=kmax)
    rng = mhd_inputs.SplitMix64(77)
    X, Y = mhd_inputs.grid(nx, ny)
    vx = np.zeros((ny, nx)); vy = np.zeros((ny, nx))
    for kx, ky in mhd_inputs._spectral_modes(kmax):
        a = math.hypot(kx, ky) ** (-7.0 / 3.0)
        s = np.sin(kx * X + ky * Y + 2 * math.pi * rng.uniform())
        vx += -a * ky * s
        vy += a * kx * s
    scale = 1.0 / math.sqrt(np.mean(vx ** 2 + vy ** 2))
    np.testing.assert_allclose(ux, vx * scale, rtol=0, atol=1e-12)
    np.testing.assert_allclose(uy, vy * scale, rtol=0, atol=1e-12)


def test_ensemble_draws():
    import mhd_inputs
    e = mhd_inputs.ensemble(512)
    assert len(e) == 512
    assert {d["n"] for d in e} <= set(mhd_inputs.ENSEMBLE_SIZES)
    assert all(1e-4 <= d["nu"] <= 1e-2 and 1e-4 <= d["eta"] <= 1e-2 for d in e)
    assert e == mhd_inputs.ensemble(512)
    nodes = sum(d["n"] ** 2 for d in e)
    assert 2.0e7 < nodes < 6.0e7


def test_tune_cache_holds_only_valid_launch_shapes():
    """The autotuner's committed cache (read by mhd_create / mhd_autotune and
    by the benchmark) may only name shapes the library accepts: 1, 2 or 4
    nodes per thread dividing nx (at most 2 for FP64), 1..16 rows per block
    (at most 8 for FP64 and for FP16S in place), and a staging depth of 0
    (the built-in rule) or 1..64 resident warps per SM."""
    import json
    with open(os.path.join(ROOT, "paper_2602_14667_gb300", "tune_cache.json")) as fh:
        cache = json.load(fh)
    assert cache
    for key, shape in cache.items():
        assert len(shape) in (2, 3), key
        V, BY = shape[:2]
        W = shape[2] if len(shape) == 3 else 0
        assert W == 0 or 1 <= W <= 64, key
        gpu, prec, size, bc, *rest = key.split("|")
        nx = int(size.split("x")[0])
        p = int(prec[1:])
        in_place = rest == ["inplace"]
        assert rest in ([], ["inplace"]) and bc == "bc00", key
        assert V in (1, 2, 4) and nx % V == 0, key
        assert 1 <= BY <= 16, key
        if p == 0:
            assert V <= 2 and BY <= 8, key
        if p == 2 and in_place:
            assert BY <= 8, key


def test_bench_reads_profile_keys_only_for_matching_sources_and_shapes():
    """bench.py reports a kernel's measured DRAM traffic (and the FP64 and
    diagnostics instruction counts) from the committed ncu summaries only
    while their recorded source hash and launch shape match."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h != bench.kernel_source_hash(bench.DIAG_KERNEL_SOURCES)
    # a summary with the current hash and shape is read; another shape or hash is not
    tmp = os.path.join(ROOT, "profiles", f"rr_step_testonly{os.getpid()}_ncu.md")
    try:
        with open(tmp, "w") as fh:
            fh.write(f"- kernel_source_sha: `{h}`\n- shape: `4,1`\n- dram_bytes_per_node: `150.5`\n")
        name = f"testonly{os.getpid()}"
        assert bench.profiled(name, (4, 1), "dram_bytes_per_node") == 150.5
        assert bench.profiled(name, (2, 16), "dram_bytes_per_node") is None
        assert bench.profiled(name, (4, 1), "missing_key") is None
        assert bench.profiled(name, (4, 1), "dram_bytes_per_node", sources=bench.DIAG_KERNEL_SOURCES) is None
        assert bench.profiled_traffic(name, 4096, (4, 1)) == 150.5 * 4096 * 4096
    finally:
        os.remove(tmp)
    assert bench.profiled("nonexistent", (4, 1), "dram_bytes_per_node") is None


def test_launch_shapes_take_two_or_three_numbers():
    """A launch shape is (nodes_per_thread, rows_per_block[, warps_per_sm]);
    two numbers keep the built-in staging depth (warps_per_sm = 0)."""
    from paper_2602_14667_gb300 import _abi
    c = _abi._shape_in((4, 1))
    assert (c.nodes_per_thread, c.rows_per_block, c.warps_per_sm) == (4, 1, 0)
    assert _abi._shape_out(_abi._shape_in([2, 8, 16])) == (2, 8, 16)
    for bad in ((4,), (1, 2, 3, 4)):
        with pytest.raises(ValueError):
            _abi._shape_in(bad)


def test_totals_arrays_follow_the_struct_fields():
    """The batch totals as one array per field read the ctypes records field
    by field (no GPU: the records are filled here)."""
    from paper_2602_14667_gb300 import _abi
    ts = (_abi.mhd_totals * 5)()
    for i in range(5):
        for j, name in enumerate(_abi.TOTAL_FIELDS):
            setattr(ts[i], name, 100.0 * i + j)
        ts[i].step = 40 + i
    a = _abi._totals_arrays(ts)
    assert sorted(a) == sorted(_abi.TOTAL_FIELDS + ("step",))
    for j, name in enumerate(_abi.TOTAL_FIELDS):
        assert list(a[name]) == [100.0 * i + j for i in range(5)], name
    assert list(a["step"]) == [40, 41, 42, 43, 44]
    assert [_abi._totals_dict(t) for t in ts][3] == {k: v[3] for k, v in a.items()}
