"""The allocation-free diagnostics entry point (mhd_totals_noalloc).

It exists for callers that cannot allocate device memory when they need the
totals (a framework that has reserved the GPU for its own pool and lends out
only its own pointers, or a latency-critical loop that must not call
cudaMalloc).  The state lives in caller-owned device memory (here a torch
tensor); the call reduces through a scratch array compiled into the library.
Its totals must match mhd_get_totals on the same state, on two calls in a
row (the second call reuses the scratch the first one left behind).
This file is collected last so that a failure here stops a run that has
already executed every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("mass", "mom_x", "mom_y", "e_kin", "e_mag", "cross_hel", "bsum_x", "bsum_y", "divb_max",
        "divb_rms", "jz_max", "omega_max")


def _close(a, b, n):
    for k in KEYS:
        if k in ("mass", "mom_x", "mom_y", "bsum_x", "bsum_y"):
            assert abs(a[k] - b[k]) <= 1e-12 * n, (k, a[k], b[k])
        else:
            assert abs(a[k] - b[k]) <= 1e-11 * max(abs(b[k]), 1e-6), (k, a[k], b[k])


def _device_copy(buf):
    import torch
    return torch.from_numpy(buf).to("cuda")


@pytest.mark.parametrize("prec,wall_y", [("fp32", False), ("fp64", False), ("fp16s", True)])
def test_noalloc_totals_match_get_totals(prec, wall_y):
    import torch

    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice, _abi
    nx, ny = 96, 80
    fields = mhd_inputs.orszag_tang(nx, 0.05, 0.05, ny)
    stream = torch.cuda.current_stream().cuda_stream
    with Lattice(nx, ny, 0.56, 0.62, precision=prec, wall_y=wall_y) as lat:
        lat.set_fields(*fields)
        lat.advance(40)
        prev = lat.get_state()
        lat.advance(1)
        ref_gather = lat.get_totals()          # gathers g from the state step 41 read
        cur = lat.get_state()
        lat.set_state(cur)
        ref_local = lat.get_totals()           # recovers g - g_eq from the stored state
        params = lat.params
    d_cur, d_prev = _device_copy(cur), _device_copy(prev)
    torch.cuda.synchronize()
    free_before = None
    for call in range(2):                       # two calls in a row share the scratch
        got = _abi.totals_noalloc(d_cur.data_ptr(), nx, ny, params, stream=stream)
        _close(got, ref_local, nx * ny)
        got = _abi.totals_noalloc(d_cur.data_ptr(), nx, ny, params, prev_ptr=d_prev.data_ptr(),
                                  stream=stream)
        _close(got, ref_gather, nx * ny)
        if call == 0:
            # the first call on a device also looks up the scratch address (and
            # may load the library's module holding it); after that no call
            # changes the device's free memory
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_matches_get_totals_beyond_2048_squared():
    """The scratch bounds the diagnostics grid (its blocks walk the tiles),
    not the lattice: a 2304 x 2112 lattice, more nodes than 2048^2, reduces
    through the same array."""
    import torch

    import mhd_inputs
    from paper_2602_14667_gb300 import Lattice, _abi
    nx, ny = 2304, 2112
    fields = mhd_inputs.orszag_tang(nx, 0.04, 0.04, ny)
    stream = torch.cuda.current_stream().cuda_stream
    with Lattice(nx, ny, 0.53, 0.55, precision="fp32") as lat:
        lat.set_fields(*fields)
        lat.advance(5)
        prev = lat.get_state()
        lat.advance(1)
        ref = lat.get_totals()
        cur = lat.get_state()
        params = lat.params
    d_cur, d_prev = _device_copy(cur), _device_copy(prev)
    for _ in range(2):
        got = _abi.totals_noalloc(d_cur.data_ptr(), nx, ny, params, prev_ptr=d_prev.data_ptr(),
                                  stream=stream)
        _close(got, ref, nx * ny)


def test_noalloc_rejects_invalid_sizes():
    import torch

    from paper_2602_14667_gb300 import MhdError, _abi
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")  # never read: rejected first
    params = _abi.mhd_params(1.0, 0.6, 0.6, 0, 0, _abi.MHD_FP32, 0, 0, 0, 0)
    with pytest.raises(MhdError, match="too large"):
        _abi.totals_noalloc(dummy.data_ptr(), 1 << 30, 1 << 30, params)
    with pytest.raises(MhdError, match="EINVAL"):
        _abi.totals_noalloc(dummy.data_ptr(), 1, 4, params)
