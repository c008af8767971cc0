"""lbm_residual_static: the residual statistics for callers that cannot allocate
device memory when they need them (their device memory belongs to another
allocator, or their runtime forbids allocation after start-up).

It must return what lbm_residual returns on the same state, call after call,
although its scratch lives in one array compiled into the library that every
call reuses.  This file is collected last so that a failure here does not hide
any other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2604_27158_gb300")
from paper_2604_27158_gb300 import _abi  # noqa: E402
from paper_2604_27158_gb300.lbm import GridSpec, Lattice, _stream_ptr  # noqa: E402


def _requires_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _static_call(lat, update_prev):
    lib = _abi.lib()
    fn = lib.lbm_residual_static
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    out = np.zeros((len(lat.grids), _abi.LBM_NSTAT), dtype=np.float64)
    code = fn(lat.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(update_prev),
              _stream_ptr(None))
    return code, out


def _lattice():
    specs = []
    for k in range(3):
        solid, _, _ = synth.porous_media(96, 48, 3, 5, seed=20 + k)
        specs.append((GridSpec(96, 48, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                               west_value=1.001, east_value=1.0), solid))
    solid, _ = synth.channel_with_disks(70, 30, 2, 3, 4, seed=3)
    specs.append((GridSpec(70, 30, 0.8, fx=1e-5), solid))
    return Lattice([a for a, _ in specs], [b for _, b in specs])


def test_static_scratch_residual_matches_workspace_residual():
    _requires_gpu()
    lat = _lattice()
    lat.step(100)
    lat.residual(update_prev=True)       # u_prev <- u(100)
    lat.step(50)
    for _ in range(2):                   # two calls in a row on the same state
        code, got = _static_call(lat, update_prev=0)
        assert code == _abi.LBM_OK, _abi.last_error()
        want = lat.residual(update_prev=False)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0.0)
        assert np.all(got[:, _abi.LBM_STAT_RESIDUAL] > 0)
    # the static variant updates the stored velocity like lbm_residual does
    code, got = _static_call(lat, update_prev=1)
    assert code == _abi.LBM_OK
    after = lat.residual(update_prev=False)
    assert np.all(after[:, _abi.LBM_STAT_RESIDUAL] == 0.0)
    lat.step(30)
    for _ in range(2):
        code, got = _static_call(lat, update_prev=0)
        assert code == _abi.LBM_OK
        np.testing.assert_allclose(got, lat.residual(update_prev=False), rtol=1e-12, atol=0.0)


def test_static_scratch_rejects_batches_beyond_its_size():
    _requires_gpu()
    # 5000 x 5000 cells are 200,000 row segments of 128 cells: ~9.6 MB of partials, more than
    # the 4 MiB array holds
    lat = Lattice([GridSpec(5000, 5000, 0.8)], [np.zeros((5000, 5000), bool)])
    code, _ = _static_call(lat, update_prev=0)
    assert code == _abi.LBM_ERR_INVALID_ARG
    assert "static array" in _abi.last_error()
