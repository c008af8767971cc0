"""Failure detection without a GPU fault: the bounded device-side wait used by the step
kernel and the tensor-core FNO kernels expires, the kernel returns, the host reports
LBM_ERR_TIMEOUT, and the GPU context stays usable for the next launches."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2604_27158_gb300")
from paper_2604_27158_gb300 import _abi  # noqa: E402
from paper_2604_27158_gb300.lbm import GridSpec, Lattice, wait_selftest  # noqa: E402


def _requires_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_bounded_wait_expires_and_reports_timeout():
    _requires_gpu()
    assert wait_selftest(arrive=False, limit_ms=5.0) == _abi.LBM_ERR_TIMEOUT
    assert "expired" in _abi.lib().lbm_last_error().decode()


def test_bounded_wait_completes_when_the_barrier_completes():
    _requires_gpu()
    assert wait_selftest(arrive=True, limit_ms=5.0) == _abi.LBM_OK


def test_context_stays_usable_after_an_expired_wait():
    _requires_gpu()
    assert wait_selftest(arrive=False, limit_ms=2.0) == _abi.LBM_ERR_TIMEOUT
    solid, _, _ = synth.porous_media(64, 32, 3, 4, seed=3)
    lat = Lattice([GridSpec(64, 32, 0.7, bc_west=P.BC_PRESSURE, bc_east=P.BC_PRESSURE,
                            west_value=1.001, east_value=1.0)], [solid])
    lat.step(50)
    st = lat.residual(update_prev=True)
    assert np.all(np.isfinite(st)) and st[0, _abi.LBM_STAT_BAD] == 0
    lat.close()


def test_invalid_limits_are_rejected_on_the_host():
    _requires_gpu()
    assert wait_selftest(arrive=False, limit_ms=0.0) == _abi.LBM_ERR_INVALID_ARG
    assert wait_selftest(arrive=False, limit_ms=1e6) == _abi.LBM_ERR_INVALID_ARG
