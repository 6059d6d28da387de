"""Failure detection without a GPU fault: a bounded device wait made to run out (nothing
completes the barrier) reports MVN_ERR_TIMEOUT through the status word and leaves the context
usable; an injected workspace-allocation failure (host side) returns MVN_ERR_OOM; a non-PD matrix
returns the LAPACK-style column; invalid limits are reported by the device check."""
import os

import numpy as np
import pytest

import oracle
from paper_2405_14892_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mvn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_14892_gb300 import mvn as m
    return m


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _small(mvn):
    c = inputs.grid_coords(5)
    S = mvn.mvn_matern(_t(c), 1.0, 0.2, 0.5)
    assert mvn.mvn_cholesky(S) == 0
    return S, np.full(25, -np.inf), np.full(25, 0.5)


def test_bounded_wait_times_out_and_context_survives(mvn):
    c = mvn.context()
    assert mvn.lib().mvn_wait_selftest(c.h, 2_000_000) == mvn.MVN_OK  # ~1 ms budget
    st, _ = c.sync()
    assert st == mvn.MVN_ERR_TIMEOUT
    S, a, b = _small(mvn)
    out = mvn.mvn_sov(_t(a), _t(b), S, 64, 2, 1).cpu().numpy()
    assert mvn.sync() == 0 and np.isfinite(out[0])
    assert mvn.lib().mvn_wait_selftest(c.h, 10) == mvn.MVN_ERR_ARG


def test_workspace_allocation_failure_injection(mvn):
    S, a, b = _small(mvn)
    fresh = mvn.Context(torch.cuda.current_device())  # empty workspace
    import ctypes
    q = mvn._qmc(64, 2, 1)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    ad, bd = _t(a), _t(b)  # kept alive for the calls below
    args = (fresh.h, 25, mvn._P(ad.data_ptr()), mvn._P(bd.data_ptr()),
            mvn._P(S.data_ptr()), 25, ctypes.byref(q), 0, mvn._P(out.data_ptr()), None)
    os.environ["MVN_FAULT_WS_ALLOC"] = "1"
    try:
        assert mvn.lib().mvn_sov(*args) == mvn.MVN_ERR_OOM
        assert b"injected" in mvn.lib().mvn_last_error(fresh.h)
    finally:
        del os.environ["MVN_FAULT_WS_ALLOC"]
    assert mvn.lib().mvn_sov(*args) == mvn.MVN_OK
    assert fresh.sync()[0] == mvn.MVN_OK
    fresh.close()


def test_invalid_limits_reported_by_device_check(mvn):
    S, a, b = _small(mvn)
    b[7] = -1.0
    a[7] = 0.0      # a > b
    mvn.mvn_sov(_t(a), _t(b), S, 64, 2, 1)
    st, info = mvn.context().sync()
    assert st == mvn.MVN_ERR_ARG and info == 8
    assert mvn.sync() == 0  # cleared
