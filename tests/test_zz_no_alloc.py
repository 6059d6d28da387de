"""The FP64 SOV entry point that allocates nothing (mvn_sov_fp64_noalloc), for callers that
cannot allocate device memory at call time (under a caching allocator that must not see
foreign cudaMalloc calls, in a real-time loop that cannot take an allocation's implicit
synchronisation, or in an embedding that only hands over device buffers).  It keeps its scratch in a fixed array inside the
library; this test checks it through the C ABI against the regular entry point (mvn_sov,
MVN_FP64) and against the CPU oracle (per-path log-weights on the same factor and lattice) on
two calls in a row, and that sizes beyond its fixed limits are refused.

Collected last on purpose (file name), so a run that stops at the first failure has run every
other test first; it also passes alone in a fresh process."""
import ctypes

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


def _factor(mvn, n, g):
    c = inputs.grid_coords(g)[:n]
    S = mvn.mvn_matern(_t(c), 1.0, 0.1, 0.5, nugget=1e-8)
    assert mvn.mvn_cholesky(S) == 0
    return S


def test_noalloc_matches_regular_entry_point_twice(mvn):
    n = 256
    L = _factor(mvn, n, 16)
    a = np.full(n, -np.inf)
    b = inputs.uniform_limits(n, -1.0, 1.0, 1)
    Ns, M = 1000, 8
    for call, seed in enumerate((11, 12)):  # two calls in a row share the fixed scratch
        lw_ref = torch.empty(Ns * M, dtype=torch.float64, device="cuda")
        ref = mvn.mvn_sov(_t(a), _t(b), L, Ns, M, seed, prec="fp64", path_logw=lw_ref)
        lw = torch.empty(Ns * M, dtype=torch.float64, device="cuda")
        got = mvn.mvn_sov_fp64_noalloc(_t(a), _t(b), L, Ns, M, seed, path_logw=lw)
        torch.cuda.synchronize()
        mvn.sync()
        g, r = lw.cpu().numpy(), lw_ref.cpu().numpy()
        assert np.all(np.abs(g - r) <= 1e-9 * np.maximum(1.0, np.abs(r))), (call, np.abs(g - r).max())
        go, ro = got.cpu().numpy(), ref.cpu().numpy()
        assert abs(go[0] - ro[0]) <= 1e-9 and abs(go[1] - ro[1]) <= 1e-10, (call, go, ro)
        assert abs(go[2] - ro[2]) <= 1e-9 * max(ro[2], 1e-300) + 1e-14
        # the oracle on the same factor and lattice: every path, and the estimate
        Lh = np.tril(L.cpu().numpy())
        lo = oracle.sov_logw(a, b, Lh, oracle.QMC(Ns, M, seed))
        assert np.all(np.abs(g - lo) <= 1e-9 * np.maximum(1.0, np.abs(lo))), (call, np.abs(g - lo).max())
        eo = oracle.estimate(lo, M)
        assert abs(go[0] - eo[0]) <= 1e-9 and abs(go[1] - eo[1]) <= 1e-10, (call, go, eo)


def test_noalloc_without_path_output_and_ragged(mvn):
    n = 77
    L = _factor(mvn, n, 9)
    rng = np.random.default_rng(3)
    a = rng.uniform(-2.0, 0.0, n)
    b = a + rng.uniform(0.5, 3.0, n)
    a[::4] = -np.inf
    for seed in (5, 6):
        ref = mvn.mvn_sov(_t(a), _t(b), L, 333, 3, seed, prec="fp64").cpu().numpy()
        got = mvn.mvn_sov_fp64_noalloc(_t(a), _t(b), L, 333, 3, seed).cpu().numpy()
        mvn.sync()
        assert abs(got[0] - ref[0]) <= 1e-9 and abs(got[1] - ref[1]) <= 1e-10


def test_noalloc_refuses_sizes_beyond_its_scratch(mvn):
    lib = mvn.lib()
    L = _factor(mvn, 256, 16)
    a = _t(np.full(257, -np.inf))
    b = _t(np.zeros(257))
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    big_n = mvn.mvn_qmc(100, 2, 0, 1, 3.0)
    P = ctypes.c_void_p
    # n = 257 > 256
    assert lib.mvn_sov_fp64_noalloc(257, P(a.data_ptr()), P(b.data_ptr()), P(L.data_ptr()), 257,
                                    ctypes.byref(big_n), P(out.data_ptr()), None, None) \
        == mvn.MVN_ERR_ARG
    # 65 shifts > 64; 262,145 paths > 262,144
    for q in (mvn.mvn_qmc(10, 65, 0, 1, 3.0), mvn.mvn_qmc(262145, 1, 0, 1, 3.0)):
        assert lib.mvn_sov_fp64_noalloc(8, P(a.data_ptr()), P(b.data_ptr()), P(L.data_ptr()), 256,
                                        ctypes.byref(q), P(out.data_ptr()), None, None) \
            == mvn.MVN_ERR_ARG
