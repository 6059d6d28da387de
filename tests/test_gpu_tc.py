"""Tensor-core path (MVN_MIXED): the limit-update GEMM self-test against an FP64 product, and
the mixed sweep's stated error against the FP64 path/oracle (|d log P| <= 1e-4)."""
import math

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


@pytest.mark.parametrize("K", [16, 64, 100, 640, 1000, 4100])
def test_tc_gemm_selftest(mvn, K):
    rng = np.random.default_rng(K)
    Y = rng.standard_normal((128, K)) * 1.5
    # entries spanning the magnitudes of a Cholesky factor (1 down to 1e-9), and rows of very
    # different scale (the per-row power-of-two scaling keeps the FP16 slices in range)
    L = rng.standard_normal((128, K)) * 10.0 ** rng.uniform(-9, 0, (128, K))
    L *= 10.0 ** rng.uniform(-6, 6, (128, 1))
    S = mvn.mvn_tc_selftest(_t(Y), _t(L)).cpu().numpy().astype(np.float64)
    mvn.sync()
    ref = Y @ L.T
    scale = np.abs(Y) @ np.abs(L).T
    err = np.abs(S - ref) / (scale + 1e-300)
    # two FP16 slices per operand and FP32 accumulation: ~2^-21 of the absolute-value product
    assert err.max() < 4e-6, err.max()


def _w_case(name, n_override=None):
    w = dict(inputs.WORKLOADS[name])
    c = inputs.grid_coords(w["g"])
    n = c.shape[0]
    a, b = inputs.limits_for(w, n)
    S = oracle.matern_closed(c, w["sigma2"], w["range"], w["nu"], w["nugget"])
    return w, c, a, b, S


def test_mixed_tc_error_w4(mvn):
    w, c, a, b, S = _w_case("W4")
    Lo = oracle.cholesky_lapack(S)
    L = mvn.to_colmajor(_t(Lo))
    Ntot = w["Ns"] * w["M"]
    lw64 = torch.empty(Ntot, dtype=torch.float64, device="cuda")
    lwtc = torch.empty(Ntot, dtype=torch.float64, device="cuda")
    o64 = mvn.mvn_sov(_t(a), _t(b), L, w["Ns"], w["M"], w["seed"], path_logw=lw64).cpu().numpy()
    otc = mvn.mvn_sov(_t(a), _t(b), L, w["Ns"], w["M"], w["seed"], prec="mixed",
                      path_logw=lwtc).cpu().numpy()
    mvn.sync()
    d = np.abs(lwtc.cpu().numpy() - lw64.cpu().numpy())
    print(f"W4 mixed (tcgen05): logP64={o64[0]:.8f} dlogP={otc[0] - o64[0]:.3e} "
          f"per-path median {np.median(d):.3e} max {d.max():.3e}")
    assert abs(otc[0] - o64[0]) <= 1e-4
    assert abs(otc[1] - o64[1]) <= 1e-4  # the literal |dP| criterion
    ref = oracle.sov_logw(a, b, Lo, oracle.QMC(w["Ns"], w["M"], w["seed"]), paths=(0, 8))
    assert np.all(np.abs(lw64.cpu().numpy()[:8] - ref) <= 1e-9 * np.maximum(1, np.abs(ref)))


@pytest.mark.parametrize("n,Ns,M", [(1, 50, 3), (63, 129, 2), (130, 300, 5), (300, 64, 4)])
def test_mixed_tc_ragged_vs_oracle(mvn, n, Ns, M):
    g = int(math.ceil(math.sqrt(n)))
    c = inputs.grid_coords(g)[:n]
    S = oracle.matern(c, 1.0, 0.15, 0.5, nugget=1e-6)
    rng = np.random.default_rng(n)
    a = rng.uniform(-2.5, 0.3, n)
    b = a + rng.uniform(0.2, 3.0, n)
    a[::3] = -np.inf
    b[1::4] = np.inf
    Lo, _ = oracle.cholesky(S)
    L = mvn.to_colmajor(_t(Lo))
    lw = torch.empty(Ns * M, dtype=torch.float64, device="cuda")
    out = mvn.mvn_sov(_t(a), _t(b), L, Ns, M, 3 + n, prec="mixed", path_logw=lw).cpu().numpy()
    mvn.sync()
    ref = oracle.sov_logw(a, b, Lo, oracle.QMC(Ns, M, 3 + n))
    est = oracle.estimate(ref, M)
    d = np.abs(lw.cpu().numpy() - ref)
    assert np.all(np.isfinite(lw.cpu().numpy()))
    assert abs(out[0] - est[0]) <= 1e-4, (out, est, d.max())
    # per path: each dimension's factor carries the FP32 step's error (~2e-7 relative in a',
    # times the Mills ratio) and the limit shift the two-slice GEMM's (~2^-21 of sum |L||y|),
    # accumulated over the path's n factors; stated bound 1e-6 max(1, |logw|) (measured up to
    # 3.4e-8 relative at n = 300)
    rel = d / np.maximum(1.0, np.abs(ref))
    print(f"n={n}: mixed per-path max |d logw| {d.max():.3e}, max relative {rel.max():.3e}")
    assert rel.max() <= 1e-6


def test_mixed_tc_batched_and_excursion(mvn):
    g = 12
    c = inputs.grid_coords(g)
    n = g * g
    S = oracle.matern(c, 1.0, 0.15, 0.5)
    mu = 0.9 + 0.7 * inputs.standard_normals(n, 31)
    ks = [1, 3, 17, 50, 51, 100, n]
    r = mvn.mvn_excursion(_t(mu), mvn.to_colmajor(_t(S)), 0.8, 0.9, 128, 4, 17, prefix_dims=ks,
                          prec="mixed")
    mvn.sync()
    ref = oracle.excursion(mu, S, 0.8, 0.9, oracle.QMC(128, 4, 17), prefix_dims=ks)
    assert np.array_equal(r["order"].cpu().numpy(), ref["order"])
    F = r["F"].cpu().numpy()
    assert np.all(np.abs(F - ref["F"]) <= 1e-4 * np.maximum(ref["F"], 1e-300) + 1e-12)
    Lo = ref["L"]
    L = mvn.to_colmajor(_t(Lo))
    a = 0.8 - mu[ref["order"]]
    b = np.full(n, np.inf)
    dims = [n, 64, 65, 1, 100]
    out = mvn.mvn_sov_batched(dims, [0] * 5, _t(a), _t(b), L, 128, 4, 17, prec="mixed").cpu().numpy()
    mvn.sync()
    for p, k in enumerate(dims):
        e = oracle.sov(a[:k], b[:k], Lo[:k, :k], oracle.QMC(128, 4, 17))
        assert abs(out[p, 0] - e[0]) <= 1e-4, (p, out[p], e)


# ------------------------------------------------------------------ tensor-core Cholesky (A2 mixed)

@pytest.mark.parametrize("n", [1, 63, 64, 100, 128, 130, 700, 2500])
def test_cholesky_mixed_vs_oracle(mvn, n):
    g = int(math.ceil(math.sqrt(n)))
    c = inputs.grid_coords(g)[:n]
    S = oracle.matern(c, 1.0, 0.1, 1.5, nugget=1e-4)
    A = mvn.to_colmajor(_t(S))
    assert mvn.mvn_cholesky(A, prec="mixed") == 0
    L = np.tril(A.cpu().numpy())
    Lo, _ = oracle.cholesky(S)
    bwd = np.linalg.norm(L @ L.T - S) / np.linalg.norm(S)
    print(f"n={n}: mixed Cholesky backward error {bwd:.3e}, max |L - L_oracle| "
          f"{np.abs(L - Lo).max():.3e}")
    # each digit product is exact; the digits keep x_ik = L_ik 2^-E_i to 2^-43 and the dropped
    # levels (s + t >= 6) cost another ~2^-43 per term, so one update term is off by ~2^-41
    # relative to 2^(E_i+E_j) = 4 here; over K <= 700 terms of random sign that is
    # ~sqrt(700) 2^-41 4 ~ 5e-11 at most
    assert bwd < 5e-11, bwd
    assert np.abs(L - Lo).max() < 1e-6


def test_cholesky_mixed_not_pd(mvn):
    S = oracle.matern(inputs.random_coords(300, 4), 1.0, 0.2, 0.5)
    S[200, 200] = -1.0
    A = mvn.to_colmajor(_t(S))
    with pytest.raises(mvn.MVNError) as e:
        mvn.mvn_cholesky(A, prec="mixed")
    assert e.value.status == mvn.MVN_ERR_NOT_PD
    B = mvn.to_colmajor(_t(np.eye(3) * 4.0))
    assert mvn.mvn_cholesky(B, prec="mixed") == 0
    assert abs(B.cpu().numpy()[2, 2] - 2.0) < 1e-15


def test_cholesky_mixed_w2_full_size(mvn):
    """W2 (n=16,384): tensor-core factor of the GPU covariance vs the oracle covariance (backward
    error by random matrix-vector products) and its effect on the W2 log P against the FP64
    factor on identical lattice points (the stated bound |d log P| <= 1e-4)."""
    w = dict(inputs.WORKLOADS["W2"])
    c = inputs.grid_coords(w["g"])
    n = c.shape[0]
    a, b = inputs.limits_for(w, n)
    So = oracle.matern_closed(c, w["sigma2"], w["range"], w["nu"], w["nugget"])
    S = mvn.mvn_matern(_t(c), w["sigma2"], w["range"], w["nu"], w["nugget"])
    S64 = S.clone()
    assert mvn.mvn_cholesky(S, prec="mixed") == 0
    assert mvn.mvn_cholesky(S64, prec="fp64") == 0
    Lg = torch.tril(S)
    rng = np.random.default_rng(1)
    for _ in range(3):
        v = rng.standard_normal(n)
        LLv = (Lg @ (Lg.t() @ _t(v))).cpu().numpy()
        Sv = So @ v
        bwd = np.linalg.norm(LLv - Sv) / np.linalg.norm(Sv)
        # products carry 42 bits (2^-42 ~ 2.3e-13) relative to the row maxima; accumulated over
        # n = 16,384 terms the bound is ~n 2^-43 ~ 2e-9
        assert bwd < 5e-10, bwd
    del Lg
    Ns, M = 200, 10
    o_mx = mvn.mvn_sov(_t(a), _t(b), S, Ns, M, w["seed"], prec="fp64").cpu().numpy()
    o_64 = mvn.mvn_sov(_t(a), _t(b), S64, Ns, M, w["seed"], prec="fp64").cpu().numpy()
    mvn.sync()
    print(f"W2 log P with tensor-core factor {o_mx[0]:.10f} vs FP64 factor {o_64[0]:.10f}")
    assert abs(o_mx[0] - o_64[0]) <= 1e-4
