"""Adjoints on the GPU vs the oracle and vs central finite differences (workload W4):
the reverse SOV sweep (d log P / d a, b, L), the blocked Cholesky adjoint, the Matern
contraction, and the autograd.Function chain d log P / d (b, sigma2, range)."""
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


@pytest.mark.parametrize("n", [1, 7, 64, 200, 333])
def test_cholesky_grad_vs_oracle(mvn, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    S = A @ A.T / n + np.eye(n)
    Lo, _ = oracle.cholesky(S)
    G = np.tril(rng.standard_normal((n, n)))
    ref = oracle.cholesky_grad(Lo, G)
    L = mvn.to_colmajor(_t(Lo))
    Gd = mvn.to_colmajor(_t(G))
    mvn.mvn_cholesky_grad(L, Gd)
    mvn.sync()
    got = np.tril(Gd.cpu().numpy())
    err = np.abs(got - ref).max() / max(1.0, np.abs(ref).max())
    assert err < 1e-11, err


def _problem(n, seed, finite_a=True):
    g = int(math.ceil(math.sqrt(n)))
    c = inputs.grid_coords(g)[:n]
    S = oracle.matern(c, 1.0, 0.25, 1.5, nugget=1e-3)
    rng = np.random.default_rng(seed)
    a = rng.uniform(-2, 0, n)
    if finite_a:
        a[::2] = -np.inf
    else:
        a[:] = -np.inf
    b = a + rng.uniform(1, 3, n)
    inf = np.isinf(a)
    b[inf] = rng.uniform(-0.5, 1.5, np.count_nonzero(inf))
    b[3::7] = np.inf
    return S, a, b


@pytest.mark.parametrize("n,Ns,M", [(1, 64, 4), (20, 100, 3), (37, 129, 2), (150, 64, 4)])
def test_sov_grad_vs_oracle(mvn, n, Ns, M):
    S, a, b = _problem(n, n)
    Lo, _ = oracle.cholesky(S)
    q = oracle.QMC(Ns, M, 5 + n)
    logP, ga, gb, gL = oracle.sov_grad(a, b, Lo, q)
    L = mvn.to_colmajor(_t(Lo))
    out3, ga_g, gb_g, gL_g = mvn.mvn_sov_grad(_t(a), _t(b), L, Ns, M, 5 + n, want_L=True)
    mvn.sync()
    assert abs(out3.cpu().numpy()[0] - logP) < 1e-9
    scale = max(1.0, np.abs(gb).max(), np.abs(ga).max())
    np.testing.assert_allclose(ga_g.cpu().numpy(), ga, atol=1e-9 * scale)
    np.testing.assert_allclose(gb_g.cpu().numpy(), gb, atol=1e-9 * scale)
    gLg = np.tril(gL_g.cpu().numpy())
    assert np.abs(gLg - np.tril(gL)).max() <= 1e-9 * max(1.0, np.abs(gL).max())


@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_matern_grad_vs_oracle(mvn, nu):
    c = inputs.random_coords(150, 7)
    Sb = np.tril(np.random.default_rng(8).standard_normal((150, 150)))
    ref = oracle.matern_theta_grad(Sb, c, 1.3, 0.2, nu)
    got = mvn.mvn_matern_grad(_t(c), 1.3, 0.2, nu, mvn.to_colmajor(_t(Sb))).cpu().numpy()
    mvn.sync()
    np.testing.assert_allclose(got, ref, rtol=1e-11)


def test_theta_chain_small_vs_oracle(mvn):
    """The whole chain (SOV adjoint -> Cholesky adjoint -> Matern contraction) on a 6 x 6 grid
    against the oracle's chain."""
    from paper_2405_14892_gb300.autograd import mvn_log_prob
    g = 6
    c = inputs.grid_coords(g)
    n = g * g
    b = np.full(n, 0.5)
    q = oracle.QMC(128, 4, 21)
    s2, rg = 1.0, 0.3
    Lo, _ = oracle.cholesky(oracle.matern(c, s2, rg, 1.5, nugget=1e-4))
    logP, ga, gb, gL = oracle.sov_grad(np.full(n, -np.inf), b, Lo, q)
    Sbar = oracle.cholesky_grad(Lo, gL)
    th = oracle.matern_theta_grad(Sbar, c, s2, rg, 1.5)
    bt = _t(b).requires_grad_(True)
    s2t = torch.tensor(s2, dtype=torch.float64, device="cuda", requires_grad=True)
    rgt = torch.tensor(rg, dtype=torch.float64, device="cuda", requires_grad=True)
    lp = mvn_log_prob(bt, s2t, rgt, _t(c), nu=1.5, nugget=1e-4, n_points=128, n_shifts=4, seed=21)
    lp.backward()
    assert abs(lp.item() - logP) < 1e-9
    np.testing.assert_allclose(bt.grad.cpu().numpy(), gb, rtol=1e-8, atol=1e-12)
    assert abs(s2t.grad.item() - th[0]) < 1e-8 * max(1, abs(th[0]))
    assert abs(rgt.grad.item() - th[1]) < 1e-8 * max(1, abs(th[1]))


def test_w4_gradients_vs_central_fd(mvn):
    """Workload W4 (n=4,096 Matern 3/2, 10,000 paths): the autograd gradients of log P with
    respect to (sigma2, range), a 16-coordinate subset of b and a random direction in b, against
    central finite differences (h = 1e-5) of the GPU estimate on identical lattice points."""
    from paper_2405_14892_gb300.autograd import mvn_log_prob
    w = inputs.WORKLOADS["W4"]
    c = _t(inputs.grid_coords(w["g"]))
    n = c.shape[0]
    _, b = inputs.limits_for(w, n)
    kw = dict(nu=w["nu"], nugget=w["nugget"], n_points=w["Ns"], n_shifts=w["M"], seed=w["seed"])
    bt = _t(b).requires_grad_(True)
    s2t = torch.tensor(w["sigma2"], dtype=torch.float64, device="cuda", requires_grad=True)
    rgt = torch.tensor(w["range"], dtype=torch.float64, device="cuda", requires_grad=True)
    lp = mvn_log_prob(bt, s2t, rgt, c, **kw)
    lp.backward()

    def f(bb, s2, rg):
        with torch.no_grad():
            return mvn_log_prob(bb, torch.tensor(s2), torch.tensor(rg), c, **kw).item()
    s2, rg = w["sigma2"], w["range"]
    b0 = _t(b)
    # theta enters through the Cholesky factor of a matrix with condition number ~1e6 (nugget
    # 1e-4): the computed log P(theta) carries rounding roughness of order 1e-7, which a central
    # difference divides by 2h.  At h = 1e-5 that is ~1e-2 absolute.  A step of 1e-3 of each
    # parameter's value keeps the roughness term ~1e-4 absolute and the O(h^2) truncation below it.
    g_s2, g_rg = s2t.grad.item(), rgt.grad.item()
    for hs2, hrg, rtol in ((1e-5, 1e-5, 3e-3), (1e-3 * s2, 1e-3 * rg, 2e-4)):
        fd_s2 = (f(b0, s2 + hs2, rg) - f(b0, s2 - hs2, rg)) / (2 * hs2)
        fd_rg = (f(b0, s2, rg + hrg) - f(b0, s2, rg - hrg)) / (2 * hrg)
        print(f"W4 h=({hs2:g},{hrg:g}): logP={lp.item():.8f} dsigma2 {g_s2:.8e} fd {fd_s2:.8e} | "
              f"drange {g_rg:.8e} fd {fd_rg:.8e}")
        assert abs(g_s2 - fd_s2) <= rtol * max(1.0, abs(fd_s2))
        assert abs(g_rg - fd_rg) <= rtol * max(1.0, abs(fd_rg))
    # b enters only the sweep (the factor is fixed): the estimate is smooth to rounding there
    h = 1e-5
    rng = np.random.default_rng(4)
    gbv = bt.grad.cpu().numpy()
    for i in rng.choice(n, 16, replace=False):
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        e[i] = h
        fd = (f(b0 + e, s2, rg) - f(b0 - e, s2, rg)) / (2 * h)
        assert abs(gbv[i] - fd) <= 1e-5 * max(1.0, abs(fd)), (i, gbv[i], fd)
    v = _t(np.random.default_rng(5).standard_normal(n))
    fd = (f(b0 + h * v, s2, rg) - f(b0 - h * v, s2, rg)) / (2 * h)
    dd = float((bt.grad * v).sum())
    assert abs(dd - fd) <= 1e-5 * max(1.0, abs(fd)), (dd, fd)


@pytest.mark.parametrize("n,Ns,M", [(20, 100, 3), (150, 64, 4), (600, 97, 3)])
def test_sov_grad_mixed_vs_oracle(mvn, n, Ns, M):
    """The mixed adjoint (FP32 limit sums and transformed variables, FP64 elementwise terms)
    against the FP64 oracle on identical lattice points.  The test field is strongly correlated
    (conditional standard deviations L_ii down to 0.07, so FP32 errors of the limit sums grow
    ~15x in a' and b') and the per-dimension errors add up along log P: the bound is
    |d log P| <= 1e-4 + 2e-7 n (one unblocked FP32 chain of limit sums gives 6.6e-4 at n = 600,
    log P = -938, in a CPU emulation; the kernels sum 16-dimension partials per 128-dimension
    group).  Every gradient entry within 5e-5 of the largest."""
    S, a, b = _problem(n, n)
    Lo, _ = oracle.cholesky(S)
    q = oracle.QMC(Ns, M, 5 + n)
    logP, ga, gb, gL = oracle.sov_grad(a, b, Lo, q)
    L = mvn.to_colmajor(_t(Lo))
    out3, ga_g, gb_g, gL_g = mvn.mvn_sov_grad(_t(a), _t(b), L, Ns, M, 5 + n, prec="mixed",
                                              want_L=True)
    mvn.sync()
    o = out3.cpu().numpy()
    scale = max(1.0, np.abs(gb).max(), np.abs(ga).max())
    e_lp = abs(o[0] - logP)
    e_a = np.abs(ga_g.cpu().numpy() - ga).max() / scale
    e_b = np.abs(gb_g.cpu().numpy() - gb).max() / scale
    e_L = np.abs(np.tril(gL_g.cpu().numpy()) - np.tril(gL)).max() / max(1.0, np.abs(gL).max())
    print(f"mixed adjoint n={n}: dlogP {e_lp:.2e} da {e_a:.2e} db {e_b:.2e} dL {e_L:.2e}")
    assert e_lp <= 1e-4 + 2e-7 * n
    assert max(e_a, e_b, e_L) <= 5e-5


def test_w4_mixed_gradients_vs_fp64(mvn):
    """Workload W4 through the autograd chain with prec="mixed" (tensor-core Cholesky, mixed
    sweep adjoint) against prec="fp64" (whose gradients the oracle and finite-difference tests
    pin): log P within 1e-4 and every gradient within 1e-3 relative."""
    from paper_2405_14892_gb300.autograd import mvn_log_prob
    w = inputs.WORKLOADS["W4"]
    c = _t(inputs.grid_coords(w["g"]))
    n = c.shape[0]
    _, b = inputs.limits_for(w, n)
    kw = dict(nu=w["nu"], nugget=w["nugget"], n_points=w["Ns"], n_shifts=w["M"], seed=w["seed"])
    res = {}
    for prec in ("fp64", "mixed"):
        bt = _t(b).requires_grad_(True)
        s2t = torch.tensor(w["sigma2"], dtype=torch.float64, device="cuda", requires_grad=True)
        rgt = torch.tensor(w["range"], dtype=torch.float64, device="cuda", requires_grad=True)
        lp = mvn_log_prob(bt, s2t, rgt, c, prec=prec, **kw)
        lp.backward()
        res[prec] = (lp.item(), bt.grad.cpu().numpy(), s2t.grad.item(), rgt.grad.item())
    l64, gb64, s64, r64 = res["fp64"]
    lmx, gbmx, smx, rmx = res["mixed"]
    e_b = np.abs(gbmx - gb64).max() / max(1.0, np.abs(gb64).max())
    e_s = abs(smx - s64) / max(1.0, abs(s64))
    e_r = abs(rmx - r64) / max(1.0, abs(r64))
    print(f"W4 mixed vs fp64: logP {lmx:.8f} vs {l64:.8f} (d {abs(lmx - l64):.2e}); "
          f"db {e_b:.2e} dsigma2 {e_s:.2e} drange {e_r:.2e}")
    assert abs(lmx - l64) <= 1e-4
    assert max(e_b, e_s, e_r) <= 1e-3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sov_grad_batched_under_a_memory_limit(mvn, prec):
    """A y-buffer limit of 3 path tiles splits 2,000 paths (16 tiles) into 6 batches that recompute
    their forward sweep: the estimate and d log P / d(a, b) are bit-identical to the unbatched
    call, d log P / dL equal to rounding; and the FP64 result still matches the oracle."""
    n, Ns, M, seed = 90, 400, 5, 77
    S, a, b = _problem(n, 3)
    Lo, _ = oracle.cholesky(S)
    L = mvn.to_colmajor(_t(Lo))
    ref = mvn.mvn_sov_grad(_t(a), _t(b), L, Ns, M, seed, prec=prec, want_L=True)
    mvn.sync()
    elt = 8 if prec == "fp64" else 4
    mvn.mvn_grad_set_ylimit(3 * 2 * n * 128 * elt)
    try:
        got = mvn.mvn_sov_grad(_t(a), _t(b), L, Ns, M, seed, prec=prec, want_L=True)
        mvn.sync()
    finally:
        mvn.mvn_grad_set_ylimit(0)
    for k in range(3):
        assert torch.equal(got[k], ref[k]), k
    gl, rl = np.tril(got[3].cpu().numpy()), np.tril(ref[3].cpu().numpy())
    assert np.abs(gl - rl).max() <= 1e-12 * max(1.0, np.abs(rl).max())
    if prec == "fp64":
        logP, ga, gb, gL = oracle.sov_grad(a, b, Lo, oracle.QMC(Ns, M, seed))
        assert abs(got[0].cpu().numpy()[0] - logP) < 1e-9
        scale = max(1.0, np.abs(gb).max(), np.abs(ga).max())
        np.testing.assert_allclose(got[2].cpu().numpy(), gb, atol=1e-9 * scale)
        assert np.abs(gl - np.tril(gL)).max() <= 1e-9 * max(1.0, np.abs(gL).max())
