"""Confidence-region detection at the paper's synthetic scale (Sec. V-B; workload W6: 40,000
sites of an exponential field, 6,250 noisy observations): the MVN_MIXED posterior (Eqs. 7-8) and
Alg. 1 over every prefix on the GPU, checked against the oracle where it can compute at this size:
posterior entries and means on sampled sites (the site-subset form of Eqs. 7-8), the order of the
first sites by the marginals, and F on sampled prefixes (the oracle's own Cholesky and sweep of
the prefix problem).  The oracle works from its own covariance and posterior throughout."""
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


def _cov(c, w, rows, cols):
    """Oracle covariance between two site sets (Eq. 6, exponential closed form)."""
    h = np.sqrt(((c[rows][:, None, :] - c[cols][None, :, :]) ** 2).sum(-1))
    C = w["sigma2"] * np.exp(-h / w["range"])
    return C


def test_crd_w6_scale(mvn):
    w = inputs.WORKLOADS["W6"]
    c = inputs.grid_coords(w["g"])
    n = c.shape[0]
    obs, y, _ = inputs.observations_at_sites(
        n, w["n_obs"], w["noise_sd"], w["field_seed"],
        lambda idx: oracle.matern_closed(c[idx], w["sigma2"], w["range"], w["nu"]))
    t2 = w["noise_sd"] ** 2
    S = mvn.mvn_matern(torch.as_tensor(c, device="cuda"), w["sigma2"], w["range"], w["nu"],
                       w["nugget"])
    Sp = mvn.colmajor_empty(n, n, "cuda")
    mu, _ = mvn.mvn_posterior(None, S, torch.as_tensor(obs, dtype=torch.int32, device="cuda"),
                              torch.as_tensor(y, device="cuda"), t2, out_Sigma=Sp, prec="mixed")
    del S
    # oracle: K^-1 [Sigma[obs, :], y] in column chunks -> mu_post and diag Sigma_post everywhere
    Koo = _cov(c, w, obs, obs) + t2 * np.eye(obs.size)
    Lk = np.linalg.cholesky(Koo)
    from scipy.linalg import solve_triangular
    zy = solve_triangular(Lk, y, lower=True)
    mu_o = np.empty(n)
    var_o = np.empty(n)
    for j0 in range(0, n, 4000):
        cols = np.arange(j0, min(n, j0 + 4000))
        Z = solve_triangular(Lk, _cov(c, w, obs, cols), lower=True)
        mu_o[cols] = Z.T @ zy
        var_o[cols] = w["sigma2"] - np.sum(Z * Z, axis=0)
    mu_g = mu.cpu().numpy()
    dg = torch.diagonal(Sp).cpu().numpy()
    print(f"W6 posterior: max |d mu| {np.abs(mu_g - mu_o).max():.3e}, max |d var| "
          f"{np.abs(dg - var_o).max():.3e}")
    # the trailing update's digit products carry 42 bits relative to the rows' scales: the
    # border row (y) is scaled by its norm bound 2^8 here, so mu_post's update, summed over the
    # 6,272 factor columns, is good to ~5e-9 and Sigma_post's to ~1e-10 (measured 6.5e-9 and
    # 6.0e-10, the double-float panel included); gates 5e-8 and 5e-9
    assert np.abs(mu_g - mu_o).max() <= 5e-8
    assert np.abs(dg - var_o).max() <= 5e-9
    # sampled off-diagonal entries by the site-subset form
    R = np.array([0, 1, 201, 12345, 20000, 39999])
    mp, Spp = oracle.posterior_parts(_cov(c, w, R, R), Koo - t2 * np.eye(obs.size),
                                     _cov(c, w, obs, R), y, t2)
    Rd = torch.as_tensor(R, device="cuda")      # R ascending: (i >= j) entries are stored
    Sg = np.tril(Sp[Rd][:, Rd].cpu().numpy())
    Sg = Sg + np.tril(Sg, -1).T
    assert np.abs(Sg - Spp).max() <= 5e-9 and np.abs(mu_g[R] - mp).max() <= 5e-8
    # Alg. 1 over every prefix on the GPU
    r = mvn.mvn_excursion(mu, Sp, w["u"], w["level"], w["Ns"], w["M"], w["seed"], prec="mixed")
    mvn.sync()
    order = r["order"].cpu().numpy()
    F = r["F"].cpu().numpy()
    assert F.size == n and np.all(np.isfinite(F))
    # the oracle's marginals and order (first 300 sites), then F on sampled prefixes
    pM = oracle.Q((w["u"] - mu_o) / np.sqrt(var_o))
    o_ref = np.argsort(-pM, kind="stable")
    assert np.array_equal(order[:300], o_ref[:300])
    np.testing.assert_allclose(r["marginal"].cpu().numpy(), pM, rtol=1e-6, atol=1e-12)
    kmax = 300
    P = o_ref[:kmax]
    mpk, Spk = oracle.posterior_parts(_cov(c, w, P, P), Koo - t2 * np.eye(obs.size),
                                      _cov(c, w, obs, P), y, t2)
    Lp, info = oracle.cholesky(Spk)
    assert info == 0
    q = oracle.QMC(w["Ns"], w["M"], w["seed"])
    a = w["u"] - mpk
    b = np.full(kmax, np.inf)
    ks = [1, 2, 10, 100, 300]
    _, lp = oracle.sov_logw(a, b, Lp, q, prefixes=ks)
    for t, k in enumerate(ks):
        Fo = oracle.estimate(lp[:, t], q.M)[1]
        print(f"F(o_{k}): GPU {F[k - 1]:.8f} oracle {Fo:.8f}")
        assert abs(math.log(F[k - 1]) - math.log(Fo)) <= 1e-4
    # the region is the longest prefix whose F reaches the level (Eq. 4)
    region = r["region"].cpu().numpy()
    K = int(region.sum())
    assert K == 0 or F[K - 1] >= w["level"]
    assert np.all(F[K:] < w["level"])
    assert np.array_equal(np.sort(np.nonzero(region)[0]), np.sort(order[:K]))
    print(f"W6: region of {K} sites; F(o_n) = {F[-1]:.3e}")
