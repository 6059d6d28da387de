"""Posterior field (Sec. V-B, Eqs. 7-8) on the GPU through the C ABI (mvn_posterior) against the
oracle, which evaluates Eqs. 7-8 as printed (explicit inverses).  FP64: entries of Sigma_post
within 1e-10 and of mu_post within 1e-10 (the prior variances are 1; the oracle and the Schur
form differ by < 5e-13 on these cases in numpy).  Only the lower triangle of Sigma is given (the
strict upper part is NaN), so a read of the wrong triangle shows up."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_14892_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-10


@pytest.fixture(scope="module")
def mvn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_14892_gb300 import mvn as m
    m.context().sync()  # start from a clear device status word
    return m


def _lower_nan(mvn, S):
    """Column-major CUDA copy of S with its strict upper triangle set to NaN."""
    Sl = np.where(np.tril(np.ones_like(S, dtype=bool)), S, np.nan)
    return mvn.to_colmajor(torch.as_tensor(Sl, dtype=torch.float64, device="cuda"))


def _case(g, n, rng_, nu, n_obs, seed):
    c = inputs.grid_coords(g)[:n]
    S = oracle.matern(c, 1.0, rng_, nu)
    obs, y, _ = inputs.observations(S, n_obs, 0.5, seed)
    return S, obs, y


def _run(mvn, mu, S, obs, y, t2):
    Sd = _lower_nan(mvn, S)
    mud = None if mu is None else torch.as_tensor(mu, device="cuda")
    out = mvn.colmajor_empty(S.shape[0], S.shape[0], "cuda").fill_(0.0)
    mp, Sp = mvn.mvn_posterior(mud, Sd, torch.as_tensor(obs, dtype=torch.int32, device="cuda"),
                               torch.as_tensor(y, device="cuda"), t2, out_Sigma=out)
    return mp.cpu().numpy(), np.tril(Sp.cpu().numpy())


@pytest.mark.parametrize("g,n,rng_,nu,n_obs", [(18, 300, 0.15, 0.5, 70), (40, 1600, 0.1, 1.5, 200),
                                               (3, 5, 0.3, 0.5, 1), (9, 81, 0.2, 0.5, 64)])
def test_posterior_vs_oracle(mvn, g, n, rng_, nu, n_obs):
    S, obs, y = _case(g, n, rng_, nu, n_obs, 7 + n)
    mu = inputs.standard_normals(n, 8)
    mp, Sp = _run(mvn, mu, S, obs, y, 0.25)
    mo, So = oracle.posterior(mu, S, obs, y, 0.25)
    assert np.all(np.isfinite(Sp)) and np.all(np.isfinite(mp))
    assert np.abs(Sp - np.tril(So)).max() <= TOL
    assert np.abs(mp - mo).max() <= TOL


def test_posterior_w3_size(mvn):
    """The confidence-region workload's posterior: n = 4,096 (64 x 64 grid, exponential kernel,
    range 0.1), 640 observations with noise sd 0.5, zero prior mean; timed with CUDA events."""
    w = inputs.WORKLOADS["W3"]
    S, obs, y = _case(w["g"], w["g"] ** 2, w["range"], w["nu"], w["n_obs"], w["field_seed"])
    n = S.shape[0]
    t2 = w["noise_sd"] ** 2
    Sd = _lower_nan(mvn, S)
    od = torch.as_tensor(obs, dtype=torch.int32, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    out = mvn.colmajor_empty(n, n, "cuda")
    mvn.mvn_posterior(None, Sd, od, yd, t2, out_Sigma=out)  # warm-up (workspace growth)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    mp, Sp = mvn.mvn_posterior(None, Sd, od, yd, t2, out_Sigma=out, check=False)
    e1.record()
    torch.cuda.synchronize()
    assert mvn.sync() == 0
    ms = e0.elapsed_time(e1)
    k = w["n_obs"]
    flops = float(n) * n * k + float(n) * k * k + k ** 3 / 3.0
    print(f"mvn_posterior n={n} n_obs={k}: {ms:.2f} ms, {flops / (ms * 1e-3) / 1e12:.3f} TFLOP/s "
          f"of minimal FP64 work (n^2 k + n k^2 + k^3/3)")
    mo, So = oracle.posterior(None, S, obs, y, t2)
    assert np.abs(np.tril(Sp.cpu().numpy()) - np.tril(So)).max() <= TOL
    assert np.abs(mp.cpu().numpy() - mo).max() <= TOL


def test_posterior_edge_cases(mvn):
    S, obs, y = _case(8, 60, 0.2, 0.5, 20, 3)
    mu = inputs.standard_normals(60, 4)
    # no observations: the prior comes back (copied bit for bit)
    mp, Sp = _run(mvn, mu, S, np.zeros(0, np.int32), np.zeros(0), 0.3)
    assert np.array_equal(mp, mu) and np.array_equal(Sp, np.tril(S))
    # repeated observations of a site
    obs2 = np.array([5, 5, 17, 0, 59, 17], dtype=np.int32)
    y2 = inputs.standard_normals(6, 5)
    mp, Sp = _run(mvn, mu, S, obs2, y2, 0.3)
    mo, So = oracle.posterior(mu, S, obs2, y2, 0.3)
    assert np.abs(Sp - np.tril(So)).max() <= TOL and np.abs(mp - mo).max() <= TOL
    # in place: outputs over the inputs
    Sd = _lower_nan(mvn, S)
    mud = torch.as_tensor(mu, device="cuda")
    mvn.mvn_posterior(mud, Sd, torch.as_tensor(obs, device="cuda"),
                      torch.as_tensor(y, device="cuda"), 0.3, out_Sigma=Sd, out_mu=mud)
    mo, So = oracle.posterior(mu, S, obs, y, 0.3)
    assert np.abs(np.tril(Sd.cpu().numpy()) - np.tril(So)).max() <= TOL
    assert np.abs(mud.cpu().numpy() - mo).max() <= TOL
    assert np.all(np.isnan(np.triu(Sd.cpu().numpy(), 1)[np.triu_indices(60, 1)]))  # untouched


def test_posterior_bad_arguments(mvn):
    S, obs, y = _case(5, 25, 0.2, 0.5, 4, 9)
    Sd = _lower_nan(mvn, S)
    yd = torch.as_tensor(y, device="cuda")
    bad = torch.as_tensor(np.array([1, 2, 25, 3], dtype=np.int32), device="cuda")
    with pytest.raises(mvn.MVNError) as e:
        mvn.mvn_posterior(None, Sd, bad, yd, 0.25)
    assert e.value.status == mvn.MVN_ERR_ARG
    assert mvn.sync() == 0  # status cleared, context usable
    good = torch.as_tensor(obs, dtype=torch.int32, device="cuda")
    with pytest.raises(mvn.MVNError) as e:
        mvn.mvn_posterior(None, Sd, good, yd, 0.0)
    assert e.value.status == mvn.MVN_ERR_ARG
    mp, Sp = mvn.mvn_posterior(None, Sd, good, yd, 0.25)
    mo, _ = oracle.posterior(None, S, obs, y, 0.25)
    assert math.isfinite(float(mp[0])) and np.abs(mp.cpu().numpy() - mo).max() <= TOL


@pytest.mark.parametrize("g,n,rng_,nu,n_obs", [(18, 300, 0.15, 0.5, 70), (40, 1600, 0.1, 1.5, 200),
                                               (9, 81, 0.2, 0.5, 64), (20, 400, 0.1, 0.5, 129)])
def test_posterior_mixed_vs_oracle(mvn, g, n, rng_, nu, n_obs):
    """MVN_MIXED posterior (the tensor-core factorisation's partial mode: the observations'
    columns in double-float with exact-digit updates, every trailing column updated once by all of
    them on the tensor cores) against the oracle's Eqs. 7-8: within 1e-9 of the largest prior
    entry (the digit products carry 42 bits; measured in the printout), n_obs not a multiple of
    64 exercises the padding variables."""
    S, obs, y = _case(g, n, rng_, nu, n_obs, 7 + n)
    Sd = mvn.to_colmajor(torch.as_tensor(S, device="cuda"))
    out = mvn.colmajor_empty(n, n, "cuda").fill_(0.0)
    mp, Sp = mvn.mvn_posterior(None, Sd, torch.as_tensor(obs, dtype=torch.int32, device="cuda"),
                               torch.as_tensor(y, device="cuda"), 0.25, out_Sigma=out,
                               prec="mixed")
    mo, So = oracle.posterior(None, S, obs, y, 0.25)
    dS = np.abs(np.tril(Sp.cpu().numpy()) - np.tril(So)).max()
    dm = np.abs(mp.cpu().numpy() - mo).max()
    print(f"mixed posterior n={n} n_obs={n_obs}: max |d Sigma_post| {dS:.3e}, max |d mu_post| "
          f"{dm:.3e}")
    assert dS <= 1e-9 and dm <= 1e-9


def test_posterior_mixed_w3_size(mvn):
    """W3 size (n = 4,096, 640 observations) in MVN_MIXED: against the FP64 path, and timed."""
    w = inputs.WORKLOADS["W3"]
    c = inputs.grid_coords(w["g"])
    n = c.shape[0]
    S = oracle.matern_closed(c, w["sigma2"], w["range"], w["nu"], w["nugget"])
    obs, y, _ = inputs.observations(S, w["n_obs"], w["noise_sd"], w["field_seed"])
    Sd = mvn.to_colmajor(torch.as_tensor(S, device="cuda"))
    od = torch.as_tensor(obs, dtype=torch.int32, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    t2 = w["noise_sd"] ** 2
    o64 = mvn.colmajor_empty(n, n, "cuda")
    omx = mvn.colmajor_empty(n, n, "cuda")
    m64, _ = mvn.mvn_posterior(None, Sd, od, yd, t2, out_Sigma=o64)
    mvn.mvn_posterior(None, Sd, od, yd, t2, out_Sigma=omx, prec="mixed")  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    mmx, _ = mvn.mvn_posterior(None, Sd, od, yd, t2, out_Sigma=omx, prec="mixed", check=False)
    e1.record()
    torch.cuda.synchronize()
    assert mvn.sync() == 0
    ms = e0.elapsed_time(e1)
    dS = (torch.tril(omx) - torch.tril(o64)).abs().max().item()
    dm = (mmx - m64).abs().max().item()
    print(f"mixed posterior W3 size: {ms:.2f} ms, |d Sigma_post| {dS:.3e}, |d mu_post| {dm:.3e}")
    assert dS <= 1e-9 and dm <= 1e-9
