"""GPU path vs the CPU oracle, element by element on the same seeded inputs, through the C ABI.

Tolerances (FP64 path): per-path |d logw| <= 1e-9 max(1, |logw|), |d log P| <= 1e-9 and
|d P| <= 1e-10 absolute; integer work (lattice tables, order, region) bit-exact."""
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


DEV = "cuda"


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def _gpu_factor(mvn, Sigma_np):
    A = mvn.to_colmajor(_t(Sigma_np))
    info = mvn.mvn_cholesky(A)
    assert info == 0
    return A


def _check_logw(got, ref, tol=1e-9):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    err = np.abs(got[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))
    assert err.max(initial=0.0) <= tol, err.max()


# ------------------------------------------------------------------ lattice tables (bit-exact)

def test_lattice_alpha_and_shifts_bit_exact(mvn):
    n = 70000
    got = mvn.mvn_lattice_alpha(n).cpu().numpy().view(np.uint64)
    ref = oracle.lattice_alpha(n)
    assert np.array_equal(got, ref)
    for seed in (0, 12, 2 ** 63 + 5):
        d = mvn.mvn_lattice_shifts(seed, 7, 333).cpu().numpy().view(np.uint64)
        assert np.array_equal(d, oracle.lattice_shifts(seed, 7, 333))


# ------------------------------------------------------------------ Matern (Eq. 6)

@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_vs_oracle(mvn, nu):
    c = inputs.random_coords(300, 3)
    S = mvn.mvn_matern(_t(c), 1.3, 0.2, nu, nugget=1e-4).cpu().numpy()
    ref = oracle.matern(c, 1.3, 0.2, nu, nugget=1e-4)
    low = np.tril_indices(300)
    np.testing.assert_allclose(S[low], ref[low], rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ Cholesky (Alg. 1)

@pytest.mark.parametrize("n", [1, 5, 64, 130, 1000])
def test_cholesky_vs_oracle(mvn, n):
    g = int(math.ceil(math.sqrt(n)))
    c = inputs.grid_coords(g)[:n]
    S = oracle.matern(c, 1.0, 0.1, 1.5, nugget=1e-4)
    A = _gpu_factor(mvn, S)
    L = np.tril(A.cpu().numpy())
    Lo, info = oracle.cholesky(S)
    assert info == 0
    # both are backward stable: compare factors relative to the conditioning-free bound
    assert np.abs(L - Lo).max() <= 1e-9, np.abs(L - Lo).max()
    assert np.linalg.norm(L @ L.T - S) / np.linalg.norm(S) < 1e-14 * n + 1e-15


def test_cholesky_not_pd_info(mvn):
    S = oracle.matern(inputs.random_coords(200, 4), 1.0, 0.2, 0.5)
    S[150, 150] = -1.0
    A = mvn.to_colmajor(_t(S))
    with pytest.raises(mvn.MVNError) as e:
        mvn.mvn_cholesky(A)
    assert e.value.status == mvn.MVN_ERR_NOT_PD
    _, info_ref = oracle.cholesky(S)
    assert info_ref == 151
    A = mvn.to_colmajor(_t(S))
    import ctypes
    info = ctypes.c_int(0)
    n = 200
    st = mvn.lib().mvn_cholesky(mvn.context().h, n, ctypes.c_void_p(A.data_ptr()), n, 0, 0,
                                ctypes.byref(info))
    assert st == mvn.MVN_ERR_NOT_PD and info.value == 151
    # the context stays usable
    B = _gpu_factor(mvn, np.eye(4) * 2.0)
    assert abs(B.cpu().numpy()[0, 0] - math.sqrt(2.0)) < 1e-15


# ------------------------------------------------------------------ SOV (Eqs. 2-3, Algs. 2-3)

def _sov_case(mvn, n, Ns, M, seed, a, b, Sigma, prec="fp64"):
    L = _gpu_factor(mvn, Sigma)
    lw = torch.empty(Ns * M, dtype=torch.float64, device=DEV)
    out = mvn.mvn_sov(_t(a), _t(b), L, Ns, M, seed, prec=prec, path_logw=lw)
    mvn.sync()
    Lo, _ = oracle.cholesky(Sigma)
    return lw.cpu().numpy(), out.cpu().numpy(), Lo


@pytest.mark.parametrize("n,Ns,M", [(1, 50, 3), (31, 129, 2), (100, 300, 5), (257, 64, 4)])
def test_sov_fp64_per_path_ragged(mvn, n, Ns, M):
    g = int(math.ceil(math.sqrt(n)))
    c = inputs.grid_coords(g)[:n]
    S = oracle.matern(c, 1.0, 0.15, 0.5, nugget=1e-6)
    rng = np.random.default_rng(n)
    a = rng.uniform(-2.5, 0.3, n)
    b = a + rng.uniform(0.2, 3.0, n)
    a[::3] = -np.inf
    b[1::4] = np.inf
    lw, out, Lo = _sov_case(mvn, n, Ns, M, 5 + n, a, b, S)
    ref = oracle.sov_logw(a, b, Lo, oracle.QMC(Ns, M, 5 + n))
    _check_logw(lw, ref)
    est = oracle.estimate(ref, M)
    assert abs(out[0] - est[0]) <= 1e-9
    assert abs(out[1] - est[1]) <= 1e-10
    assert abs(out[2] - est[2]) <= 1e-9 * max(est[2], 1e-300) + 1e-14


def test_sov_fp64_tails_and_infinite_dims(mvn):
    n = 40
    c = inputs.grid_coords(7)[:n]
    S = oracle.matern(c, 1.0, 0.3, 1.5, nugget=1e-3)
    a = np.full(n, -np.inf)
    b = np.full(n, np.inf)
    a[:10] = 2.5          # upper tail branch (a' > 0)
    b[10:20] = -2.5       # deep lower tail
    a[20:25] = -0.1
    b[20:25] = 0.1        # narrow two-sided intervals
    lw, out, Lo = _sov_case(mvn, n, 200, 3, 99, a, b, S)
    ref = oracle.sov_logw(a, b, Lo, oracle.QMC(200, 3, 99))
    _check_logw(lw, ref)


def test_sov_zero_dimension_and_all_infinite(mvn):
    lw, out, _ = _sov_case(mvn, 0, 10, 2, 1, np.zeros(0), np.zeros(0), np.zeros((0, 0)))
    assert np.all(lw == 0.0) and out[0] == 0.0 and out[1] == 1.0
    n = 9
    S = oracle.matern(inputs.grid_coords(3), 1.0, 0.3, 0.5)
    lw, out, _ = _sov_case(mvn, n, 10, 2, 1, np.full(n, -np.inf), np.full(n, np.inf), S)
    assert np.all(lw == 0.0) and out[1] == 1.0


def test_sov_w1_full_size(mvn):
    """Workload W1 at its full size (n=256, 10,000 points x 20 shifts), every path."""
    w = inputs.WORKLOADS["W1"]
    c = inputs.grid_coords(w["g"])
    n = c.shape[0]
    a, b = inputs.limits_for(w, n)
    S = oracle.matern(c, w["sigma2"], w["range"], w["nu"], w["nugget"])
    lw, out, Lo = _sov_case(mvn, n, w["Ns"], w["M"], w["seed"], a, b, S)
    ref = oracle.sov_logw(a, b, Lo, oracle.QMC(w["Ns"], w["M"], w["seed"]))
    _check_logw(lw, ref)
    est = oracle.estimate(ref, w["M"])
    assert abs(out[0] - est[0]) <= 1e-9 and abs(out[1] - est[1]) <= 1e-10


@pytest.fixture(scope="module")
def w2_oracle():
    """Oracle covariance and factor of workload W2 (n=16,384): Eq. 6 closed form, LAPACK."""
    w = inputs.WORKLOADS["W2"]
    c = inputs.grid_coords(w["g"])
    So = oracle.matern_closed(c, w["sigma2"], w["range"], w["nu"], w["nugget"])
    Lo = oracle.cholesky_lapack(So)
    return w, c, So, Lo


def test_matern_and_cholesky_w2_full_size(mvn, w2_oracle):
    """W2 covariance and factor on the GPU vs the oracle: sampled entries of Sigma, sampled
    columns of L, and the backward error ||(L L^T - Sigma) v|| / ||Sigma v|| for random v."""
    w, c, So, Lo = w2_oracle
    n = c.shape[0]
    S = mvn.mvn_matern(_t(c), w["sigma2"], w["range"], w["nu"], w["nugget"])
    Sg_cols = S[:, ::997].cpu().numpy()
    for t, j in enumerate(range(0, n, 997)):
        np.testing.assert_allclose(Sg_cols[j:, t], So[j:, j], rtol=1e-12, atol=1e-15)
    assert mvn.mvn_cholesky(S) == 0
    Lg = torch.tril(S)  # logical lower triangle (the strict upper part was never written)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal(n)
        vt = _t(v)
        LLv = (Lg @ (Lg.t() @ vt)).cpu().numpy()
        Sv = So @ v
        assert np.linalg.norm(LLv - Sv) / np.linalg.norm(Sv) < 1e-13
    cols = list(range(0, n, 1531)) + [n - 1]
    Lg_cols = Lg[:, cols].cpu().numpy()
    for t, j in enumerate(cols):
        err = np.abs(Lg_cols[j:, t] - Lo[j:, j]).max()
        assert err < 1e-7, (j, err)


def test_sov_w2_full_size_sampled_paths(mvn, w2_oracle):
    """Workload W2 at its full size (n=16,384, 20,000 paths, the bench's launch) on the GPU with
    the oracle's factor as input; the oracle recomputes a sample of paths one by one."""
    w, c, So, Lo = w2_oracle
    n = c.shape[0]
    a, b = inputs.limits_for(w, n)
    L = mvn.to_colmajor(_t(Lo))
    Ntot = w["Ns"] * w["M"]
    lw = torch.empty(Ntot, dtype=torch.float64, device=DEV)
    out = mvn.mvn_sov(_t(a), _t(b), L, w["Ns"], w["M"], w["seed"], path_logw=lw)
    mvn.sync()
    lw = lw.cpu().numpy()
    q = oracle.QMC(w["Ns"], w["M"], w["seed"])
    for p0 in (0, 2000 * 7 + 1000, Ntot - 8):
        ref = oracle.sov_logw(a, b, Lo, q, paths=(p0, p0 + 8))
        err = np.abs(lw[p0:p0 + 8] - ref) / np.maximum(1, np.abs(ref))
        assert err.max() <= 1e-9, (p0, err.max())
    assert np.all(np.isfinite(lw)) and np.all(lw <= 0)
    est = oracle.estimate(lw, w["M"])
    o = out.cpu().numpy()
    assert abs(o[0] - est[0]) <= 1e-9 and abs(o[1] - est[1]) <= 1e-10


def test_bench_w2_mixed_launch_vs_oracle_and_fp64(mvn, w2_oracle):
    """The bench's W2 step exactly as it is timed (mvn_matern -> mvn_cholesky MVN_MIXED ->
    mvn_sov MVN_MIXED at n = 16,384 with all 20,000 paths): per-path log-weights against the
    oracle (its own covariance and LAPACK factor) on three windows of sampled paths, and the
    estimate against the all-FP64 GPU path (FP64 Cholesky and FP64 sweep of the same covariance)
    on identical lattice points, gated at |d log P| <= 1e-4 (and the literal |d P| <= 1e-4).
    Per path the mixed error is the factor's (the exact-digit update carries ~42 bits) plus the
    sweep's; stated bound 1e-5 max(1, |logw|)."""
    w, c, So, Lo = w2_oracle
    n = c.shape[0]
    a, b = inputs.limits_for(w, n)
    Ns, M = w["Ns"], w["M"]
    Ntot = Ns * M
    S = mvn.mvn_matern(_t(c), w["sigma2"], w["range"], w["nu"], w["nugget"])
    S64 = S.clone()
    assert S64.stride() == S.stride()
    assert mvn.mvn_cholesky(S, prec="mixed") == 0
    lw_mx = torch.empty(Ntot, dtype=torch.float64, device=DEV)
    o_mx = mvn.mvn_sov(_t(a), _t(b), S, Ns, M, w["seed"], prec="mixed", path_logw=lw_mx)
    mvn.sync()
    o_mx = o_mx.cpu().numpy()
    lw_mx = lw_mx.cpu().numpy()
    del S
    assert mvn.mvn_cholesky(S64, prec="fp64") == 0
    lw_64 = torch.empty(Ntot, dtype=torch.float64, device=DEV)
    o_64 = mvn.mvn_sov(_t(a), _t(b), S64, Ns, M, w["seed"], prec="fp64", path_logw=lw_64)
    mvn.sync()
    o_64 = o_64.cpu().numpy()
    lw_64 = lw_64.cpu().numpy()
    del S64
    q = oracle.QMC(Ns, M, w["seed"])
    worst = 0.0
    for p0 in (0, 2000 * 3 + 517, Ntot - 8):
        ref = oracle.sov_logw(a, b, Lo, q, paths=(p0, p0 + 8))
        rel = np.abs(lw_mx[p0:p0 + 8] - ref) / np.maximum(1.0, np.abs(ref))
        rel64 = np.abs(lw_64[p0:p0 + 8] - ref) / np.maximum(1.0, np.abs(ref))
        print(f"W2 paths {p0}..{p0 + 7}: mixed max rel {rel.max():.3e}, FP64 GPU (its own "
              f"factor) max rel {rel64.max():.3e}")
        worst = max(worst, rel.max())
        assert rel.max() <= 1e-5, (p0, rel.max())
    assert np.all(np.isfinite(lw_mx)) and np.all(lw_mx <= 0)
    d = abs(o_mx[0] - o_64[0])
    print(f"W2 bench launch: log P mixed {o_mx[0]:.10f} FP64 {o_64[0]:.10f} |d log P| {d:.3e} "
          f"|dP| {abs(o_mx[1] - o_64[1]):.3e} err/P {o_64[2] / o_64[1]:.3e}")
    assert d <= 1e-4
    assert abs(o_mx[1] - o_64[1]) <= 1e-4
    est = oracle.estimate(lw_mx, M)
    assert abs(o_mx[0] - est[0]) <= 1e-9


# ------------------------------------------------------------------ batched problems (Alg. 1 loop)

def test_sov_batched_vs_oracle_loop(mvn):
    n = 150
    c = inputs.grid_coords(13)[:n]
    S = oracle.matern(c, 1.0, 0.2, 0.5)
    L = _gpu_factor(mvn, S)
    Lo, _ = oracle.cholesky(S)
    rng = np.random.default_rng(6)
    a = np.concatenate([np.full(n, -np.inf), rng.uniform(-1, 0, n)])
    b = np.concatenate([rng.uniform(0, 1.5, n), np.full(n, np.inf)])
    dims = [150, 1, 37, 0, 128, 129, 64]
    offs = [0, 5, 150, 0, 150, 3, 100]
    out = mvn.mvn_sov_batched(dims, offs, _t(a), _t(b), L, 97, 3, 41).cpu().numpy()
    mvn.sync()
    for p, (k, o) in enumerate(zip(dims, offs)):
        ref = oracle.sov(a[o:o + k], b[o:o + k], Lo[:k, :k], oracle.QMC(97, 3, 41))
        assert abs(out[p, 0] - ref[0]) <= 1e-9, (p, out[p], ref)
        assert abs(out[p, 1] - ref[1]) <= 1e-10


# ------------------------------------------------------------------ confidence region (Alg. 1)

def test_excursion_vs_oracle(mvn):
    g = 12
    c = inputs.grid_coords(g)
    n = g * g
    S = oracle.matern(c, 1.0, 0.15, 0.5)
    mu = 0.9 + 0.7 * inputs.standard_normals(n, 31)
    ks = [1, 3, 17, 50, 51, 100, n]
    r = mvn.mvn_excursion(_t(mu), mvn.to_colmajor(_t(S)), 0.8, 0.9, 128, 4, 17, prefix_dims=ks)
    mvn.sync()
    ref = oracle.excursion(mu, S, 0.8, 0.9, oracle.QMC(128, 4, 17), prefix_dims=ks)
    np.testing.assert_allclose(r["marginal"].cpu().numpy(), ref["marginal"], rtol=1e-14,
                               atol=1e-300)
    assert np.array_equal(r["order"].cpu().numpy(), ref["order"])
    np.testing.assert_allclose(r["F"].cpu().numpy(), ref["F"], rtol=1e-9, atol=1e-10)
    assert np.array_equal(r["region"].cpu().numpy(), ref["region"])


def test_excursion_all_prefixes_and_ties(mvn):
    g = 8
    c = inputs.grid_coords(g)
    n = g * g
    S = oracle.matern(c, 1.0, 0.2, 1.5, nugget=1e-4)
    mu = np.full(n, 1.2)      # every marginal equal: ties broken by index on both sides
    r = mvn.mvn_excursion(_t(mu), mvn.to_colmajor(_t(S)), 0.8, 0.5, 64, 4, 3)
    mvn.sync()
    ref = oracle.excursion(mu, S, 0.8, 0.5, oracle.QMC(64, 4, 3))
    assert np.array_equal(r["order"].cpu().numpy(), np.arange(n))
    np.testing.assert_allclose(r["F"].cpu().numpy(), ref["F"], rtol=1e-9, atol=1e-10)
    assert np.all(np.diff(r["F"].cpu().numpy()) <= 0)
    assert np.array_equal(r["region"].cpu().numpy(), ref["region"])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_excursion_graph_replays_match_eager(mvn, prec):
    """The captured confidence-region pipeline (mvn_excursion_graph) gives bit-identical results
    to the eager call, on the field it was captured with and, after the field is updated in
    place, on the new field; two launches in a row."""
    g = 11
    c = inputs.grid_coords(g)
    n = g * g
    S = mvn.to_colmajor(_t(oracle.matern(c, 1.0, 0.15, 0.5, nugget=1e-6)))
    mu0 = 0.9 + 0.7 * inputs.standard_normals(n, 41)
    mu1 = 1.0 + 0.6 * inputs.standard_normals(n, 42)
    ks = [2, 9, 40, 41, 77, n]
    mud = _t(mu0)
    G = mvn.mvn_excursion_graph(mud, S, 0.8, 0.9, 96, 4, 23, prefix_dims=ks, prec=prec)
    try:
        for mu in (mu0, mu1, mu1):
            mud.copy_(_t(mu))
            G.launch()
            assert G.sync() == 0
            ref = mvn.mvn_excursion(_t(mu), S, 0.8, 0.9, 96, 4, 23, prefix_dims=ks, prec=prec)
            mvn.sync()
            for k in ("order", "marginal", "F", "region"):
                assert torch.equal(G.result[k], ref[k]), k
        assert G.kernels > 10
    finally:
        G.close()


def test_excursion_mixed_vs_oracle(mvn):
    """MVN_MIXED confidence region (tensor-core Cholesky of the permuted covariance and
    tensor-core sweep) against the FP64 oracle: order bit-exact, |d log F| <= 1e-4 (the bound
    stated for the mixed paths), and the region equal wherever F is not within that bound of
    the level."""
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
    d = np.abs(np.log(F) - np.log(ref["F"]))
    print(f"mixed excursion: max |d log F| {d.max():.2e}")
    assert d.max() <= 1e-4
    if np.all(np.abs(np.log(ref["F"]) - np.log(0.9)) > 1e-4):
        assert np.array_equal(r["region"].cpu().numpy(), ref["region"])


# ------------------------------------------------------------------ mixed path: stated error

def test_mixed_simt_error_w4(mvn):
    """Workload W4 (n=4096, Matern 3/2): the mixed path's error against the FP64 oracle,
    |d log P| <= 1e-4 (the stated bound of the mixed path)."""
    w = inputs.WORKLOADS["W4"]
    c = inputs.grid_coords(w["g"])
    n = c.shape[0]
    a, b = inputs.limits_for(w, n)
    S = oracle.matern_closed(c, w["sigma2"], w["range"], w["nu"], w["nugget"])
    Lo = oracle.cholesky_lapack(S)
    L = mvn.to_colmajor(_t(Lo))
    Ntot = w["Ns"] * w["M"]
    lw64 = torch.empty(Ntot, dtype=torch.float64, device=DEV)
    lwmx = torch.empty(Ntot, dtype=torch.float64, device=DEV)
    o64 = mvn.mvn_sov(_t(a), _t(b), L, w["Ns"], w["M"], w["seed"], path_logw=lw64).cpu().numpy()
    omx = mvn.mvn_sov(_t(a), _t(b), L, w["Ns"], w["M"], w["seed"], prec="mixed_simt",
                      path_logw=lwmx).cpu().numpy()
    mvn.sync()
    ref = oracle.sov_logw(a, b, Lo, oracle.QMC(w["Ns"], w["M"], w["seed"]), paths=(0, 16))
    _check_logw(lw64.cpu().numpy()[:16], ref)
    d = np.abs(lwmx.cpu().numpy() - lw64.cpu().numpy())
    print(f"W4 mixed_simt: dlogP={omx[0] - o64[0]:.3e} per-path max {d.max():.3e}")
    assert abs(omx[0] - o64[0]) <= 1e-4
