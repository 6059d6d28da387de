"""Pins of the CPU oracle against things other than itself: textbook values, closed forms,
quadrature, brute-force Monte Carlo, library routines of a different implementation, and
invariants of the method.  Each test names the paper passage the pinned function follows."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2405_14892_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------- Phi, Q, Phi^-1 (Eq. 2)

def test_normal_textbook_values():
    for kind, arg, val in _read_golden("normal_quantiles.txt"):
        x, v = float(arg), float(val)
        got = oracle.Phinv([x])[0] if kind == "quantile" else oracle.Phi([x])[0]
        # Phi(x) has relative condition number ~ x^2 in the tail (the x/sqrt(2) scaling is
        # rounded before erfc), so the tolerance grows with x^2
        rtol = 2e-15 if kind == "quantile" else 4e-16 * (4 + x * x)
        assert abs(got - v) <= rtol * abs(v) + 1e-300, (kind, arg, got, v)


def test_phinv_round_trip_and_other_implementation():
    from scipy.special import ndtr, ndtri
    u = np.concatenate([10.0 ** -np.linspace(300, 1, 400), np.linspace(0.01, 0.99, 199)])
    z = oracle.Phinv(u)
    # round trip through Phi (lower tail): exact to a few ulps of u times the condition
    # number of Phi at z (~ z^2 in the tail)
    assert np.all(np.abs(oracle.Phi(z) - u) <= 5e-16 * (8 + 2 * z * z) * u)
    # a different implementation (Cephes ndtri / ndtr)
    np.testing.assert_allclose(z, ndtri(u), rtol=2e-15, atol=1e-300)
    x = np.linspace(-37, 8, 1000)
    assert np.all(np.abs(oracle.Phi(x) - ndtr(x)) <= 5e-16 * (8 + 2 * x * x) * ndtr(x))
    # symmetry Q(x) = Phi(-x), and the upper-tail form is accurate where 1-Phi cancels
    np.testing.assert_array_equal(oracle.Q(x), oracle.Phi(-x))
    assert oracle.Phi([0.0])[0] == 0.5
    assert oracle.Phinv([0.5])[0] == 0.0
    assert oracle.Phinv([0.0])[0] == -np.inf and oracle.Phinv([1.0])[0] == np.inf


# ----------------------------------------------------------------- lattice (Alg. 2 "R")

def test_splitmix64_reference_outputs():
    for c, h in _read_golden("splitmix64.txt"):
        assert oracle.splitmix64(0, int(c)) == int(h, 16)


def test_lattice_alpha_exact():
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    al = oracle.lattice_alpha(200)
    ps = oracle.primes(200)
    assert ps[:10] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29] and ps[-1] == 1223
    for p, a in zip(ps, al):
        s = Decimal(p).sqrt()
        frac = s - int(s)
        assert int(a) == int(frac * (Decimal(2) ** 64))


def test_lattice_points_fixed_point_rule():
    rng = np.random.default_rng(0)
    j = rng.integers(1, 10 ** 6, size=1000).astype(np.uint64)
    al = oracle.lattice_alpha(1000)
    de = rng.integers(0, 2 ** 63, size=1000).astype(np.uint64) * np.uint64(2)
    w = oracle.lattice_points(j, al, de)
    for t in range(0, 1000, 37):
        W = (int(j[t]) * int(al[t]) + int(de[t])) % 2 ** 64
        assert w[t] == ((W >> 11) + 0.5) / 2.0 ** 53
    assert np.all((w > 0) & (w < 1))


def test_lattice_rank1_structure():
    # for one dimension, the Ns points of a shift are an equispaced-in-the-torus orbit:
    # sorted fractional parts have gaps taking at most 3 distinct values (three-gap theorem)
    al = oracle.lattice_alpha(3)
    w = np.sort(oracle.lattice_points(np.arange(1, 1001, dtype=np.uint64), al[2], np.uint64(0)))
    gaps = np.diff(np.concatenate([w, [w[0] + 1]]))
    assert len(np.unique(np.round(gaps, 12))) <= 3


# ----------------------------------------------------------------- Cholesky (Alg. 1 dpotrf)

def _spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A @ A.T / n + np.eye(n)


def test_cholesky_vs_lapack_and_backward_error():
    A = _spd(150, 1)
    L, info = oracle.cholesky(A)
    assert info == 0
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-13)
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) < 150 * 2.2e-16


def test_cholesky_threads_do_not_change_the_result():
    """The column loop shares the rows of each column among OpenMP threads; every entry is the
    same serial sum, so one thread and all threads give identical bits."""
    import subprocess
    import sys
    A = _spd(700, 5)
    L, info = oracle.cholesky(A)
    assert info == 0
    code = ("import numpy as np, oracle, sys; A = np.load(sys.argv[1]); "
            "L, _ = oracle.cholesky(A); np.save(sys.argv[2], L)")
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        fa, fl = os.path.join(d, "a.npy"), os.path.join(d, "l.npy")
        np.save(fa, A)
        env = dict(os.environ, OMP_NUM_THREADS="1")
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
        subprocess.check_call([sys.executable, "-c", code, fa, fl], env=env)
        L1 = np.load(fl)
    assert np.array_equal(L, L1)


def test_cholesky_equicorrelated_closed_form():
    n, rho = 40, 0.37
    A = (1 - rho) * np.eye(n) + rho * np.ones((n, n))
    L, info = oracle.cholesky(A)
    assert info == 0
    for j in range(n):
        ljj = math.sqrt((1 - rho) * (1 + j * rho) / (1 + (j - 1) * rho))
        assert abs(L[j, j] - ljj) < 1e-14
        lij = rho * (1 - rho) / ((1 + (j - 1) * rho) * ljj)
        np.testing.assert_allclose(L[j + 1:, j], lij, rtol=1e-13)


def test_cholesky_not_pd_info():
    A = np.diag([1.0, 2.0, -1.0, 1.0])
    assert oracle.cholesky(A)[1] == 3
    B = np.array([[1.0, 2.0], [2.0, 1.0]])
    assert oracle.cholesky(B)[1] == 2


def test_cholesky_grad_vs_finite_differences():
    n = 7
    A = _spd(n, 2)
    G = np.tril(np.random.default_rng(3).standard_normal((n, n)))
    L, _ = oracle.cholesky(A)
    Abar = oracle.cholesky_grad(L, G)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 1), (6, 6), (5, 2), (6, 0)]:
        E = np.zeros((n, n))
        E[i, j] = h
        if i != j:
            pass  # the factorisation reads only the lower triangle
        Lp, _ = oracle.cholesky(A + E)
        Lm, _ = oracle.cholesky(A - E)
        fd = ((Lp - Lm) * G).sum() / (2 * h)
        assert abs(fd - Abar[i, j]) < 1e-7 * max(1, abs(fd)), (i, j, fd, Abar[i, j])
    # n = 1: L = sqrt(A), dL/dA = 1/(2 sqrt A)
    g = oracle.cholesky_grad(np.array([[2.0]]), np.array([[1.0]]))
    assert abs(g[0, 0] - 1 / (2 * 2.0)) < 1e-16


# ----------------------------------------------------------------- Matern (Eq. 6)

def test_matern_bessel_form_matches_closed_forms():
    c = inputs.random_coords(30, 5)
    h = np.sqrt(((c[:, None] - c[None]) ** 2).sum(-1))
    for nu, f in [(0.5, lambda x: np.exp(-x)), (1.5, lambda x: (1 + x) * np.exp(-x)),
                  (2.5, lambda x: (1 + x + x * x / 3) * np.exp(-x))]:
        C = oracle.matern(c, 1.7, 0.2, nu)
        np.testing.assert_allclose(C, 1.7 * f(h / 0.2), rtol=1e-12, atol=1e-15)


def test_matern_closed_vs_bessel_and_lapack_vs_loop():
    c = inputs.grid_coords(9)
    for nu in (0.5, 1.5, 2.5):
        np.testing.assert_allclose(oracle.matern_closed(c, 1.2, 0.3, nu, 1e-3),
                                   oracle.matern(c, 1.2, 0.3, nu, 1e-3), rtol=1e-12, atol=1e-15)
    S = oracle.matern(c, 1.0, 0.3, 1.5, 1e-4)
    np.testing.assert_allclose(oracle.cholesky_lapack(S), oracle.cholesky(S)[0], rtol=1e-9,
                               atol=1e-12)


def test_matern_param_grad_vs_fd():
    c = inputs.random_coords(12, 6)
    for nu in (0.5, 1.5):
        base, dA = oracle.matern_grad_params(c, 1.3, 0.15, nu)
        h = 1e-6
        fd = (oracle.matern(c, 1.3, 0.15 + h, nu) - oracle.matern(c, 1.3, 0.15 - h, nu)) / (2 * h)
        np.testing.assert_allclose(dA, fd, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(base * 1.3, oracle.matern(c, 1.3, 0.15, nu), rtol=1e-12)


# ----------------------------------------------------------------- SOV (Eqs. 2-3, Alg. 2-3)

Q1 = oracle.QMC(256, 8, 77)


def test_sov_n1_exact_per_path():
    for a, b, l in [(-np.inf, 0.3, 1.0), (-0.7, 1.2, 2.0), (3.0, 9.0, 1.0), (-9.0, -6.0, 1.5)]:
        lw = oracle.sov_logw([a], [b], np.array([[l]]), Q1)
        ex = math.log(oracle.Phi([b / l])[0] - oracle.Phi([a / l])[0]) if a / l <= 0 else \
            math.log(oracle.Q([a / l])[0] - oracle.Q([b / l])[0])
        np.testing.assert_array_equal(lw, ex)


def test_sov_independent_product_per_path():
    n = 12
    rng = np.random.default_rng(4)
    sd = rng.uniform(0.5, 2.0, n)
    a = rng.uniform(-3, 0, n)
    b = a + rng.uniform(0.1, 4, n)
    a[::3] = -np.inf
    lw = oracle.sov_logw(a, b, np.diag(sd), Q1)
    ex = sum(math.log(oracle.Phi([b[i] / sd[i]])[0] - oracle.Phi([a[i] / sd[i]])[0])
             if a[i] / sd[i] <= 0 else
             math.log(oracle.Q([a[i] / sd[i]])[0] - oracle.Q([b[i] / sd[i]])[0]) for i in range(n))
    np.testing.assert_allclose(lw, ex, rtol=1e-14)


def _bvn_quad(a1, b1, a2, b2, rho):
    from scipy.integrate import quad
    from scipy.special import ndtr
    s = math.sqrt(1 - rho * rho)
    f = lambda x: math.exp(-0.5 * x * x) / math.sqrt(2 * math.pi) * (
        ndtr((b2 - rho * x) / s) - ndtr((a2 - rho * x) / s))
    return quad(f, a1, b1, epsabs=1e-14, epsrel=1e-13, limit=200)[0]


def test_sov_bivariate_vs_quadrature():
    for (a1, b1, a2, b2, rho) in [(-1.0, 0.5, -0.3, 2.0, 0.6), (-np.inf, 0.0, -np.inf, 0.0, -0.4),
                                  (0.2, 3.0, -1.0, 1.0, 0.9)]:
        S = np.array([[1.0, rho], [rho, 1.0]])
        L, _ = oracle.cholesky(S)
        lo1 = a1 if np.isfinite(a1) else -40
        lo2 = a2 if np.isfinite(a2) else -40
        ref = _bvn_quad(lo1, b1, lo2, b2, rho)
        logP, P, err = oracle.sov([a1, a2], [b1, b2], L, oracle.QMC(4096, 10, 3))
        assert abs(P - ref) <= max(err, 1e-12), (P, ref, err)


def test_sov_trivariate_orthant_closed_form():
    for r12, r13, r23 in [(0.5, 0.3, 0.2), (-0.3, 0.4, 0.1), (0.8, 0.7, 0.6)]:
        S = np.array([[1, r12, r13], [r12, 1, r23], [r13, r23, 1.0]])
        L, info = oracle.cholesky(S)
        assert info == 0
        ref = 0.125 + (math.asin(r12) + math.asin(r13) + math.asin(r23)) / (4 * math.pi)
        logP, P, err = oracle.sov(np.full(3, -np.inf), np.zeros(3), L, oracle.QMC(4096, 10, 5))
        assert abs(P - ref) <= err and err < 2e-3, (P, ref, err)


def _equi(n, rho):
    return (1 - rho) * np.eye(n) + rho * np.ones((n, n))


@pytest.mark.parametrize("n", [5, 20, 100])
def test_sov_equicorrelated_half_orthant(n):
    # rho = 1/2: P(X <= 0) = 1/(n+1)
    L, _ = oracle.cholesky(_equi(n, 0.5))
    logP, P, err = oracle.sov(np.full(n, -np.inf), np.zeros(n), L, oracle.QMC(2000, 10, 9))
    assert abs(P - 1 / (n + 1)) <= err, (P, 1 / (n + 1), err)


def _equi_quad(a, b, rho):
    """P(a <= X <= b), X equicorrelated rho >= 0, by 1-D quadrature over the common factor
    X_i = sqrt(rho) Z + sqrt(1-rho) E_i (log domain inside the integrand)."""
    from scipy.integrate import quad
    from scipy.special import log_ndtr, ndtr
    r, s = math.sqrt(rho), math.sqrt(1 - rho)

    def f(z):
        hi = (b - r * z) / s
        lo = (a - r * z) / s
        lg = np.sum(np.log(np.maximum(ndtr(hi) - ndtr(lo), 1e-300)))
        return math.exp(lg - 0.5 * z * z) / math.sqrt(2 * math.pi)
    return quad(f, -12, 12, epsabs=0, epsrel=1e-12, limit=400)[0]


def test_sov_equicorrelated_quadrature_n200():
    n, rho = 200, 0.3
    rng = np.random.default_rng(8)
    b = rng.uniform(1.0, 3.0, n)
    a = np.full(n, -np.inf)
    a[:50] = -b[:50]
    ref = _equi_quad(a, b, rho)
    L, _ = oracle.cholesky(_equi(n, rho))
    logP, P, err = oracle.sov(a, b, L, oracle.QMC(1000, 10, 10))
    assert abs(P - ref) <= err, (P, ref, err)


def test_sov_bruteforce_mc_small_n():
    n = 6
    c = inputs.random_coords(n, 11)
    S = oracle.matern(c, 1.0, 0.3, 0.5)
    L, _ = oracle.cholesky(S)
    rng = np.random.default_rng(12)
    a = rng.uniform(-2.0, -0.5, n)
    b = rng.uniform(0.5, 2.0, n)
    a[0] = -np.inf
    hits = 0
    tot = 0
    for _ in range(10):
        x = rng.standard_normal((1_000_000, n)) @ L.T
        hits += np.count_nonzero(np.all((x >= a) & (x <= b), axis=1))
        tot += x.shape[0]
    pmc = hits / tot
    se_mc = math.sqrt(pmc * (1 - pmc) / tot)
    logP, P, err = oracle.sov(a, b, L, oracle.QMC(4096, 10, 13))
    assert abs(P - pmc) <= 4 * math.hypot(se_mc, err / 3), (P, pmc, se_mc, err)


def test_sov_invariants():
    n = 30
    c = inputs.random_coords(n, 14)
    S = oracle.matern(c, 1.0, 0.2, 1.5, nugget=1e-3)
    L, _ = oracle.cholesky(S)
    rng = np.random.default_rng(15)
    a = rng.uniform(-2, 0, n)
    b = a + rng.uniform(0.5, 3, n)
    a[::4] = -np.inf
    lw = oracle.sov_logw(a, b, L, Q1)
    assert np.all(lw <= 0.0) and np.all(np.isfinite(lw))  # 0 <= e^logw <= 1
    # diagonal scaling: D Sigma D with D a, D b gives the same weights per path
    d = rng.uniform(0.3, 3.0, n)
    Ld, _ = oracle.cholesky(S * np.outer(d, d))
    lw2 = oracle.sov_logw(a * d, b * d, Ld, Q1)
    np.testing.assert_allclose(lw2, lw, rtol=1e-10, atol=1e-10)
    # prefix: trailing dimensions with both limits infinite leave the weights unchanged exactly
    S3 = oracle.matern(np.vstack([c, inputs.random_coords(5, 16)]), 1.0, 0.2, 1.5, nugget=1e-3)
    L3, _ = oracle.cholesky(S3)
    lw3 = oracle.sov_logw(np.concatenate([a, np.full(5, -np.inf)]),
                          np.concatenate([b, np.full(5, np.inf)]), L3, Q1)
    np.testing.assert_array_equal(lw3, lw)
    # monotone in b for steps well above the error
    p1 = oracle.sov(a, b, L, Q1)
    p2 = oracle.sov(a, b + 0.5, L, Q1)
    assert p2[1] - p1[1] > p1[2] + p2[2]


# ----------------------------------------------------------------- Eq. 2 edge cases: underflow and clamp

TINY = 2.0 ** -1074  # smallest subnormal double: the absolute quantum of a subnormal Delta


def test_sov_zero_weight_branch_every_path():
    """Delta underflowing to 0 in a dimension (a' = 40: Q(40) ~ 3.7e-350; b' = -40 likewise)
    gives weight 0 on every path: log-weight -inf exactly, y = the finite limit, no NaN in the
    later dimensions, and the estimate (log P, P, err) = (-inf, 0, 0)."""
    n = 5
    c = inputs.random_coords(n, 21)
    S = oracle.matern(c, 1.0, 0.3, 1.5, nugget=1e-3)
    L, _ = oracle.cholesky(S)
    for a0, b0, y0 in [(40.0 * L[0, 0], np.inf, 40.0), (-np.inf, -40.0 * L[0, 0], -40.0)]:
        a = np.full(n, -np.inf)
        b = np.full(n, 0.5)
        a[0], b[0] = a0, b0
        lw, Y = oracle.sov_logw(a, b, L, Q1, return_y=True)
        assert np.all(lw == -np.inf)
        assert np.all(np.isfinite(Y))
        np.testing.assert_allclose(Y[:, 0], y0, rtol=1e-15)
        assert oracle.estimate(lw, Q1.M) == (-np.inf, 0.0, 0.0)
    # the underflow lies where the mathematics puts it: log Q(40) < log of the smallest double
    from scipy.special import log_ndtr
    assert log_ndtr(-40.0) < math.log(TINY) - 1.0


def test_sov_zero_weight_on_some_paths_vs_scipy():
    """Bivariate case whose second dimension underflows on some paths only: with
    X2 | y1 ~ N(rho y1, 1 - rho^2) and y1 = Phi^-1(w1) (a = -inf, b = +inf in dimension 1), the
    factor of dimension 2 is Q((a2 - rho y1)/sqrt(1 - rho^2)) per path, recomputed here with
    scipy's ndtri and log_ndtr (Cephes and an asymptotic series, implementations other than the
    oracle's AS241 and libm erfc; exp of log_ndtr reaches the subnormal range where Cephes' ndtr
    already returns 0).  Paths whose factor is 0 must carry log-weight -inf exactly; the others
    log(Delta)."""
    from scipy.special import log_ndtr, ndtri
    rho = 0.99
    S = np.array([[1.0, rho], [rho, 1.0]])
    L, _ = oracle.cholesky(S)
    s2 = math.sqrt(1 - rho * rho)
    a = np.array([-np.inf, 5.4])
    b = np.array([np.inf, np.inf])
    q = oracle.QMC(512, 4, 23)
    lw, D = oracle.sov_logw(a, b, L, q, return_delta=True)
    alpha = oracle.lattice_alpha(2)
    delta = oracle.lattice_shifts(q.seed, q.M, 2)
    p = np.arange(q.Ntot)
    j = (p % q.Ns + 1).astype(np.uint64)
    w1 = oracle.lattice_points(j, alpha[0], delta[p // q.Ns, 0])
    y1 = ndtri(w1)
    ap = (a[1] - rho * y1) / s2
    lref = log_ndtr(-ap)
    ref = np.exp(lref)
    zero = ref == 0.0
    assert zero.any() and (~zero).any()          # the case exercises both outcomes
    assert np.all(D[:, 0] == 1.0)
    # a subnormal factor is known to one quantum absolute; a normal one to ~1e-13 relative
    # (the condition number of Q at a' ~ 40 is ~a'^2 times the ~1e-16 error of y1)
    tol = 4 * TINY + 1e-12 * ref
    assert np.all(np.abs(D[:, 1] - ref) <= tol)
    clear = (ref > 8 * TINY) | (ap > 39.0)        # away from the underflow boundary
    assert np.all(lw[clear & zero] == -np.inf)
    fin = clear & ~zero & (ref > 2.0 ** -1022)
    np.testing.assert_allclose(lw[fin], lref[fin], rtol=0, atol=1e-12)
    sub = clear & ~zero & ~fin                    # subnormal factors: one quantum absolute
    assert sub.any()
    assert np.all(np.abs(np.exp(lw[sub]) - ref[sub]) <= 4 * TINY + 1e-12 * ref[sub])


def test_sov_near_underflow_closed_form_per_path():
    """Independent dimensions deep in the upper tail (normal Q(37) ~ 5.7e-300 and subnormal
    Q(38) ~ 2.9e-316): every path's log-weight equals sum_i log Q(a_i/sd_i), against scipy's
    log_ndtr; the subnormal factor carries one quantum of absolute error (relative 2e-8 here)."""
    from scipy.special import log_ndtr
    sd = np.array([1.0, 2.0, 0.5, 1.3])
    a = np.array([37.0, 38.0, 10.0, -np.inf]) * np.where(np.isfinite([1, 1, 1, np.inf]), sd, 1)
    b = np.array([np.inf, np.inf, np.inf, 1.0])
    lw = oracle.sov_logw(a, b, np.diag(sd), Q1)
    ref = log_ndtr(-37.0) + log_ndtr(-38.0) + log_ndtr(-10.0) + log_ndtr(1.0 / 1.3)
    tol = 1e-12 * abs(ref) + 2 * TINY / math.exp(log_ndtr(-38.0))
    assert np.all(np.abs(lw - ref) <= tol), (lw[:3], ref)
    logP = oracle.estimate(lw, Q1.M)[0]
    assert abs(logP - ref) <= tol


def test_sov_step_interior_clamp():
    """The Phi^-1 argument of Eq. 2 rounded to exactly 1 or 0 is moved to the nearest interior
    double, so y stays finite.  The lattice reaches w = 1 exactly: W = 2^64 - 1 gives
    (2^53 - 1) + 1/2, which rounds to 2^53 (ties to even)."""
    from scipy.special import ndtr, ndtri
    W1 = np.uint64(2 ** 64 - 1)
    assert oracle.lattice_points(1, W1, 0)[0] == 1.0
    # a' <= 0 branch: Phi(a') + w Delta = 0 + 1 * 1 = 1  ->  1 - 2^-53  ->  y = -Phi^-1(2^-53)
    y, d = oracle.sov_step(-np.inf, np.inf, 0.0, 1.0, W1)
    assert d == 1.0 and np.isfinite(y)
    np.testing.assert_allclose(y, -ndtri(2.0 ** -53), rtol=1e-14)
    # a' > 0 branch: Q(a') - w Delta = Q(1) - Q(1) = 0  ->  2^-1074  ->  y = -Phi^-1(2^-1074)
    y, d = oracle.sov_step(1.0, np.inf, 0.0, 1.0, W1)
    np.testing.assert_allclose(d, ndtr(-1.0), rtol=1e-15)
    assert np.isfinite(y)
    np.testing.assert_allclose(y, -ndtri(TINY), rtol=1e-14)
    # a' <= 0 branch at an ordinary w: w Delta underflows when Delta is a deep subnormal
    # (Phi(-38.4) is a few quanta), and the clamp gives y = Phi^-1(2^-1074) with Delta > 0
    Wsmall = np.uint64(1 << 40)   # w ~ 2^-24
    y, d = oracle.sov_step(-np.inf, -38.4, 0.0, 1.0, Wsmall)
    assert 0.0 < d < 64 * TINY and np.isfinite(y)
    np.testing.assert_allclose(y, ndtri(TINY), rtol=1e-14)
    # away from the clamp the step is Eq. 2 itself: scipy's ndtri of Phi(a') + w Delta
    rng = np.random.default_rng(24)
    a = rng.uniform(-3, 1, 200)
    b = a + rng.uniform(0.1, 3, 200)
    s = rng.uniform(-1, 1, 200)
    lii = rng.uniform(0.3, 2, 200)
    W = rng.integers(0, 2 ** 63, 200).astype(np.uint64) * np.uint64(2)
    y, d = oracle.sov_step(a, b, s, lii, W)
    ap, bp = (a - s) / lii, (b - s) / lii
    w = oracle.lattice_points(1, W, 0)
    dref = ndtr(bp) - ndtr(ap)
    np.testing.assert_allclose(d, dref, rtol=1e-12)
    np.testing.assert_allclose(y, ndtri(ndtr(ap) + w * dref), rtol=1e-9, atol=1e-12)


def test_estimate_log_domain():
    rng = np.random.default_rng(17)
    lw = rng.uniform(-5, 0, 40)
    logP, P, err = oracle.estimate(lw, 4)
    pq = np.exp(lw).reshape(4, 10).mean(1)
    assert abs(P - pq.mean()) < 1e-15
    assert abs(err - 3 * pq.std(ddof=1) / 2) < 1e-15
    # underflow-safe: the same set shifted by -2000 in log space
    logP2, P2, _ = oracle.estimate(lw - 2000, 4)
    assert abs(logP2 - (logP - 2000)) < 1e-12 and P2 == 0.0
    assert oracle.estimate(np.full(8, -np.inf), 2) == (-np.inf, 0.0, 0.0)


def test_shard_partials_combine_to_the_estimate():
    """Splitting the paths into shards (whole shifts, or cuts inside a shift) and combining the
    per-shift statistics gives the estimate of all paths: the log-sum-exp decomposes exactly, so
    only rounding differs."""
    rng = np.random.default_rng(41)
    M, Ns = 7, 53
    lw = rng.uniform(-60, -40, M * Ns)
    lw[5] = -np.inf
    lw[Ns:2 * Ns] = -np.inf        # a shift whose paths all have weight 0
    ref = oracle.estimate(lw, M)
    for cuts in ([0, M * Ns], [0, 3 * Ns, M * Ns], [0, 17, 100, 101, 250, M * Ns],
                 [0, 1, Ns, 2 * Ns + 5, M * Ns - 1, M * Ns]):
        parts = [oracle.shift_partials(lw[c0:c1], c0, Ns, M) for c0, c1 in zip(cuts, cuts[1:])]
        got = oracle.combine_partials(parts, Ns, M)
        assert abs(got[0] - ref[0]) <= 1e-13 * abs(ref[0])
        assert abs(got[1] - ref[1]) <= 1e-13 * ref[1]
        assert abs(got[2] - ref[2]) <= 1e-10 * ref[2]
    # a shard with no path of a shift reports (-inf, 0) for it
    part = oracle.shift_partials(lw[:10], 0, Ns, M)
    assert part[0, 0] == np.max(lw[:10]) and np.all(part[1:, 0] == -np.inf)
    assert np.all(part[1:, 1] == 0.0)
    # every weight zero
    z = [oracle.shift_partials(np.full(M * Ns, -np.inf), 0, Ns, M)]
    assert oracle.combine_partials(z, Ns, M) == (-np.inf, 0.0, 0.0)


# ----------------------------------------------------------------- univariate variable reordering

def _crit(ap, bp):
    """Conditional interval probability, tail-stable, by scipy (Cephes ndtr)."""
    from scipy.special import ndtr
    return np.where(ap > 0, ndtr(-ap) - ndtr(-bp), ndtr(bp) - ndtr(ap))


def test_reorder_independent_is_sorted_by_interval_probability():
    """With a diagonal covariance nothing is conditioned: the order is the interval
    probabilities sorted ascending (ties in index order), and every path's weight is the exact
    product, as without reordering."""
    n = 15
    rng = np.random.default_rng(51)
    sd = rng.uniform(0.5, 2.0, n)
    a = rng.uniform(-3, 0, n)
    b = a + rng.uniform(0.1, 4, n)
    a[::3] = -np.inf
    b[5] = np.inf
    L, perm, ap, bp, info = oracle.cholesky_reorder(np.diag(sd ** 2), a, b)
    assert info == 0
    ref = np.argsort(_crit(a / sd, b / sd), kind="stable")
    assert np.array_equal(perm, ref)
    np.testing.assert_allclose(np.diag(L), sd[perm], rtol=1e-15)
    assert np.all(np.tril(L, -1) == 0.0)
    lw = oracle.sov_logw(ap, bp, L, Q1)
    np.testing.assert_allclose(lw, np.sum(np.log(_crit(a / sd, b / sd))), rtol=1e-13)
    L1, perm1, *_ = oracle.cholesky_reorder(np.array([[4.0]]), [-1.0], [1.0])
    assert perm1.tolist() == [0] and L1[0, 0] == 2.0


def test_reorder_factor_is_the_cholesky_of_the_permuted_matrix():
    n = 60
    A = _spd(n, 52)
    rng = np.random.default_rng(53)
    a = rng.uniform(-2, 0, n)
    b = a + rng.uniform(0.3, 3, n)
    a[::4] = -np.inf
    L, perm, ap, bp, info = oracle.cholesky_reorder(A, a, b)
    assert info == 0 and sorted(perm.tolist()) == list(range(n))
    Ap = A[np.ix_(perm, perm)]
    np.testing.assert_allclose(L, np.linalg.cholesky(Ap), rtol=0, atol=1e-12)
    assert np.array_equal(ap, a[perm]) and np.array_equal(bp, b[perm])


def test_reorder_greedy_rule_against_schur_complements():
    """Each step's choice has the smallest conditional interval probability among the remaining
    variables, with the conditional variance taken as the Schur complement
    Sigma_rr - Sigma_rI Sigma_II^-1 Sigma_Ir and the shift as Sigma_rI L_II^-T y_I (numpy solves,
    not the oracle's column loop) and y the truncated-normal means (scipy)."""
    from scipy.linalg import solve_triangular
    from scipy.special import ndtr
    n = 14
    A = _spd(n, 54)
    rng = np.random.default_rng(55)
    a = rng.uniform(-1.5, 0.5, n)
    b = a + rng.uniform(0.2, 2.5, n)
    a[::3] = -np.inf
    L, perm, ap, bp, info = oracle.cholesky_reorder(A, a, b)
    Lp = np.linalg.cholesky(A[np.ix_(perm, perm)])
    y = np.zeros(n)
    for i in range(n):
        I = perm[:i]
        rest = [r for r in range(n) if r not in set(I.tolist())]
        if i:
            LI = Lp[:i, :i]
            W = solve_triangular(LI, A[np.ix_(I, rest)], lower=True)   # L_II^-1 Sigma_Ir
            d = A[rest, rest] - np.sum(W * W, axis=0)
            s = W.T @ y[:i]
        else:
            d, s = A[rest, rest], np.zeros(len(rest))
        c = _crit((a[rest] - s) / np.sqrt(d), (b[rest] - s) / np.sqrt(d))
        chosen = rest.index(perm[i])
        assert c[chosen] <= c.min() * (1 + 1e-10), (i, c[chosen], c.min())
        lo, hi = (ap[i] - Lp[i, :i] @ y[:i]) / Lp[i, i], (bp[i] - Lp[i, :i] @ y[:i]) / Lp[i, i]
        phi = lambda x: 0.0 if np.isinf(x) else math.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)
        y[i] = (phi(lo) - phi(hi)) / (ndtr(hi) - ndtr(lo))


def test_reorder_keeps_the_probability_and_reduces_the_error():
    """P(a <= X <= b) does not depend on the order of the variables: the reordered estimate of
    an equicorrelated case matches 1-D quadrature within its error, and its error is smaller
    than without reordering (the purpose of the ordering); the trivariate orthant closed form
    holds as well."""
    n, rho = 100, 0.3
    rng = np.random.default_rng(56)
    b = rng.uniform(0.0, 3.0, n)
    a = np.full(n, -np.inf)
    a[:30] = -b[:30] - rng.uniform(0, 1, 30)
    S = _equi(n, rho)
    ref = _equi_quad(a, b, rho)
    q = oracle.QMC(500, 10, 57)
    L0, _ = oracle.cholesky(S)
    e0 = oracle.sov(a, b, L0, q)
    L, perm, ap, bp, info = oracle.cholesky_reorder(S, a, b)
    e1 = oracle.sov(ap, bp, L, q)
    assert abs(e1[1] - ref) <= e1[2], (e1, ref)
    assert e1[2] < 0.5 * e0[2], (e1[2], e0[2])
    for r12, r13, r23 in [(0.5, 0.3, 0.2), (0.8, 0.7, 0.6)]:
        T = np.array([[1, r12, r13], [r12, 1, r23], [r13, r23, 1.0]])
        L3, p3, a3, b3, _ = oracle.cholesky_reorder(T, np.full(3, -np.inf), np.zeros(3))
        ref3 = 0.125 + (math.asin(r12) + math.asin(r13) + math.asin(r23)) / (4 * math.pi)
        e3 = oracle.sov(a3, b3, L3, oracle.QMC(4096, 10, 5))
        assert abs(e3[1] - ref3) <= e3[2]


# ----------------------------------------------------------------- SOV adjoint

def test_sov_grad_n1_closed_form():
    for a, b in [(-np.inf, 0.4), (-1.0, 0.7)]:
        logP, ga, gb, gL = oracle.sov_grad([a], [b], np.array([[1.0]]), Q1)
        den = oracle.Phi([b])[0] - oracle.Phi([a])[0]
        phi = lambda x: math.exp(-x * x / 2) / math.sqrt(2 * math.pi)
        # all paths carry the same weight; summing 2048 softmax weights costs ~1e-14
        assert abs(gb[0] - phi(b) / den) < 1e-13
        assert abs(ga[0] - (-phi(a) / den if np.isfinite(a) else 0.0)) < 1e-13


def test_sov_grad_independent_closed_form():
    n = 6
    sd = np.array([0.5, 1.0, 2.0, 1.5, 0.8, 1.2])
    b = np.array([0.2, 1.0, -0.3, 0.5, 2.0, 0.0])
    a = np.full(n, -np.inf)
    logP, ga, gb, gL = oracle.sov_grad(a, b, np.diag(sd), Q1)
    from scipy.special import ndtr
    phi = np.exp(-0.5 * (b / sd) ** 2) / math.sqrt(2 * math.pi)
    np.testing.assert_allclose(gb, phi / ndtr(b / sd) / sd, rtol=1e-13)
    # d/dsd_i of log Phi(b/sd) = -phi b / (Phi sd^2)
    np.testing.assert_allclose(np.diag(gL), -phi * b / ndtr(b / sd) / sd ** 2, rtol=1e-12,
                               atol=1e-15)


def test_sov_grad_vs_central_fd():
    n = 10
    c = inputs.random_coords(n, 18)
    S = oracle.matern(c, 1.0, 0.25, 1.5, nugget=1e-3)
    L, _ = oracle.cholesky(S)
    rng = np.random.default_rng(19)
    a = rng.uniform(-2, 0, n)
    a[::2] = -np.inf
    b = a + rng.uniform(1, 3, n)
    b[np.isinf(a)] = rng.uniform(-0.5, 1.5, np.count_nonzero(np.isinf(a)))
    q = oracle.QMC(64, 4, 20)
    logP, ga, gb, gL = oracle.sov_grad(a, b, L, q)
    h = 1e-5
    f = lambda aa, bb, LL: oracle.sov(aa, bb, LL, q)[0]
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd = (f(a, b + e, L) - f(a, b - e, L)) / (2 * h)
        assert abs(fd - gb[i]) < 1e-6 * max(1, abs(fd)), (i, fd, gb[i])
        if np.isfinite(a[i]):
            fd = (f(a + e, b, L) - f(a - e, b, L)) / (2 * h)
            assert abs(fd - ga[i]) < 1e-6 * max(1, abs(fd))
    for (i, k) in [(3, 3), (5, 2), (9, 0), (9, 8)]:
        E = np.zeros((n, n))
        E[i, k] = h
        fd = (f(a, b, L + E) - f(a, b, L - E)) / (2 * h)
        assert abs(fd - gL[i, k]) < 1e-6 * max(1, abs(fd)), (i, k, fd, gL[i, k])


def test_theta_grad_chain_vs_fd():
    """d logP / d(sigma2, range) through Sigma -> L -> SOV, vs central FD on the whole chain."""
    g = 4
    c = inputs.grid_coords(g)
    n = g * g
    b = np.full(n, 0.5)
    a = np.full(n, -np.inf)
    q = oracle.QMC(64, 4, 21)

    def logp(s2, rg):
        L, _ = oracle.cholesky(oracle.matern(c, s2, rg, 1.5, nugget=1e-4))
        return oracle.sov(a, b, L, q)[0]
    s2, rg = 1.0, 0.3
    L, _ = oracle.cholesky(oracle.matern(c, s2, rg, 1.5, nugget=1e-4))
    _, ga, gb, gL = oracle.sov_grad(a, b, L, q)
    Sbar = oracle.cholesky_grad(L, gL)
    d_s2, d_rg = oracle.matern_theta_grad(Sbar, c, s2, rg, 1.5)
    h = 1e-5
    fd_s2 = (logp(s2 + h, rg) - logp(s2 - h, rg)) / (2 * h)
    fd_rg = (logp(s2, rg + h) - logp(s2, rg - h)) / (2 * h)
    assert abs(fd_s2 - d_s2) < 1e-5 * max(1, abs(fd_s2)), (fd_s2, d_s2)
    assert abs(fd_rg - d_rg) < 1e-5 * max(1, abs(fd_rg)), (fd_rg, d_rg)


# ----------------------------------------------------------------- Alg. 1 (confidence region)

def test_excursion_prefix_identity_and_monotone():
    g = 8
    c = inputs.grid_coords(g)
    S = oracle.matern(c, 1.0, 0.2, 0.5)
    mu = inputs.standard_normals(g * g, 22) * 0.8 + 0.9
    q = oracle.QMC(128, 8, 23)
    ks = [1, 5, 17, 40, 64]
    r = oracle.excursion(mu, S, 0.8, 0.95, q, prefix_dims=ks)
    # marginals: P(X_i > u) and descending order
    from scipy.special import ndtr
    np.testing.assert_allclose(r["marginal"], 1 - ndtr((0.8 - mu) / np.sqrt(np.diag(S))),
                               rtol=1e-12, atol=1e-15)
    assert np.all(np.diff(r["marginal"][r["order"]]) <= 0)
    # F_k is exactly the k-prefix SOV problem on the same lattice (Alg. 1 loop)
    L = r["L"]
    a = 0.8 - mu[r["order"]]
    for t, k in enumerate(ks):
        P = oracle.sov(a[:k], np.full(k, np.inf), L[:k, :k], q)[1]
        assert P == r["F"][t]
    assert np.all(np.diff(r["F"]) <= 0)
    K = max([k for k, f in zip(ks, r["F"]) if f >= 0.95], default=0)
    assert r["region"].sum() == K
    assert np.all(r["region"][r["order"][:K]] == 1)


def test_excursion_mc_validation():
    """Sec. V-C MC validation: the detected region D at level 1-alpha satisfies
    P(X > u on all of D) ~ 1 - alpha (checked on D for a few levels by brute-force sampling)."""
    g = 6
    c = inputs.grid_coords(g)
    S = oracle.matern(c, 1.0, 0.3, 0.5)
    mu = 1.6 + 0.5 * inputs.standard_normals(g * g, 24)
    q = oracle.QMC(1024, 10, 25)
    r = oracle.excursion(mu, S, 0.8, 0.9, q)
    Lc = np.linalg.cholesky(S)
    rng = np.random.default_rng(26)
    x = mu + rng.standard_normal((200_000, g * g)) @ Lc.T
    for k in (3, 10, 20):
        D = r["order"][:k]
        pmc = np.mean(np.all(x[:, D] > 0.8, axis=1))
        se = math.sqrt(pmc * (1 - pmc) / x.shape[0])
        assert abs(pmc - r["F"][k - 1]) < 4 * se + 3e-3, (k, pmc, r["F"][k - 1])


# ----------------------------------------------------------------- posterior (Sec. V-B, Eqs. 7-8)

def test_posterior_scalar_closed_form():
    """One site observed once: precision adds, var = 1/(1/s2 + 1/t2), and the mean moves by
    var/t2 of the residual (conjugate normal update)."""
    s2, t2, m, yv = 2.0, 0.25, 0.3, 1.1
    mp, P = oracle.posterior(np.array([m]), np.array([[s2]]), [0], [yv], t2)
    var = 1.0 / (1.0 / s2 + 1.0 / t2)
    assert P[0, 0] == pytest.approx(var, rel=1e-14)
    assert mp[0] == pytest.approx(m + var / t2 * (yv - m), rel=1e-14)


def _random_spd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    return G @ G.T / n + 0.1 * np.eye(n), rng


def test_posterior_is_the_gaussian_conditional():
    """(x, y) is jointly Gaussian with Cov(y) = A Sigma A^T + t2 I and Cov(x, y) = Sigma A^T, so
    the posterior is the textbook conditional (Schur-complement form, no inverse of Sigma);
    includes a site observed twice and an unobserved mean offset."""
    n = 30
    S, rng = _random_spd(n, 40)
    mu = rng.standard_normal(n)
    obs = np.array([3, 7, 7, 0, 29, 12, 18, 5, 22, 9, 14, 26])
    y = rng.standard_normal(obs.size)
    t2 = 0.3
    mp, P = oracle.posterior(mu, S, obs, y, t2)
    A = np.zeros((obs.size, n))
    A[np.arange(obs.size), obs] = 1.0
    Cyy = A @ S @ A.T + t2 * np.eye(obs.size)
    Cxy = S @ A.T
    P_ref = S - Cxy @ np.linalg.solve(Cyy, Cxy.T)
    mp_ref = mu + Cxy @ np.linalg.solve(Cyy, y - A @ mu)
    assert np.abs(P - P_ref).max() < 1e-12 * np.abs(S).max() * 100
    assert np.abs(mp - mp_ref).max() < 1e-11


def test_posterior_leaves_an_independent_block_unchanged():
    S1, rng = _random_spd(8, 41)
    S2, _ = _random_spd(5, 42)
    S = np.zeros((13, 13))
    S[:8, :8], S[8:, 8:] = S1, S2
    mu = rng.standard_normal(13)
    mp, P = oracle.posterior(mu, S, [1, 4, 6], rng.standard_normal(3), 0.5)
    assert np.allclose(P[8:, 8:], S2, atol=1e-13)
    assert np.allclose(P[8:, :8], 0.0, atol=1e-13)
    assert np.allclose(mp[8:], mu[8:], atol=1e-13)
    assert not np.allclose(P[:8, :8], S1)


def test_posterior_repeated_observation_is_an_average():
    """Observing a site twice (values y1, y2, noise t2 each) equals observing it once with the
    mean of the two values and noise t2 / 2."""
    S, rng = _random_spd(10, 43)
    mu = rng.standard_normal(10)
    m2, P2 = oracle.posterior(mu, S, [4, 4, 2], [0.7, 1.5, -0.2], 0.4)
    m1, P1 = oracle.posterior(mu, S, [4], [1.1], 0.2)
    m1b, P1b = oracle.posterior(m1, P1, [2], [-0.2], 0.4)   # then the third observation
    assert np.allclose(P2, P1b, atol=1e-12) and np.allclose(m2, m1b, atol=1e-12)


def test_posterior_noiseless_limit():
    S, rng = _random_spd(12, 44)
    obs = [2, 5, 11]
    y = rng.standard_normal(3)
    mp, P = oracle.posterior(None, S, obs, y, 1e-9)
    assert np.allclose(mp[obs], y, atol=1e-6)
    assert np.all(np.abs(np.diag(P)[obs]) < 1e-8)


# ----------------------------------------------------------------- TLR (Sec. III-E)

def test_posterior_parts_equal_eqs_7_8_as_printed():
    """The site-subset form of the posterior (Woodbury) against Eqs. 7-8 with explicit inverses,
    on every site and on a subset, with and without a prior mean."""
    n = 90
    c = inputs.random_coords(n, 71)
    S = oracle.matern(c, 1.0, 0.2, 0.5)
    rng = np.random.default_rng(72)
    obs = np.sort(rng.choice(n, 25, replace=False))
    y = rng.standard_normal(25)
    mu = 0.3 * rng.standard_normal(n)
    for m in (None, mu):
        mo, So = oracle.posterior(m, S, obs, y, 0.25)
        R = np.array([0, 5, 17, 40, 89])
        mp, Sp = oracle.posterior_parts(S[np.ix_(R, R)], S[np.ix_(obs, obs)], S[np.ix_(obs, R)], y,
                                        0.25, None if m is None else m[R],
                                        None if m is None else m[obs])
        np.testing.assert_allclose(mp, mo[R], rtol=0, atol=1e-12)
        np.testing.assert_allclose(Sp, So[np.ix_(R, R)], rtol=0, atol=1e-12)


def test_tlr_truncation_eckart_young_and_planted_rank():
    rng = np.random.default_rng(30)
    A = rng.standard_normal((60, 7)) @ rng.standard_normal((7, 60))  # rank 7 exactly
    u, v, k, capped = oracle.tlr_truncate(A, 1e-9, 50)
    assert k == 7 and not capped
    np.testing.assert_allclose(u @ v.T, A, atol=1e-10)
    B = rng.standard_normal((50, 50))
    s = np.linalg.svd(B, compute_uv=False)
    acc = s[10] * 1.0000001  # keeps exactly 10 values
    u, v, k, _ = oracle.tlr_truncate(B, acc, 50)
    assert k == 10
    assert abs(np.linalg.norm(B - u @ v.T, 2) - s[10]) < 1e-12 * s[0]  # Eckart-Young
    u, v, k, capped = oracle.tlr_truncate(B, 0.0, 5)
    assert k == 5 and capped


def test_tlr_compress_and_cholesky_reduce_to_dense():
    c = inputs.grid_coords(12)
    S = oracle.matern(c, 1.0, 0.2, 0.5, nugget=1e-6)
    T = oracle.tlr_compress(S, 32, 1e-15, 32)
    assert T["nt"] == 5 and len(T["ranks"]) == 10
    np.testing.assert_allclose(oracle.tlr_to_dense(T), np.tril(S), atol=1e-12)
    L = oracle.tlr_to_dense(oracle.tlr_cholesky(T))
    np.testing.assert_allclose(L, np.linalg.cholesky(S), atol=1e-9)


def test_tlr_cholesky_planted_low_rank_is_exact():
    """Sigma = D + U U^T with D block-diagonal on the tiles and U of rank r: every off-diagonal
    tile of Sigma and of its Cholesky factor has rank r, so the TLR factorisation capped at rank r
    loses nothing and must equal the dense factor to rounding, with factor ranks r (ragged last
    tile included); compressed at a cap of r - 1 every tile reports the cap and loses its
    smallest singular value."""
    rng = np.random.default_rng(31)
    m, nt, r = 24, 5, 3
    n = m * nt - 7
    D = np.zeros((n, n))
    for i in range(nt):
        b = slice(i * m, min(n, (i + 1) * m))
        k = b.stop - b.start
        G = rng.standard_normal((k, k))
        D[b, b] = G @ G.T / k + np.eye(k)
    U = rng.standard_normal((n, r))
    S = D + U @ U.T
    T = oracle.tlr_compress(S, m, 1e-12, r)
    assert np.all(T["ranks"] == r) and T["capped"] == 0
    F = oracle.tlr_cholesky(T)
    assert np.all(F["ranks"] == r)
    np.testing.assert_allclose(oracle.tlr_to_dense(F), np.linalg.cholesky(S), atol=1e-12)
    T2 = oracle.tlr_compress(S, m, 1e-12, r - 1)
    assert T2["capped"] == len(T2["ranks"]) and np.all(T2["ranks"] == r - 1)
    A = S[2 * m:3 * m, 0:m]
    E = A - T2["U"][(2, 0)] @ T2["V"][(2, 0)].T
    assert np.linalg.norm(E, 2) == pytest.approx(np.linalg.svd(A, compute_uv=False)[r - 1],
                                                 rel=1e-10)


def test_tlr_cholesky_error_follows_accuracy():
    c = inputs.grid_coords(16, order="morton")
    S = oracle.matern(c, 1.0, 0.1, 0.5, nugget=1e-6)
    errs = []
    for acc in (1e-2, 1e-4, 1e-6):
        T = oracle.tlr_cholesky(oracle.tlr_compress(S, 32, acc, 32))
        L = oracle.tlr_to_dense(T)
        errs.append(np.linalg.norm(L @ L.T - S, 2))
        assert errs[-1] < 50 * acc, (acc, errs[-1])
    assert errs[0] > errs[1] > errs[2]
