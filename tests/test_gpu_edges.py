"""Edge cases of the SOV recurrence (Eq. 2, Alg. 3) on the GPU against the CPU oracle, through
the C ABI: the elementwise step itself (tails, the underflow branch Delta = 0, the interior
clamp of the Phi^-1 argument), whole sweeps in which every path or only some paths get weight 0
(log-weight -inf exactly, P-hat = 0, MVN_ERR_NUMERIC from mvn_sync), for the FP64 path and the
two mixed sweeps.

Tolerances.  FP64: y and Delta as the library routines allow (CUDA's erfc / normcdfinv against
the oracle's libm erfc / AS241: a few ulps; a subnormal Delta is known to a few quanta of
2^-1074 absolute); per path |d logw| <= 1e-9 max(1, |logw|).  Mixed: the step rounds s and L_ii
to FP32 and evaluates a', Phi and Phi^-1 in FP32 with FP64 only in the deep tails, so a' carries
~3 FP32 roundings (~2e-7 relative) and log Delta moves by ~(|a'| + 1) |d a'| (the Mills ratio)
plus a few ulps of erfcf: the stated bound is |d log Delta| <= 2e-6 (1 + a'^2) with a' the
larger finite standardised limit, and |d y| <= 2e-6 (1 + |y|)."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_14892_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TINY = 2.0 ** -1074


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


def _step_inputs():
    """Step inputs covering both tail branches, infinite limits, the deep tails, the underflow
    branch and the clamp (W = 2^64 - 1 gives w = 1 exactly; small W with a subnormal Delta makes
    w Delta underflow)."""
    rng = np.random.default_rng(31)
    rows = []
    W1 = 2 ** 64 - 1
    # clamp: argument rounded to 1 (a' <= 0 branch) and to 0 (a' > 0 branch)
    rows += [(-np.inf, np.inf, 0.0, 1.0, W1), (1.0, np.inf, 0.0, 1.0, W1),
             (-np.inf, -38.4, 0.0, 1.0, 1 << 40), (-np.inf, -38.0, 0.0, 1.0, 1 << 30)]
    # underflow: Delta = 0 in the upper and in the lower tail
    rows += [(40.0, np.inf, 0.0, 1.0, 1 << 62), (-np.inf, -40.0, 0.0, 1.0, 1 << 62),
             (10.0, np.inf, -30.0, 1.0, 1 << 61)]
    # deep but normal tails and the far fallbacks of the FP32 steps
    for x in (9.5, 12.0, 20.0, 30.0, 37.0):
        rows.append((x, np.inf, 0.0, 1.0, int(rng.integers(0, 2 ** 63)) * 2))
        rows.append((-np.inf, -x, 0.0, 1.0, int(rng.integers(0, 2 ** 63)) * 2))
    # random one-sided and two-sided intervals, shifted and scaled
    for _ in range(2000):
        a = rng.uniform(-6, 4)
        b = a + rng.uniform(0.05, 6)
        kind = rng.integers(0, 4)
        if kind == 0:
            a = -np.inf
        elif kind == 1:
            b = np.inf
        rows.append((a, b, rng.uniform(-2, 2), rng.uniform(0.05, 2.0),
                     int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))))
    cols = list(zip(*rows))
    a, b, s, l = (np.array(c, dtype=np.float64) for c in cols[:4])
    W = np.array(cols[4], dtype=np.uint64)   # exact 64-bit integers (2^64 - 1 included)
    return a, b, s, l, W


def _gpu_step(mvn, prec, a, b, s, l, W):
    Wt = torch.as_tensor(W.view(np.int64), device="cuda")
    y, d = mvn.mvn_sov_step_test(_t(a), _t(b), _t(s), _t(l), Wt, prec=prec)
    mvn.sync()
    return y.cpu().numpy(), d.cpu().numpy()


def test_step_fp64_vs_oracle(mvn):
    a, b, s, l, W = _step_inputs()
    y, d = _gpu_step(mvn, "fp64", a, b, s, l, W)
    yo, do = oracle.sov_step(a, b, s, l, W)
    assert np.all(np.isfinite(y)) and np.all(np.isfinite(yo))
    # the clamp rows give the same finite y on both sides
    np.testing.assert_allclose(y[:4], yo[:4], rtol=1e-13)
    # Delta: a few ulps of the larger tail probability (the difference may cancel), a few quanta
    # where it is subnormal; exactly 0 on both sides where it underflows
    pa = np.where(a - s > 0, oracle.Q((a - s) / l), oracle.Phi((a - s) / l))
    tol_d = 1e-14 * np.maximum(do, pa) + 8 * TINY
    assert np.all(np.abs(d - do) <= tol_d), np.max(np.abs(d - do) / tol_d)
    assert np.array_equal(d == 0.0, do == 0.0)
    # y: the Phi^-1 argument differs by a few ulps (more where a subnormal Delta differs by
    # quanta); y's error is that over phi(y)
    arg_rel = 1e-14 + 8 * TINY / np.maximum(do, TINY)
    tol_y = 1e-13 * (1 + np.abs(yo)) + np.minimum(arg_rel, 1.0) / np.maximum(np.abs(yo), 1.0)
    assert np.all(np.abs(y - yo) <= tol_y), np.max(np.abs(y - yo) / tol_y)


@pytest.mark.parametrize("prec", ["mixed", "mixed_simt"])
def test_step_mixed_stated_bound(mvn, prec):
    a, b, s, l, W = _step_inputs()
    # the mixed steps take s and L_ii in FP32 and the limits in FP32 on their common path: give
    # the oracle the same rounded inputs, so the comparison measures the step's own arithmetic
    # (a' to ~3 FP32 roundings, erfcf and normcdfinvf to a few ulps)
    a, b, s, l = (x.astype(np.float32).astype(np.float64) for x in (a, b, s, l))
    y, d = _gpu_step(mvn, prec, a, b, s, l, W)
    yo, do = oracle.sov_step(a, b, s, l, W)
    assert np.all(np.isfinite(y))
    # the first two rows have W = 2^64 - 1, whose point (2^53 - 1/2) 2^-53 rounds to 1 in FP64
    # (the FP64 step and the oracle clamp the Phi^-1 argument there); the FP32 steps keep
    # 1 - w = 2^-54 unrounded, so their y is the rule's own value, finite and beyond the clamp's
    assert 8.2 < y[0] < 8.4 and 8.4 < y[1] < 8.7
    a, b, s, l, W, y, d, yo, do = (x[2:] for x in (a, b, s, l, W, y, d, yo, do))
    assert np.array_equal(d == 0.0, do == 0.0)
    ok = do > 0
    ap = np.abs(np.where(np.isfinite(a), (a - s) / l, 0.0))
    bp = np.abs(np.where(np.isfinite(b), (b - s) / l, 0.0))
    lim = np.maximum(ap, bp)
    dl = np.abs(np.log(d[ok]) - np.log(do[ok]))
    bound = 2e-6 * (1 + lim[ok] ** 2)
    print(f"{prec} step: max |d log Delta| / bound = {np.max(dl / bound):.3f}, "
          f"max |d log Delta| = {dl.max():.3e}")
    assert np.all(dl <= bound)
    fin = do > 1e-290  # away from the subnormal Delta, where y's argument has few digits
    dy = np.abs(y[fin] - yo[fin])
    boundy = 2e-6 * (1 + np.abs(yo[fin]))
    print(f"{prec} step: max |d y| / bound = {np.max(dy / boundy):.3f}")
    assert np.all(dy <= boundy)


def _matern_case(n, seed):
    g = int(math.ceil(math.sqrt(n)))
    c = inputs.grid_coords(g)[:n]
    S = oracle.matern(c, 1.0, 0.15, 1.5, nugget=1e-4)
    L, info = oracle.cholesky(S)
    assert info == 0
    return S, L


@pytest.mark.parametrize("prec", ["fp64", "mixed_simt", "mixed"])
def test_sweep_every_weight_zero(mvn, prec):
    """One dimension with a' = 40 (Q(40) underflows): every path has log-weight -inf exactly,
    out3 = (-inf, 0, 0), mvn_sync returns MVN_ERR_NUMERIC, and the context stays usable.  The
    dimension sits in the second block of the CUDA-core sweeps and the second super-block of
    the tensor-core sweep (index 150)."""
    n = 200
    S, L = _matern_case(n, 1)
    a = np.full(n, -np.inf)
    b = np.full(n, 1.0)
    # a' = 60 - s/L_ii stays beyond the underflow (~38.5) for every path (|s|/L_ii < 20 here)
    a[150], b[150] = 60.0 * L[150, 150], np.inf
    ref = oracle.sov_logw(a, b, L, oracle.QMC(100, 3, 5))
    assert np.all(ref == -np.inf)
    Lg = mvn.to_colmajor(_t(L))
    lw = torch.empty(300, dtype=torch.float64, device="cuda")
    out = mvn.mvn_sov(_t(a), _t(b), Lg, 100, 3, 5, prec=prec, path_logw=lw)
    st, _ = mvn.context().sync()
    assert st == mvn.MVN_ERR_NUMERIC
    assert np.all(lw.cpu().numpy() == -np.inf)
    o = out.cpu().numpy()
    assert o[0] == -np.inf and o[1] == 0.0 and o[2] == 0.0
    # the context stays usable: the same problem without the impossible dimension
    a[150] = -np.inf
    b[150] = 1.0
    out = mvn.mvn_sov(_t(a), _t(b), Lg, 100, 3, 5, prec=prec)
    assert mvn.context().sync()[0] == 0
    assert np.isfinite(out.cpu().numpy()[0])


@pytest.mark.parametrize("prec", ["fp64", "mixed_simt", "mixed"])
def test_sweep_every_weight_zero_batched(mvn, prec):
    """Batched launch: the problem whose prefix holds the impossible dimension gets
    (-inf, 0, 0), the others their normal estimates; mvn_sync reports MVN_ERR_NUMERIC."""
    n = 140
    S, L = _matern_case(n, 2)
    a = np.full(n, -np.inf)
    b = np.full(n, 1.2)
    b[100] = -60.0 * L[100, 100]       # deep lower tail: Phi(b') underflows on every path
    Lg = mvn.to_colmajor(_t(L))
    dims = [n, 100, 64, 101]
    out = mvn.mvn_sov_batched(dims, [0] * 4, _t(a), _t(b), Lg, 64, 4, 9, prec=prec)
    st, _ = mvn.context().sync()
    assert st == mvn.MVN_ERR_NUMERIC
    o = out.cpu().numpy()
    for p, k in enumerate(dims):
        ref = oracle.sov(a[:k], b[:k], L[:k, :k], oracle.QMC(64, 4, 9))
        if k > 100:
            assert ref[0] == -np.inf and o[p, 0] == -np.inf and o[p, 1] == 0.0
        else:
            tol = 1e-9 if prec == "fp64" else 1e-4
            assert abs(o[p, 0] - ref[0]) <= tol, (p, o[p], ref)


def _straddle_case(n, i_cut):
    """Matern field with a limit a_i at dimension i_cut placed so that the underflow of
    Delta = Q(a') splits the paths: a_i = median of the limit shifts s_i + 38.5 L_ii."""
    S, L = _matern_case(n, 3)
    a = np.full(n, -np.inf)
    b = np.full(n, 1.5)
    q = oracle.QMC(256, 4, 13)
    _, Y = oracle.sov_logw(a, b, L, q, return_y=True)
    s = Y[:, :i_cut] @ L[i_cut, :i_cut]
    a[i_cut] = float(np.median(s)) + 38.5 * L[i_cut, i_cut]
    b[i_cut] = np.inf
    # after an extreme y_i the later correlated dimensions would underflow on every path:
    # leave them unrestricted (factor 1; their steps still run)
    b[i_cut + 1:] = np.inf
    return S, L, a, b, q


@pytest.mark.parametrize("prec", ["fp64", "mixed_simt", "mixed"])
def test_sweep_weight_zero_on_some_paths(mvn, prec):
    """About half of the paths underflow at dimension 150: those carry -inf exactly on both
    sides, the others match the oracle (FP64: 1e-9 relative; mixed: the stated per-path bound
    1e-4 max(1, |logw|)).  Paths whose factor at that dimension is within a few quanta of 2^-1074
    on the oracle's side (the underflow boundary, where the two libraries may round differently)
    or subnormal (y's argument then has few digits) are checked for validity only: -inf or a
    log-weight <= 0, never NaN."""
    n, i_cut = 200, 150
    S, L, a, b, q = _straddle_case(n, i_cut)
    ref, D = oracle.sov_logw(a, b, L, q, return_delta=True)
    zero = ref == -np.inf
    assert zero.any() and (~zero).any()
    Lg = mvn.to_colmajor(_t(L))
    lw = torch.empty(q.Ntot, dtype=torch.float64, device="cuda")
    out = mvn.mvn_sov(_t(a), _t(b), Lg, q.Ns, q.M, q.seed, prec=prec, path_logw=lw)
    assert mvn.context().sync()[0] == 0
    got = lw.cpu().numpy()
    assert not np.any(np.isnan(got)) and np.all(got <= 0.0)
    dmin = D[:, i_cut]
    # FP64: away from the underflow boundary and from subnormal factors; mixed: FP32 limits move
    # a' by ~1e-5 near a' = 38, so keep the factor above 1e-300 (or exactly 0)
    floor = 2.0 ** -1022 if prec == "fp64" else 1e-300
    clear = (dmin == 0.0) | (dmin > floor)
    assert clear.sum() > 0.6 * q.Ntot
    z = clear & zero
    if prec == "fp64":
        assert np.all(got[z] == -np.inf)
    else:
        # the FP32 a' can cross the boundary only within ~1e-5 of it
        assert np.mean(got[z] == -np.inf) > 0.99
    f = clear & ~zero
    assert np.all(np.isfinite(got[f]))
    tol = (1e-9 if prec == "fp64" else 1e-4) * np.maximum(1.0, np.abs(ref[f]))
    err = np.abs(got[f] - ref[f])
    print(f"{prec}: {z.sum()} zero paths, {f.sum()} finite, max |d logw| {err.max():.3e}")
    assert np.all(err <= tol), (err / tol).max()
    est = oracle.estimate(ref, q.M)
    o = out.cpu().numpy()
    assert abs(o[0] - est[0]) <= (1e-9 if prec == "fp64" else 1e-4)
