"""Plain FP64 CPU oracle for the SOV estimator of MVN probabilities and the confidence-region
loop built on it.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, obviously-correct reference the GPU library
is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library (``paper_2405_14892_gb300``)
and never imports it; both sides are fed by the seeded generators in
``paper_2405_14892_gb300.inputs``, which hold none of the method's arithmetic.

Every function names the passage of the paper it follows (Eq. / Alg. / Sec. numbers of
arXiv 2405.14892).  Library primitives used as single steps: libm ``erfc``, scipy's Bessel
``kv`` and ``gamma`` (Eq. 6), numpy's ``argsort`` (Alg. 1 ordering), ``svd`` (TLR
compression) and ``inv`` (the inverses printed in Eq. 7), Python's exact integer ``isqrt``
(lattice generators).

Pins (tests/test_oracle_*.py) tie each function to something other than itself: closed forms,
quadrature, brute-force Monte Carlo, textbook special cases and invariants.  Parts with no such
pin say "parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mvn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

U64_MASK = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP, strict IEEE: no fast-math, no FMA
    contraction, so results do not depend on the host ISA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-std=c11", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    d, i64, i32, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
    P = ctypes.c_void_p
    lib.orc_Phi.restype = d
    lib.orc_Phi.argtypes = [d]
    lib.orc_Q.restype = d
    lib.orc_Q.argtypes = [d]
    lib.orc_Phinv.restype = d
    lib.orc_Phinv.argtypes = [d]
    for f in (lib.orc_Phi_vec, lib.orc_Q_vec, lib.orc_Phinv_vec):
        f.restype = None
        f.argtypes = [i64, P, P]
    lib.orc_splitmix64.restype = u64
    lib.orc_splitmix64.argtypes = [u64, u64]
    lib.orc_shifts.restype = None
    lib.orc_shifts.argtypes = [u64, i32, i32, P]
    lib.orc_points.restype = None
    lib.orc_points.argtypes = [i64, P, P, P, P]
    lib.orc_cholesky.restype = i32
    lib.orc_cholesky.argtypes = [i32, P, i64]
    lib.orc_cholesky_grad.restype = None
    lib.orc_cholesky_grad.argtypes = [i32, P, i64, P]
    lib.orc_sov_paths.restype = None
    lib.orc_sov_paths.argtypes = [i32, P, P, P, i64, i64, P, P, i64, i64, P, P, P, i32, P, P,
                                  i32]
    lib.orc_cholesky_reorder.restype = i32
    lib.orc_cholesky_reorder.argtypes = [i32, P, P, i64, P, P, P]
    lib.orc_sov_step_vec.restype = None
    lib.orc_sov_step_vec.argtypes = [i64, P, P, P, P, P, P, P]
    lib.orc_sov_grad.restype = None
    lib.orc_sov_grad.argtypes = [i32, P, P, P, i64, i64, i64, P, P, P, P, P, P]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------- univariate normal

def Phi(x):
    """Phi(x) = P(Z <= x) (Table I; Eq. 2), as erfc(-x/sqrt 2)/2."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    _load().orc_Phi_vec(x.size, _ptr(x), _ptr(out))
    return out


def Q(x):
    """Q(x) = P(Z > x) = 1 - Phi(x), the upper tail without cancellation."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    _load().orc_Q_vec(x.size, _ptr(x), _ptr(out))
    return out


def Phinv(p):
    """Phi^-1(p) (Eq. 2) by Wichura's AS241 (PPND16)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty_like(p)
    _load().orc_Phinv_vec(p.size, _ptr(p), _ptr(out))
    return out


# --------------------------------------------------------------------------- lattice

def primes(count: int) -> list[int]:
    """The first `count` primes 2, 3, 5, ... (sieve of Eratosthenes)."""
    if count <= 0:
        return []
    limit = 16
    while True:
        sieve = bytearray([1]) * (limit + 1)
        sieve[0:2] = b"\x00\x00"
        for p in range(2, math.isqrt(limit) + 1):
            if sieve[p]:
                sieve[p * p::p] = bytearray(len(range(p * p, limit + 1, p)))
        ps = [i for i in range(limit + 1) if sieve[i]]
        if len(ps) >= count:
            return ps[:count]
        limit *= 2


def lattice_alpha(n: int) -> np.ndarray:
    """Richtmyer rank-1 lattice generators in 64-bit fixed point:
    alpha_i = floor(sqrt(p_i) * 2^64) mod 2^64 = isqrt(p_i * 2^128) mod 2^64, p_i the i-th prime
    (p_0 = 2).  These replace the i.i.d. uniforms R of Alg. 2 (reading stated in the module of
    the C oracle)."""
    return np.array([math.isqrt(p << 128) & U64_MASK for p in primes(n)], dtype=np.uint64)


def lattice_shifts(seed: int, M: int, n: int) -> np.ndarray:
    """Random shifts Delta[q, i] = SplitMix64(seed, counter q*2^32 + i), shape (M, n) uint64."""
    out = np.empty((M, n), dtype=np.uint64)
    if M * n:
        _load().orc_shifts(ctypes.c_uint64(seed & U64_MASK), M, n, _ptr(out))
    return out


def splitmix64(seed: int, counter: int) -> int:
    return int(_load().orc_splitmix64(ctypes.c_uint64(seed & U64_MASK),
                                      ctypes.c_uint64(counter & U64_MASK)))


def lattice_points(j, alpha, delta) -> np.ndarray:
    """w = ((W >> 11) + 1/2) 2^-53, W = j*alpha + delta mod 2^64 (elementwise, broadcast)."""
    j, alpha, delta = np.broadcast_arrays(np.asarray(j, dtype=np.uint64),
                                          np.asarray(alpha, dtype=np.uint64),
                                          np.asarray(delta, dtype=np.uint64))
    j = np.ascontiguousarray(j)
    alpha = np.ascontiguousarray(alpha)
    delta = np.ascontiguousarray(delta)
    out = np.empty(j.shape, dtype=np.float64)
    _load().orc_points(j.size, _ptr(j), _ptr(alpha), _ptr(delta), _ptr(out))
    return out


# --------------------------------------------------------------------------- covariance (Eq. 6)

def matern(coords: np.ndarray, sigma2: float, rng: float, nu: float, nugget: float = 0.0):
    """Matern covariance of Eq. 6 written out with the Bessel function K_nu:
    C(h) = sigma2 / (2^(nu-1) Gamma(nu)) (h/a)^nu K_nu(h/a), C(0) = sigma2, plus `nugget` on
    the diagonal.  Returns the dense n x n matrix (float64)."""
    from scipy.special import gamma, kv
    c = np.asarray(coords, dtype=np.float64)
    h = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    x = h / rng
    with np.errstate(invalid="ignore", divide="ignore"):
        C = sigma2 / (2.0 ** (nu - 1.0) * gamma(nu)) * x ** nu * kv(nu, x)
    C[h == 0.0] = sigma2
    C[np.isnan(C)] = 0.0
    C += nugget * np.eye(len(c))
    return C


def matern_closed(coords: np.ndarray, sigma2: float, rng: float, nu: float, nugget: float = 0.0,
                  dtype=np.float64):
    """Eq. 6 for half-integer nu through the closed forms of K_nu (nu = 1/2: e^-x; 3/2:
    (1+x) e^-x; 5/2: (1 + x + x^2/3) e^-x), for sizes where the Bessel form is too slow.
    Pinned against `matern` (tests/test_oracle_pins.py)."""
    c = np.asarray(coords, dtype=np.float64)
    n = len(c)
    C = np.empty((n, n), dtype=dtype)
    step = max(1, (1 << 24) // max(n, 1))
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        h = np.sqrt(((c[r0:r1, None, :] - c[None, :, :]) ** 2).sum(-1))
        x = h / rng
        if nu == 0.5:
            v = np.exp(-x)
        elif nu == 1.5:
            v = (1.0 + x) * np.exp(-x)
        elif nu == 2.5:
            v = (1.0 + x + x * x / 3.0) * np.exp(-x)
        else:
            raise ValueError("closed forms only for nu in {0.5, 1.5, 2.5}")
        C[r0:r1] = sigma2 * v
    C[np.diag_indices(n)] = sigma2 + nugget
    return C


def cholesky_lapack(A: np.ndarray) -> np.ndarray:
    """Lower Cholesky factor from LAPACK (numpy), used as a library step where the plain column
    loop of `cholesky` is too slow (n in the thousands); pinned against `cholesky` at small n."""
    return np.linalg.cholesky(A)


def matern_grad_params(coords, sigma2, rng, nu):
    """dC/dsigma2 and dC/drange of Eq. 6 for nu in {1/2, 3/2}, from the closed forms
    K_1/2 -> exp(-x) and K_3/2 -> (1 + x) exp(-x):
      nu=1/2: dC/da = sigma2 x e^-x / a;   nu=3/2: dC/da = sigma2 x^2 e^-x / a;
      dC/dsigma2 = C / sigma2 (nugget excluded)."""
    c = np.asarray(coords, dtype=np.float64)
    h = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    x = h / rng
    if nu == 0.5:
        base = np.exp(-x)
        dA = sigma2 * x * np.exp(-x) / rng
    elif nu == 1.5:
        base = (1.0 + x) * np.exp(-x)
        dA = sigma2 * x * x * np.exp(-x) / rng
    else:
        raise ValueError("closed-form derivatives only for nu in {0.5, 1.5}")
    return base, dA


# --------------------------------------------------------------------------- Cholesky

def cholesky(A: np.ndarray):
    """Lower Cholesky factor (Alg. 1 "dpotrf"), plain column loop.  Returns (L, info) with
    info = 0, or the 1-based column of the first non-positive pivot."""
    n = A.shape[0]
    F = np.asfortranarray(np.array(A, dtype=np.float64, copy=True))
    info = _load().orc_cholesky(n, _ptr(F), max(n, 1))
    L = np.tril(F)
    return L, int(info)


def cholesky_reorder(A: np.ndarray, a, b):
    """Cholesky factor with the univariate variable reordering (Gibson, Glasbey and Elston 1994;
    Genz and Bretz 2009, Sec. 4.1.3; not in the paper: a variance-reducing variant of the SOV
    estimator of Eq. 2): at step i the variable with the smallest conditional interval
    probability given the truncated-normal means of the variables already placed goes next.
    Returns (L, perm, a[perm], b[perm], info) with L the lower factor of A[perm, perm]."""
    n = A.shape[0]
    S = np.asfortranarray(np.array(A, dtype=np.float64, copy=True))
    S = np.asfortranarray(np.tril(S) + np.tril(S, -1).T)
    L = np.zeros((n, n), order="F")
    ap = np.ascontiguousarray(a, dtype=np.float64).copy()
    bp = np.ascontiguousarray(b, dtype=np.float64).copy()
    perm = np.zeros(n, dtype=np.int32)
    info = _load().orc_cholesky_reorder(n, _ptr(S), _ptr(L), max(n, 1), _ptr(ap), _ptr(bp),
                                        _ptr(perm))
    return np.array(L), perm, ap, bp, int(info)


def cholesky_grad(L: np.ndarray, Lbar: np.ndarray) -> np.ndarray:
    """Reverse mode of `cholesky`: given dF/dL (lower), return dF/dA for the lower-triangle
    entries of A read by the factorisation (strict upper part zero)."""
    n = L.shape[0]
    Lf = np.asfortranarray(np.tril(L), dtype=np.float64)
    G = np.asfortranarray(np.tril(Lbar), dtype=np.float64)
    _load().orc_cholesky_grad(n, _ptr(Lf), max(n, 1), _ptr(G))
    return np.tril(np.array(G))


# --------------------------------------------------------------------------- SOV

class QMC:
    """Lattice rule: M random shifts x Ns points per shift, total M*Ns paths."""

    def __init__(self, n_points: int, n_shifts: int, seed: int):
        self.Ns = int(n_points)
        self.M = int(n_shifts)
        self.seed = int(seed)

    @property
    def Ntot(self):
        return self.Ns * self.M


def sov_step(a, b, s, lii, W):
    """One dimension of Eq. 2 (Alg. 3's inner step) on independent inputs: the standardised
    limits a' = (a - s)/L_ii, b' = (b - s)/L_ii, the factor Delta = Phi(b') - Phi(a') (upper-tail
    form Q(a') - Q(b') when a' > 0) and y = Phi^-1(Phi(a') + w Delta) (-Phi^-1(Q(a') - w Delta)
    when a' > 0), with w = ((W >> 11) + 1/2) 2^-53 from the 64-bit lattice integer W.  Delta = 0
    gives y = the finite limit; a Phi^-1 argument rounded to 0 or 1 is moved inside (0, 1).
    Returns (y, Delta), broadcast over the inputs."""
    a, b, s, lii, W = np.broadcast_arrays(np.asarray(a, dtype=np.float64),
                                          np.asarray(b, dtype=np.float64),
                                          np.asarray(s, dtype=np.float64),
                                          np.asarray(lii, dtype=np.float64),
                                          np.asarray(W, dtype=np.uint64))
    a, b, s, lii, W = (np.ascontiguousarray(x) for x in (a, b, s, lii, W))
    y = np.empty(a.shape)
    d = np.empty(a.shape)
    _load().orc_sov_step_vec(a.size, _ptr(a), _ptr(b), _ptr(s), _ptr(lii), _ptr(W), _ptr(y),
                             _ptr(d))
    return y, d


def sov_logw(a, b, L, qmc: QMC, paths: Sequence[int] | None = None, return_y: bool = False,
             prefixes: Sequence[int] | None = None, nthreads: int = 0,
             return_delta: bool = False):
    """Per-path log-weights logw_p = sum_i log(Phi(b'_i) - Phi(a'_i)) of Eq. 2/3 (Alg. 3 on one
    path), on the shifted lattice.  `paths` is a contiguous range (p0, p1) or None = all.
    With `return_y` / `return_delta`, also returns y and the factors Delta (paths x n), and with
    `prefixes` the log-weight after each prefix length (for Alg. 1), in that order."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = a.size
    Lf = np.asfortranarray(L, dtype=np.float64)
    alpha = lattice_alpha(n)
    delta = lattice_shifts(qmc.seed, qmc.M, n)
    p0, p1 = (0, qmc.Ntot) if paths is None else (int(paths[0]), int(paths[1]))
    logw = np.empty(p1 - p0)
    Y = np.empty((p1 - p0, n)) if return_y else None
    D = np.empty((p1 - p0, n)) if return_delta else None
    kp = None
    lp = None
    if prefixes is not None:
        kp = np.ascontiguousarray(np.sort(np.asarray(prefixes, dtype=np.int32)))
        lp = np.empty((p1 - p0, kp.size))
    _load().orc_sov_paths(n, _ptr(a), _ptr(b), _ptr(Lf), max(n, 1), qmc.Ns, _ptr(alpha),
                          _ptr(delta), p0, p1, _ptr(logw),
                          _ptr(Y) if Y is not None else None,
                          _ptr(D) if D is not None else None,
                          0 if kp is None else kp.size, _ptr(kp) if kp is not None else None,
                          _ptr(lp) if lp is not None else None, int(nthreads))
    out = [logw]
    if return_y:
        out.append(Y)
    if return_delta:
        out.append(D)
    if prefixes is not None:
        out.append(lp)
    return out[0] if len(out) == 1 else tuple(out)


def _lse(v: np.ndarray) -> float:
    m = np.max(v)
    if not np.isfinite(m):
        return float(m)
    return float(m + np.log(np.sum(np.exp(v - m))))


def estimate(logw: np.ndarray, M: int, err_k: float = 3.0):
    """Alg. 2 "mean(p)" for the shifted rule, in the log domain:
    log P_q = LSE_j(logw_qj) - log Ns per shift; P = mean_q P_q; err = err_k sd_q(P_q)/sqrt(M).
    Returns (logP, P, err)."""
    logw = np.asarray(logw, dtype=np.float64).reshape(M, -1)
    Ns = logw.shape[1]
    lq = np.array([_lse(r) for r in logw]) - math.log(Ns)
    logP = _lse(lq) - math.log(M)
    if not np.isfinite(logP):
        return float(logP), 0.0, 0.0
    rel = np.exp(lq - logP)  # P_q / P
    sd_rel = float(np.std(rel, ddof=1)) if M > 1 else 0.0
    P = math.exp(logP)
    return float(logP), P, err_k * sd_rel / math.sqrt(M) * P


def shift_partials(logw_shard, p0: int, Ns: int, M: int) -> np.ndarray:
    """Per-shift statistics of a shard of the lattice paths (Sec. IV-C: the QMC samples are
    independent, so a problem's paths can be split over workers): the shard holds the
    log-weights of the global paths [p0, p0 + len); for each shift q returns
    (max_p logw_p, sum_p exp(logw_p - max)) over the shard's paths of that shift, (-inf, 0) for a
    shift with none.  Shape (M, 2)."""
    lw = np.asarray(logw_shard, dtype=np.float64)
    p1 = p0 + lw.size
    out = np.zeros((M, 2))
    out[:, 0] = -np.inf
    for q in range(M):
        lo, hi = max(p0, q * Ns), min(p1, (q + 1) * Ns)
        if hi <= lo:
            continue
        r = lw[lo - p0:hi - p0]
        m = float(np.max(r))
        out[q] = (m, float(np.sum(np.exp(r - m))) if np.isfinite(m) else 0.0)
    return out


def combine_partials(parts, Ns: int, M: int, err_k: float = 3.0):
    """Alg. 2 "mean(p)" from the shards' per-shift statistics (a list of (M, 2) arrays from
    `shift_partials` over disjoint path ranges covering the rule): per shift
    log P_q = LSE over the shards of (m_r + log s_r) - log Ns, then the estimate of `estimate`.
    Returns (logP, P, err)."""
    P = np.stack([np.asarray(x, dtype=np.float64).reshape(M, 2) for x in parts])
    with np.errstate(divide="ignore"):
        lr = np.where(P[:, :, 1] > 0, P[:, :, 0] + np.log(P[:, :, 1]), -np.inf)  # (R, M)
    lq = np.array([_lse(lr[:, q]) for q in range(M)]) - math.log(Ns)
    logP = _lse(lq) - math.log(M)
    if not np.isfinite(logP):
        return float(logP), 0.0, 0.0
    rel = np.exp(lq - logP)
    sd_rel = float(np.std(rel, ddof=1)) if M > 1 else 0.0
    Pm = math.exp(logP)
    return float(logP), Pm, err_k * sd_rel / math.sqrt(M) * Pm


def sov(a, b, L, qmc: QMC, err_k: float = 3.0, nthreads: int = 0):
    """P(a <= X <= b), X ~ N(0, L L^T), by the SOV estimator (Eqs. 2-3, Alg. 2-3).
    Returns (logP, P, err)."""
    return estimate(sov_logw(a, b, L, qmc, nthreads=nthreads), qmc.M, err_k)


def sov_grad(a, b, L, qmc: QMC, want_L: bool = True):
    """Gradient of log P-hat with respect to a, b and L (lower) by reverse mode of the per-path
    recurrence, weighted by softmax(logw) (not in the paper: chain rule of Eq. 2).
    Returns (logP, dlogP_da, dlogP_db, dlogP_dL or None)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = a.size
    logw = sov_logw(a, b, L, qmc)
    m = np.max(logw)
    wts = np.exp(logw - m)
    wts /= wts.sum()
    Lf = np.asfortranarray(L, dtype=np.float64)
    alpha = lattice_alpha(n)
    delta = lattice_shifts(qmc.seed, qmc.M, n)
    ga = np.zeros(n)
    gb = np.zeros(n)
    gL = np.zeros((n, n), order="F") if want_L else None
    _load().orc_sov_grad(n, _ptr(a), _ptr(b), _ptr(Lf), max(n, 1), qmc.Ns, qmc.Ntot,
                         _ptr(alpha), _ptr(delta), _ptr(np.ascontiguousarray(wts)), _ptr(ga),
                         _ptr(gb), _ptr(gL) if gL is not None else None)
    logP = estimate(logw, qmc.M)[0]
    return logP, ga, gb, (np.array(gL) if gL is not None else None)


def matern_theta_grad(Sbar_lower, coords, sigma2, rng, nu):
    """theta-bar = sum_{i>=j} Sbar_ij dSigma_ij/dtheta for theta = (sigma2, range), with
    Sbar the gradient with respect to the lower triangle (from `cholesky_grad`)."""
    base, dA = matern_grad_params(coords, sigma2, rng, nu)
    S = np.tril(Sbar_lower)
    return float((S * base).sum()), float((S * dA).sum())


# --------------------------------------------------------------------------- batched + Alg. 1

def sov_batched(dims, offsets, a, b, L, qmc: QMC, err_k: float = 3.0):
    """Independent problems p: P(a[o_p:o_p+k_p] <= X <= b[...]) with X ~ N(0, L_k L_k^T), L_k
    the leading k_p x k_p block of the shared factor.  A loop of single `sov` calls."""
    out = np.zeros((len(dims), 3))
    for p, (k, o) in enumerate(zip(dims, offsets)):
        k, o = int(k), int(o)
        out[p] = sov(a[o:o + k], b[o:o + k], L[:k, :k], qmc, err_k)
    return out


def excursion(mu, Sigma, u, one_minus_alpha, qmc: QMC, prefix_dims=None, err_k: float = 3.0):
    """Confidence-region detection, Alg. 1 with the readings of its limits:
      p_M,i = P(X_i > u) = Q((u - mu_i)/sqrt(Sigma_ii))            (Alg. 1 marginals)
      o = indices of p_M in descending order (stable for ties)      (Alg. 1 ordering)
      L = chol(Sigma[o, o]); a = u - mu[o], b = +inf                (unstandardised limits)
      F_k = P-hat(X_{o_1..o_k} > u) for each prefix length k        (Alg. 1 PMVN loop; Eq. 5)
      region = {o_1..o_K}, K = max{k : F_k >= 1 - alpha}             (Eq. 4)
    Returns dict(order, marginal, F (one per prefix), prefixes, region mask over locations)."""
    mu = np.asarray(mu, dtype=np.float64)
    n = mu.size
    pM = Q((u - mu) / np.sqrt(np.diag(Sigma)))
    order = np.argsort(-pM, kind="stable")
    L, info = cholesky(Sigma[np.ix_(order, order)])
    if info:
        raise np.linalg.LinAlgError(f"not positive definite at column {info}")
    a = u - mu[order]
    b = np.full(n, np.inf)
    ks = np.arange(1, n + 1) if prefix_dims is None else np.asarray(prefix_dims, dtype=np.int64)
    ks_sorted = np.unique(ks)
    _, lp = sov_logw(a, b, L, qmc, prefixes=ks_sorted)
    Fk = {}
    for t, k in enumerate(ks_sorted):
        Fk[int(k)] = estimate(lp[:, t], qmc.M, err_k)[1]
    F = np.array([Fk[int(k)] for k in ks])
    region = np.zeros(n, dtype=np.uint8)
    ok = [int(k) for k in ks_sorted if Fk[int(k)] >= one_minus_alpha]
    K = max(ok) if ok else 0
    region[order[:K]] = 1
    return dict(order=order, marginal=pM, F=F, prefixes=ks, region=region, L=L)


def posterior(mu, Sigma, obs, y, noise_var: float):
    """Posterior of the field x ~ N(mu, Sigma) given y = A x + e, e ~ N(0, noise_var I), where the
    indicator matrix A (n_obs x n) has A[k, obs[k]] = 1 (Sec. V-B):
      Sigma_post = (Sigma^-1 + A^T A / noise_var)^-1                        (Eq. 7)
      mu_post    = mu + Sigma_post A^T (y - A mu) / noise_var                 (Eq. 8)
    written as printed, with explicit inverses (numpy's inv as the library step).  mu may be
    None (zero mean).  Returns (mu_post, Sigma_post), Sigma_post full and symmetric."""
    Sigma = np.asarray(Sigma, dtype=np.float64)
    n = Sigma.shape[0]
    obs = np.asarray(obs, dtype=np.int64)
    y = np.asarray(y, dtype=np.float64)
    mu = np.zeros(n) if mu is None else np.asarray(mu, dtype=np.float64)
    A = np.zeros((obs.size, n))
    A[np.arange(obs.size), obs] = 1.0
    Sigma_post = np.linalg.inv(np.linalg.inv(Sigma) + A.T @ A / noise_var)
    Sigma_post = 0.5 * (Sigma_post + Sigma_post.T)
    mu_post = mu + Sigma_post @ (A.T @ (y - A @ mu)) / noise_var
    return mu_post, Sigma_post


def posterior_parts(Sigma_rows, Sigma_oo, Sigma_o_rows, y, noise_var: float, mu_rows=None,
                    mu_obs=None):
    """Entries of the posterior of Eqs. 7-8 for a subset of sites, where the n x n inverse of
    Eq. 7 cannot be formed: with K = Sigma[obs, obs] + noise_var I, the matrix of Eq. 7 equals
    Sigma - Sigma[:, obs] K^-1 Sigma[obs, :] and Eq. 8 equals mu + Sigma[:, obs] K^-1 (y - mu[obs])
    (the Woodbury identity; pinned against `posterior` as printed).
      Sigma_rows   : Sigma[R, R] for the requested sites R (r x r)
      Sigma_oo     : Sigma[obs, obs] (k x k);  Sigma_o_rows: Sigma[obs, R] (k x r)
    Returns (mu_post[R], Sigma_post[R, R]) (numpy's solve as the library step)."""
    K = np.asarray(Sigma_oo, dtype=np.float64) + noise_var * np.eye(len(y))
    B = np.asarray(Sigma_o_rows, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    resid = y - (0.0 if mu_obs is None else np.asarray(mu_obs))
    sol = np.linalg.solve(K, np.column_stack([B, resid]))
    mu = (0.0 if mu_rows is None else np.asarray(mu_rows)) + B.T @ sol[:, -1]
    S = np.asarray(Sigma_rows, dtype=np.float64) - B.T @ sol[:, :-1]
    return mu, 0.5 * (S + S.T)


# --------------------------------------------------------------------------- tile low rank (Sec. III-E)

def tlr_tile_index(i: int, j: int, nt: int) -> int:
    """Position of off-diagonal tile (i, j), i > j, in column order (1,0),(2,0),..,(nt-1,0),(2,1).."""
    return j * nt - j * (j + 1) // 2 + (i - j - 1)


def tlr_truncate(A: np.ndarray, acc: float, max_rank: int):
    """Truncated SVD of one tile (Sec. III-E: "the ranks of the tiles correspond to the most
    significant singular values"): the smallest rank k with sigma_{k+1} <= acc, capped at
    max_rank.  Returns (U sigma, V, k, capped) with A ~= (U sigma) V^T; by Eckart-Young the
    2-norm error is sigma_{k+1} (numpy's SVD as the library step)."""
    Uf, s, Vt = np.linalg.svd(A, full_matrices=False)
    k = int(np.count_nonzero(s > acc))
    capped = k > max_rank
    k = min(k, max_rank)
    return Uf[:, :k] * s[:k], Vt[:k].T.copy(), k, capped


def tlr_compress(Sigma: np.ndarray, tile: int, acc: float, max_rank: int):
    """TLR form of the lower triangle of Sigma: dense diagonal tiles D[i], and for i > j the
    truncated SVD of tile (i, j).  Returns dict(D, U, V, ranks (column order), capped, nt, m)."""
    n = Sigma.shape[0]
    m = tile
    nt = (n + m - 1) // m
    D, U, V, ranks = [], {}, {}, []
    capped = 0
    for i in range(nt):
        r = slice(i * m, min(n, (i + 1) * m))
        D.append(np.array(Sigma[r, r]))
    for j in range(nt):
        for i in range(j + 1, nt):
            A = Sigma[i * m:min(n, (i + 1) * m), j * m:min(n, (j + 1) * m)]
            u, v, k, cp = tlr_truncate(A, acc, max_rank)
            U[(i, j)], V[(i, j)] = u, v
            ranks.append(k)
            capped += int(cp)
    return dict(D=D, U=U, V=V, ranks=np.array(ranks, dtype=np.int32), capped=capped, nt=nt, m=m,
                n=n, acc=acc, max_rank=max_rank)


def tlr_cholesky(T: dict):
    """TLR Cholesky (Alg. 1 "dpotrf" on TLR tiles, HiCMA-style, Akbudak et al. 2017), left-looking:
      D_kk -= sum_{l<k} U_kl (V_kl^T V_kl) U_kl^T;  L_kk = chol(D_kk)
      A_ik  = U_ik V_ik^T - sum_{l<k} U_il (V_il^T V_kl) U_kl^T   (accumulated densely)
      A_ik ~= U' V'^T truncated at acc (recompression);  L_ik = U' (L_kk^-1 V')^T.
    Returns a new dict with the factor in the same form (D holds the L_kk).
    Pinned by its exact cases: acc -> 0 reduces to the dense Cholesky, and a covariance
    D + U U^T (D block-diagonal on the tiles, U of rank r), whose tiles and factor tiles all have
    rank r, is factorised exactly with the rank capped at r.  At a truncating acc the result is
    an approximation; its reconstruction error is checked to be of the order of acc."""
    nt, acc, kmax = T["nt"], T["acc"], T["max_rank"]
    D = [d.copy() for d in T["D"]]
    U = dict(T["U"])
    V = dict(T["V"])
    ranks = {}
    for k in range(nt):
        Dk = D[k]
        for l in range(k):
            W = V[(k, l)].T @ V[(k, l)]
            Dk -= U[(k, l)] @ W @ U[(k, l)].T
        Lkk = np.linalg.cholesky(0.5 * (Dk + Dk.T))
        D[k] = Lkk
        for i in range(k + 1, nt):
            A = U[(i, k)] @ V[(i, k)].T
            for l in range(k):
                A -= U[(i, l)] @ (V[(i, l)].T @ V[(k, l)]) @ U[(k, l)].T
            u, v, r, _ = tlr_truncate(A, acc, kmax)
            U[(i, k)] = u
            V[(i, k)] = np.linalg.solve(Lkk, v) if r else v   # (u v^T) L^-T = u (L^-1 v)^T
            ranks[(i, k)] = r
    out = dict(T)
    out.update(D=D, U=U, V=V,
               ranks=np.array([ranks[(i, j)] for j in range(nt) for i in range(j + 1, nt)],
                              dtype=np.int32))
    return out


def tlr_to_dense(T: dict) -> np.ndarray:
    """Lower-triangular dense matrix of a TLR object (diagonal tiles lower part, U V^T below)."""
    n, m, nt = T["n"], T["m"], T["nt"]
    A = np.zeros((n, n))
    for i in range(nt):
        r = slice(i * m, min(n, (i + 1) * m))
        A[r, r] = np.tril(T["D"][i])
    for j in range(nt):
        for i in range(j + 1, nt):
            A[i * m:min(n, (i + 1) * m), j * m:min(n, (j + 1) * m)] = T["U"][(i, j)] @ T["V"][(i, j)].T
    return A
