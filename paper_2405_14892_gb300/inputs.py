"""Seeded synthetic inputs shared by the GPU library's tests/bench and the CPU oracle.

This module holds none of the method's arithmetic: it only makes locations, limits, seeds,
problem lists and the synthetic field observations of the paper's protocol (Sec. V-B), from
numpy PCG64 generators.  The posterior of Eqs. 7-8 is not computed here.

Workloads (the paper's Sec. V uses fields on regular grids in [0,1]^2; its datasets are not
available, so these seeded inputs stand in for them):
  W1  n=256   : 16x16 grid, exponential (Matern nu=1/2) sigma2=1, range 0.1; a=-inf,
                b_i ~ U(-1,1) (seed 1); tile 64; 10,000 lattice points x 20 shifts.
  W2  n=16384 : 128x128 grid, Matern nu=3/2, range 0.05, nugget 1e-4; a=-inf, b_i=0.5;
                tile 512; 20,000 paths = 10 shifts x 2,000 points.
  W3  n=4096  : 64x64 grid, Matern nu=1/2, range 0.1; posterior field (Eqs. 7-8) from 640
                noisy observations (noise sd 0.5); threshold u=0.8, level 0.95; 256 prefix problems
                with dims ~ U{64..4096} (seed 3); 10,000 paths = 10 x 1,000.
  W4  n=4096  : 64x64 grid, Matern nu=3/2, sigma2=1, range 0.1, nugget 1e-4; a=-inf, b_i=0.5;
                10,000 paths = 10 x 1,000.
  W5  n=65536 : 256x256 grid (Morton order), exponential range 0.05; tile 1024; TLR acc 1e-5,
                max rank 256; a=-inf, b_i=0.5; 10,000 paths = 10 x 1,000.
  W6  n=40000 : 200x200 grid, exponential range 0.1, 6,250 noisy observations (sd 0.5): the
                paper's synthetic confidence-region protocol at its size (posterior + Alg. 1).
"""
from __future__ import annotations

import numpy as np


def grid_coords(g: int, order: str = "row") -> np.ndarray:
    """Locations s = (i/(g-1), j/(g-1)) of a g x g regular grid in [0,1]^2, shape (g*g, 2).
    order="row": row-major (i outer); order="morton": Z-order of (i, j)."""
    if g == 1:
        return np.zeros((1, 2))
    i, j = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    if order == "morton":
        key = np.zeros(g * g, dtype=np.int64)
        for bit in range(int(np.ceil(np.log2(max(g, 2)))) + 1):
            key |= ((i >> bit) & 1) << (2 * bit + 1)
            key |= ((j >> bit) & 1) << (2 * bit)
        perm = np.argsort(key, kind="stable")
        i, j = i[perm], j[perm]
    elif order != "row":
        raise ValueError(order)
    return np.stack([i / (g - 1), j / (g - 1)], axis=1).astype(np.float64)


def random_coords(n: int, seed: int) -> np.ndarray:
    """n uniform locations in [0,1]^2 (irregular set, Table I "geom")."""
    return np.random.default_rng(seed).random((n, 2))


def uniform_limits(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def prefix_problem_dims(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Problem dimensions k ~ U{lo..hi} (inclusive), int32."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=count).astype(np.int32)


def standard_normals(shape, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


def observations(Sigma_prior: np.ndarray, n_obs: int, noise_sd: float, seed: int):
    """Synthetic observations of the protocol of Sec. V-B: a truth field x ~ N(0, Sigma_prior)
    (drawn through a Cholesky factor of Sigma_prior + 1e-10 I), n_obs distinct sites chosen at
    random (sorted), and y = x[sites] + N(0, noise_sd^2) noise.  Returns (sites int32, y, x).
    The posterior given these (Eqs. 7-8) is computed by the library (mvn_posterior) and by the
    oracle, not here."""
    rng = np.random.default_rng(seed)
    n = Sigma_prior.shape[0]
    C = np.linalg.cholesky(Sigma_prior + 1e-10 * np.eye(n))
    x = C @ rng.standard_normal(n)
    idx = np.sort(rng.choice(n, size=n_obs, replace=False))
    y = x[idx] + noise_sd * rng.standard_normal(n_obs)
    return idx.astype(np.int32), y, x


def observations_at_sites(n: int, n_obs: int, noise_sd: float, seed: int, Sigma_block=None):
    """The same protocol for fields too large to draw whole: n_obs distinct sites chosen at random
    (sorted) first; the truth field is then needed only there, x[sites] ~ N(0, Sigma[sites,
    sites]), drawn through a Cholesky factor of the block (+ 1e-10 I) that the caller supplies
    (Sigma_block(sites) -> the block).  Returns (sites int32, y, x[sites])."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(n, size=n_obs, replace=False))
    B = np.asarray(Sigma_block(idx), dtype=np.float64)
    C = np.linalg.cholesky(B + 1e-10 * np.eye(n_obs))
    x = C @ rng.standard_normal(n_obs)
    y = x + noise_sd * rng.standard_normal(n_obs)
    return idx.astype(np.int32), y, x


WORKLOADS = {
    "W1": dict(name="sov-n256-exp", g=16, nu=0.5, sigma2=1.0, range=0.1, nugget=0.0, tile=64,
               Ns=10_000, M=20, seed=11, limits="uniform", b_seed=1),
    "W2": dict(name="sov-n16384-matern32", g=128, nu=1.5, sigma2=1.0, range=0.05, nugget=1e-4,
               tile=512, Ns=2_000, M=10, seed=12, limits="b=0.5"),
    "W3": dict(name="excursion-n4096-exp", g=64, nu=0.5, sigma2=1.0, range=0.1, nugget=0.0,
               Ns=1_000, M=10, seed=13, u=0.8, level=0.95, nprob=256, dims_lo=64,
               dims_hi=4096, dims_seed=3, n_obs=640, noise_sd=0.5, field_seed=30),
    "W4": dict(name="adjoint-n4096-matern32", g=64, nu=1.5, sigma2=1.0, range=0.1, nugget=1e-4,
               Ns=1_000, M=10, seed=14, limits="b=0.5"),
    "W5": dict(name="tlr-n65536-exp", g=256, nu=0.5, sigma2=1.0, range=0.05, nugget=0.0,
               tile=1024, acc=1e-5, max_rank=256, Ns=1_000, M=10, seed=15, limits="b=0.5",
               order="morton"),
    # the paper's synthetic confidence-region protocol at its own size (Sec. V-B): 40,000 sites
    # of an exponential field of medium correlation (range 0.1), 6,250 observations with noise
    # N(0, 0.5^2), the posterior (Eqs. 7-8), then Alg. 1 over every prefix
    "W6": dict(name="crd-n40000-exp", g=200, nu=0.5, sigma2=1.0, range=0.1, nugget=0.0,
               Ns=1_000, M=10, seed=16, u=0.8, level=0.95, n_obs=6250, noise_sd=0.5,
               field_seed=31),
}


def limits_for(w: dict, n: int):
    """(a, b) of a workload: a = -inf; b as the workload states."""
    a = np.full(n, -np.inf)
    if w.get("limits") == "uniform":
        b = uniform_limits(n, -1.0, 1.0, w["b_seed"])
    else:
        b = np.full(n, 0.5)
    return a, b
