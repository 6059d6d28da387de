"""torch.autograd.Function for log P(a <= X <= b), X ~ N(0, Sigma(theta)) with a Matern
covariance (Eq. 6) on given locations: gradients with respect to the upper limits b and to the
covariance parameters theta = (sigma2, range).

The forward pass runs the library's chain Matern -> Cholesky -> SOV sweep; the gradient comes
from the library's adjoints (reverse SOV sweep -> Cholesky adjoint -> Matern contraction), all in
CUDA kernels.  The gradients are those of the estimator on its fixed lattice points (the exact
derivative of the estimate).

prec="fp64": every step in FP64.  prec="mixed": the tensor-core Cholesky (MVN_MIXED), the sweep
and its reverse with FP32 limit sums and transformed variables (FP64 elementwise steps,
log-weights and derivative terms), the Cholesky adjoint and the Matern contraction in FP64.
"""
from __future__ import annotations

import torch

from . import mvn


class MVNLogProb(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, sigma2, rng, coords, a, nu, nugget, n_points, n_shifts, seed, prec):
        s2 = float(sigma2)
        rg = float(rng)
        S = mvn.mvn_matern(coords, s2, rg, nu, nugget)
        mvn.mvn_cholesky(S, prec=prec)
        want_theta = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        out3, ga, gb, gL = mvn.mvn_sov_grad(a.contiguous(), b.contiguous(), S, n_points, n_shifts,
                                            seed, prec=prec, want_L=want_theta)
        if want_theta:
            Sbar = mvn.mvn_cholesky_grad(S, gL)
            th = mvn.mvn_matern_grad(coords, s2, rg, nu, Sbar)
        else:
            th = torch.zeros(2, dtype=torch.float64, device=b.device)
        ctx.save_for_backward(gb, th)
        return out3[0].clone()

    @staticmethod
    def backward(ctx, g):
        gb, th = ctx.saved_tensors
        return (g * gb, g * th[0], g * th[1], None, None, None, None, None, None, None, None)


def mvn_log_prob(b, sigma2, rng, coords, a=None, nu=1.5, nugget=0.0, n_points=1000,
                 n_shifts=10, seed=0, prec="fp64"):
    """log P-hat(a <= X <= b) with autograd support for b, sigma2 and range."""
    if prec not in ("fp64", "mixed"):
        raise ValueError("prec must be 'fp64' or 'mixed'")
    if a is None:
        a = torch.full_like(b, float("-inf"))
    return MVNLogProb.apply(b, sigma2, rng, coords, a, nu, nugget, n_points, n_shifts, seed, prec)
