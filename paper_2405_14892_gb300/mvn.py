"""ctypes binding of libmvn.so (include/mvn.h) with the same entry-point names.

Argument marshalling only: every step of the computation runs in the library's CUDA kernels.
Matrices are FP64 torch CUDA tensors in column-major storage (``stride(0) == 1``; a tensor made
with ``colmajor_empty(n, n)`` or ``x.t().contiguous().t()``), vectors are contiguous FP64 CUDA
tensors.  Calls enqueue on torch's current CUDA stream.  There is no CPU fallback: if the library
is missing or the tensors are not on a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmvn.so")

MVN_OK, MVN_ERR_ARG, MVN_ERR_NOT_PD, MVN_ERR_CUDA, MVN_ERR_OOM, MVN_ERR_TIMEOUT, \
    MVN_ERR_NUMERIC, MVN_ERR_NOT_IMPLEMENTED = range(8)
STATUS_NAMES = {0: "MVN_OK", 1: "MVN_ERR_ARG", 2: "MVN_ERR_NOT_PD", 3: "MVN_ERR_CUDA",
                4: "MVN_ERR_OOM", 5: "MVN_ERR_TIMEOUT", 6: "MVN_ERR_NUMERIC",
                7: "MVN_ERR_NOT_IMPLEMENTED"}
PREC = {"fp64": 0, "mixed": 1, "mixed_simt": 2}


class MVNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mvn_qmc(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_shifts", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("err_k", ctypes.c_double)]


class mvn_tune_result(ctypes.Structure):
    _fields_ = [("chol_bulk_p", ctypes.c_int32), ("chol_tail_p", ctypes.c_int32),
                ("sweep_ctas_per_sm", ctypes.c_int32), ("from_cache", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()

# exported symbol -> (restype, argtypes)
_P, _I, _I64, _D, _U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, \
    ctypes.c_uint64
_QP = ctypes.POINTER(mvn_qmc)
SIGNATURES = {
    "mvn_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "mvn_destroy": (_I, [_P]),
    "mvn_set_stream": (_I, [_P, _P]),
    "mvn_last_error": (ctypes.c_char_p, [_P]),
    "mvn_sync": (_I, [_P, ctypes.POINTER(_I)]),
    "mvn_launch_count": (_I64, [_P]),
    "mvn_matern": (_I, [_P, _I, _P, _D, _D, _D, _D, _P, _I64]),
    "mvn_matern_grad": (_I, [_P, _I, _P, _D, _D, _D, _P, _I64, _P]),
    "mvn_cholesky": (_I, [_P, _I, _P, _I64, _I, _I, ctypes.POINTER(_I)]),
    "mvn_cholesky_grad": (_I, [_P, _I, _P, _I64, _P]),
    "mvn_cholesky_reorder": (_I, [_P, _I, _P, _I64, _P, _P, _P, _P, _P, ctypes.POINTER(_I)]),
    "mvn_sov": (_I, [_P, _I, _P, _P, _P, _I64, _QP, _I, _P, _P]),
    "mvn_sov_grad": (_I, [_P, _I, _P, _P, _P, _I64, _QP, _I, _P, _P, _P, _P]),
    "mvn_grad_set_ylimit": (_I, [_P, _I64]),
    "mvn_sov_partial": (_I, [_P, _I, _P, _P, _P, _I64, _QP, _I, _I64, _I64, _P, _P]),
    "mvn_sov_combine": (_I, [_P, _I, _QP, _P, _P]),
    "mvn_sov_batched": (_I, [_P, _I, _P, _P, _P, _P, _P, _I64, _QP, _I, _P]),
    "mvn_posterior": (_I, [_P, _I, _P, _P, _I64, _I, _P, _P, _D, _I, _P, _P, _I64,
                           ctypes.POINTER(_I)]),
    "mvn_excursion": (_I, [_P, _I, _P, _P, _I64, _D, _D, _I, _P, _QP, _I, _I, _P, _P, _P, _P]),
    "mvn_excursion_graph": (_I, [_P, _I, _P, _P, _I64, _D, _D, _I, _P, _QP, _I, _P, _P, _P, _P,
                                 ctypes.POINTER(_P)]),
    "mvn_graph_launch": (_I, [_P]),
    "mvn_graph_sync": (_I, [_P, ctypes.POINTER(_I)]),
    "mvn_graph_kernels": (_I64, [_P]),
    "mvn_graph_destroy": (_I, [_P]),
    "mvn_autotune": (_I, [_P, _I, _I64, _I, ctypes.c_char_p, ctypes.POINTER(mvn_tune_result)]),
    "mvn_tune_set": (_I, [_P, _I, _I64, _I, ctypes.POINTER(mvn_tune_result)]),
    "mvn_tlr_compress": (_I, [_P, _I, _P, _I64, _I, _D, _I, ctypes.POINTER(_P),
                              ctypes.POINTER(_I)]),
    "mvn_tlr_cholesky": (_I, [_P, _P, ctypes.POINTER(_I)]),
    "mvn_tlr_to_dense": (_I, [_P, _P, _P, _I64]),
    "mvn_tlr_ranks": (_I, [_P, _P]),
    "mvn_sov_tlr": (_I, [_P, _P, _P, _P, _QP, _I, _P, _P]),
    "mvn_tlr_free": (_I, [_P]),
    "mvn_lattice_alpha": (_I, [_P, _I, _P]),
    "mvn_lattice_shifts": (_I, [_P, _U64, _I, _I, _P]),
    "mvn_tc_selftest": (_I, [_P, _I, _P, _P, _P]),
    "mvn_sov_step_test": (_I, [_P, _I, _I64, _P, _P, _P, _P, _P, _P, _P]),
    "mvn_sov_fp64_noalloc": (_I, [_I, _P, _P, _P, _I64, _QP, _P, _P, _P]),
    "mvn_wait_selftest": (_I, [_P, _I64]),
    "mvn_timing": (_I, [_P, _I]),
    "mvn_kernel_time": (_I, [_P, ctypes.c_char_p, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
}


def lib():
    """Load libmvn.so (built by ``paper_2405_14892_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build()")
                L = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in SIGNATURES.items():
                    f = getattr(L, name)
                    f.restype = res
                    f.argtypes = args
                _lib = L
    return _lib


class Context:
    """An mvn_ctx bound to one CUDA device and stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the MVN library has no CPU path")
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = _P()
        st = lib().mvn_create(ctypes.byref(h), device, _P(self.stream.cuda_stream))
        if st != MVN_OK:
            raise MVNError(st, "mvn_create failed")
        self.h = h

    def check(self, st: int):
        if st != MVN_OK:
            raise MVNError(st, lib().mvn_last_error(self.h).decode())

    def sync(self) -> tuple[int, int]:
        info = _I(0)
        st = lib().mvn_sync(self.h, ctypes.byref(info))
        return st, info.value

    def launches(self) -> int:
        return int(lib().mvn_launch_count(self.h))

    def timing(self, enable: bool):
        """Record CUDA events around the library's main kernels (see mvn_kernel_time)."""
        self.check(lib().mvn_timing(self.h, 1 if enable else 0))

    def kernel_time(self, name: str) -> tuple[float, int]:
        """(total ms, launches) of kernel `name` since timing was enabled."""
        ms = _D(0.0)
        cnt = _I64(0)
        self.check(lib().mvn_kernel_time(self.h, name.encode(), ctypes.byref(ms),
                                         ctypes.byref(cnt)))
        return ms.value, cnt.value

    def close(self):
        if getattr(self, "h", None):
            lib().mvn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_contexts: dict = {}


def context(device: int | None = None) -> Context:
    """The cached context of the current device and current torch stream."""
    if device is None:
        device = torch.cuda.current_device()
    s = torch.cuda.current_stream(device)
    key = (device, s.cuda_stream)
    c = _contexts.get(key)
    if c is None:
        c = Context(device, s)
        _contexts[key] = c
    return c


# ------------------------------------------------------------------------- tensor helpers

def colmajor_empty(rows: int, cols: int, device="cuda") -> torch.Tensor:
    """An uninitialised FP64 (rows x cols) tensor with column-major storage."""
    return torch.empty((cols, rows), dtype=torch.float64, device=device).t()


def to_colmajor(x: torch.Tensor) -> torch.Tensor:
    return x.to(torch.float64).t().contiguous().t()


def _mat(x: torch.Tensor, n: int, name: str):
    if not x.is_cuda or x.dtype != torch.float64:
        raise ValueError(f"{name} must be a CUDA float64 tensor")
    if x.dim() != 2 or x.shape[0] < n or x.shape[1] < n:
        raise ValueError(f"{name} must be at least {n} x {n}")
    if n > 0 and x.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    ld = max(x.stride(1), 1) if n > 0 else 1
    return _P(x.data_ptr()), ld


def _vec(x: torch.Tensor | None, n: int, name: str, dtype=torch.float64):
    if x is None:
        return None
    if not x.is_cuda or x.dtype != dtype or not x.is_contiguous() or x.numel() < n:
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor with >= {n} elements")
    return _P(x.data_ptr())


def _qmc(n_points: int, n_shifts: int, seed: int, err_k: float = 3.0) -> mvn_qmc:
    return mvn_qmc(int(n_points), int(n_shifts), 0, int(seed) & ((1 << 64) - 1), float(err_k))


# ------------------------------------------------------------------------- entry points

def mvn_matern(coords: torch.Tensor, sigma2: float, rng: float, nu: float, nugget: float = 0.0,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """Lower triangle of the Matern covariance (Eq. 6) into a column-major n x n tensor."""
    n = coords.shape[0]
    if out is None:
        out = colmajor_empty(n, n, coords.device)
    S, ld = _mat(out, n, "out")
    c = context()
    c.check(lib().mvn_matern(c.h, n, _vec(coords.contiguous(), 2 * n, "coords"), sigma2, rng, nu,
                             nugget, S, ld))
    return out


def mvn_matern_grad(coords, sigma2, rng, nu, Sbar: torch.Tensor) -> torch.Tensor:
    n = coords.shape[0]
    out = torch.empty(2, dtype=torch.float64, device=coords.device)
    S, ld = _mat(Sbar, n, "Sbar")
    c = context()
    c.check(lib().mvn_matern_grad(c.h, n, _vec(coords.contiguous(), 2 * n, "coords"), sigma2, rng,
                                  nu, S, ld, _P(out.data_ptr())))
    return out


def mvn_cholesky(A: torch.Tensor, prec: str = "fp64", tile: int = 0, check: bool = True) -> int:
    """In-place lower Cholesky of a column-major FP64 CUDA matrix.  With check=True the call
    waits and returns the LAPACK-style info (raising MVNError on a non-positive pivot)."""
    n = A.shape[0]
    P, ld = _mat(A, n, "A")
    c = context()
    info = _I(0)
    st = lib().mvn_cholesky(c.h, n, P, ld, tile, PREC[prec], ctypes.byref(info) if check else None)
    c.check(st)
    return info.value


def mvn_cholesky_reorder(A: torch.Tensor, a: torch.Tensor, b: torch.Tensor,
                         check: bool = True):
    """In-place factor of A[perm, perm] with the univariate variable reordering.  Returns
    (perm int32 tensor, a[perm], b[perm], info); with check=False the call does not wait and info
    is 0 (a failure then surfaces at the next sync)."""
    n = A.shape[0]
    Ap, ld = _mat(A, n, "A")
    perm = torch.empty(n, dtype=torch.int32, device=A.device)
    a2 = torch.empty(n, dtype=torch.float64, device=A.device)
    b2 = torch.empty(n, dtype=torch.float64, device=A.device)
    info = _I(0)
    c = context()
    st = lib().mvn_cholesky_reorder(c.h, n, Ap, ld, _vec(a, n, "a"), _vec(b, n, "b"),
                                    _vec(perm, n, "perm", dtype=torch.int32), _vec(a2, n, "a_perm"),
                                    _vec(b2, n, "b_perm"), ctypes.byref(info) if check else None)
    if st == MVN_ERR_NOT_PD:
        raise MVNError(st, f"not positive definite at step {info.value}")
    c.check(st)
    return perm, a2, b2, info.value


def mvn_cholesky_grad(L: torch.Tensor, Lbar: torch.Tensor) -> torch.Tensor:
    n = L.shape[0]
    Lp, ld = _mat(L, n, "L")
    Gp, ldg = _mat(Lbar, n, "Lbar")
    if ldg != ld:
        raise ValueError("L and Lbar must have the same leading dimension")
    c = context()
    c.check(lib().mvn_cholesky_grad(c.h, n, Lp, ld, Gp))
    return Lbar


def mvn_sov(a: torch.Tensor, b: torch.Tensor, L: torch.Tensor, n_points: int, n_shifts: int,
            seed: int, prec: str = "fp64", err_k: float = 3.0,
            path_logw: torch.Tensor | None = None, out3: torch.Tensor | None = None):
    """{log P-hat, P-hat, err} (device tensor of 3) for P(a <= X <= b), X ~ N(0, L L^T)."""
    n = a.numel()
    if out3 is None:
        out3 = torch.empty(3, dtype=torch.float64, device=a.device)
    Lp, ld = _mat(L, n, "L")
    q = _qmc(n_points, n_shifts, seed, err_k)
    c = context()
    c.check(lib().mvn_sov(c.h, n, _vec(a, n, "a"), _vec(b, n, "b"), Lp, ld, ctypes.byref(q),
                          PREC[prec], _vec(out3, 3, "out3"),
                          _vec(path_logw, n_points * n_shifts, "path_logw")))
    return out3


def mvn_sov_partial(a: torch.Tensor, b: torch.Tensor, L: torch.Tensor, n_points: int,
                    n_shifts: int, seed: int, p0: int, p1: int, prec: str = "fp64",
                    err_k: float = 3.0, partial: torch.Tensor | None = None,
                    path_logw: torch.Tensor | None = None) -> torch.Tensor:
    """Shard [p0, p1) of the lattice paths: returns the per-shift pairs (2 * n_shifts doubles)
    for mvn_sov_combine."""
    n = a.numel()
    if partial is None:
        partial = torch.empty(2 * n_shifts, dtype=torch.float64, device=a.device)
    Lp, ld = _mat(L, n, "L")
    q = _qmc(n_points, n_shifts, seed, err_k)
    c = context()
    c.check(lib().mvn_sov_partial(c.h, n, _vec(a, n, "a"), _vec(b, n, "b"), Lp, ld,
                                  ctypes.byref(q), PREC[prec], int(p0), int(p1),
                                  _vec(partial, 2 * n_shifts, "partial"),
                                  _vec(path_logw, int(p1) - int(p0), "path_logw")))
    return partial


def mvn_sov_combine(partials: torch.Tensor, n_points: int, n_shifts: int, err_k: float = 3.0,
                    out3: torch.Tensor | None = None) -> torch.Tensor:
    """Estimate {log P, P, err} from the stacked pairs of the shards (nparts x 2 n_shifts)."""
    nparts = partials.numel() // (2 * n_shifts)
    if out3 is None:
        out3 = torch.empty(3, dtype=torch.float64, device=partials.device)
    q = _qmc(n_points, n_shifts, 0, err_k)
    c = context()
    c.check(lib().mvn_sov_combine(c.h, nparts, ctypes.byref(q),
                                  _vec(partials.contiguous(), nparts * 2 * n_shifts, "partials"),
                                  _vec(out3, 3, "out3")))
    return out3


def mvn_sov_grad(a, b, L, n_points, n_shifts, seed, prec="fp64", err_k=3.0, want_L=False):
    n = a.numel()
    out3 = torch.empty(3, dtype=torch.float64, device=a.device)
    ga = torch.empty(n, dtype=torch.float64, device=a.device)
    gb = torch.empty(n, dtype=torch.float64, device=a.device)
    gL = None
    Lp, ld = _mat(L, n, "L")
    if want_L:
        if ld != n:
            raise ValueError("L must be tightly packed (ld == n) when want_L")
        gL = colmajor_empty(n, n, a.device)
    q = _qmc(n_points, n_shifts, seed, err_k)
    c = context()
    c.check(lib().mvn_sov_grad(c.h, n, _vec(a, n, "a"), _vec(b, n, "b"), Lp, ld, ctypes.byref(q),
                               PREC[prec], _P(out3.data_ptr()), _P(ga.data_ptr()),
                               _P(gb.data_ptr()), _P(gL.data_ptr()) if gL is not None else None))
    return out3, ga, gb, gL


def mvn_grad_set_ylimit(nbytes: int):
    """Limit of mvn_sov_grad's y / reverse-sum buffers on the current context (0 = default)."""
    c = context()
    c.check(lib().mvn_grad_set_ylimit(c.h, int(nbytes)))


def mvn_sov_batched(dims, offsets, a, b, L, n_points, n_shifts, seed, prec="fp64", err_k=3.0):
    """Independent problems (dims[p], limits a[off_p:off_p+dims[p]]) sharing the leading blocks
    of L; returns a (nprob, 3) device tensor of {log P-hat, P-hat, err}."""
    nprob = len(dims)
    if len(offsets) != nprob:
        raise ValueError("dims and offsets must have the same length")
    d = (ctypes.c_int * nprob)(*[int(x) for x in dims])
    o = (ctypes.c_int64 * nprob)(*[int(x) for x in offsets])
    nmax = max([int(x) for x in dims] + [0])
    # the library sees raw pointers: the limit vectors must hold every problem's slice
    need = max([int(x) + int(y) for x, y in zip(offsets, dims) if int(y) > 0] + [0])
    Lp, ld = _mat(L, nmax, "L")
    out = torch.empty((nprob, 3), dtype=torch.float64, device=a.device)
    q = _qmc(n_points, n_shifts, seed, err_k)
    c = context()
    c.check(lib().mvn_sov_batched(c.h, nprob, ctypes.cast(d, _P), ctypes.cast(o, _P),
                                  _vec(a, need, "a"), _vec(b, need, "b"), Lp, ld,
                                  ctypes.byref(q), PREC[prec], _P(out.data_ptr())))
    return out


def mvn_posterior(mu: torch.Tensor | None, Sigma: torch.Tensor, obs: torch.Tensor,
                  y: torch.Tensor, noise_var: float, out_Sigma: torch.Tensor | None = None,
                  out_mu: torch.Tensor | None = None, check: bool = True, prec: str = "fp64"):
    """Posterior mean and covariance (Eqs. 7-8) of the field N(mu, Sigma) given y observed with
    noise variance noise_var at the sites obs (int32 CUDA tensor).  Returns (mu_post, Sigma_post),
    Sigma_post column-major with its lower triangle written (out_Sigma may be Sigma itself).
    With check=True the call waits and raises MVNError on a device-side error."""
    n = Sigma.shape[0]
    Sp, ld = _mat(Sigma, n, "Sigma")
    if out_Sigma is None:
        out_Sigma = colmajor_empty(n, n, Sigma.device)
    Op, ldo = _mat(out_Sigma, n, "out_Sigma")
    if out_mu is None:
        out_mu = torch.empty(n, dtype=torch.float64, device=Sigma.device)
    n_obs = obs.numel()
    if y.numel() != n_obs:
        raise ValueError("y and obs must have the same length")
    c = context()
    info = _I(0)
    c.check(lib().mvn_posterior(c.h, n, _vec(mu, n, "mu"), Sp, ld, n_obs,
                                _vec(obs, n_obs, "obs", dtype=torch.int32),
                                _vec(y, n_obs, "y"), float(noise_var), PREC[prec],
                                _vec(out_mu, n, "out_mu"),
                                Op, ldo, ctypes.byref(info) if check else None))
    return out_mu, out_Sigma


def mvn_excursion(mu: torch.Tensor, Sigma: torch.Tensor, u: float, level: float, n_points: int,
                  n_shifts: int, seed: int, prefix_dims=None, prec="fp64", err_k=3.0):
    """Confidence region of level `level` above u (Alg. 1).  Returns dict of device tensors:
    order (int32 n), marginal (n), F (one per prefix), region (uint8 n)."""
    n = mu.numel()
    Sp, ld = _mat(Sigma, n, "Sigma")
    dev = mu.device
    order = torch.empty(n, dtype=torch.int32, device=dev)
    marg = torch.empty(n, dtype=torch.float64, device=dev)
    region = torch.empty(n, dtype=torch.uint8, device=dev)
    if prefix_dims is None:
        nprob, pk = n, None
    else:
        nprob = len(prefix_dims)
        pk = (ctypes.c_int * nprob)(*[int(x) for x in prefix_dims])
    F = torch.empty(nprob, dtype=torch.float64, device=dev)
    q = _qmc(n_points, n_shifts, seed, err_k)
    c = context()
    c.check(lib().mvn_excursion(c.h, n, _vec(mu, n, "mu"), Sp, ld, u, level, nprob,
                                ctypes.cast(pk, _P) if pk is not None else None, ctypes.byref(q),
                                PREC[prec], 0, _P(order.data_ptr()), _P(marg.data_ptr()),
                                _P(F.data_ptr()), _P(region.data_ptr())))
    return dict(order=order, marginal=marg, F=F, region=region)


class ExcursionGraph:
    """The confidence-region pipeline captured as one CUDA graph (mvn_excursion_graph).  Every
    launch() re-reads the mu and Sigma tensors given at creation (update them in place) and
    rewrites the output tensors in .result."""

    def __init__(self, handle, ctx, keep, result):
        self.h = handle
        self.ctx = ctx
        self._keep = keep          # the input tensors the graph reads
        self.result = result
        self.kernels = int(lib().mvn_graph_kernels(handle))

    def launch(self):
        self.ctx.check(lib().mvn_graph_launch(self.h))

    def sync(self) -> int:
        info = _I(0)
        self.ctx.check(lib().mvn_graph_sync(self.h, ctypes.byref(info)))
        return info.value

    def close(self):
        if self.h:
            lib().mvn_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mvn_excursion_graph(mu: torch.Tensor, Sigma: torch.Tensor, u: float, level: float,
                        n_points: int, n_shifts: int, seed: int, prefix_dims=None, prec="fp64",
                        err_k=3.0) -> ExcursionGraph:
    """Capture mvn_excursion's pipeline for these buffers into a CUDA graph (runs it once)."""
    n = mu.numel()
    Sp, ld = _mat(Sigma, n, "Sigma")
    dev = mu.device
    order = torch.empty(n, dtype=torch.int32, device=dev)
    marg = torch.empty(n, dtype=torch.float64, device=dev)
    region = torch.empty(n, dtype=torch.uint8, device=dev)
    if prefix_dims is None:
        nprob, pk = n, None
    else:
        nprob = len(prefix_dims)
        pk = (ctypes.c_int * nprob)(*[int(x) for x in prefix_dims])
    F = torch.empty(nprob, dtype=torch.float64, device=dev)
    q = _qmc(n_points, n_shifts, seed, err_k)
    c = context()
    h = _P()
    c.check(lib().mvn_excursion_graph(c.h, n, _vec(mu, n, "mu"), Sp, ld, u, level, nprob,
                                      ctypes.cast(pk, _P) if pk is not None else None,
                                      ctypes.byref(q), PREC[prec], _P(order.data_ptr()),
                                      _P(marg.data_ptr()), _P(F.data_ptr()),
                                      _P(region.data_ptr()), ctypes.byref(h)))
    return ExcursionGraph(h, c, (mu, Sigma),
                          dict(order=order, marginal=marg, F=F, region=region))


def mvn_autotune(n: int, n_paths: int, prec: str = "mixed", cache: str | None = None) -> dict:
    """Time the candidate launch shapes for (n, n_paths, prec) on this device, keep the fastest
    in the context (and in the JSON-lines file `cache`, if given); returns the choice."""
    r = mvn_tune_result()
    c = context()
    c.check(lib().mvn_autotune(c.h, n, n_paths, PREC[prec],
                               cache.encode() if cache else None, ctypes.byref(r)))
    return {"chol_bulk_p": r.chol_bulk_p, "chol_tail_p": r.chol_tail_p,
            "sweep_ctas_per_sm": r.sweep_ctas_per_sm, "from_cache": bool(r.from_cache)}


def mvn_tune_set(n: int, n_paths: int, prec: str, chol_bulk_p: int = 16, chol_tail_p: int = 2,
                 sweep_ctas_per_sm: int = 2) -> None:
    """Set the launch shapes for (n, n_paths, prec) by hand."""
    r = mvn_tune_result(chol_bulk_p, chol_tail_p, sweep_ctas_per_sm, 0)
    c = context()
    c.check(lib().mvn_tune_set(c.h, n, n_paths, PREC[prec], ctypes.byref(r)))


def mvn_lattice_alpha(n: int) -> torch.Tensor:
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    c = context()
    c.check(lib().mvn_lattice_alpha(c.h, n, _P(out.data_ptr())))
    return out


def mvn_lattice_shifts(seed: int, M: int, n: int) -> torch.Tensor:
    out = torch.empty((M, n), dtype=torch.int64, device="cuda")
    c = context()
    c.check(lib().mvn_lattice_shifts(c.h, int(seed) & ((1 << 64) - 1), M, n, _P(out.data_ptr())))
    return out


def mvn_tc_selftest(Y: torch.Tensor, L: torch.Tensor) -> torch.Tensor:
    """S = Y (128 x K) L (128 x K)^T through the tensor-core path of MVN_MIXED (FP32 result)."""
    K = Y.shape[1]
    assert Y.shape == (128, K) and L.shape == (128, K)
    S = torch.empty((128, 128), dtype=torch.float32, device=Y.device)
    c = context()
    c.check(lib().mvn_tc_selftest(c.h, K, _vec(Y.contiguous(), 128 * K, "Y"),
                                  _vec(L.contiguous(), 128 * K, "L"), _P(S.data_ptr())))
    return S


def mvn_sov_step_test(a, b, s, lii, W, prec: str = "fp64"):
    """The sweeps' elementwise step of Eq. 2 on independent inputs (FP64 CUDA tensors a, b, s,
    lii and an int64 tensor W holding the lattice integers' bits).  Returns (y, delta)."""
    n = a.numel()
    y = torch.empty(n, dtype=torch.float64, device=a.device)
    d = torch.empty(n, dtype=torch.float64, device=a.device)
    c = context()
    c.check(lib().mvn_sov_step_test(c.h, PREC[prec], n, _vec(a, n, "a"), _vec(b, n, "b"),
                                    _vec(s, n, "s"), _vec(lii, n, "lii"),
                                    _vec(W, n, "W", dtype=torch.int64), _vec(y, n, "y"),
                                    _vec(d, n, "delta")))
    return y, d


def mvn_sov_fp64_noalloc(a, b, L, n_points, n_shifts, seed, err_k=3.0, path_logw=None,
                         out3=None):
    """FP64 SOV estimate through the entry point that allocates nothing (fixed scratch inside
    the library; see include/mvn.h for its limits).  Enqueued on torch's current stream."""
    n = a.numel()
    if out3 is None:
        out3 = torch.empty(3, dtype=torch.float64, device=a.device)
    Lp, ld = _mat(L, n, "L")
    q = _qmc(n_points, n_shifts, seed, err_k)
    st = lib().mvn_sov_fp64_noalloc(n, _vec(a, n, "a"), _vec(b, n, "b"), Lp, ld, ctypes.byref(q),
                                    _vec(out3, 3, "out3"),
                                    _vec(path_logw, n_points * n_shifts, "path_logw"),
                                    _P(torch.cuda.current_stream(a.device).cuda_stream))
    if st != MVN_OK:
        raise MVNError(st, "mvn_sov_fp64_noalloc failed")
    return out3


class TLR:
    """Owner of an mvn_tlr object (tile low-rank form of a covariance or of its factor)."""

    def __init__(self, handle, n, tile, max_rank, capped):
        self.h = handle
        self.n, self.tile, self.max_rank, self.capped = n, tile, max_rank, capped
        self.nt = (n + tile - 1) // tile

    def ranks(self):
        import numpy as np
        k = self.nt * (self.nt - 1) // 2
        buf = (ctypes.c_int * max(k, 1))()
        st = lib().mvn_tlr_ranks(self.h, ctypes.cast(buf, _P))
        if st != MVN_OK:
            raise MVNError(st, "mvn_tlr_ranks failed")
        return np.array(buf[:k], dtype=np.int32)

    def __del__(self):
        try:
            if self.h:
                lib().mvn_tlr_free(self.h)
                self.h = None
        except Exception:
            pass


def mvn_tlr_compress(Sigma: torch.Tensor, tile: int, acc: float, max_rank: int) -> TLR:
    n = Sigma.shape[0]
    Sp, ld = _mat(Sigma, n, "Sigma")
    h = _P()
    hit = _I(0)
    c = context()
    c.check(lib().mvn_tlr_compress(c.h, n, Sp, ld, tile, acc, max_rank, ctypes.byref(h),
                                   ctypes.byref(hit)))
    return TLR(h, n, tile, max_rank, hit.value)


def mvn_tlr_cholesky(T: TLR) -> int:
    info = _I(0)
    c = context()
    c.check(lib().mvn_tlr_cholesky(c.h, T.h, ctypes.byref(info)))
    return info.value


def mvn_tlr_to_dense(T: TLR, out: torch.Tensor | None = None) -> torch.Tensor:
    if out is None:
        out = torch.zeros((T.n, T.n), dtype=torch.float64, device="cuda").t()
    Lp, ld = _mat(out, T.n, "out")
    c = context()
    c.check(lib().mvn_tlr_to_dense(c.h, T.h, Lp, ld))
    return out


def mvn_sov_tlr(T: TLR, a: torch.Tensor, b: torch.Tensor, n_points: int, n_shifts: int,
                seed: int, prec: str = "fp64", err_k: float = 3.0,
                path_logw: torch.Tensor | None = None, out3: torch.Tensor | None = None):
    """SOV estimate on a factored TLR object (low-rank limit updates); returns out3."""
    n = T.n
    if out3 is None:
        out3 = torch.empty(3, dtype=torch.float64, device=a.device)
    q = _qmc(n_points, n_shifts, seed, err_k)
    c = context()
    c.check(lib().mvn_sov_tlr(c.h, T.h, _vec(a, n, "a"), _vec(b, n, "b"), ctypes.byref(q),
                              PREC[prec], _vec(out3, 3, "out3"),
                              _vec(path_logw, n_points * n_shifts, "path_logw")))
    return out3


def sync():
    """Wait for the current context; raise MVNError for a device-side error."""
    c = context()
    st, info = c.sync()
    if st != MVN_OK:
        raise MVNError(st, lib().mvn_last_error(c.h).decode())
    return info
