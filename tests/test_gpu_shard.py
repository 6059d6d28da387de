"""One SOV problem split into path ranges (mvn_sov_partial + mvn_sov_combine), as the ranks of a
multi-GPU run would split it, here as consecutive calls on one GPU: per-path log-weights equal to
the unsplit call's bit for bit, the combined estimate equal to it (bit for bit for one shard;
to rounding when a cut falls inside a shift), and to the oracle."""
import ctypes

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


def _case(n=300):
    g = int(np.ceil(np.sqrt(n)))
    c = inputs.grid_coords(g)[:n]
    S = oracle.matern(c, 1.0, 0.12, 1.5, nugget=1e-4)
    L, _ = oracle.cholesky(S)
    a = np.full(n, -np.inf)
    b = inputs.uniform_limits(n, -0.3, 1.8, 8)
    return L, a, b


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_simt"])
def test_shards_reproduce_the_whole_call(mvn, prec):
    L, a, b = _case()
    n = a.size
    Ns, M, seed = 333, 6, 29
    Ntot = Ns * M
    Lg = mvn.to_colmajor(_t(L))
    ad, bd = _t(a), _t(b)
    lw = torch.empty(Ntot, dtype=torch.float64, device="cuda")
    whole = mvn.mvn_sov(ad, bd, Lg, Ns, M, seed, prec=prec, path_logw=lw)
    # one shard with every path: the same pairs as the single call's reduction, bit for bit
    one = mvn.mvn_sov_partial(ad, bd, Lg, Ns, M, seed, 0, Ntot, prec=prec)
    out1 = mvn.mvn_sov_combine(one, Ns, M)
    # three shards, two cuts inside shifts and one on a shift boundary
    cuts = [0, 500, 2 * Ns, 1700, Ntot]
    parts, lws = [], []
    for p0, p1 in zip(cuts, cuts[1:]):
        lwp = torch.empty(p1 - p0, dtype=torch.float64, device="cuda")
        parts.append(mvn.mvn_sov_partial(ad, bd, Lg, Ns, M, seed, p0, p1, prec=prec,
                                         path_logw=lwp))
        lws.append(lwp)
    out3 = mvn.mvn_sov_combine(torch.stack(parts), Ns, M)
    mvn.sync()
    w = whole.cpu().numpy()
    assert np.array_equal(out1.cpu().numpy(), w)
    assert torch.equal(torch.cat(lws), lw)
    o = out3.cpu().numpy()
    assert abs(o[0] - w[0]) <= 1e-14 * abs(w[0])
    assert abs(o[1] - w[1]) <= 1e-14 * w[1]
    assert abs(o[2] - w[2]) <= 1e-11 * w[2]
    if prec == "fp64":
        ref = oracle.estimate(oracle.sov_logw(a, b, L, oracle.QMC(Ns, M, seed)), M)
        assert abs(o[0] - ref[0]) <= 1e-9 and abs(o[1] - ref[1]) <= 1e-10


def test_empty_shard_and_bad_ranges(mvn):
    L, a, b = _case(40)
    Lg = mvn.to_colmajor(_t(L))
    ad, bd = _t(a), _t(b)
    p = mvn.mvn_sov_partial(ad, bd, Lg, 50, 3, 1, 70, 70).cpu().numpy().reshape(3, 2)
    mvn.sync()
    assert np.all(p[:, 0] == -np.inf) and np.all(p[:, 1] == 0.0)
    # a shard inside one shift leaves the other shifts empty
    p = mvn.mvn_sov_partial(ad, bd, Lg, 50, 3, 1, 60, 90).cpu().numpy().reshape(3, 2)
    mvn.sync()
    assert np.isfinite(p[1, 0]) and p[1, 1] >= 1.0
    assert p[0, 0] == -np.inf and p[2, 0] == -np.inf
    lib = mvn.lib()
    q = mvn.mvn_qmc(50, 3, 0, 1, 3.0)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    P = ctypes.c_void_p
    for p0, p1 in ((-1, 10), (20, 10), (0, 151)):
        assert lib.mvn_sov_partial(mvn.context().h, 40, P(ad.data_ptr()), P(bd.data_ptr()),
                                   P(Lg.data_ptr()), 40, ctypes.byref(q), 0, p0, p1,
                                   P(out.data_ptr()), None) == mvn.MVN_ERR_ARG
    assert lib.mvn_sov_combine(mvn.context().h, 0, ctypes.byref(q), P(out.data_ptr()),
                               P(out.data_ptr())) == mvn.MVN_ERR_ARG


def test_sharded_helper_on_one_rank(mvn):
    """paper_2405_14892_gb300.shard.sov_sharded without a process group is one shard."""
    from paper_2405_14892_gb300 import shard
    L, a, b = _case(100)
    Lg = mvn.to_colmajor(_t(L))
    ref = mvn.mvn_sov(_t(a), _t(b), Lg, 200, 4, 3)
    got = shard.sov_sharded(_t(a), _t(b), Lg, 200, 4, 3)
    mvn.sync()
    assert torch.equal(got, ref)
