"""The autotuner of launch shapes (mvn_autotune / mvn_tune_set): its choices come from the
candidate sets, are cached and reloaded from a JSON-lines file, and no choice changes a result
bit (the MVN_MIXED Cholesky update sums exact integers in any order; the sweeps compute each
path independently of the grid)."""
import json

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


def test_autotune_choice_and_cache(mvn, tmp_path):
    cache = str(tmp_path / "tune.jsonl")
    r = mvn.mvn_autotune(700, 3000, "mixed", cache=cache)
    assert r["chol_bulk_p"] in (4, 8, 16, 32, 64) and r["chol_tail_p"] in (1, 2)
    assert r["sweep_ctas_per_sm"] in (1, 2) and not r["from_cache"]
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and json.loads(lines[0])["chol_bulk_p"] == r["chol_bulk_p"]
    r2 = mvn.mvn_autotune(700, 3000, "mixed", cache=cache)   # same buckets: from the file
    assert r2["from_cache"] and {k: r2[k] for k in r if k != "from_cache"} == \
        {k: r[k] for k in r if k != "from_cache"}
    r3 = mvn.mvn_autotune(300, 3000, "mixed_simt", cache=cache)
    assert r3["sweep_ctas_per_sm"] in (1, 2, 3) and not r3["from_cache"]
    assert len(open(cache).read().splitlines()) == 2


@pytest.mark.parametrize("prec", ["mixed", "mixed_simt", "fp64"])
def test_every_launch_shape_gives_identical_results(mvn, prec):
    g = 26
    c = inputs.grid_coords(g)
    n = g * g                     # 676: ragged against the 64-wide panels and 128-wide blocks
    S = oracle.matern_closed(c, 1.0, 0.1, 1.5, 1e-4)
    a, b = np.full(n, -np.inf), np.full(n, 0.5)
    Ns, M = 300, 7                # 2,100 paths: 17 tiles, ragged last tile
    res = []
    shapes = [(16, 2, 2), (4, 1, 1), (64, 2, 1), (8, 1, 2)]
    if prec != "mixed":
        shapes += [(16, 2, 3)]
    for bulk, tail, ctas in shapes:
        mvn.mvn_tune_set(n, Ns * M, prec, bulk, tail, ctas)
        A = mvn.to_colmajor(_t(S))
        mvn.mvn_cholesky(A, prec="mixed" if prec == "mixed" else "fp64")
        lw = torch.empty(Ns * M, dtype=torch.float64, device="cuda")
        out = mvn.mvn_sov(_t(a), _t(b), A, Ns, M, 9, prec=prec, path_logw=lw)
        mvn.sync()
        res.append((torch.tril(A).clone(), lw.clone(), out.clone()))
    for L, lw, out in res[1:]:
        assert torch.equal(L, res[0][0])
        assert torch.equal(lw, res[0][1])
        assert torch.equal(out, res[0][2])
    mvn.mvn_tune_set(n, Ns * M, prec)   # back to the defaults
