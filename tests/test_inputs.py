"""The seeded input recipe on CPU: grid layout and Morton order, limits, problem lists and the
synthetic observations of Sec. V-B, each checked against a property that does not restate the
generator's own code."""
import numpy as np
import pytest

from paper_2405_14892_gb300 import inputs


@pytest.mark.parametrize("g", [2, 5, 16])
def test_row_grid_layout(g):
    c = inputs.grid_coords(g)
    assert c.shape == (g * g, 2)
    assert np.array_equal(c[0], [0.0, 0.0]) and np.array_equal(c[-1], [1.0, 1.0])
    # row-major: point i*g + j sits at (i, j) / (g - 1)
    i, j = 3 % g, (g - 1) // 2
    assert np.allclose(c[i * g + j], [i / (g - 1), j / (g - 1)])
    # nearest-neighbour spacing is 1/(g-1) everywhere
    d = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(d, np.inf)
    assert np.allclose(d.min(1), 1.0 / (g - 1))


@pytest.mark.parametrize("g,block", [(64, 256), (64, 1024), (16, 64)])
def test_morton_order_tiles_are_squares(g, block):
    """Morton order is a permutation of the grid in which every run of 4^k consecutive points
    is a 2^k x 2^k square of neighbouring grid points (what makes TLR tiles compact)."""
    row = inputs.grid_coords(g)
    mor = inputs.grid_coords(g, order="morton")
    key = lambda c: set(map(tuple, np.round(c * (g - 1)).astype(int)))  # noqa: E731
    assert key(row) == key(mor) and len(key(mor)) == g * g
    side = int(round(np.sqrt(block)))
    ij = np.round(mor * (g - 1)).astype(int)
    for t in range(g * g // block):
        sq = ij[t * block:(t + 1) * block]
        assert sq[:, 0].max() - sq[:, 0].min() == side - 1
        assert sq[:, 1].max() - sq[:, 1].min() == side - 1
        assert sq[:, 0].min() % side == 0 and sq[:, 1].min() % side == 0


def test_limits_of_the_workloads():
    n = 256
    a, b = inputs.limits_for(inputs.WORKLOADS["W1"], n)
    assert np.all(np.isneginf(a)) and np.all((b > -1) & (b < 1))
    assert np.array_equal(b, inputs.limits_for(inputs.WORKLOADS["W1"], n)[1])  # seeded
    assert abs(b.mean()) < 0.15 and b.std() == pytest.approx(np.sqrt(1 / 3), rel=0.15)
    for w in ("W2", "W4", "W5"):
        a, b = inputs.limits_for(inputs.WORKLOADS[w], 10)
        assert np.all(np.isneginf(a)) and np.all(b == 0.5)


def test_prefix_problem_dims():
    w = inputs.WORKLOADS["W3"]
    d = inputs.prefix_problem_dims(w["nprob"], w["dims_lo"], w["dims_hi"], w["dims_seed"])
    assert d.dtype == np.int32 and d.shape == (256,)
    assert d.min() >= 64 and d.max() <= 4096
    assert np.array_equal(d, inputs.prefix_problem_dims(256, 64, 4096, 3))
    # uniform on {64..4096}: mean 2080, sd ~1164
    assert abs(d.mean() - 2080) < 3 * 1164 / np.sqrt(256)


def test_observations_of_the_synthetic_protocol():
    """Sec. V-B protocol: distinct sorted sites, y = truth at the sites plus N(0, sd^2) noise;
    seeded.  (The posterior given them is the oracle's and the library's, not the input
    module's.)"""
    w = inputs.WORKLOADS["W3"]
    g = 32
    c = inputs.grid_coords(g)
    h = np.sqrt(((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    S = np.exp(-h / w["range"])
    idx, y, x = inputs.observations(S, 400, w["noise_sd"], w["field_seed"])
    assert idx.dtype == np.int32 and idx.shape == (400,) and y.shape == (400,)
    assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < g * g
    e = y - x[idx]
    assert abs(e.std() - w["noise_sd"]) < 0.1 * w["noise_sd"] and abs(e.mean()) < 0.1
    i2, y2, _ = inputs.observations(S, 400, w["noise_sd"], w["field_seed"])
    assert np.array_equal(idx, i2) and np.array_equal(y, y2)
