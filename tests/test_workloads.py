"""The synthetic inputs have the sizes, value ranges and structure stated for
them (the stand-ins for the paper's datasets, Sec. 4.1 and Appx. D): checked here
from each recipe's definition, on the CPU."""
import numpy as np
import pytest

import workloads as W


def test_grid_784_recipe():
    p = W.grid_problem_784(0)
    C, r, c = p["C"], p["r"], p["c"]
    assert C.shape == (784, 784) and C.dtype == np.float64
    assert C.max() == 1.0 and np.all(np.diag(C) == 0.0) and np.allclose(C, C.T)
    # squared Euclidean between pixel centres (a, b) / 27, divided by its max (2)
    assert C[0, 1] == pytest.approx((1 / 27) ** 2 / 2, rel=1e-12)
    assert C[0, 28] == pytest.approx((1 / 27) ** 2 / 2, rel=1e-12)
    assert C[0, 783] == 1.0
    for h in (r, c):
        assert h.shape == (784,) and h.sum() == pytest.approx(1.0, abs=1e-12)
        assert h.min() > 0.0 and h.min() >= 1e-6 / (1 + 784e-6) * (1 - 1e-12)  # the floor


@pytest.mark.parametrize("kind", ["sqeuclid", "l1"])
def test_grid_4096_recipe(kind):
    p = W.grid_problem_4096(3, kind)
    C, r, c = p["C"], p["r"], p["c"]
    assert C.shape == (4096, 4096) and C.dtype == np.float32 and C.max() == 1.0
    if kind == "l1":
        assert C[0, 1] == pytest.approx((1 / 63) / 2, rel=1e-6)
    else:
        assert C[0, 1] == pytest.approx((1 / 63) ** 2 / 2, rel=1e-6)
    for h in (r, c):
        assert h.sum() == pytest.approx(1.0, abs=1e-12)
        assert (h == 0.0).sum() == 410  # 10% of the bins zeroed
        assert h.min() >= 0.0
    assert not np.array_equal(r == 0, c == 0)  # separate seeded choices


def test_points_and_batch_recipes():
    p = W.uniform_points_problem(1, 300, 200)
    assert p["X"].shape == (300, 2) and p["Y"].shape == (200, 2) and p["X"].dtype == np.float32
    assert 0.0 <= p["X"].min() and p["X"].max() <= 1.0
    assert p["r"].sum() == pytest.approx(1.0) and p["c"].sum() == pytest.approx(1.0)
    n = W.batch_sizes(0)
    assert n.shape == (256,) and n.min() >= 256 and n.max() <= 4096
    assert abs(n.mean() - (256 + 4096) / 2) < 250  # uniform on {256, ..., 4096}


def test_high_dimensional_and_colour_recipes():
    p = W.gmm_problem_d64(0, n=4096)
    assert p["X"].shape == (4096, 64) and p["X"].dtype == np.float32
    assert np.allclose(p["r"], 1 / 4096) and np.allclose(p["c"], 1 / 4096)
    # 8 components with means ~ N(0, 4 I) and unit widths: the per-coordinate
    # variance is about 4 + 1
    assert 2.5 < p["X"].var() < 8.0
    q = W.colour_problem(0, n=1 << 14)
    assert q["X"].shape == (1 << 14, 3) and q["X"].dtype == np.float32
    assert q["X"].min() >= 0.0 and q["X"].max() <= 1.0
    assert np.allclose(q["r"], 1 / (1 << 14))


def test_generators_are_seeded():
    a, b = W.grid_problem_784(5), W.grid_problem_784(5)
    assert np.array_equal(a["r"], b["r"]) and np.array_equal(a["c"], b["c"])
    assert not np.array_equal(W.grid_problem_784(6)["r"], a["r"])
