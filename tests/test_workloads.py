"""The seeded input recipes: shapes, sizes and structure of the synthetic
workloads as the design notes state them (so that a change to an input
generator shows up here, not as a shifted benchmark).  CPU only."""

import math

import numpy as np

from paper_1211_4752_gb300 import workloads as W


def test_ecs_const_is_the_benchmark_problem():
    w = W.ecs_const()
    assert (w["n"], w["dim"], w["layers"]) == (1024, 2, 32)
    assert w["k2"] == (0.625 * 1024) ** 2
    assert w["rhs"].shape == (1, 1023, 1023) and w["rhs"].dtype == np.complex128
    assert np.argwhere(w["rhs"][0] != 0).tolist() == [[511, 511]]
    assert w["rhs"][0, 511, 511] == 1.0


def test_batch_sources_split_and_seed():
    g = W.batch_sources()
    assert [x["n"] for x in g] == [256, 512, 1024]
    assert [x["rhs"].shape[0] for x in g] == [22, 21, 21]
    assert sorted(i for x in g for i in x["ids"]) == list(range(64))
    for x in g:
        assert x["layers"] == x["n"] // 32 and x["k2"] == (0.625 * x["n"]) ** 2
        lo, hi = x["layers"], x["n"] - x["layers"] - 2   # sources inside the physical region
        pos = np.argwhere(x["rhs"] != 0)
        assert len(pos) == x["rhs"].shape[0] and pos[:, 1:].min() >= lo and pos[:, 1:].max() <= hi
    g2 = W.batch_sources()
    assert all(np.array_equal(a["rhs"], b["rhs"]) for a, b in zip(g, g2))


def test_ionization_model_recipe():
    for k0, n in W.ION_GRIDS.items():
        w = W.ionization(k0)
        assert w["n"] == n and w["layers"] == (0, n // 8)
    w = W.ionization(2, n=64)
    r = 50.0
    x = (np.arange(1, 64) / 64) * r
    # the coefficient of u and the source, times r^2 (x = r xi), [y][x] layout
    assert math.isclose(w["k2"][0, 5], r * r * (math.exp(-x[5] ** 2) + math.exp(-x[0] ** 2) + 4.0))
    assert math.isclose(w["rhs"][0, 3, 5].real, r * r * math.exp(-(x[5] ** 2 + x[3] ** 2)))
    assert np.all(np.diff(w["k2"][10]) <= 0)     # decreasing away from x = 0


def test_bump_and_cube():
    w = W.bump()
    assert (w["n"], w["layers"]) == (512, 16) and w["rhs"].shape == (16, 511, 511)
    kb = (0.5 * 512) ** 2
    assert w["k2"].min() >= kb * (1 - 1e-12) and w["k2"].max() <= kb * 1.1 + 1e-6
    c = W.cube()
    assert (c["n"], c["dim"], c["layers"], c["k2"]) == (128, 3, 16, 6400.0)
    assert np.argwhere(c["rhs"][0] != 0).tolist() == [[63, 63, 63]]
