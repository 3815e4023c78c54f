"""Values the paper prints: the dtheta schedule of Tables 1, 2 and 5, and
the level count of Sec. 4.1 (n = 2^p grid points <-> p levels)."""

import math
from pathlib import Path

import pytest

import oracle as O

ROWS = [tuple(int(v) for v in line.split()[:3])
        for line in (Path(__file__).parent / "golden" / "shift_schedule.txt").read_text().splitlines()
        if line.strip() and not line.startswith("#")]


@pytest.mark.parametrize("n,tmax_den,dth_den", ROWS)
def test_dtheta_matches_tables(n, tmax_den, dth_den):
    H = O.build_hierarchy(n, 1, 10.0, theta_max=math.pi / tmax_den)
    assert H.info["dtheta"] == pytest.approx(math.pi / dth_den, rel=1e-14)
    # finest level keeps the original operator; level l carries e^{i l dtheta}
    assert H.levels[0].beta == 1.0
    assert H.levels[3].beta == pytest.approx(complex(math.cos(3 * math.pi / dth_den),
                                                     math.sin(3 * math.pi / dth_den)))


@pytest.mark.parametrize("p", [3, 5, 8])
def test_level_count(p):
    n = 2 ** p
    assert len(O.build_hierarchy(n, 1, 1.0, coarsest=2).levels) == p
    assert len(O.build_hierarchy(n, 1, 1.0).levels) == p - 1   # 3-point coarsest
