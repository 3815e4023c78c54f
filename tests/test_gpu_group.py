"""Group solves (hh_solve_group): problems of different grid sizes, media,
precisions and smoothers in one call, run concurrently on the device.  The
kernels are the same as in separate solves and deterministic, so every
result must equal the separate solve's bit for bit; the full-size case is
the many-source workload over 255^2, 511^2 and 1023^2 grids."""

import math

import numpy as np
import pytest

from paper_1211_4752_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _small_group():
    from paper_1211_4752_gb300 import HelmholtzMG
    probs = []
    mg = HelmholtzMG(64, k2=1600.0, layers=16, precision="mixed", max_batch=2)
    f = np.stack([W.point_sources(64, 2, [(31, 31)])[0], W.random_field((63, 63), 3)])
    probs.append((mg, dev(f)))
    k2 = W.smooth_k2(128, 2, 4, 30.0, 40.0)
    mg = HelmholtzMG(128, k2=dev(k2), layers=(8, 24), precision="fp64", max_batch=3,
                     smoother="gmres")
    f = W.random_field((3, 127, 127), 9)
    probs.append((mg, dev(f)))
    mg = HelmholtzMG(16, dim=3, k2=49.0, layers=2, precision="mixed", max_batch=1)
    f = W.point_sources(16, 3, [(7, 7, 7)])
    probs.append((mg, dev(f)))
    return probs


def test_group_equals_separate_solves():
    from paper_1211_4752_gb300 import solve_group
    probs = _small_group()
    sep = [mg.solve(f, tol=1e-7) for mg, f in probs]
    grp = solve_group(probs, tol=1e-7)
    for (us, infs), (ug, infg) in zip(sep, grp):
        assert infs == infg
        assert all(i["status"] == "OK" for i in infg)
        assert torch.equal(us, ug)
    # an initial guess is honoured per problem
    mg, f = probs[0]
    u0 = grp[0][0].clone()
    (u1, i1), = solve_group([(mg, f, u0)], tol=1e-7)
    assert all(i["cycles"] <= 1 for i in i1) and torch.equal(u1, u0)
    for mg, _ in probs:
        mg.close()


def test_group_arguments_are_checked():
    from paper_1211_4752_gb300 import solve_group
    from paper_1211_4752_gb300._binding import HHError
    probs = _small_group()
    with pytest.raises(HHError):
        solve_group([probs[0], probs[0]])   # the same handle twice
    with pytest.raises(HHError):
        solve_group(probs, tol=2.0)
    assert solve_group([]) == []
    for mg, _ in probs:
        mg.close()


def test_group_many_sources_full_size():
    """64 point sources over 255^2, 511^2 and 1023^2 grids (kh = 0.625, ECS
    n/32) in one call: every right-hand side reaches 1e-6 (FP64 residual by an
    independent apply), and the 255^2 group equals its separate solve."""
    from paper_1211_4752_gb300 import HelmholtzMG, solve_group
    groups = W.batch_sources()
    probs = []
    for g in groups:
        B = g["rhs"].shape[0]
        mg = HelmholtzMG(g["n"], k2=g["k2"], layers=g["layers"], precision="mixed", max_batch=B)
        probs.append((mg, dev(g["rhs"])))
    res = solve_group(probs, tol=1e-6)
    assert sum(f.shape[0] for _, f in probs) == 64
    for (mg, f), (u, info) in zip(probs, res):
        assert all(i["status"] == "OK" for i in info)
        rho = mg.rel_residual_static(u, f).cpu().numpy()
        assert np.all(rho <= 1e-6)
        assert np.allclose(rho, [i["rel_residual"] for i in info], rtol=1e-6, atol=1e-13)
    mg, f = probs[0]
    us, infs = mg.solve(f, tol=1e-6)
    assert infs == res[0][1] and torch.equal(us, res[0][0])
    for mg, _ in probs:
        mg.close()
