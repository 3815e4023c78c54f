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


def _worklist_handles(monkeypatch, sizes=(64, 128, 256), batches=(2, 1, 3)):
    """Mixed-precision handles with the group's tile shape (60 x 16) and the
    per-level coarse schedule, so that separate solves run the same per-tile
    arithmetic as the work-list group."""
    from paper_1211_4752_gb300 import HelmholtzMG
    monkeypatch.setenv("HH_TILE_VARIANT", "0")
    out = []
    for i, (n, nb) in enumerate(zip(sizes, batches)):
        coarse = int(round(math.log2(n))) - 6          # fused levels above 63^2 .. 31^2 tail
        if coarse > 0:
            monkeypatch.setenv("HH_COARSE", ",".join(["1"] * coarse))
        else:
            monkeypatch.delenv("HH_COARSE", raising=False)
        # media on which the weighted-Jacobi cycle converges: k = 40 with ECS 16 at
        # 64^2, a smooth k^2 field (k from 76 to 80) with ECS 8 at 128^2, kh =
        # 0.625 with ECS n/32 otherwise
        if n == 64:
            k2, layers = 1600.0, 16
        elif n == 128:
            k2, layers = dev(W.smooth_k2(n, 2, 4, 76.0, 80.0)), 8
        else:
            k2, layers = (0.625 * n) ** 2, n // 32
        mg = HelmholtzMG(n, k2=k2, layers=layers, precision="mixed", max_batch=nb)
        rng = np.random.default_rng(n)
        pos = [tuple(rng.integers(n // 4, 3 * n // 4, size=2)) for _ in range(nb)]
        out.append((mg, dev(W.point_sources(n, 2, pos))))
    monkeypatch.delenv("HH_TILE_VARIANT")
    monkeypatch.delenv("HH_COARSE", raising=False)
    return out


def test_worklist_group_equals_separate_solves(monkeypatch):
    """hh_group_create / hh_group_solve: one launch per level size over the
    tiles of every problem, one tail launch and one stop test for all; the
    per-tile arithmetic is that of the single-problem kernels, so every
    right-hand side's solution, cycle count and refinements equal its
    separate solve's bit for bit; a second solve repeats them."""
    from paper_1211_4752_gb300 import HelmholtzGroup
    probs = _worklist_handles(monkeypatch)
    sep = [mg.solve(f, tol=1e-7) for mg, f in probs]
    assert all(i["status"] == "OK" for _, infs in sep for i in infs), sep
    grp = HelmholtzGroup([mg for mg, _ in probs], [f.shape[0] for _, f in probs])
    for _ in range(2):
        res = grp.solve([f for _, f in probs], tol=1e-7)
        for (us, infs), (ug, infg) in zip(sep, res):
            assert infs == infg, (infs, infg)
            assert torch.equal(us, ug)
    # kernels: per cycle one launch per size class and direction, tail, stop test
    assert grp.kernels > 0
    # an initial guess is honoured per problem
    res2 = grp.solve([f for _, f in probs], tol=1e-7, u0=[u for u, _ in res])
    assert all(i["cycles"] <= 1 for _, info in res2 for i in info)
    grp.close()
    for mg, _ in probs:
        mg.close()


def test_worklist_group_arguments():
    from paper_1211_4752_gb300 import HelmholtzGroup, HelmholtzMG
    from paper_1211_4752_gb300._binding import HHError, HH_ERR_ARG, HH_ERR_UNSUPPORTED
    a = HelmholtzMG(64, k2=1600.0, layers=16, precision="mixed", max_batch=2)
    b = HelmholtzMG(64, k2=1600.0, layers=16, precision="fp64", max_batch=1)
    with pytest.raises(HHError) as ei:
        HelmholtzGroup([a, b], [1, 1])
    assert ei.value.status == HH_ERR_UNSUPPORTED
    with pytest.raises(HHError) as ei:
        HelmholtzGroup([a, a], [1, 1])
    assert ei.value.status == HH_ERR_ARG
    with pytest.raises(HHError) as ei:
        HelmholtzGroup([a], [3])                      # above max_batch
    assert ei.value.status == HH_ERR_ARG
    g = HelmholtzGroup([a], [2])
    with pytest.raises(HHError) as ei:                # a batch other than the group's
        g.solve([dev(W.point_sources(64, 2, [(31, 31)]))])
    assert ei.value.status == HH_ERR_ARG
    g.close()
    a.close()
    b.close()


def test_worklist_group_full_size_many_sources():
    """The 64-source workload (22 x 255^2, 21 x 511^2, 21 x 1023^2, kh =
    0.625, ECS width 1/32) as one work-list group: every right-hand side
    reaches 1e-6 by an independent FP64 residual, and agrees with the
    concurrent-stream group solve (same problems, autotuned tiles) to the
    mixed path's 1e-5."""
    from paper_1211_4752_gb300 import HelmholtzGroup, HelmholtzMG, solve_group
    groups = W.batch_sources()
    probs = []
    for g in groups:
        mg = HelmholtzMG(g["n"], k2=g["k2"], layers=g["layers"], precision="mixed",
                         max_batch=g["rhs"].shape[0])
        probs.append((mg, dev(g["rhs"])))
    grp = HelmholtzGroup([mg for mg, _ in probs], [f.shape[0] for _, f in probs])
    res = grp.solve([f for _, f in probs], tol=1e-6)
    ref = solve_group(probs, tol=1e-6)
    for (mg, f), (u, info), (ur, _) in zip(probs, res, ref):
        assert all(i["status"] == "OK" for i in info)
        rho = mg.rel_residual_static(u, f).cpu().numpy()
        assert np.all(rho <= 1e-6)
        a, b = u.cpu().numpy(), ur.cpu().numpy()
        for k in range(a.shape[0]):
            assert np.linalg.norm(a[k] - b[k]) <= 1e-5 * np.linalg.norm(b[k])
    grp.close()
    for mg, _ in probs:
        mg.close()
