"""Pins of the oracle's flexible GMRES (the cycle used as a preconditioner,
Table 3): with the identity preconditioner it is GMRES, whose k-th iterate
minimises the residual over K_k(A, f) (checked by least squares on the
monomial Krylov basis); with the exact inverse it takes one iteration; with
the V-cycle it converges to the direct solution."""

import numpy as np
import pytest

import oracle as O
from paper_1211_4752_gb300 import workloads as W


def _small():
    H = O.build_hierarchy(16, 2, 150.0, layers=3)
    f = W.random_field(H.levels[0].shape, 3)
    return H, f


@pytest.mark.parametrize("k", [1, 2, 4])
def test_identity_preconditioner_is_gmres_minimiser(k):
    H, f = _small()
    lv = H.levels[0]
    res = O.fgmres(H, f, tol=1e-300, m=k, max_iter=k,
                   precond=lambda v: v.copy(), strict=False)
    K, AK = [], []
    q = f.ravel()
    for _ in range(k):
        K.append(q)
        q = O.apply_operator(lv, q.reshape(f.shape)).ravel()
        AK.append(q)
    y = np.linalg.lstsq(np.stack(AK, 1), f.ravel(), rcond=None)[0]
    ref = (np.stack(K, 1) @ y).reshape(f.shape)
    assert res.cycles == k
    assert np.linalg.norm(res.u - ref) <= 1e-9 * np.linalg.norm(ref)


def test_exact_preconditioner_takes_one_iteration():
    H, f = _small()
    A = O.dense_matrix(H.levels[0])
    res = O.fgmres(H, f, tol=1e-12, m=5,
                   precond=lambda v: np.linalg.solve(A, v.ravel()).reshape(v.shape))
    assert res.cycles == 1
    assert np.linalg.norm(f - O.apply_operator(H.levels[0], res.u)) <= 1e-12 * np.linalg.norm(f)


@pytest.mark.parametrize("smoother", ["jacobi", "gmres"])
def test_vcycle_preconditioned_fgmres_converges_to_direct_solution(smoother):
    H = O.build_hierarchy(32, 2, 300.0, layers=4, smoother=smoother)
    f = W.point_sources(32, 2, [(15, 15)])[0]
    res = O.fgmres(H, f, tol=1e-10, m=8)
    A = O.dense_matrix(H.levels[0])
    ref = np.linalg.solve(A, f.ravel()).reshape(f.shape)
    assert np.linalg.norm(res.u - ref) <= 1e-8 * np.linalg.norm(ref)
    assert res.history[-1] <= 1e-10


def _gmres_minimiser(lv, f, u0, k):
    """u0 + the element of K_k(A, r0) that minimises |f - A u|, by least
    squares on the monomial basis."""
    r0 = (f - O.apply_operator(lv, u0)).ravel()
    K, AK = [], []
    q = r0
    for _ in range(k):
        K.append(q)
        q = O.apply_operator(lv, q.reshape(f.shape)).ravel()
        AK.append(q)
    y = np.linalg.lstsq(np.stack(AK, 1), r0, rcond=None)[0]
    return u0 + (np.stack(K, 1) @ y).reshape(f.shape)


def test_restart_minimises_from_the_previous_iterate():
    H, f = _small()
    lv = H.levels[0]
    res = O.fgmres(H, f, tol=1e-300, m=2, max_iter=6,
                   precond=lambda v: v.copy(), strict=False)
    ref = np.zeros_like(f)
    for _ in range(3):
        ref = _gmres_minimiser(lv, f, ref, 2)
    assert res.cycles == 6
    assert np.linalg.norm(res.u - ref) <= 1e-9 * np.linalg.norm(ref)
