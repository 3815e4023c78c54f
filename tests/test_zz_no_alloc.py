"""hh_rel_residual_static, whose partial sums live in a fixed device array
(no allocation), against the existing entry points: the residual that
hh_solve reports for the iterate it returns, and f - hh_apply(u).

The file name sorts last so that it also runs after every other test in the
same process (the scratch array is shared process-wide)."""

import numpy as np
import pytest

from paper_1211_4752_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _apply_residuals(mg, u, f):
    r = (f - mg.apply(u)).cpu().numpy()
    fn = f.cpu().numpy()
    return np.array([np.linalg.norm(r[b]) / np.linalg.norm(fn[b]) for b in range(f.shape[0])])


def test_static_residual_matches_solve_and_apply_on_consecutive_calls():
    from paper_1211_4752_gb300 import HelmholtzMG
    n, k, layers = 64, 40.0, 4
    mg = HelmholtzMG(n, k2=k * k, layers=layers, max_batch=3)
    rng = np.random.default_rng(5)
    pos = [tuple(rng.integers(n // 4, 3 * n // 4, size=2)) for _ in range(3)]
    f = torch.from_numpy(W.point_sources(n, 2, pos) + 0.1 * W.random_field((3, n - 1, n - 1), 6)).cuda()
    seen = []
    for tol in (1e-4, 1e-9):              # two calls in a row, different iterates
        u, info = mg.solve(f, tol=tol)
        rho = mg.rel_residual_static(u, f).cpu().numpy()
        # the residual cancels ||f|| ~ ||A u|| down to rho ||f||: two evaluation
        # orders differ by a few eps * (||f|| + || |A| |u| ||) / ||f||, ~1e-14
        for b in range(3):
            assert info[b]["status"] == "OK"
            assert abs(rho[b] - info[b]["rel_residual"]) <= 1e-10 * rho[b] + 1e-13
        ref = _apply_residuals(mg, u, f)
        assert np.allclose(rho, ref, rtol=1e-10, atol=1e-13)
        seen.append(rho)
    assert np.all(seen[1] < 1e-9) and np.all(seen[0] > 1e-9)
    # a smaller batch right after a larger one reads only what it wrote
    one = mg.rel_residual_static(u[:1].contiguous(), f[:1].contiguous()).cpu().numpy()
    assert abs(one[0] - seen[1][0]) <= 1e-12 * seen[1][0]
    mg.close()


def test_static_residual_edge_cases():
    from paper_1211_4752_gb300 import HelmholtzMG
    from paper_1211_4752_gb300 import _binding as B
    n = 32
    mg = HelmholtzMG(n, k2=400.0, layers=2, max_batch=2)
    z = torch.zeros((2, n - 1, n - 1), dtype=torch.complex128, device="cuda")
    u = torch.from_numpy(W.random_field((2, n - 1, n - 1), 1)).cuda()
    rho = mg.rel_residual_static(z, z).cpu().numpy()
    assert np.all(rho == 0.0)                 # f = 0, r = 0
    rho = mg.rel_residual_static(u, z).cpu().numpy()
    assert np.all(np.isinf(rho))              # f = 0, r != 0
    big = torch.zeros((65, n - 1, n - 1), dtype=torch.complex128, device="cuda")
    rr = torch.empty(65, dtype=torch.float64, device="cuda")
    st = B.lib().hh_rel_residual_static(mg._h, big.data_ptr(), big.data_ptr(), 65,
                                        rr.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == B.HH_ERR_ARG
    mg.close()
