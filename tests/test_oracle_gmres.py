"""Pins of the oracle's GMRES(m) smoother (Sec. 3.2) and of the cycle built
on it: the minimal-residual property against an independent least-squares
solve on the monomial Krylov basis, exactness when the Krylov space is the
whole space, monotone residuals, and the cycle counts of Tables 1 and 2."""

import math
from pathlib import Path

import numpy as np
import pytest

import oracle as O
from paper_1211_4752_gb300 import workloads as W

GOLDEN = Path(__file__).resolve().parent / "golden"


def _level(n, dim, k2, layers):
    return O.build_hierarchy(n, dim, k2, layers=layers).levels


@pytest.mark.parametrize("m", [1, 2, 3])
def test_gmres_step_minimises_residual_over_krylov_space(m):
    lv = _level(16, 2, 300.0, 3)[1]           # 7 x 7 level with a shift and ECS
    rng = np.random.default_rng(m)
    shape = lv.shape
    u = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    got = O.gmres_smooth(lv, u, f, m)
    # independent: least squares on [A r0, A^2 r0, ...] (monomial basis)
    r0 = (f - O.apply_operator(lv, u)).ravel()
    K, AK = [], []
    q = r0
    for _ in range(m):
        K.append(q)
        q = O.apply_operator(lv, q.reshape(shape)).ravel()
        AK.append(q)
    y = np.linalg.lstsq(np.stack(AK, 1), r0, rcond=None)[0]
    ref = u + (np.stack(K, 1) @ y).reshape(shape)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    r_new = np.linalg.norm(f - O.apply_operator(lv, got))
    assert r_new <= np.linalg.norm(r0) * (1 + 1e-14)


def test_gmres_three_steps_solve_a_three_unknown_system():
    lv = _level(4, 1, 7.0, 0)[0]              # 1-D, 3 interior points
    f = np.array([1.0, -2.0 + 1j, 0.5])
    u = O.gmres_smooth(lv, np.zeros(3, complex), f, 3)
    assert np.linalg.norm(f - O.apply_operator(lv, u)) <= 1e-12 * np.linalg.norm(f)


def test_gmres_cycle_converges_where_jacobi_diverges():
    """The 511^2 bump medium at kh = 0.5 makes the Jacobi cycle diverge
    (Sec. 3.2); a smaller copy (127^2, same kh) with GMRES(3) smoothing
    converges to the direct solution."""
    w = W.bump(n=128, layers=4, nsrc=1)
    H = O.build_hierarchy(128, 2, w["k2"], layers=4, smoother="gmres")
    f = w["rhs"][0]
    res = O.solve(H, f, tol=1e-8, max_cycles=200)
    Hj = O.build_hierarchy(128, 2, w["k2"], layers=4)
    with pytest.raises(O.DivergedError):
        O.solve(Hj, f, tol=1e-8, max_cycles=200)
    lv = H.levels[0]
    from scipy.sparse import diags, identity, kron
    def op1(ax):
        N = lv.n - 1
        return diags([-lv.lo[ax][1:], lv.dg[ax], -lv.up[ax][:-1]], [-1, 0, 1], shape=(N, N))
    N = lv.n - 1
    A = (kron(identity(N), op1(0)) + kron(op1(1), identity(N))) * lv.alpha \
        - diags(lv.beta * lv.k2.ravel())
    from scipy.sparse.linalg import spsolve
    ref = spsolve(A.tocsc(), f.ravel()).reshape(f.shape)
    assert np.linalg.norm(res.u - ref) <= 1e-6 * np.linalg.norm(ref)


def test_cycle_counts_follow_tables_1_and_2():
    """GMRES(3)-smoothed V(1,1) cycles to 1e-7 for the constant-k model: at
    128^2 and 256^2 within a factor 2 of the counts the paper prints, more
    cycles for k = 80 than for k = 40, and the 64^2 grid at k = 80 (kh = 1.25)
    far slower than 128^2.  Exact agreement is not expected: the paper gives
    neither the ECS angle nor where its layer lies (our readings: pi/6, inside
    the unit square)."""
    table = {}
    for line in (GOLDEN / "table12_gmres_cycles.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k, n, c = map(int, line.split())
            table[(k, n)] = c
    got = {}
    for k in (40, 80):
        for n in (64, 128, 256):
            H = O.build_hierarchy(n, 2, float(k * k), layers=n // 4, smoother="gmres")
            f = W.point_sources(n, 2, [(n // 2 - 1, n // 2 - 1)])[0]
            got[(k, n)] = O.solve(H, f, tol=1e-7, max_cycles=400).cycles
    for k in (40, 80):
        for n in (128, 256):
            assert table[(k, n)] / 2 <= got[(k, n)] <= table[(k, n)] * 2, (k, n, got)
        for n in (64, 128, 256):
            assert got[(80, n)] > got[(40, n)]
    assert got[(80, 64)] >= 2 * got[(80, 128)]


def _table5():
    rows = []
    for line in (GOLDEN / "table5_theta_sweep.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            d, c = map(int, line.split())
            rows.append((d, c))
    return rows


def theta_sweep_cycles(d_values, n=128, k=30.0):
    f = W.point_sources(n, 2, [(n // 2 - 1, n // 2 - 1)])[0]
    out = []
    for d in d_values:
        H = O.build_hierarchy(n, 2, k * k, layers=n // 4, smoother="gmres",
                              theta_max=math.pi / d)
        out.append(O.solve(H, f, tol=1e-7, max_cycles=400).cycles)
    return out


def test_theta_sweep_follows_table_5():
    """Cycles as a function of theta_max (Table 5, k = 30, n = 128): within a
    factor 2 of the printed counts, falling from the smallest rotation to a
    minimum at pi/8 .. pi/5 and rising again at pi/4 (too small a shift leaves
    coarse spectra near zero; too large a one corrupts the smooth modes)."""
    table = _table5()
    got = theta_sweep_cycles([d for d, _ in table])
    for (d, c), g in zip(table, got):
        assert c / 2 <= g <= c * 2, (d, g, c)
    i_min = int(np.argmin(got))
    assert [d for d, _ in table][i_min] in (8, 6, 5)
    assert got[0] > got[i_min] and got[-1] > got[i_min]


def _table8():
    rows = {}
    for line in (GOLDEN / "table8_ionization.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            k0, n, c = map(int, line.split())
            rows[k0] = (n, c)
    return rows


def test_ionization_model_matches_table8():
    """Sec. 4.3's ionization model (Dirichlet on two sides, ECS on the others,
    a space-dependent coefficient and source; the layer reading n/8 cells):
    the oracle's GMRES(3)-smoothed cycle counts fall within 25 % of the
    LVL-MG row of Table 8 for k0 = 1, 2, 3 and grow with k0, and the
    weighted-Jacobi cycle diverges on this medium (the instability of
    Eq. (jacstab))."""
    table = _table8()
    got = {}
    for k0 in (1, 2, 3):
        w = W.ionization(k0)
        assert w["n"] == table[k0][0]
        H = O.build_hierarchy(w["n"], 2, w["k2"], layers=w["layers"], smoother="gmres")
        got[k0] = O.solve(H, w["rhs"][0], tol=1e-7, max_cycles=600).cycles
        assert 0.75 * table[k0][1] <= got[k0] <= 1.25 * table[k0][1], (k0, got)
    assert got[1] < got[2] < got[3]
    w = W.ionization(1)
    H = O.build_hierarchy(w["n"], 2, w["k2"], layers=w["layers"])
    with pytest.raises(O.DivergedError):
        O.solve(H, w["rhs"][0], tol=1e-7, max_cycles=600)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_last_krylov_norm_follows_from_the_arnoldi_sums(level):
    """A GMRES(3) step needs its last Krylov vector q_3 only through |q_3|
    (the entry h_{3,2} of the least-squares problem).  With the classical
    Gram-Schmidt basis q_{j+1} = A q_j - sum_i c_ij q_i, c_ij = <q_i, A q_j> /
    |q_i|^2, the q_i are orthogonal, so |q_3|^2 = |A q_2|^2 - sum_i |c_i2|^2
    |q_i|^2: the sums of the last Arnoldi product determine it without
    forming q_3 (the CUDA path's reading).  Checked on every level of a
    shifted ECS hierarchy with a k^2 field (63^2 .. 3^2), where |q_3|^2 /
    |A q_2|^2 ranges from about 0.5 down to 1e-2, for a random residual and
    for a point source."""
    n = 64
    k2 = W.smooth_k2(n, 2, 4, 30.0, 50.0)
    lv = O.build_hierarchy(n, 2, k2, layers=8, smoother="gmres").levels[level]
    rng = np.random.default_rng(level)
    shape = lv.shape
    point = np.zeros(shape, complex)
    point[shape[0] // 2, shape[1] // 3] = 1.0
    for r0 in (rng.standard_normal(shape) + 1j * rng.standard_normal(shape), point):
        q = [r0.ravel()]
        for j in range(3):
            w = O.apply_operator(lv, q[j].reshape(shape)).ravel()
            c = [np.vdot(q[i], w) / np.vdot(q[i], q[i]).real for i in range(j + 1)]
            q.append(w - sum(c[i] * q[i] for i in range(j + 1)))
        explicit = np.vdot(q[3], q[3]).real
        by_sums = np.vdot(w, w).real - sum(abs(c[i]) ** 2 * np.vdot(q[i], q[i]).real
                                           for i in range(3))
        assert explicit > 0.0
        assert abs(by_sums - explicit) <= 1e-9 * explicit, (level, explicit, by_sums)
