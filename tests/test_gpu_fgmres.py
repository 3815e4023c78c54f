"""Flexible GMRES(m) with one level-dependent V-cycle as the preconditioner
(the LVL-MG-FGMRES of Table 3) on the GPU against the oracle's fgmres.

Both sides run the same Arnoldi process on the same preconditioner; the GPU
orthogonalises with two classical Gram-Schmidt passes and solves the small
least-squares problem by Givens rotations, the oracle uses modified
Gram-Schmidt and a library least-squares solve.  In FP64 the iterates agree
to rounding, so the iteration counts are equal and the solutions agree far
below the stopping tolerance.  With complex64 cycles the preconditioner
differs from the oracle's by complex64 rounding; flexible GMRES absorbs
that, and the counts may differ by a step or two."""

import math

import numpy as np
import pytest

import oracle as O
from paper_1211_4752_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.ravel(b))


CASES = [
    dict(n=64, dim=2, k2=("const", 1600.0), layers=16, smoother="jacobi", m=10, form="csl"),
    dict(n=64, dim=2, k2=("const", 1600.0), layers=16, smoother="gmres", m=10, form="csl"),
    dict(n=128, dim=2, k2=("field", 40.0, 60.0), layers=(8, 24), smoother="jacobi", m=6,
         form="csg"),
    dict(n=256, dim=2, k2=("const", 25600.0), layers=64, smoother="jacobi", m=32, form="csl"),
    dict(n=16, dim=3, k2=("field", 5.0, 9.0), layers=2, smoother="jacobi", m=5, form="csl"),
    dict(n=32, dim=3, k2=("const", 300.0), layers=(2, 3), smoother="gmres", m=4, form="csl"),
]


def _pair(case, precision="fp64", batch=3):
    from paper_1211_4752_gb300 import HelmholtzMG
    n, dim = case["n"], case["dim"]
    spec = case["k2"]
    k2 = spec[1] if spec[0] == "const" else W.smooth_k2(n, dim, 4, spec[1], spec[2])
    P = int(round(math.log2(n)))
    c = [np.exp(-1j * (math.pi / 6) / P)] * (P - 2) if case["form"] == "csg" else None
    H = O.build_hierarchy(n, dim, k2, layers=case["layers"], form=case["form"], c=c,
                          smoother=case["smoother"])
    k2_t = dev(k2) if isinstance(k2, np.ndarray) else float(k2)
    mg = HelmholtzMG(n, dim=dim, k2=k2_t, layers=case["layers"], form=case["form"], c=c,
                     precision=precision, max_batch=batch, smoother=case["smoother"])
    return H, mg


def _rhs(H, n, dim):
    """A centre point source, a random field and a zero right-hand side."""
    shape = H.levels[0].shape
    f = np.zeros((3,) + shape, dtype=np.complex128)
    f[0] = W.point_sources(n, dim, [tuple([n // 2 - 1] * dim)])[0]
    f[1] = W.random_field(shape, 77)
    return f


def _rho(H, u, f):
    return np.linalg.norm(f - O.apply_operator(H.levels[0], u)) / np.linalg.norm(f)


@pytest.mark.parametrize("case", CASES,
                         ids=lambda c: f"{c['dim']}d-n{c['n']}-{c['smoother']}-m{c['m']}")
def test_fgmres_matches_oracle(case):
    H, mg = _pair(case)
    n, dim, m, tol = case["n"], case["dim"], case["m"], 1e-8
    f = _rhs(H, n, dim)
    u, info = mg.fgmres(dev(f), tol=tol, restart=m)
    u = host(u)
    for b in range(2):
        ref = O.fgmres(H, f[b], tol=tol, m=m)
        assert info[b]["status"] == "OK", (b, info[b])
        assert abs(info[b]["cycles"] - ref.cycles) <= 1, (b, info[b], ref.cycles)
        assert info[b]["refinements"] == (info[b]["cycles"] - 1) // m, (b, info[b])
        assert relerr(u[b], ref.u) < 1e-7, b
        assert _rho(H, u[b], f[b]) <= 1.01 * tol
        assert abs(info[b]["rel_residual"] - _rho(H, u[b], f[b])) <= 1e-3 * tol
    # the zero right-hand side returns u = 0 without iterating
    assert info[2]["status"] == "OK" and info[2]["cycles"] == 0
    assert not np.any(u[2])
    mg.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4]],
                         ids=lambda c: f"{c['dim']}d-n{c['n']}-{c['smoother']}")
def test_fgmres_complex64_preconditioner(case):
    """Complex64 cycles as the preconditioner of the FP64 Krylov process:
    the same solution to the tolerance, within two iterations of the FP64
    oracle."""
    H, mg = _pair(case, precision="mixed")
    n, dim, m, tol = case["n"], case["dim"], case["m"], 1e-8
    f = _rhs(H, n, dim)
    u, info = mg.fgmres(dev(f), tol=tol, restart=m)
    u = host(u)
    for b in range(2):
        ref = O.fgmres(H, f[b], tol=tol, m=m)
        assert info[b]["status"] == "OK", (b, info[b])
        assert abs(info[b]["cycles"] - ref.cycles) <= 2, (b, info[b], ref.cycles)
        assert _rho(H, u[b], f[b]) <= 1.01 * tol
        assert relerr(u[b], ref.u) < 1e-5
    mg.close()


def test_fgmres_iteration_limit_and_guess():
    """max_iter stops every right-hand side with NOT_CONVERGED and the
    iterate the oracle reaches after the same number of iterations (across a
    restart); an initial guess starts the oracle's process from it."""
    case = CASES[0]
    H, mg = _pair(case)
    n, dim = case["n"], case["dim"]
    f = _rhs(H, n, dim)
    u, info = mg.fgmres(dev(f[:2]), tol=1e-12, restart=4, max_iter=6)
    u = host(u)
    for b in range(2):
        ref = O.fgmres(H, f[b], tol=1e-12, m=4, max_iter=6, strict=False)
        assert info[b]["status"] == "ERR_NOT_CONVERGED" and info[b]["cycles"] == 6
        assert relerr(u[b], ref.u) < 1e-10
    g = W.random_field(f[:2].shape, 5, scale=1e-3)
    u, info = mg.fgmres(dev(f[:2]), tol=1e-8, restart=7, u0=dev(g))
    u = host(u)
    for b in range(2):
        ref = O.fgmres(H, f[b], tol=1e-8, m=7, u0=g[b])
        assert info[b]["status"] == "OK" and info[b]["cycles"] == ref.cycles
        assert relerr(u[b], ref.u) < 1e-9
    mg.close()


def test_fgmres_needs_fewer_cycles_than_the_stand_alone_cycle():
    """Table 3's comparison on the constant-k model (k = 40, n = 128, ECS
    n/4, GMRES(3) smoothing, tol 1e-7): LVL-MG-FGMRES takes no more V-cycles
    than LVL-MG alone."""
    from paper_1211_4752_gb300 import HelmholtzMG
    n = 128
    f = W.point_sources(n, 2, [(n // 2 - 1, n // 2 - 1)])
    mg = HelmholtzMG(n, k2=1600.0, layers=n // 4, smoother="gmres")
    _, i_mg = mg.solve(dev(f), tol=1e-7)
    _, i_fg = mg.fgmres(dev(f), tol=1e-7, restart=30)
    assert i_mg[0]["status"] == "OK" and i_fg[0]["status"] == "OK"
    assert i_fg[0]["cycles"] <= i_mg[0]["cycles"]
    mg.close()


def test_fgmres_options_are_checked():
    from paper_1211_4752_gb300 import HelmholtzMG
    from paper_1211_4752_gb300._binding import HHError
    mg = HelmholtzMG(64, k2=100.0)
    f = dev(np.ones((1, 63, 63), dtype=np.complex128))
    for kw in (dict(restart=0), dict(restart=33), dict(max_iter=-1), dict(tol=0.0)):
        with pytest.raises(HHError):
            mg.fgmres(f, **kw)
    mg.close()
