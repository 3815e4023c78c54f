"""GMRES(m) smoothing (Sec. 3.2) on the GPU against the oracle's GMRES cycle.

The GPU builds the Krylov basis with classical Gram-Schmidt on unnormalised
vectors and solves the small least-squares problem by Givens rotations; the
oracle uses modified Gram-Schmidt and a library least-squares solve.  Both
compute the same minimiser, so iterates agree to rounding."""

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
    dict(n=64, dim=2, k2=("field", 30.0, 36.0), layers=4, form="csl", m=3),
    dict(n=128, dim=2, k2=("const", 6400.0), layers=(8, 12), form="csg", m=3),
    dict(n=64, dim=2, k2=("const", 1600.0), layers=8, form="csl", m=2),
    dict(n=16, dim=3, k2=("field", 5.0, 9.0), layers=2, form="csl", m=3),
    dict(n=32, dim=3, k2=("const", 300.0), layers=(2, 3), form="csg", m=1),
]


def _pair(case, precision="fp64", batch=2):
    from paper_1211_4752_gb300 import HelmholtzMG
    n, dim = case["n"], case["dim"]
    spec = case["k2"]
    k2 = spec[1] if spec[0] == "const" else W.smooth_k2(n, dim, 4, spec[1], spec[2])
    P = int(round(math.log2(n)))
    c = [np.exp(-1j * (math.pi / 6) / P)] * (P - 2) if case["form"] == "csg" else None
    H = O.build_hierarchy(n, dim, k2, layers=case["layers"], form=case["form"], c=c,
                          smoother="gmres", m=case["m"])
    k2_t = dev(k2) if isinstance(k2, np.ndarray) else float(k2)
    mg = HelmholtzMG(n, dim=dim, k2=k2_t, layers=case["layers"], form=case["form"], c=c,
                     precision=precision, max_batch=batch, smoother="gmres", gmres_m=case["m"])
    return H, mg


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dim']}d-n{c['n']}-m{c['m']}")
def test_gmres_cycles_match_oracle(case):
    H, mg = _pair(case)
    f = W.random_field((2,) + H.levels[0].shape, 31)
    got = host(mg.cycles(dev(f), dev(np.zeros_like(f)), 2))
    for b in range(2):
        u = np.zeros_like(f[b])
        for _ in range(2):
            u = O.vcycle(H, 0, u, f[b])
        assert relerr(got[b], u) < 1e-9, b
    mg.close()
    # complex64 cycles on the same hierarchy
    H, mg = _pair(case, precision="mixed")
    got = host(mg.cycles(dev(f), dev(np.zeros_like(f)), 2))
    u = np.zeros_like(f[0])
    for _ in range(2):
        u = O.vcycle(H, 0, u, f[0])
    assert relerr(got[0], u) < 1e-4
    mg.close()


@pytest.mark.parametrize("n", [64, 128])
def test_gmres_solve_matches_oracle_constant_k(n):
    """The constant-k model of Table 1 (k = 40, centre source, ECS n/4):
    FP64 cycle for cycle against the oracle, mixed to the same residual."""
    from paper_1211_4752_gb300 import HelmholtzMG
    H = O.build_hierarchy(n, 2, 1600.0, layers=n // 4, smoother="gmres")
    f = W.point_sources(n, 2, [(n // 2 - 1, n // 2 - 1)])
    ref = O.solve(H, f[0], tol=1e-7, max_cycles=400)
    mg = HelmholtzMG(n, k2=1600.0, layers=n // 4, smoother="gmres")
    u, info = mg.solve(dev(f), tol=1e-7)
    assert info[0]["status"] == "OK"
    assert abs(info[0]["cycles"] - ref.cycles) <= 1
    assert relerr(host(u)[0], ref.u) < 1e-8
    mg.close()
    mg = HelmholtzMG(n, k2=1600.0, layers=n // 4, smoother="gmres", precision="mixed")
    u, info = mg.solve(dev(f), tol=1e-7)
    assert info[0]["status"] == "OK"
    rho = np.linalg.norm(f[0] - O.apply_operator(H.levels[0], host(u)[0])) / np.linalg.norm(f[0])
    assert rho <= 1e-7
    assert relerr(host(u)[0], ref.u) < 1e-5
    mg.close()


def test_gmres_adjoint_and_gradient():
    """Adjoint solve with GMRES-smoothed cycles on the conjugate-transposed
    hierarchy, and the gradient, against the oracle, on a medium where the
    Jacobi cycle diverges (kh = 0.5)."""
    from paper_1211_4752_gb300 import HelmholtzMG
    w = W.bump(n=64, layers=4, nsrc=2)
    k2 = w["k2"]
    H = O.build_hierarchy(64, 2, k2, layers=4, smoother="gmres")
    Ha = O.adjoint_hierarchy(H)
    mg = HelmholtzMG(64, k2=dev(k2), layers=4, max_batch=2, smoother="gmres")
    f = w["rhs"]
    g = W.random_field(f.shape, 41)
    u, iu = mg.solve(dev(f), tol=1e-10)
    lam, il = mg.adjoint(dev(g), tol=1e-10)
    assert all(i["status"] == "OK" for i in iu + il)
    u_ref = np.stack([O.solve(H, f[b], tol=1e-10).u for b in range(2)])
    lam_ref = np.stack([O.solve(Ha, g[b], tol=1e-10).u for b in range(2)])
    assert relerr(host(u), u_ref) < 1e-8
    assert relerr(host(lam), lam_ref) < 1e-8
    grad = host(mg.grad_k2(u, lam))
    gref = O.grad_k2(u_ref, lam_ref)
    assert np.abs(grad - gref).max() <= 1e-7 * np.abs(gref).max()
    mg.close()


def test_gmres_options_are_checked():
    from paper_1211_4752_gb300 import HelmholtzMG
    from paper_1211_4752_gb300._binding import HHError
    with pytest.raises(HHError):
        HelmholtzMG(64, k2=100.0, smoother="gmres", gmres_m=4)
    with pytest.raises(HHError):
        HelmholtzMG(64, k2=100.0, smoother="gmres", max_batch=65)


def test_theta_sweep_matches_oracle():
    """Table 5's experiment (k = 30, n = 128, GMRES(3), theta_max from pi/15
    to pi/4): the GPU's cycle counts equal the oracle's at every rotation."""
    from paper_1211_4752_gb300 import HelmholtzMG
    n = 128
    f = W.point_sources(n, 2, [(n // 2 - 1, n // 2 - 1)])
    for d in (15, 12, 10, 8, 6, 5, 4):
        H = O.build_hierarchy(n, 2, 900.0, layers=n // 4, smoother="gmres", theta_max=math.pi / d)
        ref = O.solve(H, f[0], tol=1e-7, max_cycles=400).cycles
        mg = HelmholtzMG(n, k2=900.0, layers=n // 4, smoother="gmres", theta_max=math.pi / d)
        _, info = mg.solve(dev(f), tol=1e-7)
        assert info[0]["status"] == "OK" and abs(info[0]["cycles"] - ref) <= 1, (d, info, ref)
        mg.close()


@pytest.mark.parametrize("k0", [1, 2, 3])
def test_ionization_model_matches_oracle(k0):
    """Sec. 4.3's ionization model (Table 8 grid sizes, Dirichlet on x = 0 and
    y = 0, ECS on the other sides, space-dependent coefficient and source):
    FP64 cycle for cycle against the oracle to 1e-7, mixed to the same
    residual; the Jacobi cycle diverges on both sides."""
    from paper_1211_4752_gb300 import HelmholtzMG
    w = W.ionization(k0)
    n = w["n"]
    H = O.build_hierarchy(n, 2, w["k2"], layers=w["layers"], smoother="gmres")
    ref = O.solve(H, w["rhs"][0], tol=1e-7, max_cycles=600)
    f = dev(w["rhs"])
    mg = HelmholtzMG(n, k2=dev(w["k2"]), layers=w["layers"], smoother="gmres")
    u, info = mg.solve(f, tol=1e-7)
    assert info[0]["status"] == "OK" and abs(info[0]["cycles"] - ref.cycles) <= 1, (info, ref.cycles)
    assert relerr(host(u)[0], ref.u) < 1e-8
    mg.close()
    mg = HelmholtzMG(n, k2=dev(w["k2"]), layers=w["layers"], smoother="gmres", precision="mixed")
    u, info = mg.solve(f, tol=1e-7)
    assert info[0]["status"] == "OK"
    rho = np.linalg.norm(w["rhs"][0] - O.apply_operator(H.levels[0], host(u)[0])) / np.linalg.norm(w["rhs"][0])
    assert rho <= 1e-7
    assert relerr(host(u)[0], ref.u) < 1e-5
    mg.close()
    if k0 == 1:
        Hj = O.build_hierarchy(n, 2, w["k2"], layers=w["layers"])
        with pytest.raises(O.DivergedError):
            O.solve(Hj, w["rhs"][0], tol=1e-7, max_cycles=600)
        mg = HelmholtzMG(n, k2=dev(w["k2"]), layers=w["layers"])
        _, info = mg.solve(f, tol=1e-7)
        assert info[0]["status"] == "ERR_DIVERGED"
        mg.close()


@pytest.mark.parametrize("k,n", [(20, 32), (40, 64), (80, 128), (160, 256)])
def test_radiating_condition_matches_oracle(k, n):
    """Table 4's model (constant k, the radiating condition on every side, no
    ECS layer, centre source): GMRES(3)-smoothed solves cycle for cycle
    against the oracle (FP64) and to the same residual (mixed); the adjoint
    against the oracle's conjugate-transposed hierarchy; weighted-Jacobi
    cycles (the fused kernels and the tail operator) iterate for iterate."""
    from paper_1211_4752_gb300 import HelmholtzMG
    k2 = float(k * k)
    f = W.point_sources(n, 2, [(n // 2 - 1, n // 2 - 1)])
    H = O.build_hierarchy(n, 2, k2, sommerfeld=True, smoother="gmres")
    ref = O.solve(H, f[0], tol=1e-7, max_cycles=600)
    mg = HelmholtzMG(n, k2=k2, sommerfeld=True, smoother="gmres")
    u, info = mg.solve(dev(f), tol=1e-7)
    assert info[0]["status"] == "OK" and abs(info[0]["cycles"] - ref.cycles) <= 1, (info, ref.cycles)
    assert relerr(host(u)[0], ref.u) < 1e-8
    g = W.random_field(f.shape, 61)
    lam, il = mg.adjoint(dev(g), tol=1e-7)
    lref = O.solve(O.adjoint_hierarchy(H), g[0], tol=1e-7, max_cycles=600)
    assert il[0]["status"] == "OK" and abs(il[0]["cycles"] - lref.cycles) <= 1
    assert relerr(host(lam)[0], lref.u) < 1e-8
    mg.close()
    mg = HelmholtzMG(n, k2=k2, sommerfeld=True, smoother="gmres", precision="mixed")
    u, info = mg.solve(dev(f), tol=1e-7)
    assert info[0]["status"] == "OK"
    rho = np.linalg.norm(f[0] - O.apply_operator(H.levels[0], host(u)[0])) / np.linalg.norm(f[0])
    assert rho <= 1e-7 and relerr(host(u)[0], ref.u) < 1e-5
    mg.close()
    Hj = O.build_hierarchy(n, 2, k2, sommerfeld=True)
    uj = np.zeros_like(f[0])
    for _ in range(3):
        uj = O.vcycle(Hj, 0, uj, f[0])
    for precision, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        mg = HelmholtzMG(n, k2=k2, sommerfeld=True, precision=precision)
        got = host(mg.cycles(dev(f), dev(np.zeros_like(f)), 3))
        assert relerr(got[0], uj) < tol, precision
        mg.close()


def test_radiating_condition_3d_cycles_match_oracle():
    from paper_1211_4752_gb300 import HelmholtzMG
    n, k2 = 16, 64.0
    f = W.random_field((1, 15, 15, 15), 62)
    for sm in ("jacobi", "gmres"):
        H = O.build_hierarchy(n, 3, k2, sommerfeld=True, smoother=sm)
        u = np.zeros_like(f[0])
        for _ in range(2):
            u = O.vcycle(H, 0, u, f[0])
        mg = HelmholtzMG(n, dim=3, k2=k2, sommerfeld=True, smoother=sm)
        got = host(mg.cycles(dev(f), dev(np.zeros_like(f)), 2))
        assert relerr(got[0], u) < 1e-10, sm
        mg.close()


@pytest.mark.parametrize("fuse", ["0", "1"])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3]],
                         ids=lambda c: f"{c['dim']}d-n{c['n']}-m{c['m']}")
def test_gmres_fused_and_separate_kernels_match_oracle(case, fuse, monkeypatch):
    """The orthogonalisation of step j fused with the Arnoldi product of step
    j+1 (neighbours' q_{j+1} recomputed; HH_GMFUSE=1, the complex64 default)
    and the separate kernels (HH_GMFUSE=0, the complex128 default) both
    follow the oracle: FP64 to 1e-9, complex64 to 1e-4, after two cycles."""
    monkeypatch.setenv("HH_GMFUSE", fuse)
    f = W.random_field((2,) + (case["n"] - 1,) * case["dim"], 37)
    for precision, tol in (("fp64", 1e-9), ("mixed", 1e-4)):
        H, mg = _pair(case, precision=precision)
        assert mg.cycle_kernels > 0
        got = host(mg.cycles(dev(f), dev(np.zeros_like(f)), 2))
        for b in range(2):
            u = np.zeros_like(f[b])
            for _ in range(2):
                u = O.vcycle(H, 0, u, f[b])
            assert relerr(got[b], u) < tol, (precision, b)
        mg.close()


def test_gmres_time_hooks():
    """hh_time_kernel kernel 6 (one level-0 GMRES step) and kernel 4 (the
    one-block tail) run on a GMRES handle; kernel 6 is refused on a Jacobi
    handle."""
    import ctypes as ct
    from paper_1211_4752_gb300 import HelmholtzMG, _binding as B
    s = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    mg = HelmholtzMG(256, k2=(0.625 * 256) ** 2, layers=8, precision="mixed", smoother="gmres")
    ms = ct.c_double()
    for kernel in (6, 4):
        assert B.lib().hh_time_kernel(mg._h, kernel, 0, 1, 3, ct.byref(ms), s) == 0
        assert ms.value > 0.0
    mg.close()
    mj = HelmholtzMG(64, k2=1600.0, layers=4, precision="mixed")
    assert B.lib().hh_time_kernel(mj._h, 6, 0, 1, 1, ct.byref(ms), s) != 0
    mj.close()


@pytest.mark.parametrize("n", [128, 512])
def test_gmres_column_kernels_match_oracle(n, monkeypatch):
    """The column-marching Arnoldi and fused kernels (normally from 256^2 on;
    HH_GMCOL_MIN_N=64 turns them on here, 128: one chunk with idle lanes, 512:
    two 256-column chunks and a warp-edge neighbour exchange across them)
    against the oracle's GMRES cycle: FP64 (with HH_GMFUSE=1) to 1e-9 and
    complex64 to 1e-4, after two cycles, on a k^2 field with ECS layers."""
    monkeypatch.setenv("HH_GMCOL_MIN_N", "64")
    monkeypatch.setenv("HH_GMFUSE", "1")
    case = dict(n=n, dim=2, k2=("field", 0.3 * n * n / 4, 0.35 * n * n / 4), layers=n // 16,
                form="csl", m=3)
    f = W.random_field((2,) + (n - 1,) * 2, 41)
    for precision, tol in (("fp64", 1e-9), ("mixed", 1e-4)):
        H, mg = _pair(case, precision=precision)
        got = host(mg.cycles(dev(f), dev(np.zeros_like(f)), 2))
        for b in range(2):
            u = np.zeros_like(f[b])
            for _ in range(2):
                u = O.vcycle(H, 0, u, f[b])
            assert relerr(got[b], u) < tol, (precision, b)
        mg.close()
