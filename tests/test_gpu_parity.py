"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several thread blocks and ragged tails; ECS and Dirichlet,
constant and heterogeneous k^2, CSL and CSG forms, batches, 2-D and 3-D."""

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
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def maxrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    # n, dim, k2 spec, layers, form, c_scale
    dict(n=16, dim=2, k2=("const", 300.0), layers=0, form="csl"),
    dict(n=64, dim=2, k2=("field", 10.0, 30.0), layers=(4, 6), form="csl"),
    dict(n=128, dim=2, k2=("field", 40.0, 70.0), layers=8, form="csg", c=True),
    dict(n=16, dim=3, k2=("field", 5.0, 9.0), layers=2, form="csl"),
    dict(n=32, dim=3, k2=("const", 300.0), layers=(2, 3), form="csg"),
]


def k2_of(case, seed=0):
    spec = case["k2"]
    if spec[0] == "const":
        return spec[1]
    return W.smooth_k2(case["n"], case["dim"], seed, spec[1], spec[2])


def make_pair(case, batch=2, **kw):
    from paper_1211_4752_gb300 import HelmholtzMG
    n, dim = case["n"], case["dim"]
    k2 = k2_of(case)
    P = int(round(math.log2(n)))
    L = P - 1
    c = None
    if case.get("c"):
        c = [np.exp(-1j * (math.pi / 6) / P)] * (L - 1)
    H = O.build_hierarchy(n, dim, k2, layers=case["layers"], form=case["form"], c=c,
                          omega=kw.get("omega", 0.8), nu1=kw.get("nu1", 1), nu2=kw.get("nu2", 1))
    k2_t = dev(k2) if isinstance(k2, np.ndarray) else float(k2)
    mg = HelmholtzMG(n, dim=dim, k2=k2_t, layers=case["layers"], form=case["form"], c=c,
                     max_batch=batch, **kw)
    return H, mg


def rnd(shape, seed):
    return W.random_field(shape, seed)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dim']}d-n{c['n']}-{c['form']}")
def test_apply_forward_and_adjoint(case):
    H, mg = make_pair(case, batch=3)
    Ha = O.adjoint_hierarchy(H)
    for l in range(len(H.levels)):
        lv = H.levels[l]
        x = rnd((3,) + lv.shape, 10 + l)
        for adj, hier in ((False, H), (True, Ha)):
            y = host(mg.apply(dev(x), level=l, adjoint=adj))
            ref = np.stack([O.apply_operator(hier.levels[l], x[b]) for b in range(3)])
            assert maxrel(y, ref) < 1e-13, (l, adj)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['dim']}d-n{c['n']}-{c['form']}")
def test_step_kernels(case):
    check_step_kernels(case)


def test_step_kernels_3d_63():
    """The 3-D tile-staged kernels (8 x 8 x 8 boxes) on 63^3 with a k^2 field
    and uneven ECS layers: several boxes per axis and a ragged last box on
    every level (63, 31, 15, 7 = 8 q - 1)."""
    check_step_kernels(dict(n=64, dim=3, k2=("field", 20.0, 40.0), layers=(4, 6), form="csl"))


def check_step_kernels(case):
    H, mg = make_pair(case, batch=2)
    for l in range(len(H.levels) - 1):
        lv, lc = H.levels[l], H.levels[l + 1]
        u = rnd((2,) + lv.shape, 1 + l)
        f = rnd((2,) + lv.shape, 2 + l)
        e = rnd((2,) + lc.shape, 3 + l)
        # weighted Jacobi, Eq. (wjacobi)
        got = host(mg.smooth(l, dev(u), dev(f)))
        ref = np.stack([O.jacobi(lv, u[b], f[b], H.omega) for b in range(2)])
        assert maxrel(got, ref) < 1e-13
        # c * FW(f - A u)
        got = host(mg.residual_restrict(l, dev(u), dev(f)))
        ref = np.stack([H.c[l] * O.restrict_fw(f[b] - O.apply_operator(lv, u[b])) for b in range(2)])
        assert maxrel(got, ref) < 1e-12
        # Jacobi of u + P e
        got = host(mg.correct_smooth(l, dev(u), dev(e), dev(f)))
        ref = np.stack([O.jacobi(lv, u[b] + O.prolong(e[b]), f[b], H.omega) for b in range(2)])
        assert maxrel(got, ref) < 1e-13
    fL = rnd((2,) + H.levels[-1].shape, 99)
    got = host(mg.coarse_solve(dev(fL)))
    ref = np.stack([O.lu_solve(H.lu, fL[b].ravel()).reshape(fL[b].shape) for b in range(2)])
    assert maxrel(got, ref) < 1e-13


@pytest.mark.parametrize("nu", [(1, 1), (2, 3)])
@pytest.mark.parametrize("case", CASES[1:4], ids=lambda c: f"{c['dim']}d-n{c['n']}-{c['form']}")
def test_cycles_match_oracle_fp64(case, nu):
    H, mg = make_pair(case, batch=2, nu1=nu[0], nu2=nu[1], omega=0.8 + 0.05j)
    f = rnd((2,) + H.levels[0].shape, 5)
    u0 = rnd((2,) + H.levels[0].shape, 6) * 1e-3
    got = host(mg.cycles(dev(f), dev(u0), 3))
    ref = []
    for b in range(2):
        u = u0[b].copy()
        for _ in range(3):
            u = O.vcycle(H, 0, u, f[b])
        ref.append(u)
    assert relerr(got, np.stack(ref)) < 1e-12


def test_cycles_complex64_track_oracle():
    case = CASES[1]
    H, mg = make_pair(case, batch=1, precision="mixed")
    f = rnd((1,) + H.levels[0].shape, 5)
    got = host(mg.cycles(dev(f), dev(np.zeros_like(f)), 2))
    u = np.zeros_like(f[0])
    for _ in range(2):
        u = O.vcycle(H, 0, u, f[0])
    assert relerr(got[0], u) < 1e-5


def test_tail_operator_matches_tail_kernel(monkeypatch):
    """complex64 cycles: the dense tail operator (default) and the recursive
    tail kernel (HH_TAIL=kernel) run the same V-cycle; both track the oracle."""
    case = CASES[2]   # 128^2, heterogeneous k^2, CSG with c, ECS layers
    H, mg = make_pair(case, batch=2, precision="mixed")
    monkeypatch.setenv("HH_TAIL", "kernel")
    _, mgk = make_pair(case, batch=2, precision="mixed")
    f = rnd((2,) + H.levels[0].shape, 11)
    z = np.zeros_like(f)
    a = host(mg.cycles(dev(f), dev(z), 3))
    b = host(mgk.cycles(dev(f), dev(z), 3))
    u = np.zeros_like(f[1])
    for _ in range(3):
        u = O.vcycle(H, 0, u, f[1])
    assert relerr(a, b) < 2e-6
    assert relerr(a[1], u) < 1e-5 and relerr(b[1], u) < 1e-5


@pytest.mark.parametrize("n", [64, 256])
def test_cluster_mid_levels_match_per_level_kernels(n, monkeypatch):
    """complex64 cycles: the cluster kernel for the middle levels (HH_MID=1)
    against the per-level kernels and the dense tail (default), forward and
    adjoint, on a heterogeneous medium with ECS layers and the CSG form."""
    from paper_1211_4752_gb300 import HelmholtzMG
    import math as _m
    k2 = W.smooth_k2(n, 2, 9, 0.55 * n, 0.62 * n)
    P = int(round(_m.log2(n)))
    c = [np.exp(-1j * (_m.pi / 6) / P)] * (P - 2)
    kw = dict(k2=dev(k2), layers=n // 16, form="csg", c=c, max_batch=2, precision="mixed")
    monkeypatch.setenv("HH_MID", "1")
    mg = HelmholtzMG(n, **kw)
    monkeypatch.delenv("HH_MID")
    mg0 = HelmholtzMG(n, **kw)
    if n > 64:   # the cluster kernel replaces per-level kernels (at 64 it replaces the tail)
        assert mg.cycle_kernels < mg0.cycle_kernels
    f = rnd((2, n - 1, n - 1), 21)
    z = np.zeros_like(f)
    a = host(mg.cycles(dev(f), dev(z), 3))
    b = host(mg0.cycles(dev(f), dev(z), 3))
    assert relerr(a, b) < 2e-6
    H = O.build_hierarchy(n, 2, k2, layers=n // 16, form="csg", c=c)
    u = np.zeros_like(f[0])
    for _ in range(3):
        u = O.vcycle(H, 0, u, f[0])
    assert relerr(a[0], u) < 1e-5
    # adjoint direction: a loose tolerance that one cycle meets (the Jacobi
    # cycle diverges on random right-hand sides at this kh after a few cycles)
    g = rnd((2, n - 1, n - 1), 22)
    la, ia = mg.adjoint(dev(g), tol=0.7)
    lb, ib = mg0.adjoint(dev(g), tol=0.7)
    assert all(i["status"] == "OK" for i in ia + ib)
    assert [i["cycles"] for i in ia] == [i["cycles"] for i in ib]
    assert relerr(host(la), host(lb)) < 1e-5
    mg.close()
    mg0.close()


@pytest.mark.parametrize("n,batch", [(64, 2), (256, 3), (1024, 1)])
def test_persistent_cycle_matches_per_level_kernels(n, batch, monkeypatch):
    """complex64 cycles in one cooperative launch (HH_PERSIST=1) against the
    per-level kernels: iterates to complex64 rounding (the tile shapes differ,
    so the summation order does), solves cycle for cycle, forward and adjoint,
    on a heterogeneous medium with ECS layers; FGMRES on top of it."""
    from paper_1211_4752_gb300 import HelmholtzMG
    k2 = W.smooth_k2(n, 2, 9, 0.55 * n, 0.62 * n)
    kw = dict(k2=dev(k2), layers=n // 16, max_batch=batch, precision="mixed")
    monkeypatch.setenv("HH_PERSIST", "1")
    mg = HelmholtzMG(n, **kw)
    monkeypatch.delenv("HH_PERSIST")
    mg0 = HelmholtzMG(n, **kw)
    assert mg.cycle_kernels == 1 < mg0.cycle_kernels
    f = rnd((batch, n - 1, n - 1), 31)
    z = np.zeros_like(f)
    a = host(mg.cycles(dev(f), dev(z), 3))
    b = host(mg0.cycles(dev(f), dev(z), 3))
    assert relerr(a, b) < 2e-6
    mg.close()
    mg0.close()
    # solves on the constant-k model (k = 40 with ECS n/4 at 64, else kh =
    # 0.625 with ECS n/32), where the Jacobi cycle converges
    kc, lay = (1600.0, 16) if n == 64 else ((0.625 * n) ** 2, n // 32)
    kw = dict(k2=kc, layers=lay, max_batch=batch, precision="mixed")
    monkeypatch.setenv("HH_PERSIST", "1")
    mg = HelmholtzMG(n, **kw)
    monkeypatch.delenv("HH_PERSIST")
    mg0 = HelmholtzMG(n, **kw)
    assert mg.cycle_kernels == 1
    src = np.zeros_like(f)
    for j in range(batch):
        src[j] = W.point_sources(n, 2, [(n // 2 - 1 + 3 * j, n // 2 - 1)])[0]
    ua, ia = mg.solve(dev(src), tol=1e-6)
    ub, ib = mg0.solve(dev(src), tol=1e-6)
    assert all(i["status"] == "OK" for i in ia)
    # the per-level path's tile shapes come from the autotuner, so its
    # complex64 rounding (and at the tolerance a cycle) may differ
    assert all(abs(x["cycles"] - y["cycles"]) <= 1 for x, y in zip(ia, ib)), (ia, ib)
    assert relerr(host(ua), host(ub)) < 1e-5
    la, il = mg.adjoint(dev(src), tol=1e-6)
    assert all(i["status"] == "OK" for i in il)
    rho = np.linalg.norm((host(mg.apply(la, adjoint=True)) - src).reshape(batch, -1), axis=1)
    assert np.all(rho <= 1e-6 * np.linalg.norm(src.reshape(batch, -1), axis=1))
    uf, jf = mg.fgmres(dev(src), tol=1e-6, restart=16)
    assert all(i["status"] == "OK" for i in jf)
    assert relerr(host(uf), host(ub)) < 1e-5
    mg.close()
    mg0.close()


def test_adjoint_mixed_matches_oracle():
    """Mixed-precision adjoint solve (adjoint tail operator) vs the oracle."""
    from paper_1211_4752_gb300 import HelmholtzMG
    n, layers = 128, 8
    k2 = W.smooth_k2(n, 2, 4, 76.0, 80.0)
    H = O.build_hierarchy(n, 2, k2, layers=layers)
    Ha = O.adjoint_hierarchy(H)
    mg = HelmholtzMG(n, k2=dev(k2), layers=layers, max_batch=2, precision="mixed")
    g = rnd((2, n - 1, n - 1), 12)
    lam, il = mg.adjoint(dev(g), tol=1e-9)
    lam_ref = np.stack([O.solve(Ha, g[b], tol=1e-11).u for b in range(2)])
    assert all(i["status"] == "OK" for i in il)
    assert relerr(host(lam), lam_ref) < 1e-7


def test_loop_unroll_leaves_iterates_unchanged(monkeypatch):
    """Cycle copies after the stop test do nothing: the iterate, the cycle
    count and the residual are bit-identical for every unroll factor, and the
    device-counted kernels follow ceil((cycles + 1) / U) loop iterations."""
    from paper_1211_4752_gb300 import HelmholtzMG
    n, k, layers = 64, 40.0, 2
    f = point_rhs(n, 2, 1, 3)
    out = {}
    for U in (1, 3):
        monkeypatch.setenv("HH_UNROLL", str(U))
        mg = HelmholtzMG(n, k2=k * k, layers=layers, max_batch=1)
        u, info = mg.solve(dev(f), tol=1e-8)
        c = info[0]["cycles"]
        assert mg.solve_kernels == U * math.ceil((c + 1) / U) * mg.cycle_kernels + 3
        out[U] = (host(u), c, info[0]["rel_residual"])
        mg.close()
    assert out[1][1] == out[3][1] and out[1][2] == out[3][2]
    assert np.array_equal(out[1][0], out[3][0])


def point_rhs(n, dim, batch, seed):
    rng = np.random.default_rng(seed)
    pos = [tuple(rng.integers(n // 8, n - n // 8 - 1, size=dim)) for _ in range(batch)]
    return W.point_sources(n, dim, pos)


SOLVE_CASES = [
    dict(n=64, k=40.0, layers=2),     # kh = 0.625, thin layer
    dict(n=128, k=40.0, layers=16),
    dict(n=32, k=20.0, layers=4),
]


@pytest.mark.parametrize("sc", SOLVE_CASES, ids=lambda s: f"n{s['n']}-k{s['k']}")
def test_solve_fp64_matches_oracle(sc):
    from paper_1211_4752_gb300 import HelmholtzMG
    n, k, layers = sc["n"], sc["k"], sc["layers"]
    f = point_rhs(n, 2, 3, n)
    H = O.build_hierarchy(n, 2, k * k, layers=layers)
    mg = HelmholtzMG(n, k2=k * k, layers=layers, max_batch=3)
    u, info = mg.solve(dev(f), tol=1e-6)
    u = host(u)
    for b in range(3):
        res = O.solve(H, f[b], tol=1e-6, max_cycles=20000)
        assert info[b]["status"] == "OK"
        assert abs(info[b]["cycles"] - res.cycles) <= 1, (info[b], res.cycles)
        assert relerr(u[b], res.u) < 1e-10
        rho = np.linalg.norm(f[b] - O.apply_operator(H.levels[0], u[b])) / np.linalg.norm(f[b])
        assert rho <= 1e-6 and abs(rho - info[b]["rel_residual"]) < 1e-12


@pytest.mark.parametrize("sc", SOLVE_CASES[:2], ids=lambda s: f"n{s['n']}-k{s['k']}")
def test_solve_mixed_error_vs_oracle(sc):
    from paper_1211_4752_gb300 import HelmholtzMG
    n, k, layers = sc["n"], sc["k"], sc["layers"]
    f = point_rhs(n, 2, 2, n + 1)
    H = O.build_hierarchy(n, 2, k * k, layers=layers)
    mg = HelmholtzMG(n, k2=k * k, layers=layers, max_batch=2, precision="mixed")
    u, info = mg.solve(dev(f), tol=1e-6)
    u = host(u)
    for b in range(2):
        ref = O.solve(H, f[b], tol=1e-10, max_cycles=40000).u
        assert info[b]["status"] == "OK" and info[b]["refinements"] >= 1
        rho = np.linalg.norm(f[b] - O.apply_operator(H.levels[0], u[b])) / np.linalg.norm(f[b])
        assert rho <= 1e-6
        assert relerr(u[b], ref) <= 1e-5


def test_dirichlet_model_problem_stalls_like_oracle():
    """63^2, k = 40, Dirichlet: neither side reaches 1e-6; iterates agree."""
    from paper_1211_4752_gb300 import HelmholtzMG
    w = W.dirichlet_const()
    H = O.build_hierarchy(w["n"], 2, w["k2"], layers=0)
    mg = HelmholtzMG(w["n"], k2=w["k2"], layers=0, max_cycles=60)
    u, info = mg.solve(dev(w["rhs"]), tol=1e-6)
    assert info[0]["status"] == "ERR_NOT_CONVERGED" and info[0]["cycles"] == 60
    with pytest.raises(O.NotConvergedError):
        O.solve(H, w["rhs"][0], tol=1e-6, max_cycles=60)
    ref = np.zeros_like(w["rhs"][0])
    for _ in range(60):
        ref = O.vcycle(H, 0, ref, w["rhs"][0])
    assert relerr(host(u)[0], ref) < 1e-10


def test_adjoint_solve_and_gradient_match_oracle():
    from paper_1211_4752_gb300 import HelmholtzMG
    n, layers = 64, 8
    k2 = W.smooth_k2(n, 2, 3, 38.0, 40.0)   # kh ~ 0.6: the Jacobi cycle converges
    H = O.build_hierarchy(n, 2, k2, layers=layers)
    Ha = O.adjoint_hierarchy(H)
    mg = HelmholtzMG(n, k2=dev(k2), layers=layers, max_batch=2)
    f = point_rhs(n, 2, 2, 7)
    g = rnd((2, n - 1, n - 1), 8)
    u, iu = mg.solve(dev(f), tol=1e-10)
    lam, il = mg.adjoint(dev(g), tol=1e-10)
    u_h, lam_h = host(u), host(lam)
    lam_ref = np.stack([O.solve(Ha, g[b], tol=1e-10).u for b in range(2)])
    u_ref = np.stack([O.solve(H, f[b], tol=1e-10).u for b in range(2)])
    assert relerr(lam_h, lam_ref) < 1e-9
    assert all(i["status"] == "OK" for i in il)
    grad = host(mg.grad_k2(u, lam))
    assert maxrel(grad, O.grad_k2(u_ref, lam_ref)) < 1e-8
    # dot test on the device: <A x, y> = <x, A^H y>
    x, y = rnd((1, n - 1, n - 1), 1), rnd((1, n - 1, n - 1), 2)
    lhs = np.vdot(host(mg.apply(dev(x))), y)
    rhs = np.vdot(x, host(mg.apply(dev(y), adjoint=True)))
    assert abs(lhs - rhs) <= 1e-13 * 8 * n * n * np.linalg.norm(x) * np.linalg.norm(y)


def test_autograd_matches_central_differences():
    from paper_1211_4752_gb300 import helmholtz_solve
    n, layers = 32, 4
    k2 = dev(W.smooth_k2(n, 2, 11, 19.0, 21.0)).requires_grad_(True)
    f = dev(point_rhs(n, 2, 2, 3)).requires_grad_(True)
    rows = n - 1 - layers - 1
    d = dev(rnd((2, n - 1), 4) * 1e-4)
    kw = dict(n=n, layers=layers)

    def loss_of(k2v, fv):
        u = helmholtz_solve(k2v, fv, tol=1e-12, **kw)
        return 0.5 * (u[:, rows, :] - d).abs().pow(2).sum()

    L0 = loss_of(k2, f)
    L0.backward()
    gk = k2.grad.detach().cpu().numpy()
    gf = f.grad.detach().cpu().numpy()
    k2n = k2.detach().cpu().numpy()
    rng = np.random.default_rng(0)
    pts = [tuple(rng.integers(0, n - 1, size=2)) for _ in range(20)]
    with torch.no_grad():
        for (i, j) in pts:
            dk = 1e-4 * k2n[i, j]
            kp = k2.detach().clone(); kp[i, j] += dk
            km = k2.detach().clone(); km[i, j] -= dk
            fd = (loss_of(kp, f.detach()) - loss_of(km, f.detach())).item() / (2 * dk)
            assert abs(fd - gk[i, j]) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(gk).max())
        # d loss / d f along a random complex direction: Re <grad_f, v>
        v = dev(rnd(tuple(f.shape), 5))
        eps = 1e-3
        fd = (loss_of(k2.detach(), f.detach() + eps * v) - loss_of(k2.detach(), f.detach() - eps * v)).item() / (2 * eps)
        pred = np.real(np.vdot(gf, host(v)))
        assert abs(fd - pred) <= 1e-4 * abs(fd)


def test_edge_cases():
    from paper_1211_4752_gb300 import HelmholtzMG, HHError
    n = 32
    mg = HelmholtzMG(n, k2=400.0, layers=4, max_batch=3)
    f = point_rhs(n, 2, 3, 1)
    f[1] = 0.0                       # a zero right-hand side in the batch
    u, info = mg.solve(dev(f), tol=1e-6)
    u = host(u)
    assert info[1]["status"] == "OK" and info[1]["cycles"] == 0 and not np.any(u[1])
    assert info[0]["status"] == "OK" and info[2]["status"] == "OK"
    # the converged solution as the initial guess: no further cycle needed
    u2, info2 = mg.solve(dev(f), tol=1e-6, u0=dev(u))
    assert info2[0]["cycles"] == 0 and info2[2]["cycles"] == 0
    assert np.array_equal(host(u2)[0], u[0])
    # host-buffer entry point matches the device one
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    info3 = mg.solve_host(fh, uh, tol=1e-6)
    assert np.array_equal(uh.numpy(), u) and info3[0]["cycles"] == info[0]["cycles"]
    with pytest.raises(HHError):
        mg.solve(dev(point_rhs(n, 2, 4, 1)))      # batch > max_batch
    with pytest.raises((HHError, ValueError)):
        mg.smooth(7, dev(np.zeros((1, 3, 3), complex)), dev(np.zeros((1, 3, 3), complex)))


def test_max_cycles_and_divergence_status():
    from paper_1211_4752_gb300 import HelmholtzMG
    n = 32
    # k^2 = 250 diverges with weighted Jacobi (oracle: diverged at cycle 7)
    f = W.random_field((1, n - 1, n - 1), 2)
    H = O.build_hierarchy(n, 2, 250.0, layers=4)
    with pytest.raises(O.DivergedError):
        O.solve(H, f[0], tol=1e-10)
    mg = HelmholtzMG(n, k2=250.0, layers=4)
    u, info = mg.solve(dev(f), tol=1e-10)
    assert info[0]["status"] == "ERR_DIVERGED"
    mg2 = HelmholtzMG(n, k2=400.0, layers=4, max_cycles=5)
    u, info = mg2.solve(dev(point_rhs(n, 2, 1, 3)), tol=1e-10)
    assert info[0]["status"] == "ERR_NOT_CONVERGED" and info[0]["cycles"] == 5


OMEGAS = [0.8, 0.8 + 0.2j, 0.8 - 0.2j, 0.7 + 0.3j, 0.7 - 0.3j, 0.6 - 0.4j, 1.0 - 0.3j,
          0.5 + 0.5j]


@pytest.mark.parametrize("layers", [16, 8])
def test_complex_omega_jacobi_ablation_matches_oracle(layers):
    """The weighted-Jacobi cycle with complex weights omega (Eq. (wjacobi)) on
    Table 1's constant-k model (k = 40, 63^2, centre source, ECS n/4 and
    n/8): cycle counts to 1e-6, or the cycle at which rho passes the
    divergence limit, equal the oracle's (+-1) for every weight.  No fixed
    weight converges where the real one diverges, the instability of fixed
    Jacobi weights on the shifted levels (Eq. (jacstab)) that motivates GMRES
    smoothing."""
    from paper_1211_4752_gb300 import HelmholtzMG
    n, k2 = 64, 1600.0
    f = W.point_sources(n, 2, [(n // 2 - 1, n // 2 - 1)])
    for om in OMEGAS:
        H = O.build_hierarchy(n, 2, k2, layers=layers, omega=om)
        try:
            ref = O.solve(H, f[0], tol=1e-6, max_cycles=3000)
            want, cyc = "OK", ref.cycles
        except O.DivergedError as e:
            want, cyc = "ERR_DIVERGED", int(str(e).split("cycle ")[1].split(":")[0])
        mg = HelmholtzMG(n, k2=k2, layers=layers, omega=om)
        _, info = mg.solve(dev(f), tol=1e-6)
        assert info[0]["status"] == want and abs(info[0]["cycles"] - cyc) <= 1, (om, info, want, cyc)
        mg.close()


def test_bounded_wait_timeout_returns_status_and_handle_recovers(monkeypatch):
    """The failure path of the bounded device waits, without a fault: with the
    test hook on, one block of the cooperative cycle leaves without arriving
    at its first grid barrier; the others' waits give up after about a
    second, the solve returns HH_ERR_TIMEOUT, and the next solve on the same
    handle (hook off) converges to the same iterate as before."""
    import time
    from paper_1211_4752_gb300 import HelmholtzMG
    from paper_1211_4752_gb300 import _binding as B
    n = 64
    kw = dict(k2=1600.0, layers=16, max_batch=1, precision="mixed")
    monkeypatch.setenv("HH_PERSIST", "1")
    mg = HelmholtzMG(n, **kw)
    monkeypatch.delenv("HH_PERSIST")
    assert mg.cycle_kernels == 1          # the cooperative cycle is in use
    src = dev(W.point_sources(n, 2, [(31, 31)]))
    u0, i0 = mg.solve(src, tol=1e-6)
    assert i0[0]["status"] == "OK"
    mg.test_barrier_timeout(True)
    t0 = time.perf_counter()
    with pytest.raises(B.HHError) as ei:
        mg.solve(src, tol=1e-6)
    assert ei.value.status == B.HH_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    mg.test_barrier_timeout(False)
    u1, i1 = mg.solve(src, tol=1e-6)
    assert i1[0]["status"] == "OK" and i1[0]["cycles"] == i0[0]["cycles"]
    assert torch.equal(u0, u1)
    la, il = mg.adjoint(src, tol=1e-6)
    assert il[0]["status"] == "OK"
    mg.close()
    plain = HelmholtzMG(n, **kw)          # no cooperative cycle: the hook is refused
    with pytest.raises(B.HHError) as ei:
        plain.test_barrier_timeout(True)
    assert ei.value.status == B.HH_ERR_UNSUPPORTED
    plain.close()


def test_tuner_cache_gives_identical_handles(tmp_path):
    """hh_options.tuner_cache: the first handle times the tile shapes and
    records them under its key; a second handle built from the same file
    takes them without timing, so the two give bit-identical solutions and
    cycle counts.  A recorded choice is used as written; a malformed file is
    an argument error."""
    import json
    from paper_1211_4752_gb300 import HelmholtzMG
    from paper_1211_4752_gb300 import _binding as B
    n = 256
    path = tmp_path / "tuner.json"
    kw = dict(k2=(0.625 * n) ** 2, layers=8, max_batch=2, precision="mixed", tuner_cache=path)
    a = HelmholtzMG(n, **kw)
    data = json.loads(path.read_text())
    key = a.tuner_key
    assert key in data and key.startswith("v3 dim=2 n=256 prec=mixed")
    sched = a.coarse_schedule
    tuned = 1 + sum(sched)                    # levels 0 .. T-1 carry a tile shape
    assert data[key][tuned] == len(sched)     # then the schedule: groups, (J, b, B) each
    assert data[key][tuned + 1::3] == sched
    levels = [l for l in range(a.levels) if a.tile_shape(l) is not None]
    b = HelmholtzMG(n, **kw)
    assert b.coarse_schedule == sched
    assert [a.tile_shape(l) for l in levels] == [b.tile_shape(l) for l in levels]
    src = np.stack([W.point_sources(n, 2, [(127, 127)])[0], W.point_sources(n, 2, [(90, 160)])[0]])
    ua, ia = a.solve(dev(src), tol=1e-6)
    ub, ib = b.solve(dev(src), tol=1e-6)
    assert all(i["status"] == "OK" for i in ia)
    assert [i["cycles"] for i in ia] == [i["cycles"] for i in ib]
    assert torch.equal(ua, ub)
    a.close()
    b.close()
    data[key] = [4] * tuned + [1, tuned - 1, 4, 16]   # shape 4 is 28 x 16; one group
    path.write_text(json.dumps(data))
    c = HelmholtzMG(n, **kw)
    assert c.coarse_schedule == [tuned - 1]
    assert c.tile_shape(0) == (28, 16)
    c.close()
    path.write_text("{ not json")
    with pytest.raises(B.HHError) as ei:
        HelmholtzMG(n, **kw)
    assert ei.value.status == B.HH_ERR_ARG


def test_torch_caching_allocator_serves_the_workspace(tmp_path):
    """hh_options.dev_alloc / dev_free: with allocator='torch' the whole
    workspace (levels, tail operator, FGMRES vectors) comes from torch's
    caching allocator and goes back to it on close; solutions equal those of
    a handle on the library's own allocations (same tuner cache)."""
    from paper_1211_4752_gb300 import HelmholtzMG
    n = 128
    kw = dict(k2=(0.625 * n) ** 2, layers=4, max_batch=2, precision="mixed",
              tuner_cache=tmp_path / "t.json")
    import gc
    ref = HelmholtzMG(n, **kw)
    src = dev(np.stack([W.point_sources(n, 2, [(63, 63)])[0], W.point_sources(n, 2, [(40, 80)])[0]]))
    gc.collect()          # earlier tests' garbage must not be freed while we count
    gc.disable()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    mg = HelmholtzMG(n, allocator="torch", **kw)
    during = torch.cuda.memory_allocated()
    assert during - before > 6 * (n - 1) * n * 8   # at least the level-0 arrays
    u1, i1 = mg.solve(src, tol=1e-6)
    u0, i0 = ref.solve(src, tol=1e-6)
    assert all(i["status"] == "OK" for i in i1)
    assert torch.equal(u0, u1)
    g1, j1 = mg.fgmres(src, tol=1e-6, restart=8)
    assert all(i["status"] == "OK" for i in j1)
    results = sum(t.numel() * t.element_size() for t in (u0, u1, g1))
    assert torch.cuda.memory_allocated() > during + results   # the Krylov workspace
    mg.close()
    del u0, u1, g1
    torch.cuda.synchronize()
    after = torch.cuda.memory_allocated()
    gc.enable()
    assert after == before
    ref.close()


def test_tiled_3d_cycle_matches_pointwise(monkeypatch):
    """The 3-D cycle's tile-staged kernels and the point-wise ones
    (HH_POINTWISE3D=1) evaluate the same per-point arithmetic: FP64 cycles on
    63^3 with a k^2 field agree to rounding, complex64 to its rounding."""
    from paper_1211_4752_gb300 import HelmholtzMG
    n = 64
    k2 = W.smooth_k2(n, 3, 2, 20.0, 40.0)
    f = rnd((1,) + (n - 1,) * 3, 5)
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("HH_POINTWISE3D", mode)
        for precision in ("fp64", "mixed"):
            mg = HelmholtzMG(n, dim=3, k2=dev(k2), layers=(4, 6), precision=precision, max_batch=1)
            out[mode, precision] = host(mg.cycles(dev(f), dev(np.zeros_like(f)), 2))
            mg.close()
    assert maxrel(out["0", "fp64"], out["1", "fp64"]) < 1e-13
    assert maxrel(out["0", "mixed"], out["1", "mixed"]) < 1e-5
