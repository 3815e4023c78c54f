"""FP64 oracle: level-dependent V(1,1) multigrid for (-Delta - k^2) u = f.

TEST INFRASTRUCTURE (see the package docstring): imported only by the tests,
the smoke check and the benchmark's CPU-baseline leg.

Paper passages followed (Cools, Reps, Vanroose, arXiv 1211.4752):
  * Eq. (HH), Sec. 2: the discrete Helmholtz operator -Delta^h - k^2 on a
    vertex-centred grid with n intervals per dimension; the wavenumber may
    depend on space; coarse operators come from rediscretisation.
  * Eq. (standardtg) and the text after it: two-grid correction with
    full-weighting restriction and (bi/tri-)linear interpolation.
  * Sec. 3.1, Eqs. (cslvariant)/(csgvariant): level m uses the shift
    e^{i theta_{m-1}} on k^2 (CSL form) or the rotation e^{-i theta_{m-1}} on
    the Laplacian (CSG form); theta_m = m*dtheta, dtheta = theta_max/p,
    theta_max = pi/6, and the finest level keeps the original operator.
  * Eq. (erreq1) and the text around it: the restricted residual may be scaled
    by a constant c before the coarse solve (c = e^{-i dtheta} for CSG).
  * Eq. (wjacobi): weighted Jacobi R = I - omega D^{-1} A.
  * Sec. 2.4 and Sec. 4.1: exterior complex scaling (ECS) absorbing layers,
    i.e. a complex-valued grid distance in a border layer.
  * Sec. 4.1: V(1,1)-cycles repeated as a stand-alone solver until a residual
    tolerance is met.

Readings taken where the paper is silent (also listed in the design notes):
  * the hierarchy stops at 3 interior points per dimension (n = 4) and is
    solved there by a dense LU with partial pivoting;
  * the ECS layer lies inside the unit interval, is rotated by the angle gamma
    (default pi/6) and keeps its physical position on coarse levels;
  * coarse k^2 is the injection of the fine k^2;
  * the stopping test is ||f - A_0 u||_2 / ||f||_2 <= tol from u_0 = 0.

Array layout: interior points only (the homogeneous Dirichlet boundary is
implicit), axis order (z, y, x) / (y, x) / (x,), complex128.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Level", "Hierarchy", "ecs_coordinate", "level_spacings", "laplacian_1d",
    "apply_operator", "operator_diagonal", "jacobi", "gmres_smooth", "smooth",
    "restrict_fw", "prolong",
    "dense_matrix", "lu_factor", "lu_solve", "build_hierarchy",
    "adjoint_hierarchy", "vcycle", "solve", "residual_norm",
    "symmetrizer_weights", "adjoint_solve_symmetrized", "grad_k2", "fgmres",
    "SolveResult", "DivergedError", "NotConvergedError",
]


class DivergedError(RuntimeError):
    pass


class NotConvergedError(RuntimeError):
    pass


# --------------------------------------------------------------------------
# Grid: exterior complex scaling (Sec. 2.4, Sec. 4.1)
# --------------------------------------------------------------------------

def ecs_coordinate(x, a, b, gamma):
    """Complex coordinate z(x) on [0, 1]: z = x on the physical interval [a, b],
    rotated by e^{i gamma} about the nearer end point outside it (exterior
    complex scaling, Sec. 2.4; layer of the paper's constant-k model, Sec. 4.1).
    With a = 0, b = 1 (no layer) the grid is the real uniform grid."""
    x = np.asarray(x, dtype=np.float64)
    rot = np.exp(1j * gamma)
    z = x.astype(np.complex128)
    lo = x < a
    hi = x > b
    z[lo] = a + (x[lo] - a) * rot
    z[hi] = b + (x[hi] - b) * rot
    return z


def level_spacings(n_l, a, b, gamma):
    """The n_l complex grid distances h_i = z(x_{i+1}) - z(x_i), x_i = i/n_l, of a
    level with n_l intervals on the unit interval."""
    x = np.arange(n_l + 1, dtype=np.float64) / n_l
    return np.diff(ecs_coordinate(x, a, b, gamma))


def laplacian_1d(h, sommerfeld_k=None, ends=(True, True)):
    """Three-point second difference on a (complex, non-uniform) grid, as the
    coefficients of -D2 at the n-1 interior nodes:

        (-D2 u)_i = -lo_i u_{i-1} + dg_i u_i - up_i u_{i+1},
        lo_i = 2/((h_{i-1}+h_i) h_{i-1}),  up_i = 2/((h_{i-1}+h_i) h_i),
        dg_i = lo_i + up_i = 2/(h_{i-1} h_i).

    On the uniform real grid this is (-u_{i-1} + 2u_i - u_{i+1})/h^2, the
    Laplacian of Eq. (HH).  The end nodes are u = 0 (Dirichlet), or, with
    sommerfeld_k = k, at the ends selected by `ends` (low, high), carry the
    radiating condition du/dn = i k u of Table 4's model, discretised to
    second order by the one-sided difference on the two end cells (uniform
    spacing h there): (3 u_b - 4 u_{b-1} + u_{b-2}) / (2 h) = i k u_b, and
    eliminated, u_b = (4 u_{b-1} - u_{b-2}) / (3 - 2 i k h).  The row next
    to the end then couples to its two inner neighbours only: at the high
    end dg -= 4 up / (3 - 2ikh) and lo -= up / (3 - 2ikh); mirrored at the
    low end."""
    hm = h[:-1]
    hp = h[1:]
    lo = 2.0 / ((hm + hp) * hm)
    up = 2.0 / ((hm + hp) * hp)
    dg = lo + up
    if sommerfeld_k is not None:
        lo, dg, up = (x.astype(np.complex128) for x in (lo, dg, up))
        if ends[0]:
            d = 3.0 - 2j * sommerfeld_k * h[0]
            dg[0] -= 4.0 * lo[0] / d
            up[0] -= lo[0] / d
        if ends[1]:
            d = 3.0 - 2j * sommerfeld_k * h[-1]
            dg[-1] -= 4.0 * up[-1] / d
            lo[-1] -= up[-1] / d
    return lo, dg, up


# --------------------------------------------------------------------------
# Level operators (Eq. (HH); Sec. 3.1 Eqs. (cslvariant)/(csgvariant))
# --------------------------------------------------------------------------

@dataclass
class Level:
    """One level: A u = alpha * sum_axes(-lo u_- + dg u - up u_+) - beta k2 u.

    CSL form (Eq. (cslvariant)): alpha = 1, beta = e^{i theta}.
    CSG form (Eq. (csgvariant)): alpha = e^{-i theta}, beta = 1.
    lo/dg/up hold one 1-D coefficient array per axis (array axis order)."""
    n: int
    dim: int
    lo: list
    dg: list
    up: list
    alpha: complex
    beta: complex
    k2: np.ndarray

    @property
    def shape(self):
        return (self.n - 1,) * self.dim


@dataclass
class Hierarchy:
    levels: list
    c: list               # scale of the restricted residual, level l -> l+1
    omega: complex = 0.8  # Jacobi weight, Eq. (wjacobi)
    nu1: int = 1
    nu2: int = 1
    lu: tuple = None      # (factors, pivots) of the coarsest operator
    smoother: str = "jacobi"   # or "gmres": GMRES(m) smoothing (Sec. 3.2)
    m: int = 3                 # GMRES degree
    info: dict = field(default_factory=dict)


def _along(vec, ax, dim):
    shape = [1] * dim
    shape[ax] = vec.shape[0]
    return vec.reshape(shape)


def _shift(u, ax, s):
    """u at index i+s along axis ax, zero outside (homogeneous Dirichlet)."""
    out = np.zeros_like(u)
    n = u.shape[ax]
    src = [slice(None)] * u.ndim
    dst = [slice(None)] * u.ndim
    if s < 0:
        src[ax] = slice(0, n + s)
        dst[ax] = slice(-s, n)
    else:
        src[ax] = slice(s, n)
        dst[ax] = slice(0, n - s)
    out[tuple(dst)] = u[tuple(src)]
    return out


def apply_operator(lv: Level, u):
    """A_l u on interior points, zero Dirichlet values outside (Eq. (HH) with
    the level shift of Eq. (cslvariant) or (csgvariant))."""
    lap = np.zeros_like(u)
    for ax in range(lv.dim):
        lo = _along(lv.lo[ax], ax, lv.dim)
        dg = _along(lv.dg[ax], ax, lv.dim)
        up = _along(lv.up[ax], ax, lv.dim)
        lap += -lo * _shift(u, ax, -1) + dg * u - up * _shift(u, ax, +1)
    return lv.alpha * lap - lv.beta * lv.k2 * u


def operator_diagonal(lv: Level):
    """Pointwise diagonal D of A_l (used by Eq. (wjacobi))."""
    d = np.zeros(lv.shape, dtype=np.complex128)
    for ax in range(lv.dim):
        d = d + _along(lv.dg[ax], ax, lv.dim)
    return lv.alpha * d - lv.beta * lv.k2


def jacobi(lv: Level, u, f, omega):
    """One weighted-Jacobi sweep u <- u + omega D^{-1}(f - A u), Eq. (wjacobi);
    every point uses the old iterate."""
    return u + omega * (f - apply_operator(lv, u)) / operator_diagonal(lv)


def gmres_smooth(lv: Level, u, f, m=3):
    """One GMRES(m) smoothing step (Sec. 3.2, the smoother the paper uses):
    u + z, where z minimises ||f - A (u + z)||_2 over the Krylov space
    K_m(A, r0) = span{r0, A r0, ..., A^{m-1} r0}, r0 = f - A u.  Arnoldi with
    modified Gram-Schmidt builds an orthonormal basis V and the (m+1) x m
    Hessenberg matrix H with A V_m = V_{m+1} H; y minimises ||beta e1 - H y||
    (a small least-squares solve) and z = V_m y.  If the space has dimension
    j < m (A V_j lies in span V_j), the exact minimiser on it is taken."""
    r0 = f - apply_operator(lv, u)
    beta = np.linalg.norm(r0)
    if beta == 0.0:
        return u
    V = [r0 / beta]
    H = np.zeros((m + 1, m), dtype=np.complex128)
    k = m
    for j in range(m):
        w = apply_operator(lv, V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0.0:
            k = j + 1
            break
        V.append(w / H[j + 1, j])
    e1 = np.zeros(k + 1, dtype=np.complex128)
    e1[0] = beta
    y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
    z = sum(y[j] * V[j] for j in range(k))
    return u + z


def smooth(hier, lv: Level, u, f):
    """One smoothing step with the hierarchy's smoother."""
    if hier.smoother == "gmres":
        return gmres_smooth(lv, u, f, hier.m)
    return jacobi(lv, u, f, hier.omega)


# --------------------------------------------------------------------------
# Intergrid transfers (text after Eq. (standardtg))
# --------------------------------------------------------------------------

def restrict_fw(r):
    """Full weighting: the tensor product of the 1-D stencil [1 2 1]/4 centred
    on the fine point that coincides with each coarse point (coarse interior
    index c <-> fine interior index 2c+1, zero Dirichlet values)."""
    out = r
    for ax in range(r.ndim):
        n = out.shape[ax]
        nc = (n + 1) // 2 - 1
        sl = lambda start: tuple(  # noqa: E731
            slice(start, start + 2 * nc - 1, 2) if a == ax else slice(None)
            for a in range(out.ndim))
        out = 0.25 * out[sl(0)] + 0.5 * out[sl(1)] + 0.25 * out[sl(2)]
    return out


def prolong(e):
    """(Bi/tri-)linear interpolation: the tensor product of 1-D linear
    interpolation from coarse to fine with zero coarse boundary values;
    coincident fine points copy, in-between points average their two coarse
    neighbours along each axis."""
    out = e
    for ax in range(e.ndim):
        nc = out.shape[ax]
        pad = [(0, 0)] * out.ndim
        pad[ax] = (1, 1)
        ep = np.pad(out, pad)                 # coarse 1-based 0..nc+1
        shape = list(out.shape)
        shape[ax] = 2 * nc + 1
        fine = np.zeros(shape, dtype=out.dtype)
        odd = [slice(None)] * out.ndim
        even = [slice(None)] * out.ndim
        odd[ax] = slice(1, None, 2)           # fine 0-based odd = coincident
        even[ax] = slice(0, None, 2)
        lo = [slice(None)] * out.ndim
        hi = [slice(None)] * out.ndim
        mid = [slice(None)] * out.ndim
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        mid[ax] = slice(1, -1)
        fine[tuple(odd)] = ep[tuple(mid)]
        fine[tuple(even)] = 0.5 * (ep[tuple(lo)] + ep[tuple(hi)])
        out = fine
    return out


# --------------------------------------------------------------------------
# Coarsest level: dense LU with partial pivoting
# --------------------------------------------------------------------------

def dense_matrix(lv: Level):
    """A_l as a dense matrix, column j = A_l applied to the j-th unit vector
    (row-major flattening of the interior points)."""
    m = int(np.prod(lv.shape))
    M = np.zeros((m, m), dtype=np.complex128)
    for j in range(m):
        e = np.zeros(m, dtype=np.complex128)
        e[j] = 1.0
        M[:, j] = apply_operator(lv, e.reshape(lv.shape)).ravel()
    return M


def lu_factor(M):
    """Doolittle LU with row interchanges: at step k the pivot is the row of
    largest modulus in column k (the first such row on ties)."""
    A = np.array(M, dtype=np.complex128, copy=True)
    n = A.shape[0]
    piv = np.arange(n)
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if p != k:
            A[[k, p]] = A[[p, k]]
            piv[[k, p]] = piv[[p, k]]
        if A[k, k] == 0:
            raise ZeroDivisionError("singular coarsest operator")
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, piv


def lu_solve(lu, b):
    """Solve with the factors of lu_factor: permute, forward, back."""
    A, piv = lu
    y = np.array(b, dtype=np.complex128)[piv]
    n = A.shape[0]
    for i in range(n):
        y[i] -= A[i, :i] @ y[:i]
    for i in range(n - 1, -1, -1):
        y[i] = (y[i] - A[i, i + 1:] @ y[i + 1:]) / A[i, i]
    return y


# --------------------------------------------------------------------------
# Hierarchy (Sec. 3.1)
# --------------------------------------------------------------------------

def build_hierarchy(n, dim, k2, layers=0, gamma=math.pi / 6,
                    theta_max=math.pi / 6, p=None, form="csl", c=None,
                    omega=0.8, nu1=1, nu2=1, coarsest=4, thetas=None,
                    smoother="jacobi", m=3, sommerfeld=False):
    """Level-dependent hierarchy for (-Delta - k^2) u = f on the unit square
    (cube) with n = 2^P intervals per dimension.

    n_l = n / 2^l intervals on level l (l = 0 finest), down to `coarsest`
    intervals.  theta_l = l * dtheta with dtheta = theta_max / p, p = log2(n)
    by default (Sec. 3.1; the tables of Sec. 4.1 use dtheta = (pi/6)/log2 n).
    form 'csl': alpha_l = 1, beta_l = e^{i theta_l}  (Eq. (cslvariant));
    form 'csg': alpha_l = e^{-i theta_l}, beta_l = 1 (Eq. (csgvariant)).
    c[l] scales the residual restricted from level l to l+1 (Eq. (erreq1));
    default 1.  `layers` is the ECS layer width in fine-grid points, one
    number for every side or a (lo, hi) pair; gamma is the ECS angle.
    k2 is the real fine-grid k^2 field (array of the interior shape) or a
    constant; coarse levels inject it.  sommerfeld=True replaces the
    Dirichlet condition at every end without an ECS layer by the radiating
    condition of Table 4 (laplacian_1d; constant k only), on every level with
    that level's spacing and the unshifted k."""
    P = int(round(math.log2(n)))
    if 2 ** P != n:
        raise ValueError("n must be a power of two")
    if p is None:
        p = P
    dtheta = theta_max / p
    if np.isscalar(layers):
        layers = (layers, layers)
    a = layers[0] / n
    b = 1.0 - layers[1] / n
    k2 = np.asarray(k2, dtype=np.float64)
    ksom = None
    if sommerfeld:
        if k2.ndim != 0:
            raise ValueError("the radiating condition needs a constant k")
        ksom = math.sqrt(float(k2))
    if k2.ndim == 0:
        k2 = np.full((n - 1,) * dim, float(k2))
    levels = []
    n_l = n
    l = 0
    k2_l = k2
    while True:
        h = level_spacings(n_l, a, b, gamma)
        lo, dg, up = laplacian_1d(h, ksom, (layers[0] == 0, layers[1] == 0))
        theta = thetas[l] if thetas is not None else l * dtheta
        if form == "csl":
            alpha, beta = 1.0 + 0j, np.exp(1j * theta)
        elif form == "csg":
            alpha, beta = np.exp(-1j * theta), 1.0 + 0j
        else:
            raise ValueError(form)
        levels.append(Level(n_l, dim, [lo] * dim, [dg] * dim, [up] * dim,
                            complex(alpha), complex(beta), k2_l))
        if n_l <= coarsest:
            break
        n_l //= 2
        l += 1
        inj = tuple(slice(1, None, 2) for _ in range(dim))
        k2_l = k2_l[inj]
    if c is None:
        c = [1.0 + 0j] * (len(levels) - 1)
    if smoother not in ("jacobi", "gmres"):
        raise ValueError(smoother)
    hier = Hierarchy(levels, list(c), omega, nu1, nu2, smoother=smoother, m=m)
    hier.lu = lu_factor(dense_matrix(levels[-1]))
    hier.info = dict(dtheta=dtheta, p=p, a=a, b=b, gamma=gamma, form=form,
                     sommerfeld=bool(sommerfeld))
    return hier


def adjoint_hierarchy(hier: Hierarchy):
    """The conjugate-transposed hierarchy: level operators A_l^H (per axis the
    tridiagonal matrix is transposed and conjugated), conj(beta), conj(alpha),
    conj(c), same transfers and Jacobi weight conj(omega).  The V-cycle on it
    solves A_0^H lambda = g."""
    levels = []
    for lv in hier.levels:
        lo, dg, up = [], [], []
        for ax in range(lv.dim):
            lo_a = np.zeros_like(lv.lo[ax])
            up_a = np.zeros_like(lv.up[ax])
            lo_a[1:] = np.conj(lv.up[ax][:-1])   # (M^H)_{i,i-1} = conj(M_{i-1,i})
            up_a[:-1] = np.conj(lv.lo[ax][1:])   # (M^H)_{i,i+1} = conj(M_{i+1,i})
            lo.append(lo_a)
            up.append(up_a)
            dg.append(np.conj(lv.dg[ax]))
        levels.append(Level(lv.n, lv.dim, lo, dg, up, np.conj(lv.alpha),
                            np.conj(lv.beta), lv.k2))
    adj = Hierarchy(levels, [np.conj(x) for x in hier.c], np.conj(hier.omega),
                    hier.nu1, hier.nu2, smoother=hier.smoother, m=hier.m)
    adj.lu = lu_factor(dense_matrix(levels[-1]))
    adj.info = dict(hier.info, adjoint=True)
    return adj


# --------------------------------------------------------------------------
# Cycle and solver (Sec. 3.1, Sec. 4.1)
# --------------------------------------------------------------------------

def vcycle(hier: Hierarchy, l, u, f):
    """One level-dependent V(nu1,nu2)-cycle on level l: pre-smooth, residual,
    scaled full-weighting restriction, coarse solve (recursive, zero initial
    guess; LU on the coarsest level), interpolated correction, post-smooth."""
    lv = hier.levels[l]
    for _ in range(hier.nu1):
        u = smooth(hier, lv, u, f)
    r = f - apply_operator(lv, u)
    fc = hier.c[l] * restrict_fw(r)
    if l + 1 == len(hier.levels) - 1:
        ec = lu_solve(hier.lu, fc.ravel()).reshape(fc.shape)
    else:
        ec = vcycle(hier, l + 1, np.zeros_like(fc), fc)
    u = u + prolong(ec)
    for _ in range(hier.nu2):
        u = smooth(hier, lv, u, f)
    return u


def residual_norm(hier: Hierarchy, u, f):
    """||f - A_0 u||_2 over the interior points."""
    return float(np.linalg.norm((f - apply_operator(hier.levels[0], u)).ravel()))


@dataclass
class SolveResult:
    u: np.ndarray
    cycles: int
    history: list


def solve(hier: Hierarchy, f, tol=1e-6, max_cycles=20000, u0=None,
          div_limit=1e3):
    """Repeat V-cycles from u_0 = 0 (or u0) until
    rho_k = ||f - A_0 u_k||_2 / ||f||_2 <= tol (Sec. 4.1 uses V(1,1)-cycles as
    a stand-alone solver).  Raises DivergedError when rho_k > div_limit or is
    not finite, NotConvergedError after max_cycles."""
    f = np.asarray(f, dtype=np.complex128)
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.complex128)
    nf = float(np.linalg.norm(f.ravel()))
    if nf == 0.0:
        return SolveResult(np.zeros_like(f), 0, [])
    hist = []
    for k in range(1, max_cycles + 1):
        u = vcycle(hier, 0, u, f)
        rho = residual_norm(hier, u, f) / nf
        hist.append(rho)
        if not np.isfinite(rho) or rho > div_limit:
            raise DivergedError(f"diverged at cycle {k}: rho={rho}")
        if rho <= tol:
            return SolveResult(u, k, hist)
    raise NotConvergedError(f"no convergence in {max_cycles} cycles: rho={hist[-1]}")


# --------------------------------------------------------------------------
# Adjoint and gradient
# --------------------------------------------------------------------------

def fgmres(hier: Hierarchy, f, tol=1e-6, m=10, max_iter=2000, u0=None, precond=None,
           strict=True):
    """Right-preconditioned flexible GMRES(m) (Saad 1993) for A_0 u = f, the
    preconditioner being one level-dependent V-cycle from a zero initial
    guess on the residual equation (the use of the cycle in Table 3 of the
    paper; flexible because a GMRES-smoothed cycle is not a fixed linear
    map).  Modified Gram-Schmidt Arnoldi; stops when the least-squares
    residual estimate falls to tol * ||f||.  Returns a SolveResult whose
    `cycles` counts the preconditioner applications (= iterations).
    `precond(v)` replaces the V-cycle (for the pins); with strict=False the
    iterate reached after max_iter iterations is returned instead of raising."""
    if precond is None:
        precond = lambda v: vcycle(hier, 0, np.zeros_like(v), v)
    lv = hier.levels[0]
    nf = np.linalg.norm(f)
    u = np.zeros_like(f) if u0 is None else u0.copy()
    hist = []
    it = 0
    while True:
        r = f - apply_operator(lv, u)
        beta = np.linalg.norm(r)
        hist.append(beta / nf)
        if beta <= tol * nf:
            return SolveResult(u, it, hist)
        if it >= max_iter:
            if not strict:
                return SolveResult(u, it, hist)
            raise NotConvergedError(f"no convergence in {it} iterations")
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        e1 = np.zeros(m + 1, dtype=np.complex128)
        e1[0] = beta
        k = 0
        for j in range(m):
            Z.append(precond(V[j]))
            w = apply_operator(lv, Z[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            it += 1
            k = j + 1
            y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1[:k + 1], rcond=None)
            est = np.linalg.norm(e1[:k + 1] - H[:k + 1, :k] @ y)
            if H[j + 1, j] == 0.0 or est <= tol * nf or it >= max_iter:
                break
            V.append(w / H[j + 1, j])
        y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1[:k + 1], rcond=None)
        u = u + sum(y[i] * Z[i] for i in range(k))
        if est <= tol * nf:
            r = f - apply_operator(lv, u)
            hist.append(np.linalg.norm(r) / nf)
            return SolveResult(u, it, hist)


def symmetrizer_weights(hier: Hierarchy):
    """W = prod over axes of (h_{i-1} + h_i)/2 on the finest level.  W A_0 is
    complex symmetric for the three-point formula of laplacian_1d, so
    A_0^T = W A_0 W^{-1}."""
    info = hier.info
    lv = hier.levels[0]
    h = level_spacings(lv.n, info["a"], info["b"], info["gamma"])
    w1 = 0.5 * (h[:-1] + h[1:])
    W = np.ones(lv.shape, dtype=np.complex128)
    for ax in range(lv.dim):
        W = W * _along(w1, ax, lv.dim)
    return W


def adjoint_solve_symmetrized(hier: Hierarchy, g, tol=1e-6, max_cycles=20000):
    """A_0^H lambda = g through the forward solver:
    lambda = conj(W y) with A_0 y = W^{-1} conj(g).  (W A_0 is complex
    symmetric for Dirichlet and ECS ends; the eliminated radiating condition
    couples the end row to a second neighbour, which breaks that symmetry.)"""
    if hier.info.get("sommerfeld"):
        raise ValueError("the symmetrizer route needs Dirichlet or ECS ends")
    W = symmetrizer_weights(hier)
    res = solve(hier, np.conj(g) / W, tol=tol, max_cycles=max_cycles)
    return np.conj(W * res.u), res


def grad_k2(u, lam):
    """d loss / d k^2 = sum over right-hand sides of Re(conj(lambda) * u), from
    A_0 = L - diag(k^2) and lambda = A_0^{-H} (d loss / d u); u and lam carry
    the right-hand sides along axis 0 when 3-D (2-D grids) / 4-D."""
    return np.sum(np.real(np.conj(lam) * u), axis=0)
