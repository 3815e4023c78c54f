"""Python face of the C ABI: a handle class and a torch.autograd.Function.

Only argument marshalling happens here (tensor checks, pointers, the current
torch stream); every step of the method runs in the CUDA library.  Arrays are
torch tensors on the handle's CUDA device: complex128 [batch, N, N] (2-D) or
[batch, N, N, N] (3-D) with N = n - 1 interior points per axis, x fastest.
"""

from __future__ import annotations

import ctypes as ct
import math

import torch

from . import _binding as B


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ct.c_void_p(t.data_ptr())


class HelmholtzMG:
    """Level-dependent multigrid hierarchy for (-Delta - k^2) u = f.

    n: intervals per axis (power of two); dim: 2 or 3; k2: fine k^2 field
    (real tensor of the interior shape, any device) or a float; layers: ECS
    layer width in fine cells, one int or (lo, hi); form: 'csl' | 'csg';
    thetas / c: optional per-level angles / per-transfer residual scales;
    precision: 'fp64' | 'mixed'; sommerfeld: the radiating condition of
    Table 4 at the ends without an ECS layer (constant k only);
    tuner_cache: path of the autotuner's cache file (hh_options.tuner_cache);
    allocator: None (the library's cudaMalloc) or 'torch' (the handle's
    workspace comes from torch's caching allocator on the handle's device)."""

    def __init__(self, n, dim=2, k2=0.0, layers=0, ecs_angle=math.pi / 6,
                 form="csl", theta_max=math.pi / 6, p=0, thetas=None, c=None,
                 omega=0.8, nu1=1, nu2=1, precision="fp64", coarsest=4,
                 max_cycles=20000, div_limit=1e3, inner_tol=1e-3,
                 max_inner=20000, max_batch=1, device=None, smoother="jacobi",
                 gmres_m=3, sommerfeld=False, tuner_cache=None, allocator=None):
        L = B.lib()
        self.n, self.dim, self.N = int(n), int(dim), int(n) - 1
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.shape = (self.N,) * self.dim
        self.max_batch = int(max_batch)
        self.precision = precision
        lo, hi = (layers, layers) if isinstance(layers, int) else tuple(layers)
        g = B.HHGrid(self.dim, self.n, int(lo), int(hi), float(ecs_angle), int(bool(sommerfeld)))
        sh = B.HHShift()
        L.hh_default_shift(ct.byref(sh))
        sh.form = B.HH_FORM_CSL if form == "csl" else B.HH_FORM_CSG
        sh.theta_max = float(theta_max)
        sh.p = int(p)
        self._keep = []
        if thetas is not None:
            arr = (ct.c_double * len(thetas))(*[float(t) for t in thetas])
            self._keep.append(arr)
            sh.theta = ct.cast(arr, ct.POINTER(ct.c_double))
        if c is not None:
            flat = []
            for z in c:
                z = complex(z)
                flat += [z.real, z.imag]
            arr = (ct.c_double * len(flat))(*flat)
            self._keep.append(arr)
            sh.c = ct.cast(arr, ct.POINTER(ct.c_double))
        o = B.HHOptions()
        L.hh_default_options(ct.byref(o))
        w = complex(omega)
        o.omega_re, o.omega_im = w.real, w.imag
        o.nu1, o.nu2 = int(nu1), int(nu2)
        o.precision = B.HH_FP64 if precision == "fp64" else B.HH_MIXED
        o.coarsest = int(coarsest)
        o.max_cycles = int(max_cycles)
        o.div_limit = float(div_limit)
        o.inner_tol = float(inner_tol)
        o.max_inner = int(max_inner)
        if smoother not in ("jacobi", "gmres"):
            raise ValueError("smoother must be 'jacobi' or 'gmres'")
        o.smoother = B.HH_SMOOTH_GMRES if smoother == "gmres" else B.HH_SMOOTH_JACOBI
        o.gmres_m = int(gmres_m)
        if tuner_cache is not None:
            self._tuner_path = str(tuner_cache).encode()
            o.tuner_cache = self._tuner_path
        self._alloc_cbs = None
        if allocator == "torch":
            dev_index = self.device.index if self.device.index is not None else torch.cuda.current_device()

            def _alloc(nbytes, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev_index)
                except RuntimeError:
                    return None

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cbs = (B.DEV_ALLOC(_alloc), B.DEV_FREE(_free))
            o.dev_alloc = ct.cast(self._alloc_cbs[0], ct.c_void_p)
            o.dev_free = ct.cast(self._alloc_cbs[1], ct.c_void_p)
        elif allocator is not None:
            raise ValueError("allocator must be None or 'torch'")
        self.k2_const = 0.0
        k2_ptr = ct.c_void_p(0)
        if isinstance(k2, torch.Tensor):
            k2t = k2.detach().to(device=self.device, dtype=torch.float64).contiguous()
            if tuple(k2t.shape) != self.shape:
                raise ValueError(f"k2 must have shape {self.shape}")
            k2_ptr = _ptr(k2t)
        else:
            self.k2_const = float(k2)
        h = ct.c_void_p()
        with torch.cuda.device(self.device):
            B.check(L.hh_setup(ct.byref(g), k2_ptr, self.k2_const, ct.byref(sh),
                               ct.byref(o), self.max_batch, _stream(), ct.byref(h)))
        self._h = h
        self.levels = L.hh_num_levels(h)

    # ---- helpers ---------------------------------------------------------
    def _vec(self, x, name, level=0):
        N = self.level_points(level)
        shape = (N,) * self.dim
        if not isinstance(x, torch.Tensor) or x.dtype != torch.complex128 or x.device != self.device:
            raise TypeError(f"{name} must be a complex128 tensor on {self.device}")
        if tuple(x.shape[-self.dim:]) != shape or x.dim() != self.dim + 1:
            raise ValueError(f"{name} must have shape [batch, {', '.join(map(str, shape))}]")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return x

    def level_points(self, level):
        return B.lib().hh_level_points(self._h, int(level))

    @property
    def cycle_kernels(self):
        """Kernels one V-cycle launches (stop test included)."""
        return B.lib().hh_cycle_kernels(self._h)

    @property
    def solve_kernels(self):
        """Kernels launched by the last completed solve (-1 before one)."""
        return B.lib().hh_solve_kernels(self._h)

    @property
    def coarse_schedule(self):
        """Group sizes of the fused coarse passes (levels 1 .. T-1), [] if none."""
        n = B.lib().hh_coarse_schedule(self._h, None, 0)
        arr = (ct.c_int * max(n, 1))()
        B.lib().hh_coarse_schedule(self._h, arr, n)
        return [arr[i] for i in range(max(n, 0))]

    @property
    def tuner_key(self):
        """The autotuner's key of this handle (hh_tuner_key)."""
        n = B.lib().hh_tuner_key(self._h, None, 0)
        buf = ct.create_string_buffer(n + 1)
        B.lib().hh_tuner_key(self._h, buf, n + 1)
        return buf.value.decode()

    def tile_shape(self, level):
        """(bx, by) of the fused 2-D kernels on `level`, or None."""
        bx, by = ct.c_int(), ct.c_int()
        ok = B.lib().hh_tile_shape(self._h, int(level), ct.byref(bx), ct.byref(by))
        return (bx.value, by.value) if ok else None

    def close(self):
        if getattr(self, "_h", None):
            B.lib().hh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _infos(arr, n):
        return [dict(cycles=arr[i].cycles, refinements=arr[i].refinements,
                     rel_residual=arr[i].rel_residual,
                     status=B.STATUS_NAMES.get(arr[i].status, arr[i].status))
                for i in range(n)]

    # ---- solves ----------------------------------------------------------
    def _solve(self, fn, f, tol, u0, raise_on_fail):
        f = self._vec(f, "rhs")
        nb = f.shape[0]
        u = torch.empty_like(f) if u0 is None else self._vec(u0, "u0").clone()
        info = (B.HHSolveInfo * nb)()
        with torch.cuda.device(self.device):
            st = fn(self._h, _ptr(f), _ptr(u), nb, float(tol),
                    B.HH_USE_GUESS if u0 is not None else 0, info, _stream())
        if st not in (B.HH_OK, B.HH_ERR_NOT_CONVERGED, B.HH_ERR_DIVERGED) or (raise_on_fail and st != B.HH_OK):
            B.check(st)
        return u, self._infos(info, nb)

    def solve(self, f, tol=1e-6, u0=None, raise_on_fail=False):
        """u = A_0^{-1} f by V-cycles to ||f - A_0 u|| / ||f|| <= tol."""
        return self._solve(B.lib().hh_solve, f, tol, u0, raise_on_fail)

    def adjoint(self, g, tol=1e-6, lam0=None, raise_on_fail=False):
        """lambda = A_0^{-H} g by V-cycles on the conjugate-transposed hierarchy."""
        return self._solve(B.lib().hh_adjoint, g, tol, lam0, raise_on_fail)

    def fgmres(self, f, tol=1e-6, restart=10, max_iter=0, u0=None, raise_on_fail=False):
        """u = A_0^{-1} f by flexible GMRES(restart) with one V-cycle of this
        handle as the preconditioner per iteration (Table 3's LVL-MG-FGMRES).
        info: cycles = iterations, refinements = restarts."""
        def fn(h, fp, up, nb, t, flags, info, s):
            return B.lib().hh_fgmres(h, fp, up, nb, t, int(restart), int(max_iter), flags, info, s)
        return self._solve(fn, f, tol, u0, raise_on_fail)

    def solve_host(self, f_host, u_host, tol=1e-6, use_guess=False):
        """Solve with HOST (ideally pinned) complex128 tensors; the copies
        are part of the call.  u_host is overwritten with the solution."""
        for t, nm in ((f_host, "f_host"), (u_host, "u_host")):
            if t.device.type != "cpu" or t.dtype != torch.complex128 or not t.is_contiguous():
                raise TypeError(f"{nm} must be a contiguous complex128 CPU tensor")
        nb = f_host.shape[0]
        info = (B.HHSolveInfo * nb)()
        with torch.cuda.device(self.device):
            st = B.lib().hh_solve_host(self._h, _ptr(f_host), _ptr(u_host), nb,
                                       float(tol), B.HH_USE_GUESS if use_guess else 0,
                                       info, _stream())
        if st not in (B.HH_OK, B.HH_ERR_NOT_CONVERGED, B.HH_ERR_DIVERGED):
            B.check(st)
        return self._infos(info, nb)

    def grad_k2(self, u, lam):
        u = self._vec(u, "u")
        lam = self._vec(lam, "lam")
        g = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_grad_k2(self._h, _ptr(u), _ptr(lam), u.shape[0], _ptr(g), _stream()))
        return g

    def test_barrier_timeout(self, on):
        """Test hook of the bounded device waits (handles set up with
        HH_PERSIST=1 only): while on, solves return HH_ERR_TIMEOUT after
        about a second instead of converging; off restores normal solves."""
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_test_barrier_timeout(self._h, int(bool(on))))

    # ---- step API (complex128, FP64 tables) ------------------------------
    def rel_residual_static(self, u, f):
        """||f_b - A_0 u_b|| / ||f_b|| per right-hand side (FP64, on the device),
        computed with the library's fixed scratch array: no allocation by the
        library (the returned tensor is allocated here, by torch).  At most 64
        right-hand sides; calls that overlap in time on one device race."""
        u = self._vec(u, "u")
        f = self._vec(f, "f")
        rho = torch.empty(u.shape[0], dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_rel_residual_static(self._h, _ptr(u), _ptr(f), u.shape[0],
                                                   _ptr(rho), _stream()))
        return rho

    def apply(self, x, level=0, adjoint=False):
        x = self._vec(x, "x", level)
        y = torch.empty_like(x)
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_apply(self._h, int(level), int(bool(adjoint)), _ptr(x), _ptr(y), x.shape[0], _stream()))
        return y

    def cycles(self, f, u, ncycles):
        f = self._vec(f, "f")
        u = self._vec(u, "u").clone()
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_cycles(self._h, _ptr(f), _ptr(u), f.shape[0], int(ncycles), _stream()))
        return u

    def smooth(self, level, u, f):
        u = self._vec(u, "u", level)
        f = self._vec(f, "f", level)
        out = torch.empty_like(u)
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_smooth(self._h, int(level), _ptr(u), _ptr(f), _ptr(out), u.shape[0], _stream()))
        return out

    def residual_restrict(self, level, u, f):
        u = self._vec(u, "u", level)
        f = self._vec(f, "f", level)
        Nc = self.level_points(level + 1)
        fc = torch.empty((u.shape[0],) + (Nc,) * self.dim, dtype=torch.complex128, device=self.device)
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_residual_restrict(self._h, int(level), _ptr(u), _ptr(f), _ptr(fc), u.shape[0], _stream()))
        return fc

    def correct_smooth(self, level, u, e, f):
        u = self._vec(u, "u", level)
        e = self._vec(e, "e", level + 1)
        f = self._vec(f, "f", level)
        out = torch.empty_like(u)
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_correct_smooth(self._h, int(level), _ptr(u), _ptr(e), _ptr(f), _ptr(out), u.shape[0], _stream()))
        return out

    def coarse_solve(self, f):
        f = self._vec(f, "f", self.levels - 1)
        e = torch.empty_like(f)
        with torch.cuda.device(self.device):
            B.check(B.lib().hh_coarse_solve(self._h, _ptr(f), _ptr(e), f.shape[0], _stream()))
        return e


class HelmholtzSolve(torch.autograd.Function):
    """u = A_0(k2)^{-1} f with A_0 = -Delta - diag(k2) (finest operator).

    Backward (adjoint method): lambda = A_0^{-H} grad_u by the adjoint
    V-cycle, grad_f = lambda, grad_k2 = sum_b Re(conj(lambda_b) u_b).
    `mg_kwargs` are HelmholtzMG keyword arguments (n, dim, layers, ...)."""

    @staticmethod
    def forward(ctx, k2, f, mg_kwargs, tol=1e-6):
        kw = dict(mg_kwargs)
        kw.setdefault("max_batch", f.shape[0])
        mg = HelmholtzMG(k2=k2.detach(), device=f.device, **kw)
        u, info = mg.solve(f.detach().contiguous(), tol=tol, raise_on_fail=True)
        ctx.mg = mg
        ctx.tol = tol
        ctx.save_for_backward(u)
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        mg = ctx.mg
        lam, _ = mg.adjoint(grad_u.contiguous(), tol=ctx.tol, raise_on_fail=True)
        gk2 = mg.grad_k2(u, lam) if ctx.needs_input_grad[0] else None
        gf = lam if ctx.needs_input_grad[1] else None
        ctx.mg = None
        mg.close()
        return gk2, gf, None, None


def helmholtz_solve(k2, f, tol=1e-6, **mg_kwargs):
    """Differentiable solve: u = A_0(k2)^{-1} f (see HelmholtzSolve)."""
    return HelmholtzSolve.apply(k2, f, mg_kwargs, tol)


def solve_group(problems, tol=1e-6):
    """Solve independent problems of possibly different grid sizes in one call
    (hh_solve_group): `problems` is a list of (HelmholtzMG, f) or
    (HelmholtzMG, f, u0) with distinct handles; the problems run
    concurrently on the device.  Returns [(u, info), ...] in order."""
    items = (B.HHGroupItem * len(problems))()
    outs, keep = [], []
    for i, p in enumerate(problems):
        mg, f = p[0], p[1]
        u0 = p[2] if len(p) > 2 else None
        f = mg._vec(f, "rhs")
        nb = f.shape[0]
        u = torch.empty_like(f) if u0 is None else mg._vec(u0, "u0").clone()
        info = (B.HHSolveInfo * nb)()
        items[i] = B.HHGroupItem(mg._h, _ptr(f), _ptr(u), nb,
                                 B.HH_USE_GUESS if u0 is not None else 0, info)
        outs.append((u, info, nb))
        keep.append(f)
    dev = problems[0][0].device if problems else torch.device("cuda")
    with torch.cuda.device(dev):
        st = B.lib().hh_solve_group(items, len(problems), float(tol), _stream())
    if st not in (B.HH_OK, B.HH_ERR_NOT_CONVERGED, B.HH_ERR_DIVERGED):
        B.check(st)
    return [(u, HelmholtzMG._infos(info, nb)) for u, info, nb in outs]


class HelmholtzGroup:
    """A work-list group (hh_group_create): mixed-precision 2-D handles of
    possibly different grid sizes whose cycles run as ONE chain of launches
    (one launch per level size over every problem's level of that size, one
    tail launch, one stop test for all).  `handles` and `batches` are fixed;
    solve() takes one right-hand-side tensor per handle."""

    def __init__(self, handles, batches):
        self.handles = list(handles)
        self.batches = [int(b) for b in batches]
        n = len(self.handles)
        hs = (ct.c_void_p * n)(*[mg._h.value if isinstance(mg._h, ct.c_void_p) else mg._h
                                 for mg in self.handles])
        bs = (ct.c_int * n)(*self.batches)
        g = ct.c_void_p()
        with torch.cuda.device(self.handles[0].device):
            B.check(B.lib().hh_group_create(hs, bs, n, ct.byref(g)))
        self._g = g

    @property
    def kernels(self):
        """Kernels launched by the last solve (-1 before one)."""
        return B.lib().hh_group_kernels(self._g)

    def solve(self, rhs, tol=1e-6, u0=None):
        """rhs: one complex128 tensor per handle ([batch, N, N]); returns
        [(u, info), ...] in the handles' order."""
        n = len(self.handles)
        items = (B.HHGroupItem * n)()
        outs, keep = [], []
        for i, (mg, f) in enumerate(zip(self.handles, rhs)):
            f = mg._vec(f, "rhs")
            nb = f.shape[0]
            g0 = None if u0 is None else u0[i]
            u = torch.empty_like(f) if g0 is None else mg._vec(g0, "u0").clone()
            info = (B.HHSolveInfo * nb)()
            items[i] = B.HHGroupItem(mg._h, _ptr(f), _ptr(u), nb,
                                     B.HH_USE_GUESS if g0 is not None else 0, info)
            outs.append((u, info, nb))
            keep.append(f)
        with torch.cuda.device(self.handles[0].device):
            st = B.lib().hh_group_solve(self._g, items, float(tol), _stream())
        if st not in (B.HH_OK, B.HH_ERR_NOT_CONVERGED, B.HH_ERR_DIVERGED):
            B.check(st)
        return [(u, HelmholtzMG._infos(info, nb)) for u, info, nb in outs]

    def close(self):
        if getattr(self, "_g", None):
            B.lib().hh_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
