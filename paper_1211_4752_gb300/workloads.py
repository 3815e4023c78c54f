"""Seeded synthetic inputs shaped like the paper's model problems.

This module only builds problem data (grid size, k^2 field, ECS layer width,
right-hand sides); it holds none of the method's arithmetic, and it serves
both the CUDA path and the CPU oracle.  numpy only.

Workloads (unit square / cube, n intervals per axis, N = n - 1 interior points,
interior point i at coordinate (i + 1) / n):

* ``dirichlet_const``   63^2, k = 40, homogeneous Dirichlet, unit source at the
  centre grid point (the constant-k model of Sec. 4.1 with Dirichlet bounds).
* ``ecs_const``         1023^2, k = 640 (kh = 0.625), ECS layers of 32 cells,
  unit source at (0.5, 0.5) (constant-k model of Sec. 4.1).
* ``layered``           2047^2, k^2 = (omega / c)^2 with c piecewise constant
  over three layers (the wedge model of Sec. 4.2 made synthetic), ECS 48.
* ``batch_sources``     64 unit sources over 255^2 / 511^2 / 1023^2 grids,
  kh = 0.625, ECS layers of width 1/32.
* ``bump``              511^2, kh = 0.5 background with a 10 % Gaussian bump
  in k^2, ECS 16, 16 sources on the first physical row.
* ``cube``              127^3, k = 80 (kh = 0.625), ECS 16, centre source.
* ``ionization``        the quantum-mechanical ionization model of Sec. 4.3 on
  (0, r)^2, r = 50: coefficient e^{-x^2} + e^{-y^2} + k0^2 of u, source
  e^{-(x^2+y^2)}, u = 0 on x = 0 and y = 0, ECS on the sides x = r, y = r;
  grid sizes of Table 8 (k0 = 1 .. 5: 128^2, 256^2, 256^2, 512^2, 512^2).
  Mapped to the unit square by x = r xi: the coefficient and the source are
  multiplied by r^2.
"""

from __future__ import annotations

import math

import numpy as np


def interior_coords(n):
    return (np.arange(1, n, dtype=np.float64)) / n


def point_sources(n, dim, positions):
    """Unit point sources (value 1 at one grid point, no 1/h^d factor; the
    source of the constant-k model, Sec. 4.1) as a complex128
    [len(positions), N, ..., N] array; positions are interior index tuples
    in array axis order."""
    N = n - 1
    f = np.zeros((len(positions),) + (N,) * dim, dtype=np.complex128)
    for b, pos in enumerate(positions):
        f[(b,) + tuple(pos)] = 1.0
    return f


def dirichlet_const():
    n, k = 64, 40.0
    return dict(name="dirichlet_const_63x63_k40", n=n, dim=2, k2=k * k,
                layers=0, rhs=point_sources(n, 2, [(31, 31)]))


def ecs_const(n=1024, layers=None, kh=0.625):
    k = kh * n
    layers = n // 32 if layers is None else layers
    c = n // 2 - 1
    return dict(name=f"ecs_const_{n-1}x{n-1}_k{k:g}_ecs{layers}", n=n, dim=2,
                k2=k * k, layers=layers, rhs=point_sources(n, 2, [(c, c)]))


def layered(n=2048, layers=48, seed=0, kh=0.625):
    """Three-layer medium: two interfaces through the centre column at
    depths 1/3 and 2/3 of the physical region, each tilted by an angle drawn
    from U[-20, 20] degrees (redrawn while the lines cross inside the unit
    square); layer speeds from U[1.5, 4.5]; omega = kh * n * c_min so that the
    largest k h is kh; source on the centre column 10 points below the top
    edge of the physical region.  Depth is the slow (row) axis."""
    rng = np.random.default_rng(seed)
    a = layers / n
    b = 1.0 - layers / n
    d1 = a + (b - a) / 3.0
    d2 = a + 2.0 * (b - a) / 3.0
    while True:
        t1, t2 = np.tan(np.deg2rad(rng.uniform(-20.0, 20.0, size=2)))
        # depth(x) = d + t (x - 0.5); crossing where (d2 - d1) = (t1 - t2)(x - .5)
        if t1 == t2:
            break
        xc = 0.5 + (d2 - d1) / (t1 - t2)
        if not (0.0 <= xc <= 1.0):
            break
    speeds = rng.uniform(1.5, 4.5, size=3)
    x = interior_coords(n)
    X, Y = np.meshgrid(x, x, indexing="xy")       # Y = depth (row index)
    i1 = d1 + t1 * (X - 0.5)
    i2 = d2 + t2 * (X - 0.5)
    c = np.where(Y < i1, speeds[0], np.where(Y < i2, speeds[1], speeds[2]))
    omega = kh * n * speeds.min()
    k2 = (omega / c) ** 2
    row = layers + 10 - 1
    col = n // 2 - 1
    return dict(name=f"layered_{n-1}x{n-1}_ecs{layers}_seed{seed}", n=n, dim=2,
                k2=k2, layers=layers, rhs=point_sources(n, 2, [(row, col)]),
                speeds=speeds, tilts=(t1, t2), omega=omega)


def batch_sources(total=64, sizes=(256, 512, 1024), seed=0, kh=0.625):
    """Unit sources at seed-drawn interior points (uniform over the physical
    region) spread round-robin over the grid sizes in a seed-drawn order."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(total)
    groups = []
    for gi, n in enumerate(sizes):
        layers = n // 32
        ids = [int(j) for j in order if j % len(sizes) == gi]
        lo, hi = layers, n - layers - 2
        pos = [tuple(rng.integers(lo, hi + 1, size=2)) for _ in ids]
        k = kh * n
        groups.append(dict(name=f"batch_{n-1}x{n-1}_k{k:g}_ecs{layers}", n=n,
                           dim=2, k2=k * k, layers=layers, ids=ids,
                           rhs=point_sources(n, 2, pos)))
    return groups


def bump(n=512, layers=16, seed=0, nsrc=16, kh=0.5, amp=0.1, sigma=0.05):
    """k^2 = k_bg^2 (1 + amp exp(-|x - x_c|^2 / (2 sigma^2))), x_c ~ U[.3,.7]^2,
    k_bg = kh * n; sources on the first physical row at equispaced columns;
    receivers on the last physical row; data d: seeded complex values of the
    size of a typical receiver response."""
    rng = np.random.default_rng(seed)
    xc = rng.uniform(0.3, 0.7, size=2)
    x = interior_coords(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    kbg2 = (kh * n) ** 2
    k2 = kbg2 * (1.0 + amp * np.exp(-((X - xc[0]) ** 2 + (Y - xc[1]) ** 2) / (2 * sigma ** 2)))
    first, last = layers, n - layers - 2
    cols = np.linspace(layers, n - layers - 2, nsrc).round().astype(int)
    rhs = point_sources(n, 2, [(first, int(cc)) for cc in cols])
    rows = np.full(n - 1 - 2 * layers, last)
    rcols = np.arange(layers, n - 1 - layers)
    scale = 1.0 / n ** 2
    d = scale * (rng.standard_normal((nsrc, rcols.size)) +
                 1j * rng.standard_normal((nsrc, rcols.size)))
    return dict(name=f"bump_{n-1}x{n-1}_kh{kh}_ecs{layers}", n=n, dim=2, k2=k2,
                layers=layers, rhs=rhs, receiver_rows=rows,
                receiver_cols=rcols, data=d, center=xc)


def cube(n=128, k=80.0, layers=16):
    c = n // 2 - 1
    return dict(name=f"cube_{n-1}^3_k{k:g}_ecs{layers}", n=n, dim=3, k2=k * k,
                layers=layers, rhs=point_sources(n, 3, [(c, c, c)]))


ION_GRIDS = {1: 128, 2: 256, 3: 256, 4: 512, 5: 512}   # Table 8


def ionization(k0=1, n=None, r=50.0, layer_frac=8):
    """Sec. 4.3's ionization model (see the module docstring).  The ECS layer
    takes the last n / layer_frac cells next to x = r and y = r inside the
    grid; the sides x = 0 and y = 0 have no layer (homogeneous Dirichlet).
    Arrays are [y][x] over the interior points (i + 1) r / n."""
    n = ION_GRIDS[k0] if n is None else n
    x = interior_coords(n) * r
    X, Y = np.meshgrid(x, x, indexing="xy")
    k2 = r * r * (np.exp(-X * X) + np.exp(-Y * Y) + float(k0) ** 2)
    rhs = (r * r * np.exp(-(X * X + Y * Y)))[None].astype(np.complex128)
    layers = n // layer_frac
    return dict(name=f"ionization_{n-1}x{n-1}_k0{k0:g}_ecs0-{layers}", n=n, dim=2, k2=k2,
                layers=(0, layers), rhs=rhs)


def random_field(shape, seed, complex_=True, scale=1.0):
    """Seeded standard-normal test vectors (complex128 or float64)."""
    rng = np.random.default_rng(seed)
    if complex_:
        return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return scale * rng.standard_normal(shape)


def smooth_k2(n, dim, seed, kmin, kmax):
    """A seeded smoothly varying k^2 field in [kmin^2, kmax^2] (test input)."""
    rng = np.random.default_rng(seed)
    x = interior_coords(n)
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    ph = rng.uniform(0, 2 * math.pi, size=dim)
    s = sum(np.sin(2 * math.pi * (j + 1) * g + p) for j, (g, p) in enumerate(zip(grids, ph)))
    s = (s - s.min()) / max(s.max() - s.min(), 1e-300)
    return (kmin + (kmax - kmin) * s) ** 2
