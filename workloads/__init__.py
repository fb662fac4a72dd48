"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds the *shapes* of the paper's workloads and nothing of the method's
arithmetic: point clouds, mode (frequency) lists, coefficient vectors, triangle meshes
and quadrature weights.  It evaluates no eigenfunction, builds no tree and computes no
factorization; every consumer does that with its own code.

Recipes (each draw uses ``numpy.random.default_rng(seed)``):

* flat periodic square (Eq. ``2D-DFT``, Sec. 1): points uniform in ``[-pi, pi]^2``; modes
  are the integer box ``k in [-sqrt(m)/2, sqrt(m)/2 - 1]^2`` listed row-major (k1 slow);
* unit sphere (Sec. 1, spherical harmonics): a jittered Fibonacci lattice
  ``z_i = 1 - (2i + 1 + u_i)/n``, ``lon_i = 2 pi i / golden + v_i sqrt(4 pi / n)``
  with ``u, v ~ U(-1/2, 1/2)``; quadrature weights ``4 pi / n``;
* deformed sphere (Sec. 6.2 stand-in): icosphere of a given subdivision level with
  radius ``1 + 0.2 h / max|h|`` where ``h`` is a seeded random polynomial of total degree
  <= 6 in (x, y, z); restricted to the sphere such a polynomial is exactly a combination
  of real harmonics of degree <= 6;
* coefficients: i.i.d. standard normal (real) or ``(N(0,1) + i N(0,1))/sqrt(2)`` (complex);
  sphere coefficients decay as ``N(0,1)/(1+l)`` with ``l = floor(sqrt(j))`` for the
  degree-ordered index ``j = l^2 + l + m``.
"""
from __future__ import annotations

import numpy as np

GOLDEN = (1.0 + 5.0 ** 0.5) / 2.0


def torus_points(n: int, seed: int = 0) -> np.ndarray:
    """n points uniform in [-pi, pi]^2, shape (n, 2), float64."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi, np.pi, size=(n, 2))


def torus_modes(m: int) -> np.ndarray:
    """Integer frequencies of the box [-s/2, s/2-1]^2 with s = sqrt(m), shape (m, 2), int64.

    Listed row-major (k1 is the slow index).  ``m`` must be a perfect square with even root.
    """
    s = int(round(m ** 0.5))
    if s * s != m or s % 2:
        raise ValueError("m must be the square of an even integer")
    k = np.arange(-s // 2, s // 2, dtype=np.int64)
    k1, k2 = np.meshgrid(k, k, indexing="ij")
    return np.stack([k1.ravel(), k2.ravel()], axis=1)


def torus_modes_lowest(m: int) -> np.ndarray:
    """The m integer frequencies of smallest |k|^2 (ties by k1, then k2), shape (m, 2), int64.

    For any m (the box of :func:`torus_modes` needs a perfect square).
    """
    s = 2
    while s * s < m:
        s += 2
    k = np.arange(-s // 2 - 1, s // 2 + 2, dtype=np.int64)
    k1, k2 = np.meshgrid(k, k, indexing="ij")
    K = np.stack([k1.ravel(), k2.ravel()], axis=1)
    order = np.lexsort((K[:, 1], K[:, 0], K[:, 0] ** 2 + K[:, 1] ** 2))
    return K[order[:m]]


def torus_eigenvalues(modes: np.ndarray) -> np.ndarray:
    """|k|^2 for each integer frequency (the periodic Laplacian's eigenvalue)."""
    modes = np.asarray(modes, dtype=np.float64)
    return modes[:, 0] ** 2 + modes[:, 1] ** 2


def uniform_grid_points(s: int) -> np.ndarray:
    """The s x s uniform grid x_j = -pi + 2 pi j / s on [-pi, pi)^2, row-major (x1 slow)."""
    g = -np.pi + 2.0 * np.pi * np.arange(s) / s
    a, b = np.meshgrid(g, g, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1)


def fibonacci_points(n: int, seed: int = 0) -> np.ndarray:
    """Jittered Fibonacci lattice on the unit sphere, shape (n, 3), float64."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    u = rng.uniform(-0.5, 0.5, size=n)
    v = rng.uniform(-0.5, 0.5, size=n)
    z = 1.0 - (2.0 * i + 1.0 + u) / n
    lon = 2.0 * np.pi * i / GOLDEN + v * np.sqrt(4.0 * np.pi / n)
    s = np.sqrt(np.clip(1.0 - z * z, 0.0, 1.0))
    return np.stack([s * np.cos(lon), s * np.sin(lon), z], axis=1)


def sphere_degree_count(lmax: int) -> int:
    """Number of real harmonics of degree <= lmax."""
    return (lmax + 1) ** 2


def sphere_eigenvalues(m: int) -> np.ndarray:
    """l(l+1) for the degree-ordered index j = l^2 + l + mm, j < m."""
    l = np.floor(np.sqrt(np.arange(m, dtype=np.float64)))
    return l * (l + 1.0)


def sphere_coefficients(m: int, nrhs: int = 1, seed: int = 1) -> np.ndarray:
    """Real coefficients N(0,1)/(1+l), shape (m, nrhs), float64 (column j uses seed+j)."""
    l = np.floor(np.sqrt(np.arange(m, dtype=np.float64)))
    cols = [np.random.default_rng(seed + j).standard_normal(m) / (1.0 + l) for j in range(nrhs)]
    return np.stack(cols, axis=1)


def gaussian(shape, seed: int = 1, complex_: bool = False) -> np.ndarray:
    """i.i.d. N(0,1) (or circular complex normal with unit variance), float64/complex128."""
    rng = np.random.default_rng(seed)
    if not complex_:
        return rng.standard_normal(shape)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def gaussian_columns(rows: int, nrhs: int, seed: int = 1, complex_: bool = False) -> np.ndarray:
    """(rows, nrhs) matrix whose column j is ``gaussian(rows, seed + j)``."""
    return np.stack([gaussian(rows, seed + j, complex_) for j in range(nrhs)], axis=1)


def icosphere(level: int):
    """Unit icosphere: (vertices (V,3) float64, triangles (F,3) int64), outward orientation.

    Level 0 is the icosahedron (12 vertices); each level splits every triangle into four
    and projects new vertices to the sphere.  Level 6 has 40962 vertices, 81920 triangles.
    """
    t = GOLDEN
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    F = faces
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = V[a] + V[b]
                V.append(p / np.linalg.norm(p))
                cache[key] = len(V) - 1
            return cache[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    return np.array(V), np.array(F, dtype=np.int64)


def criss_cross_rectangle(a: float, b: float, nx: int, ny: int):
    """Flat rectangle [0, a] x [0, b] (z = 0) meshed by an nx x ny grid of cells, each split
    into four triangles by its centre vertex: (vertices (V,3), triangles (F,3) int64).  The
    mesh is symmetric under x -> a - x and y -> b - y.  Grid vertices come first (row-major in
    y, then x), then the cell centres."""
    xs, ys = np.linspace(0.0, a, nx + 1), np.linspace(0.0, b, ny + 1)
    gx, gy = np.meshgrid(xs, ys)
    grid = np.stack([gx.ravel(), gy.ravel(), np.zeros(gx.size)], axis=1)
    cx, cy = np.meshgrid(0.5 * (xs[1:] + xs[:-1]), 0.5 * (ys[1:] + ys[:-1]))
    centres = np.stack([cx.ravel(), cy.ravel(), np.zeros(cx.size)], axis=1)
    V = np.concatenate([grid, centres])
    g = lambda i, j: j * (nx + 1) + i  # noqa: E731
    F = []
    for j in range(ny):
        for i in range(nx):
            c = len(grid) + j * nx + i
            p00, p10, p11, p01 = g(i, j), g(i + 1, j), g(i + 1, j + 1), g(i, j + 1)
            F += [(p00, p10, c), (p10, p11, c), (p11, p01, c), (p01, p00, c)]
    return V, np.array(F, dtype=np.int64)


def random_polynomial_height(points: np.ndarray, degree: int = 6, seed: int = 3) -> np.ndarray:
    """h(x) = sum over monomials x^a y^b z^c (a+b+c <= degree) of seeded N(0,1) weights."""
    rng = np.random.default_rng(seed)
    x, y, z = points[:, 0], points[:, 1], points[:, 2]
    h = np.zeros(len(points))
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                h += rng.standard_normal() * x ** a * y ** b * z ** c
    return h


def deformed_icosphere(level: int, amplitude: float = 0.2, seed: int = 3):
    """Icosphere with radius 1 + amplitude * h / max|h| (h from random_polynomial_height)."""
    V, F = icosphere(level)
    h = random_polynomial_height(V, 6, seed)
    r = 1.0 + amplitude * h / np.max(np.abs(h))
    return V * r[:, None], F


def deformed_sphere_points(n: int, seed: int = 0, amplitude: float = 0.2, shape_seed: int = 3) -> np.ndarray:
    """Jittered Fibonacci points moved to radius 1 + amplitude * h / max|h| (h as in
    :func:`deformed_icosphere`), for deformed-sphere point sets of any size."""
    X = fibonacci_points(n, seed=seed)
    h = random_polynomial_height(X, 6, shape_seed)
    return X * (1.0 + amplitude * h / np.max(np.abs(h)))[:, None]


def batched_instances(count: int = 64, seed: int = 2, nmin: int = 2000, nmax: int = 40000,
                      kmax: int = 128):
    """Sizes of the batched ragged workload: list of dicts (kind, n, m, nrhs)."""
    rng = np.random.default_rng(seed)
    kinds = ("torus", "sphere", "deformed")
    out = []
    for i in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        out.append({"kind": kinds[i % 3], "n": n, "m": max(1, n // 4),
                    "nrhs": int(rng.integers(1, kmax + 1))})
    return out
