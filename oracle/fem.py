"""P1 finite elements for the Laplace-Beltrami eigenproblem (oracle; test infrastructure only).

Discretizes Eq. ``eigenproblem`` (Sec. 1) on a closed triangle mesh as the generalized
symmetric eigenproblem ``K phi = lambda M phi``:

* K, the cotangent stiffness matrix: for each triangle with vertices (a, b, c) and the
  interior angle gamma at c opposite edge (a, b), K_ab -= cot(gamma)/2 and K_aa, K_bb
  += cot(gamma)/2 (this is the P1 Galerkin matrix of the Dirichlet energy);
* M, the barycentric lumped mass matrix: M_aa = sum over incident triangles of area/3.

The lowest m eigenpairs are M-orthonormal columns Phi (Phi^T M Phi = I), sorted by
eigenvalue (ties keep solver order).  Large problems are solved in spectral slices with
shift-invert Lanczos, shifts spaced by Weyl's law N(lambda) ~ A lambda / (4 pi) for a
closed surface of area A (Sec. 7.1; the printed form there is inverted).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def triangle_areas(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)


def cotan_stiffness(V: np.ndarray, F: np.ndarray) -> sp.csr_matrix:
    """Cotangent stiffness matrix K (n x n, symmetric, rows sum to zero)."""
    n = len(V)
    rows, cols, vals = [], [], []
    for k in range(3):
        i, j, o = F[:, k], F[:, (k + 1) % 3], F[:, (k + 2) % 3]
        u = V[i] - V[o]
        w = V[j] - V[o]
        cot = np.einsum("ij,ij->i", u, w) / np.linalg.norm(np.cross(u, w), axis=1)
        h = 0.5 * cot
        rows += [i, j, i, j]
        cols += [j, i, i, j]
        vals += [-h, -h, h, h]
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return K.tocsr()


def lumped_mass(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Diagonal of the barycentric lumped mass matrix (length n)."""
    A = triangle_areas(V, F)
    m = np.zeros(len(V))
    for k in range(3):
        np.add.at(m, F[:, k], A / 3.0)
    return m


def eigenpairs_dense(K: sp.spmatrix, Mdiag: np.ndarray, m: int):
    """Lowest m pairs of K phi = lambda M phi by dense LAPACK (small meshes)."""
    lam, Phi = sla.eigh(K.toarray(), np.diag(Mdiag), subset_by_index=[0, m - 1])
    return lam, Phi


def _m_orthonormalize(Phi: np.ndarray, Mdiag: np.ndarray) -> np.ndarray:
    G = Phi.T @ (Mdiag[:, None] * Phi)
    Lc = np.linalg.cholesky(G)
    return sla.solve_triangular(Lc, Phi.T, lower=True).T


def _nearest_pairs(K, M, Mdiag, sigma, k, rng, V=None):
    """The k pairs of K phi = lambda M phi nearest sigma by shift-invert Lanczos; with V
    (M-orthonormal columns spanning found eigenvectors) the operator acts on the
    M-orthogonal complement of V, so those pairs are skipped."""
    n = K.shape[0]
    v0 = rng.standard_normal(n)
    if V is None or V.shape[1] == 0:
        lam, vec = spla.eigsh(K, k=k, M=M, sigma=sigma, which="LM", v0=v0, tol=1e-12)
    else:
        lu = spla.splu((K - sigma * M).tocsc())

        def solve(x):
            y = lu.solve(np.asarray(x, dtype=np.float64).ravel())
            return y - V @ (V.T @ (Mdiag * y))

        op = spla.LinearOperator((n, n), matvec=solve, dtype=np.float64)
        v0 = v0 - V @ (V.T @ (Mdiag * v0))
        lam, vec = spla.eigsh(K, k=k, M=M, sigma=sigma, which="LM", v0=v0, tol=1e-12, OPinv=op)
    o = np.argsort(lam)
    return lam[o], vec[:, o]


def eigenpairs_sliced(K: sp.spmatrix, Mdiag: np.ndarray, m: int, per_slice: int = 512,
                      area: float | None = None, seed: int = 0):
    """Lowest m pairs by shift-invert Lanczos in spectral slices (large meshes).

    The spectrum is covered from the bottom by slices that partition it:

    * the first slice asks for the ``per_slice`` pairs nearest a shift just below zero; K is
      positive semidefinite, so these are the lowest pairs;
    * every later slice is centred half a band above the covered part, the band width taken
      from Weyl's law N(lambda) ~ A lambda / (4 pi) at first and from the previous slice's
      observed width after that;
    * the pairs nearest a shift are a contiguous stretch of the spectrum, so a slice is used
      only if its stretch reaches well below the covered boundary (otherwise the shift moves
      down and the slice is recomputed); single-vector Lanczos can miss copies of a multiple
      eigenvalue, so the slice is searched again on the M-orthogonal complement of what it
      found until the nearest remaining eigenvalue lies outside the stretch;
    * it contributes its eigenvalues from the boundary up to just below its top, where the
      window could cut a degenerate cluster, and that point becomes the new boundary.

    The result is M-orthonormalized.
    """
    n = K.shape[0]
    if area is None:
        area = float(Mdiag.sum())
    k = min(per_slice, n - 2)
    M = sp.diags(Mdiag).tocsc()
    K = K.tocsc()
    rng = np.random.default_rng(seed)
    width = k * 4.0 * np.pi / area
    lam_parts, vec_parts = [], []
    covered = None  # every eigenvalue below `covered` has been taken, none above it
    found = 0
    while found < m:
        sigma = -1e-3 * width if covered is None else covered + 0.5 * width
        for _ in range(30):
            lam, vec = _nearest_pairs(K, M, Mdiag, sigma, k, rng)
            if covered is None or lam[0] < covered - 0.05 * (lam[-1] - lam[0]):
                break
            sigma = covered + 0.5 * (sigma - covered)  # the stretch missed the boundary
        else:
            raise RuntimeError("spectral slicing could not reach the covered part of the spectrum")
        radius = max(abs(lam[0] - sigma), abs(lam[-1] - sigma))
        for _ in range(50):  # recover copies of multiple eigenvalues the first pass missed
            V = _m_orthonormalize(vec, Mdiag)
            extra_l, extra_v = _nearest_pairs(K, M, Mdiag, sigma, min(16, n - 2 - vec.shape[1]), rng, V)
            inside = np.abs(extra_l - sigma) < radius * (1 - 1e-10)
            if not inside.any():
                break
            lam = np.concatenate([lam, extra_l[inside]])
            vec = np.concatenate([vec, extra_v[:, inside]], axis=1)
            o = np.argsort(lam)
            lam, vec = lam[o], vec[:, o]
        else:
            raise RuntimeError("spectral slicing kept finding new copies of multiple eigenvalues")
        top = lam[-1] - 1e-8 * max(abs(lam[-1]), 1.0)
        keep = lam < top if covered is None else (lam >= covered) & (lam < top)
        lam_parts.append(lam[keep])
        vec_parts.append(vec[:, keep])
        found += int(keep.sum())
        covered = top
        width = lam[-1] - lam[0]
    lam_all = np.concatenate(lam_parts)
    o = np.argsort(lam_all, kind="stable")[:m]
    Phi = np.concatenate(vec_parts, axis=1)[:, o]
    return lam_all[o], _m_orthonormalize(Phi, Mdiag)


def laplace_beltrami_basis(V: np.ndarray, F: np.ndarray, m: int, dense_limit: int = 3000):
    """(eigenvalues (m,), Phi (n, m), Mdiag (n,), K) for a closed triangle mesh."""
    K = cotan_stiffness(V, F)
    Md = lumped_mass(V, F)
    if len(V) <= dense_limit:
        lam, Phi = eigenpairs_dense(K, Md, m)
    else:
        lam, Phi = eigenpairs_sliced(K, Md, m)
    return lam, Phi, Md, K
