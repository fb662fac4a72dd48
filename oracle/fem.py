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


def eigenpairs_sliced(K: sp.spmatrix, Mdiag: np.ndarray, m: int, per_slice: int = 512,
                      area: float | None = None, seed: int = 0):
    """Lowest m pairs by shift-invert Lanczos in spectral slices (large meshes).

    Each slice asks for ``per_slice`` pairs nearest a shift sigma placed (by Weyl's law) at
    the middle of the next band of eigenvalues; pairs are merged by eigenvalue, duplicates
    at band edges are removed by M-orthogonality, and the result is M-orthonormalized.
    """
    n = K.shape[0]
    if area is None:
        area = float(Mdiag.sum())
    M = sp.diags(Mdiag).tocsc()
    K = K.tocsc()
    lam_all, vec_all = [], []
    rng = np.random.default_rng(seed)
    have = 0
    lo = 0.0
    while have < m:
        # Weyl: the count below lambda is about area * lambda / (4 pi)
        width = per_slice * 4.0 * np.pi / area
        sigma = lo + 0.5 * width - (1e-3 if lo == 0.0 else 0.0)
        v0 = rng.standard_normal(n)
        lam, vec = spla.eigsh(K, k=per_slice, M=M, sigma=sigma, which="LM", v0=v0, tol=1e-12)
        o = np.argsort(lam)
        lam, vec = lam[o], vec[:, o]
        for j in range(len(lam)):
            v = vec[:, j]
            if vec_all:
                B = np.stack(vec_all, axis=1)
                coeff = B.T @ (Mdiag * v)
                if np.max(np.abs(coeff)) > 0.5 * np.sqrt(v @ (Mdiag * v)):
                    continue  # already found in an earlier slice
            lam_all.append(lam[j])
            vec_all.append(v)
        have = sum(1 for x in lam_all if x <= lam[-1])
        lo = lam[-1] - 0.1 * width
        if len(lam_all) >= m + per_slice:
            break
    lam_all = np.array(lam_all)
    o = np.argsort(lam_all, kind="stable")[:m]
    Phi = np.stack(vec_all, axis=1)[:, o]
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
