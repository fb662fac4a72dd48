"""Closed-form columns of the transform matrix Phi (oracle; test infrastructure only).

Phi_jk = phi_k(x_j) (Eq. ``MHT-sum``, Sec. 1).

* Flat periodic square: phi_k(x) = exp(i k . x) with integer k (Eq. ``2D-DFT``); the
  Laplacian eigenvalue is |k|^2.
* Unit sphere: orthonormal real spherical harmonics of degree l and order mm, column index
  ``j = l^2 + l + mm``; eigenvalue l(l+1) (Sec. 1, the sphere's eigenfunctions).  Real form
  without Condon-Shortley phase:

      Y_l^0      = N_l0 P_l^0(cos t)
      Y_l^{mm>0} = sqrt(2) N_lm P_l^mm(cos t) cos(mm p)
      Y_l^{mm<0} = sqrt(2) N_l|mm| P_l^|mm|(cos t) sin(|mm| p)

  with N_lm = sqrt((2l+1)/(4 pi) (l-mm)!/(l+mm)!) folded into the normalized Legendre
  recurrence below.
"""
from __future__ import annotations

import numpy as np


def torus_phi(points: np.ndarray, modes: np.ndarray) -> np.ndarray:
    """Dense Phi (n, m) complex128 with Phi_jk = exp(i k_k . x_j)."""
    pts = np.asarray(points, dtype=np.float64)
    k = np.asarray(modes, dtype=np.float64)
    return np.exp(1j * (pts @ k.T))


def _normalized_legendre_columns(z: np.ndarray, lmax: int):
    """Yield (l, mm, Pbar_l^mm(z)) for 0 <= mm <= l <= lmax.

    Pbar_l^mm = N_lm P_l^mm is the fully normalized associated Legendre function (no
    Condon-Shortley phase).  Recurrences (standard, e.g. Numerical Recipes Sec. 6.7 in
    normalized form):
      Pbar_mm^mm     = sqrt((2mm+1)/(2mm)) sin(t) Pbar_{mm-1}^{mm-1},  Pbar_0^0 = 1/sqrt(4 pi)
      Pbar_{mm+1}^mm = sqrt(2mm+3) z Pbar_mm^mm
      Pbar_l^mm      = a_lm (z Pbar_{l-1}^mm - b_lm Pbar_{l-2}^mm),
        a_lm = sqrt((4l^2-1)/(l^2-mm^2)),  b_lm = sqrt(((l-1)^2-mm^2)/(4(l-1)^2-1)).
    """
    s = np.sqrt(np.clip(1.0 - z * z, 0.0, 1.0))
    pmm = np.full(z.shape, 1.0 / np.sqrt(4.0 * np.pi))
    for mm in range(lmax + 1):
        if mm > 0:
            pmm = pmm * np.sqrt((2.0 * mm + 1.0) / (2.0 * mm)) * s
        yield mm, mm, pmm
        if mm == lmax:
            break
        p_prev2 = pmm
        p_prev1 = np.sqrt(2.0 * mm + 3.0) * z * pmm
        yield mm + 1, mm, p_prev1
        for l in range(mm + 2, lmax + 1):
            a = np.sqrt((4.0 * l * l - 1.0) / (l * l - mm * mm))
            b = np.sqrt(((l - 1.0) ** 2 - mm * mm) / (4.0 * (l - 1.0) ** 2 - 1.0))
            p = a * (z * p_prev1 - b * p_prev2)
            p_prev2, p_prev1 = p_prev1, p
            yield l, mm, p


def sphere_phi(points: np.ndarray, lmax: int, ncols: int | None = None) -> np.ndarray:
    """Dense Phi (n, ncols) float64 of real spherical harmonics at unit-sphere points.

    Column j = l^2 + l + mm; ``ncols`` defaults to (lmax+1)^2 and may truncate it.
    """
    pts = np.asarray(points, dtype=np.float64)
    r = np.linalg.norm(pts, axis=1)
    z = pts[:, 2] / r
    lon = np.arctan2(pts[:, 1], pts[:, 0])
    m_all = (lmax + 1) ** 2
    ncols = m_all if ncols is None else ncols
    out = np.zeros((len(pts), ncols))
    root2 = np.sqrt(2.0)
    for l, mm, p in _normalized_legendre_columns(z, lmax):
        j0 = l * l + l
        if mm == 0:
            if j0 < ncols:
                out[:, j0] = p
        else:
            if j0 + mm < ncols:
                out[:, j0 + mm] = root2 * p * np.cos(mm * lon)
            if j0 - mm < ncols:
                out[:, j0 - mm] = root2 * p * np.sin(mm * lon)
    return out
