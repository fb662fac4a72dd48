"""The transform by direct summation (oracle; test infrastructure only).

Synthesis is the definition f_j = sum_k c_k phi_k(x_j), i.e. f = Phi c (Eq. ``MHT-sum``,
Sec. 1).  Analysis is the weighted adjoint c = Phi^H diag(w) f, the fast adjoint that maps
point values to coefficients (Sec. 1); Phi^H is the conjugate transpose (the paper's ``*``).
With w = None the plain adjoint Phi^H f is returned.
"""
from __future__ import annotations

import numpy as np


def synthesize(Phi: np.ndarray, c: np.ndarray) -> np.ndarray:
    """f = Phi c for a dense Phi (n, m) and c (m,) or (m, k)."""
    return Phi @ c


def analyze(Phi: np.ndarray, f: np.ndarray, w: np.ndarray | None = None) -> np.ndarray:
    """c = Phi^H diag(w) f for a dense Phi (n, m) and f (n,) or (n, k)."""
    g = f if w is None else (w[:, None] * f if f.ndim == 2 else w * f)
    return Phi.conj().T @ g


def inverse(Phi: np.ndarray, f: np.ndarray) -> np.ndarray:
    """The inverse transform c = argmin_c ||Phi c - f||_2 (Sec. 7.1, Eq. inverse-MHT), by the
    library least-squares routine (SVD-based), column by column for f (n, k)."""
    return np.linalg.lstsq(Phi, f, rcond=None)[0]
