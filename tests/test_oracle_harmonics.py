"""Pins for oracle/harmonics.py against FFTs, scipy's spherical harmonics and exact identities."""
import numpy as np
import pytest
import scipy.special as sps

import workloads as W
from oracle import harmonics as H


def test_torus_uniform_grid_is_fft2():
    # Eq. 2D-DFT on the uniform grid x_j = -pi + 2 pi j / s is an inverse 2D DFT:
    # f[j1, j2] = s^2 ifft2(C)[j1, j2] with C[k mod s] = c_k (-1)^(k1 + k2).
    s = 16
    X = W.uniform_grid_points(s)
    K = W.torus_modes(s * s)
    c = W.gaussian(s * s, seed=4, complex_=True)
    f = H.torus_phi(X, K) @ c
    C = np.zeros((s, s), dtype=complex)
    C[K[:, 0] % s, K[:, 1] % s] = c * (-1.0) ** (K[:, 0] + K[:, 1])
    ref = (s * s) * np.fft.ifft2(C).ravel()
    assert np.max(np.abs(f - ref)) < 1e-11 * np.max(np.abs(ref))


def test_torus_uniform_grid_orthogonal():
    s = 8
    Phi = H.torus_phi(W.uniform_grid_points(s), W.torus_modes(s * s))
    G = Phi.conj().T @ Phi
    assert np.allclose(G, s * s * np.eye(s * s), atol=1e-10)


def test_torus_closed_form_entry():
    x = np.array([[0.3, -1.2]])
    k = np.array([[2, -3]])
    assert np.isclose(H.torus_phi(x, k)[0, 0], np.cos(2 * 0.3 + 3 * 1.2) + 1j * np.sin(2 * 0.3 + 3 * 1.2))


def _real_from_scipy(l, mm, pts):
    theta = np.arccos(np.clip(pts[:, 2], -1, 1))
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    Y = sps.sph_harm_y(l, abs(mm), theta, phi)  # Condon-Shortley phase included
    if mm == 0:
        return Y.real
    cs = (-1.0) ** abs(mm)
    return np.sqrt(2.0) * cs * (Y.real if mm > 0 else Y.imag)


@pytest.mark.parametrize("l", [0, 1, 2, 5, 17, 40])
def test_sphere_matches_scipy(l):
    pts = W.fibonacci_points(200, seed=7)
    Phi = H.sphere_phi(pts, l)
    for mm in range(-l, l + 1):
        ref = _real_from_scipy(l, mm, pts)
        assert np.max(np.abs(Phi[:, l * l + l + mm] - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_sphere_low_degree_closed_forms():
    pts = W.fibonacci_points(50, seed=8)
    x, y, z = pts.T
    Phi = H.sphere_phi(pts, 2)
    c1 = np.sqrt(3 / (4 * np.pi))
    assert np.allclose(Phi[:, 0], 1 / np.sqrt(4 * np.pi))
    assert np.allclose(Phi[:, 1], c1 * y)
    assert np.allclose(Phi[:, 2], c1 * z)
    assert np.allclose(Phi[:, 3], c1 * x)
    assert np.allclose(Phi[:, 6], np.sqrt(5 / (16 * np.pi)) * (3 * z * z - 1))
    assert np.allclose(Phi[:, 8], np.sqrt(15 / (16 * np.pi)) * (x * x - y * y))


def test_sphere_addition_theorem_high_degree():
    # sum_mm Y_lm(x)^2 = (2l+1)/(4 pi) for every point and degree, up to l = 255
    pts = W.fibonacci_points(64, seed=9)
    lmax = 255
    Phi = H.sphere_phi(pts, lmax)
    for l in range(0, lmax + 1, 17):
        s = np.sum(Phi[:, l * l:(l + 1) * (l + 1)] ** 2, axis=1)
        assert np.allclose(s, (2 * l + 1) / (4 * np.pi), rtol=1e-11)


def test_sphere_quadrature_orthonormality():
    # Gauss-Legendre in cos(theta) x uniform longitude integrates degree <= 2 lmax exactly
    lmax = 20
    zq, wq = np.polynomial.legendre.leggauss(lmax + 1)
    nlon = 2 * lmax + 2
    lon = 2 * np.pi * np.arange(nlon) / nlon
    Z, LON = np.meshgrid(zq, lon, indexing="ij")
    Wt = np.repeat(wq, nlon) * (2 * np.pi / nlon)
    s = np.sqrt(1 - Z.ravel() ** 2)
    pts = np.stack([s * np.cos(LON.ravel()), s * np.sin(LON.ravel()), Z.ravel()], 1)
    Phi = H.sphere_phi(pts, lmax)
    G = Phi.T @ (Wt[:, None] * Phi)
    assert np.max(np.abs(G - np.eye(G.shape[1]))) < 1e-12


def test_sphere_is_laplacian_eigenfunction():
    # Surface Laplacian by second differences in (theta, lon): -l(l+1) Y
    l, h = 7, 1e-3
    th, ph = 1.1, 0.7

    def Y(t, p):
        pt = np.array([[np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)]])
        return H.sphere_phi(pt, l)[0, l * l:]

    d2t = (Y(th + h, ph) - 2 * Y(th, ph) + Y(th - h, ph)) / h ** 2
    dt = (Y(th + h, ph) - Y(th - h, ph)) / (2 * h)
    d2p = (Y(th, ph + h) - 2 * Y(th, ph) + Y(th, ph - h)) / h ** 2
    lap = d2t + np.cos(th) / np.sin(th) * dt + d2p / np.sin(th) ** 2
    assert np.allclose(lap, -l * (l + 1) * Y(th, ph), atol=1e-4)


def test_inverse_transform_recovers_coefficients_and_solves_normal_equations():
    # Eq. inverse-MHT: a consistent system returns its coefficients; an inconsistent one
    # leaves a residual orthogonal to the range of Phi
    from oracle import dense as D
    X = W.fibonacci_points(400)
    Phi = H.sphere_phi(X, 9)  # m = 100 < n: full column rank
    c0 = W.gaussian_columns(100, 2, 3)
    assert np.allclose(D.inverse(Phi, Phi @ c0), c0, atol=1e-11)
    f = Phi @ c0 + W.gaussian_columns(400, 2, 9)
    c = D.inverse(Phi, f)
    assert np.abs(Phi.T @ (Phi @ c - f)).max() < 1e-9 * np.abs(Phi.T @ f).max()
    assert np.linalg.norm(Phi @ c - f) <= np.linalg.norm(Phi @ c0 - f) + 1e-12
