"""Pins for oracle/fem.py: exact mesh invariants, linear precision and the sphere spectrum."""
import numpy as np

import workloads as W
from oracle import fem


def _planar_grid(s=9, jitter=0.15, seed=0):
    rng = np.random.default_rng(seed)
    g = np.linspace(0, 1, s)
    X, Y = np.meshgrid(g, g, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), np.zeros(s * s)], 1)
    interior = (P[:, 0] > 0) & (P[:, 0] < 1) & (P[:, 1] > 0) & (P[:, 1] < 1)
    P[interior, :2] += rng.uniform(-jitter, jitter, (interior.sum(), 2)) / (s - 1)
    F = []
    for i in range(s - 1):
        for j in range(s - 1):
            a, b, c, d = i * s + j, (i + 1) * s + j, (i + 1) * s + j + 1, i * s + j + 1
            F += [(a, b, c), (a, c, d)]
    return P, np.array(F), interior


def test_stiffness_symmetric_rows_sum_zero():
    V, F = W.icosphere(2)
    K = fem.cotan_stiffness(V, F)
    assert abs(K - K.T).max() < 1e-14
    assert np.max(np.abs(K @ np.ones(len(V)))) < 1e-12


def test_linear_precision_on_planar_mesh():
    # the cotan Laplacian annihilates linear functions at interior vertices
    P, F, interior = _planar_grid()
    K = fem.cotan_stiffness(P, F)
    u = 0.7 * P[:, 0] - 1.3 * P[:, 1] + 0.2
    assert np.max(np.abs((K @ u)[interior])) < 1e-12


def test_stiffness_energy_of_linear_function():
    # u^T K u = integral |grad u|^2 = |g|^2 * area for u = g . x on a planar mesh
    P, F, _ = _planar_grid(seed=3)
    K = fem.cotan_stiffness(P, F)
    u = 2.0 * P[:, 0] + 0.5 * P[:, 1]
    assert np.isclose(u @ (K @ u), (4.0 + 0.25) * 1.0, rtol=1e-12)


def test_lumped_mass_total_area():
    P, F, _ = _planar_grid()
    assert np.isclose(fem.lumped_mass(P, F).sum(), 1.0, rtol=1e-13)
    # inscribed polyhedra converge to the sphere's area 4 pi at second order
    e = [4 * np.pi - fem.lumped_mass(*W.icosphere(lv)).sum() for lv in (3, 4)]
    assert 0 < e[1] < 0.02 and 3.8 < e[0] / e[1] < 4.2


def test_sphere_spectrum_and_orthonormality():
    V, F = W.icosphere(3)  # 642 vertices
    lam, Phi, Md, K = fem.laplace_beltrami_basis(V, F, 25)
    # M-orthonormal and a true generalized eigenbasis
    assert np.max(np.abs(Phi.T @ (Md[:, None] * Phi) - np.eye(25))) < 1e-10
    assert np.max(np.abs(K @ Phi - (Md[:, None] * Phi) * lam)) < 1e-9
    # eigenvalues approach l(l+1) with multiplicity 2l+1 (l = 0..4)
    ref = np.concatenate([[l * (l + 1)] * (2 * l + 1) for l in range(5)])
    assert abs(lam[0]) < 1e-10
    assert np.max(np.abs(lam - ref) / np.maximum(ref, 1)) < 0.03


def test_deformed_mesh_radius_range():
    V, F = W.deformed_icosphere(2)
    r = np.linalg.norm(V, axis=1)
    assert r.min() >= 0.8 - 1e-12 and r.max() <= 1.2 + 1e-12
    assert np.isclose(np.max(np.abs(r - 1)), 0.2)


def test_sliced_eigensolver_matches_dense():
    # the spectral slicing used for large meshes against dense LAPACK on meshes both handle: a
    # deformed icosphere (no symmetry) and the icosphere itself, whose exactly degenerate
    # clusters single-vector Lanczos finds completely only with the deflated re-search
    for (V, F), m, per_slice in ((W.deformed_icosphere(4), 300, 64), (W.icosphere(4), 100, 48)):
        K, Md = fem.cotan_stiffness(V, F), fem.lumped_mass(V, F)
        ld, Pd = fem.eigenpairs_dense(K, Md, m)
        ls, Ps = fem.eigenpairs_sliced(K, Md, m, per_slice=per_slice)
        assert np.max(np.abs(ls - ld) / np.maximum(ld, 1)) < 1e-10
        assert np.abs(Ps.T @ (Md[:, None] * Ps) - np.eye(m)).max() < 1e-10
        # the same invariant subspace (m sits at a gap of the spectrum in both cases)
        assert np.abs(Pd @ (Pd.T @ (Md[:, None] * Ps)) - Ps).max() < 1e-8
