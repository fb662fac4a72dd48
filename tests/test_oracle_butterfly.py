"""Pins for oracle/butterfly.py: brute force, exact low rank, the paper's error claim, adjoints."""
import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from oracle import dense as D
from oracle import harmonics as H


def test_id_recovers_exact_rank_and_reconstructs():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((60, 7)) @ rng.standard_normal((7, 40))
    perm, T = B.interpolative_decomposition(A, 1e-12)
    r = T.shape[0]
    assert r == 7
    assert sorted(perm.tolist()) == list(range(40))
    R = np.zeros((r, 40)); R[:, perm[:r]] = np.eye(r); R[:, perm[r:]] = T
    assert np.linalg.norm(A - A[:, perm[:r]] @ R) < 1e-10 * np.linalg.norm(A)


def test_id_error_tracks_tolerance():
    rng = np.random.default_rng(1)
    U, _ = np.linalg.qr(rng.standard_normal((80, 50)))
    V, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    A = (U * np.logspace(0, -12, 50)) @ V.T
    for eps in (1e-3, 1e-6, 1e-9):
        perm, T = B.interpolative_decomposition(A, eps)
        r = T.shape[0]
        approx = A[:, perm[:r]] @ np.hstack([np.eye(r), T])
        err = np.linalg.norm(A[:, perm] - approx, 2) / np.linalg.norm(A, 2)
        assert err < 100 * eps
        expected = int(np.sum(np.logspace(0, -12, 50) > eps))
        assert abs(r - expected) <= 3


def test_id_complex_and_degenerate():
    rng = np.random.default_rng(2)
    A = (rng.standard_normal((30, 5)) + 1j * rng.standard_normal((30, 5))) @ \
        (rng.standard_normal((5, 12)) + 1j * rng.standard_normal((5, 12)))
    perm, T = B.interpolative_decomposition(A, 1e-12)
    r = T.shape[0]
    assert r == 5
    assert np.allclose(A[:, perm[:r]] @ np.hstack([np.eye(r), T]), A[:, perm], atol=1e-10)
    perm, T = B.interpolative_decomposition(np.zeros((4, 3)), 1e-6)
    assert T.shape == (0, 3)
    perm, T = B.interpolative_decomposition(np.zeros((0, 3)), 1e-6)
    assert T.shape == (0, 3)


def test_frequency_tree_halves_in_eigenvalue_order():
    lam = np.array([5.0, 1.0, 1.0, 0.0, 9.0, 2.0, 2.0])
    perm, off = B.frequency_tree(lam, 2)
    assert perm.tolist() == [3, 1, 2, 5, 6, 0, 4]  # stable sort, ties by index
    assert off.tolist() == [0, 1, 3, 5, 7]          # floor(size/2) to the left


def test_space_tree_rect_uniform_grid_equal_boxes():
    X = W.uniform_grid_points(16) + 1e-9
    perm, off = B.space_tree(X, 4, "rect")
    assert sorted(perm.tolist()) == list(range(256))
    assert np.all(np.diff(off) == 16)
    # every leaf is a 4x4 block of grid points: bounding boxes of side 3 * 2 pi / 16
    for i in range(16):
        P = X[perm[off[i]:off[i + 1]]]
        assert np.allclose(np.ptp(P, axis=0), 3 * 2 * np.pi / 16)


def test_space_tree_fiedler_separates_clusters():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 3)) * 0.1
    Bc = rng.standard_normal((40, 3)) * 0.1 + np.array([5.0, 0, 0])
    X = np.vstack([A, Bc])
    perm, off = B.space_tree(X, 1, "fiedler")
    left = set(perm[off[0]:off[1]].tolist())
    assert left == set(range(40)) or left == set(range(40, 80))


def _segment_points(n, seed=0):
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 10.0, n)
    return x, np.stack([x, 1e-3 * rng.standard_normal(n), 1e-3 * rng.standard_normal(n)], axis=1)


def _assert_quarters(x, perm, off):
    # Algorithm 2 on evenly spaced points of a segment: the graph is a uniform path, whose
    # Fiedler vector is monotone and changes sign at the middle, and each half is again a
    # path with free ends, so depth 2 gives four equal, contiguous quarters
    n = len(x)
    assert np.array_equal(np.diff(off), [n // 4] * 4)
    spans = sorted((x[perm[off[i]:off[i + 1]]].min(), x[perm[off[i]:off[i + 1]]].max()) for i in range(4))
    for q, (lo, hi) in enumerate(spans):
        assert np.isclose(lo, x[q * n // 4]) and np.isclose(hi, x[(q + 1) * n // 4 - 1])


@pytest.mark.parametrize("n", [64, 100])
def test_space_tree_fiedler_bisects_a_segment(n):
    x, X = _segment_points(n)
    perm, off = B.space_tree(X, 2, "fiedler")
    _assert_quarters(x, perm, off)


def test_space_tree_depth_and_nesting():
    X = W.fibonacci_points(300, seed=1)
    perm, off = B.space_tree(X, 3, "fiedler")
    assert sorted(perm.tolist()) == list(range(300))
    assert len(off) == 9 and off[0] == 0 and off[-1] == 300 and np.all(np.diff(off) >= 0)


@pytest.mark.parametrize("kind", ["sphere", "torus"])
def test_exact_factorization_on_tiny_inputs(kind):
    # with eps at rounding level the butterfly is the dense matrix (brute force)
    if kind == "sphere":
        n, lmax = 64, 7
        X = W.fibonacci_points(n)
        Phi = H.sphere_phi(X, lmax); lam = W.sphere_eigenvalues(Phi.shape[1]); tree = "fiedler"
    else:
        n = 64
        X = W.torus_points(n); K = W.torus_modes(64)
        Phi = H.torus_phi(X, K); lam = W.torus_eigenvalues(K); tree = "rect"
    F = B.build(B.dense_evaluator(Phi), n, Phi.shape[1], lam, X, 1e-15, 16, tree,
                complex_=(kind == "torus"))
    assert F.L == 2
    assert np.max(np.abs(B.to_dense(F) - Phi)) < 1e-10 * np.max(np.abs(Phi))


def test_level_zero_is_one_interpolative_decomposition():
    X = W.fibonacci_points(40)
    Phi = H.sphere_phi(X, 5)
    F = B.build(B.dense_evaluator(Phi), 40, 36, W.sphere_eigenvalues(36), X, 1e-13, 64)
    assert F.L == 0 and len(F.T) == 1 and len(F.U) == 1
    assert np.allclose(B.to_dense(F), Phi, atol=1e-10)


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_error_agrees_with_tolerance_torus(eps):
    # Sec. 6.1: relative l2 matvec error on a Gaussian vector is about eps
    n = m = 576
    X = W.torus_points(n); K = W.torus_modes(m); Phi = H.torus_phi(X, K)
    F = B.build(B.dense_evaluator(Phi), n, m, W.torus_eigenvalues(K), X, eps, 36, "rect",
                complex_=True)
    c = W.gaussian(m, 1, True)
    err = np.linalg.norm(B.synthesize(F, c) - Phi @ c) / np.linalg.norm(Phi @ c)
    assert eps / 1000 < err < 10 * eps


def test_error_agrees_with_tolerance_sphere_weighted_adjoint():
    n = 1024
    X = W.fibonacci_points(n); Phi = H.sphere_phi(X, 31)
    m = Phi.shape[1]
    F = B.build(B.dense_evaluator(Phi), n, m, W.sphere_eigenvalues(m), X, 1e-6, 64)
    c = W.sphere_coefficients(m)[:, 0]
    assert np.linalg.norm(B.synthesize(F, c) - Phi @ c) / np.linalg.norm(Phi @ c) < 1e-5
    w = np.full(n, 4 * np.pi / n); g = W.gaussian(n, 5)
    ref = D.analyze(Phi, g, w)
    assert np.linalg.norm(B.analyze(F, g, w) - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("complex_", [False, True])
def test_adjoint_is_conjugate_transpose(complex_):
    n = 256
    if complex_:
        X = W.torus_points(n); K = W.torus_modes(256); Phi = H.torus_phi(X, K)
        F = B.build(B.dense_evaluator(Phi), n, 256, W.torus_eigenvalues(K), X, 1e-4, 32,
                    "rect", complex_=True)
    else:
        X = W.fibonacci_points(n); Phi = H.sphere_phi(X, 15)
        F = B.build(B.dense_evaluator(Phi), n, 256, W.sphere_eigenvalues(256), X, 1e-4, 32)
    M = B.to_dense(F)
    g = W.gaussian(n, 6, complex_)
    w = W.gaussian(n, 7) ** 2
    assert np.allclose(B.analyze(F, g, w), M.conj().T @ (w * g), atol=1e-12 * np.abs(M).max() * n)
    c = W.gaussian(256, 8, complex_)
    lhs = np.vdot(B.synthesize(F, c), g)
    rhs = np.vdot(c, B.analyze(F, g))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs) * 100


def test_multiple_right_hand_sides_are_columnwise():
    n = 256
    X = W.fibonacci_points(n); Phi = H.sphere_phi(X, 15)
    F = B.build(B.dense_evaluator(Phi), n, 256, W.sphere_eigenvalues(256), X, 1e-6, 32)
    C = W.gaussian_columns(256, 3, 11)
    Fm = B.synthesize(F, C)
    for j in range(3):
        assert np.allclose(Fm[:, j], B.synthesize(F, C[:, j]))


def _figure_blocks():
    """Blocks of Fig. BF-levels (Sec. 2), transcribed in tests/golden/bf_levels_L3.txt."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bf_levels_L3.txt")
    rows = [tuple(int(v) for v in ln.split()) for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return {lv: {r[1:] for r in rows if r[0] == lv} for lv in range(4)}


def _expected_rank_for(blocks, L, l, tau, nu, sx, sw):
    # block (tau, nu) at level l: space node at depth l, frequency node at height l (leaf units)
    key = (nu << l, (nu + 1) << l, tau << (L - l), (tau + 1) << (L - l))
    assert key in blocks, f"level {l} block (tau={tau}, nu={nu}) is not one the figure draws"
    fl, fh, sl, sh = key
    return min((sh - sl) * sx, (fh - fl) * sw)


def test_level_structure_matches_the_papers_figure():
    G = _figure_blocks()
    for lv, blocks in G.items():  # every level tiles the 8 x 8 leaf grid with 8 equal blocks
        cover = np.zeros((8, 8), dtype=int)
        for fl, fh, sl, sh in blocks:
            cover[sl:sh, fl:fh] += 1
        assert len(blocks) == 8 and (cover == 1).all()
        assert len({(fh - fl) * (sh - sl) for fl, fh, sl, sh in blocks}) == 1
    # a Gaussian Phi with unequal leaf sizes (n = 8 * 32 points, m = 8 * 8 modes): the ID rank of
    # every block is min(|tau|, |nu|), which tells which space node meets which frequency node
    sx, sw, L = 32, 8, 3
    n, m = 8 * sx, 8 * sw
    Phi = np.random.default_rng(7).standard_normal((n, m))
    space = (np.arange(n), np.arange(0, n + 1, sx))
    F = B.build(B.dense_evaluator(Phi), n, m, np.arange(m, dtype=float), np.zeros((n, 3)), 1e-12, sx,
                space=space)
    assert F.L == L
    for l in range(L + 1):
        nb = 1 << (L - l)
        for tau in range(1 << l):
            for nu in range(nb):
                assert F.ranks[l][tau * nb + nu] == _expected_rank_for(G[l], L, l, tau, nu, sx, sw)
