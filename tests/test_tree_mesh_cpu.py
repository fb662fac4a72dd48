"""Algorithm 2's patch rule on triangle meshes (Sec. 3, Eq. neumann-eigenproblem).

Pins of the oracle against closed forms, and the library's tree against the oracle's:
  * phi_2 of the P1 Neumann problem on a 4 x 1 rectangle is the first Neumann mode
    cos(pi x / 4) (eigenvalue (pi / 4)^2);
  * the patch rule cuts that rectangle along its nodal line x = 2: triangles by the sign of the
    integral of phi_2, and the points of the closed patch set M_1 (the line itself included)
    on M_1's side;
  * two levels give the four unit strips (the 2 x 1 halves again have a simple phi_2);
  * the library (MHT_TREE_FIEDLER_MESH, Lanczos on the shifted FEM operator) builds the same
    leaves as the oracle (dense / shift-invert eigensolver).
"""
import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from oracle import fem

A, NX, NY = 4.0, 16, 4


@pytest.fixture(scope="module")
def rect():
    V, F = W.criss_cross_rectangle(A, 1.0, NX, NY)
    return V, F


def test_oracle_phi2_is_the_first_neumann_mode_of_the_rectangle(rect):
    V, F = rect
    K, M = fem.cotan_stiffness(V, F), fem.lumped_mass(V, F)
    phi = B._neumann_phi2(K, M)
    ref = np.cos(np.pi * V[:, 0] / A)
    corr = abs(np.sum(M * phi * ref)) / np.sqrt(np.sum(M * phi ** 2) * np.sum(M * ref ** 2))
    assert corr > 0.999
    lam = phi @ (K @ phi) / np.sum(M * phi ** 2)
    assert abs(lam - (np.pi / A) ** 2) < 0.02 * (np.pi / A) ** 2


def test_oracle_patch_rule_cuts_the_rectangle_along_its_nodal_line(rect):
    V, F = rect
    tri_m1, pt_m1 = B._split_patches(V, F, np.arange(len(F)), np.arange(len(V)))
    cx = V[F].mean(axis=1)[:, 0]
    x = V[:, 0]
    left = cx < A / 2
    assert tri_m1.sum() == len(F) // 2
    assert np.array_equal(tri_m1, left) or np.array_equal(tri_m1, ~left)
    if np.array_equal(tri_m1, left):  # M_1 closed: the nodal line goes with it
        assert np.array_equal(pt_m1, x <= A / 2 + 1e-12)
    else:
        assert np.array_equal(pt_m1, x >= A / 2 - 1e-12)


def test_oracle_patch_tree_two_levels_gives_the_unit_strips(rect):
    V, F = rect
    perm, off = B.space_tree(V, 2, kind="mesh", tris=F)
    assert sorted(perm.tolist()) == list(range(len(V)))
    for k in range(4):
        xs = V[perm[off[k]:off[k + 1]], 0]
        assert xs.max() - xs.min() <= 1.0 + 1e-12  # one closed strip [j, j + 1]
        assert np.floor(xs.min() + 1e-9) == np.floor(xs.max() - 1e-9) or xs.max() - xs.min() <= 1.0


def _plan(V, F, levels, tree, tris=None):
    from paper_2605_21828_gb300 import Plan
    K, M = fem.cotan_stiffness(V, F), fem.lumped_mass(V, F)
    lam, Phi = fem.eigenpairs_dense(K, M, 48)
    return Plan.build(n=len(V), m=48, eigenvalues=lam, evaluator="dense", dense=Phi, points=V,
                      tris=F if tris is None else tris, eps=1e-6, levels=levels, tree=tree)


@pytest.mark.parametrize("tree", ["mesh", "auto"])
def test_library_patch_tree_matches_the_oracle(mht_lib, rect, tree):
    V, F = rect
    E = _plan(V, F, 2, tree).export()
    perm, off = E["space_perm"], E["space_offsets"]
    po, oo = B.space_tree(V, 2, kind="mesh", tris=F)
    lib = {frozenset(perm[off[k]:off[k + 1]].tolist()) for k in range(4)}
    ora = {frozenset(po[oo[k]:oo[k + 1]].tolist()) for k in range(4)}
    assert lib == ora


def test_library_mesh_tree_rejects_bad_input(mht_lib, rect):
    from paper_2605_21828_gb300 import Plan
    from paper_2605_21828_gb300._lib import MhtError
    V, F = rect
    Fbad = F.copy()
    Fbad[3, 1] = len(V)
    with pytest.raises(MhtError, match="INVALID_ARG"):
        _plan(V, F, 2, "mesh", tris=Fbad)
    K, M = fem.cotan_stiffness(V, F), fem.lumped_mass(V, F)
    lam, Phi = fem.eigenpairs_dense(K, M, 8)
    with pytest.raises(MhtError, match="INVALID_ARG"):
        Plan.build(n=len(V), m=8, eigenvalues=lam, evaluator="dense", dense=Phi, points=V, eps=1e-6,
                   levels=1, tree="mesh")
