"""Independent FP64 row-wise butterfly factorization and its apply (oracle; test only).

Follows Sec. 2 and Algorithm 1 of the paper in its notation:

* two complete binary trees of equal depth L: the space tree T_x on points (Sec. 3,
  Algorithm 2, Fiedler bisection) and the frequency tree T_lambda on modes in eigenvalue
  order (Sec. 3, first paragraph);
* level 0: for each frequency leaf nu, a low-rank factorization
  Phi(:, nu) = U_{:nu} V_{:nu}^*; here a column interpolative decomposition (ID)
  Phi(:, nu) ~= Phi(:, J_nu) T_nu with T_nu = [I | T~] P^T;
* levels l = 1..L: for tau at depth l with parent p and nu at height l with children
  c1, c2, the ID [U_{p c1}(tau,:)  U_{p c2}(tau,:)] = U_{tau nu} R_{tau nu}^*.  With nested
  IDs U_{p c}(tau, :) = Phi(tau, J_{p c}), so the block being skeletonized is
  Phi(tau, J_{p c1} u J_{p c2}) and R_{tau nu}^* = [I | T~] P^T;
* column bases U_{tau:} = Phi(tau, J_{tau, root}) for each space leaf tau.

Readings where the paper is silent (all listed in the design notes):
* ID by Householder QR with column pivoting; rank = #{k : |R_kk| > eps |R_11|};
  T~ = R_11^{-1} R_12 (the paper leaves the low-rank type free, Sec. 2);
* the apply runs leaf stage V, then transfers R for l = 1..L, then U; the adjoint runs the
  same stages transposed in reverse order (this follows from the algebra of Sec. 2; the
  order printed in the prose at the end of Sec. 2 matches only the adjoint);
* both trees are split to exactly depth L = max(0, ceil(log2(n / leaf_size)));
  empty space nodes are allowed;
* the frequency tree halves index ranges with floor(size/2) to the left child.

Blocks at level l are numbered tau-major: b = tau * 2^(L-l) + nu.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# --------------------------------------------------------------------------- trees

def tree_depth(n: int, leaf_size: int) -> int:
    """L = max(0, ceil(log2(n / leaf_size)))."""
    if n <= leaf_size:
        return 0
    return int(np.ceil(np.log2(n / leaf_size)))


def frequency_tree(eigenvalues: np.ndarray, L: int):
    """(mode_perm, mode_off): modes in stable eigenvalue order, leaf ranges at depth L."""
    lam = np.asarray(eigenvalues, dtype=np.float64)
    perm = np.argsort(lam, kind="stable").astype(np.int64)
    ranges = [(0, len(lam))]
    for _ in range(L):
        nxt = []
        for a, b in ranges:
            h = (b - a) // 2
            nxt += [(a, a + h), (a + h, b)]
        ranges = nxt
    off = np.array([a for a, _ in ranges] + [len(lam)], dtype=np.int64)
    return perm, off


def _knn_graph_fiedler(X: np.ndarray, knn: int = 10, seed: int = 0) -> np.ndarray:
    """Second eigenvector phi_2 of a heat-kernel kNN graph Laplacian on the points X.

    Mesh-free rule of Sec. 3: graph weights exp(-d^2 / t) on the symmetrized kNN graph with
    t = mean squared kNN distance; the normalized generalized problem
    (D - K) v = lambda D v (Sec. 7.3 form) is solved and v_2 returned.
    """
    n = len(X)
    k = min(knn, n - 1)
    d2 = np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=2) if n <= 2048 else None
    if d2 is not None:
        nbr = np.argsort(d2, axis=1)[:, 1:k + 1]
        dist2 = np.take_along_axis(d2, nbr, axis=1)
    else:
        from scipy.spatial import cKDTree
        dist, nbr = cKDTree(X).query(X, k + 1)
        nbr, dist2 = nbr[:, 1:], dist[:, 1:] ** 2
    t = max(float(np.mean(dist2)), 1e-300)
    rows = np.repeat(np.arange(n), k)
    W = sp.coo_matrix((np.exp(-dist2.ravel() / t), (rows, nbr.ravel())), shape=(n, n)).tocsr()
    W = W.maximum(W.T)
    deg = np.asarray(W.sum(axis=1)).ravel()
    deg = np.where(deg > 0, deg, 1.0)
    Dm = sp.diags(1.0 / np.sqrt(deg))
    S = Dm @ W @ Dm  # symmetric, top eigenvalue 1 with eigenvector sqrt(deg)
    if n <= 1500:
        w, V = np.linalg.eigh(S.toarray())
        psi = V[:, -2]
    else:
        rng = np.random.default_rng(seed)
        w, V = spla.eigsh(S, k=2, which="LA", v0=rng.standard_normal(n), tol=1e-8)
        psi = V[:, np.argsort(w)[0]]
    return psi / np.sqrt(deg)


def _split_fiedler(X: np.ndarray):
    """Boolean mask of M_1 = {phi_2 <= 0} for a point set (Algorithm 2, mesh-free rule)."""
    n = len(X)
    if n == 0:
        return np.zeros(0, dtype=bool)
    if n == 1:
        return np.ones(1, dtype=bool)
    if n == 2:
        return np.array([True, False])
    return _knn_graph_fiedler(X) <= 0.0


def _neumann_phi2(K: sp.spmatrix, Mdiag: np.ndarray) -> np.ndarray:
    """phi_2 of K phi = lambda M phi (Eq. neumann-eigenproblem discretized by P1 elements; the
    homogeneous Neumann condition is the natural one, so no boundary rows change).  Dense
    LAPACK for small sub-meshes, else shift-invert Lanczos just below 0 (K is singular)."""
    nv = K.shape[0]
    if nv <= 1500:
        lam, Phi = sla.eigh(K.toarray(), np.diag(Mdiag), subset_by_index=[0, 1])
        return Phi[:, 1]
    shift = -1e-8 * float(np.max(K.diagonal() / Mdiag))
    lam, Phi = spla.eigsh(K.tocsc(), k=2, M=sp.diags(Mdiag).tocsc(), sigma=shift, which="LM",
                          v0=np.random.default_rng(0).standard_normal(nv), tol=1e-10)
    return Phi[:, np.argsort(lam)[1]]


def _split_patches(V: np.ndarray, F: np.ndarray, tri_ids: np.ndarray, pts: np.ndarray):
    """Algorithm 2, patch rule (Sec. 3): the node's sub-mesh is its triangles F[tri_ids];
    phi_2 is its second Neumann eigenfunction (P1 cotangent stiffness, lumped mass);
    M_1 = {P : integral of phi_2 over P <= 0}, the P1 integral being area(P)/3 times the sum of
    the vertex values; a point (a mesh vertex) belongs to M_1 when it is a vertex of a triangle
    of M_1 (M_1 as a closed set of patches), else to M_2.

    Returns (mask over tri_ids, mask over pts).  Degenerate cases (no triangles, or every point
    on one side) split the points by order, first half to M_1.
    """
    from oracle import fem
    tri_ids = np.asarray(tri_ids, dtype=np.int64)
    pts = np.asarray(pts, dtype=np.int64)
    by_order = np.arange(len(pts)) < len(pts) // 2
    if len(tri_ids) == 0 or len(pts) == 0:
        return np.ones(len(tri_ids), dtype=bool), by_order
    verts, loc = np.unique(F[tri_ids], return_inverse=True)
    loc = loc.reshape(-1, 3)
    Vl = V[verts]
    phi2 = _neumann_phi2(fem.cotan_stiffness(Vl, loc), fem.lumped_mass(Vl, loc))
    integral = fem.triangle_areas(Vl, loc) / 3.0 * phi2[loc].sum(axis=1)
    tri_m1 = integral <= 0.0
    vert_m1 = np.zeros(len(verts), dtype=bool)
    vert_m1[loc[tri_m1].ravel()] = True
    pos = np.clip(np.searchsorted(verts, pts), 0, len(verts) - 1)
    pt_m1 = (verts[pos] == pts) & vert_m1[pos]
    if pt_m1.all() or not pt_m1.any():
        pt_m1 = by_order
    return tri_m1, pt_m1


def _split_rect(X: np.ndarray, box):
    """Flat square: exact Neumann Fiedler function of the node's rectangle.

    phi_2 = cos(pi (x - a) / w) along the longer side (ties: first coordinate), i.e. a
    midpoint cut; M_1 = {phi_2 <= 0}.  At the periodic root phi_2 = sin(x_1).
    Returns (mask, box1, box2).
    """
    if box is None:  # periodic root
        mask = np.sin(X[:, 0]) <= 0.0
        return mask, ((-np.pi, 0.0), (-np.pi, np.pi)), ((0.0, np.pi), (-np.pi, np.pi))
    (a1, b1), (a2, b2) = box
    if (b1 - a1) >= (b2 - a2):
        mid = 0.5 * (a1 + b1)
        mask = np.cos(np.pi * (X[:, 0] - a1) / (b1 - a1)) <= 0.0
        return mask, ((mid, b1), (a2, b2)), ((a1, mid), (a2, b2))
    mid = 0.5 * (a2 + b2)
    mask = np.cos(np.pi * (X[:, 1] - a2) / (b2 - a2)) <= 0.0
    return mask, ((a1, b1), (mid, b2)), ((a1, b1), (a2, mid))


def space_tree(points: np.ndarray, L: int, kind: str = "fiedler", tris: np.ndarray | None = None):
    """(space_perm, space_off): Fiedler bisection (Algorithm 2) to exactly depth L.

    kind = "fiedler" (kNN graph Laplacian, mesh-free rule), "rect" (flat periodic square,
    exact rectangle Fiedler functions) or "mesh" (patch rule on the triangle mesh ``tris``
    whose vertices are the points).  M_1 becomes the first child.
    """
    X = np.asarray(points, dtype=np.float64)
    if kind == "mesh":
        F = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
        nodes = [(np.arange(len(X), dtype=np.int64), np.arange(len(F), dtype=np.int64))]
    else:
        nodes = [(np.arange(len(X), dtype=np.int64), None)]
    for _ in range(L):
        nxt = []
        for idx, box in nodes:
            if kind == "mesh":
                tmask, mask = _split_patches(X, F, box, idx)
                b1, b2 = box[tmask], box[~tmask]
            elif kind == "rect":
                mask, b1, b2 = _split_rect(X[idx], box)
            else:
                mask, b1, b2 = _split_fiedler(X[idx]), None, None
            nxt += [(idx[mask], b1), (idx[~mask], b2)]
        nodes = nxt
    perm = np.concatenate([idx for idx, _ in nodes]) if nodes else np.zeros(0, np.int64)
    sizes = [len(idx) for idx, _ in nodes]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return perm.astype(np.int64), off


# ------------------------------------------------------------------------------ ID

def interpolative_decomposition(A: np.ndarray, eps: float):
    """Column ID A ~= A(:, skel) [I | T~] P^T by column-pivoted Householder QR.

    Returns (perm, T~) where perm lists the K local column indices with the r skeleton
    columns first (pivot order) and T~ = R_11^{-1} R_12 is r x (K - r).  The rank r counts
    pivots with |R_kk| > eps |R_11|.
    """
    M, K = A.shape
    if M == 0 or K == 0:
        return np.arange(K, dtype=np.int64), np.zeros((0, K), dtype=A.dtype)
    R, piv = sla.qr(A, mode="r", pivoting=True)
    d = np.abs(np.diag(R))
    if d[0] == 0.0:
        return piv.astype(np.int64), np.zeros((0, K), dtype=A.dtype)
    r = int(np.sum(d > eps * d[0]))
    T = sla.solve_triangular(R[:r, :r], R[:r, r:]) if r < K else np.zeros((r, 0), A.dtype)
    return piv.astype(np.int64), T


# ------------------------------------------------------------------- factorization

@dataclass
class Factorization:
    """Butterfly factors as plain arrays (the same content the library imports/exports).

    ranks[l][b], perms[l][b] (K ints, skeleton first) and T[l][b] (r x (K-r)) for levels
    l = 0..L; U[tau] (|tau| x r_L) for the space leaves.
    """
    L: int
    n: int
    m: int
    complex_: bool
    space_perm: np.ndarray
    space_off: np.ndarray
    mode_perm: np.ndarray
    mode_off: np.ndarray
    ranks: list = field(default_factory=list)
    perms: list = field(default_factory=list)
    T: list = field(default_factory=list)
    U: list = field(default_factory=list)

    def space_node(self, depth: int, i: int) -> np.ndarray:
        """Original point indices of space node i at the given depth."""
        w = 1 << (self.L - depth)
        return self.space_perm[self.space_off[i * w]:self.space_off[(i + 1) * w]]

    def stored_entries(self) -> int:
        """Entries of all T~ blocks plus all column bases (the applied data)."""
        e = sum(t.size for lv in self.T for t in lv)
        return e + sum(u.size for u in self.U)

    def block_input_size(self, l: int, b: int) -> int:
        nb = 1 << (self.L - l)
        tau, nu = divmod(b, nb)
        if l == 0:
            return int(self.mode_off[nu + 1] - self.mode_off[nu])
        p = tau >> 1
        q = p * (nb << 1) + 2 * nu
        return int(self.ranks[l - 1][q] + self.ranks[l - 1][q + 1])


def build(phi_eval, n: int, m: int, eigenvalues: np.ndarray, points: np.ndarray, eps: float,
          leaf_size: int, tree: str = "fiedler", complex_: bool = False,
          space=None) -> Factorization:
    """Algorithm 1: leaf IDs, then transfer IDs for l = 1..L, then column bases.

    ``phi_eval(rows, cols)`` returns Phi(rows, cols) in FP64 (original indices).
    ``space`` may give a prebuilt (space_perm, space_off) of depth L.
    """
    L = tree_depth(n, leaf_size)
    mode_perm, mode_off = frequency_tree(eigenvalues, L)
    if space is None:
        space_perm, space_off = space_tree(points, L, tree)
    else:
        space_perm, space_off = (np.asarray(a, dtype=np.int64) for a in space)
    F = Factorization(L, n, m, complex_, space_perm, space_off, mode_perm, mode_off)
    nblk = 1 << L
    all_rows = np.arange(n, dtype=np.int64)
    J_prev = []
    r0, p0, t0 = [], [], []
    for nu in range(nblk):
        cols = mode_perm[mode_off[nu]:mode_off[nu + 1]]
        A = phi_eval(all_rows, cols)
        perm, T = interpolative_decomposition(A, eps)
        r0.append(T.shape[0]); p0.append(perm); t0.append(T)
        J_prev.append(cols[perm[:T.shape[0]]])
    F.ranks.append(np.array(r0, dtype=np.int64)); F.perms.append(p0); F.T.append(t0)
    for l in range(1, L + 1):
        nb = 1 << (L - l)
        rl, pl, tl, J = [], [], [], []
        for tau in range(1 << l):
            p = tau >> 1
            rows = F.space_node(l, tau)
            for nu in range(nb):
                q = p * (nb << 1) + 2 * nu
                cand = np.concatenate([J_prev[q], J_prev[q + 1]])
                perm, T = interpolative_decomposition(phi_eval(rows, cand), eps)
                rl.append(T.shape[0]); pl.append(perm); tl.append(T)
                J.append(cand[perm[:T.shape[0]]])
        F.ranks.append(np.array(rl, dtype=np.int64)); F.perms.append(pl); F.T.append(tl)
        J_prev = J
    F.U = [phi_eval(F.space_node(L, tau), J_prev[tau]) for tau in range(nblk)]
    return F


def dense_evaluator(Phi: np.ndarray):
    """phi_eval for a dense matrix."""
    return lambda rows, cols: Phi[np.ix_(np.asarray(rows), np.asarray(cols))]


# -------------------------------------------------------------------------- apply

def _id_apply(perm, T, x):
    """y = [I | T~] P^T x = x(skel) + T~ x(rest)."""
    r = T.shape[0]
    return x[perm[:r]] + T @ x[perm[r:]]


def _id_apply_adjoint(perm, T, z, K):
    """u = P [I ; T~^H] z: u(skel) = z, u(rest) = T~^H z."""
    r = T.shape[0]
    u = np.zeros((K,) + z.shape[1:], dtype=np.result_type(T, z))
    u[perm[:r]] = z
    u[perm[r:]] = T.conj().T @ z
    return u


def synthesize(F: Factorization, c: np.ndarray) -> np.ndarray:
    """f = Phi_eps c: stage V (leaves), transfers R for l = 1..L, then U."""
    c = np.asarray(c)
    L, nblk = F.L, 1 << F.L
    y = []
    for nu in range(nblk):
        x = c[F.mode_perm[F.mode_off[nu]:F.mode_off[nu + 1]]]
        y.append(_id_apply(F.perms[0][nu], F.T[0][nu], x))
    for l in range(1, L + 1):
        nb = 1 << (L - l)
        ynew = []
        for tau in range(1 << l):
            p = tau >> 1
            for nu in range(nb):
                q = p * (nb << 1) + 2 * nu
                b = tau * nb + nu
                ynew.append(_id_apply(F.perms[l][b], F.T[l][b],
                                      np.concatenate([y[q], y[q + 1]])))
        y = ynew
    dt = np.result_type(c, *(u for u in F.U)) if F.U else c.dtype
    f = np.zeros((F.n,) + c.shape[1:], dtype=dt)
    for tau in range(nblk):
        f[F.space_node(L, tau)] = F.U[tau] @ y[tau]
    return f


def analyze(F: Factorization, f: np.ndarray, w: np.ndarray | None = None) -> np.ndarray:
    """c = Phi_eps^H diag(w) f: stages U^H, R^H for l = L..1, then V^H (leaves last)."""
    f = np.asarray(f)
    g = f if w is None else (w[:, None] * f if f.ndim == 2 else w * f)
    L, nblk = F.L, 1 << F.L
    z = [F.U[tau].conj().T @ g[F.space_node(L, tau)] for tau in range(nblk)]
    for l in range(L, 0, -1):
        nb = 1 << (L - l)
        npair = (1 << (l - 1)) * nb
        zprev = [None] * (2 * npair)
        for p in range(1 << (l - 1)):
            for nu in range(nb):
                q = p * (nb << 1) + 2 * nu
                r1 = int(F.ranks[l - 1][q])
                K = r1 + int(F.ranks[l - 1][q + 1])
                u = 0
                for s in (0, 1):
                    b = (2 * p + s) * nb + nu
                    u = u + _id_apply_adjoint(F.perms[l][b], F.T[l][b], z[b], K)
                zprev[q], zprev[q + 1] = u[:r1], u[r1:]
        z = zprev
    dt = np.result_type(g, *(t for t in F.T[0])) if F.T[0] else g.dtype
    c = np.zeros((F.m,) + g.shape[1:], dtype=dt)
    for nu in range(nblk):
        K = int(F.mode_off[nu + 1] - F.mode_off[nu])
        c[F.mode_perm[F.mode_off[nu]:F.mode_off[nu + 1]]] = _id_apply_adjoint(
            F.perms[0][nu], F.T[0][nu], z[nu], K)
    return c


def to_dense(F: Factorization) -> np.ndarray:
    """Phi_eps as a dense matrix (columns = synthesize of unit vectors); tiny cases only."""
    dt = np.complex128 if F.complex_ else np.float64
    return synthesize(F, np.eye(F.m, dtype=dt))
