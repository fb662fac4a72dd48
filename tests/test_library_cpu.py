"""CPU tests of libmht: exported symbols, the FP64 host build, import/export, persistence
and argument checking.  No compute call here touches a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from oracle import dense as D
from oracle import fem
from oracle import harmonics as H
from tests._bridge import arrays_to_oracle, oracle_to_arrays

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _plan_cls():
    from paper_2605_21828_gb300 import Plan
    return Plan


def test_library_exports_every_declared_symbol(mht_lib):
    hdr = open(os.path.join(ROOT, "include", "mht.h")).read()
    declared = set(re.findall(r"^\s*(?:mht_status|const char\*)\s+(mht_[a-z0-9_]+)\s*\(", hdr, re.M))
    assert len(declared) >= 18
    for name in sorted(declared):
        assert hasattr(mht_lib, name), name
    from paper_2605_21828_gb300 import _lib
    assert declared == set(_lib.SIGNATURES)


def _sphere(n, lmax):
    X = W.fibonacci_points(n)
    Phi = H.sphere_phi(X, lmax)
    return X, Phi, W.sphere_eigenvalues(Phi.shape[1])


@pytest.mark.parametrize("tree", ["fiedler", "pca"])
@pytest.mark.parametrize("oversample", [0.0, 2.0])
def test_host_build_sphere_matches_dense(mht_lib, tree, oversample):
    n, eps = 1024, 1e-6
    X, Phi, lam = _sphere(n, 31)
    w = np.full(n, 4 * np.pi / n)
    p = _plan_cls().build(n=n, m=Phi.shape[1], eigenvalues=lam, evaluator="sphere", points=X,
                          eps=eps, leaf_size=64, tree=tree, oversample=oversample, weights=w)
    F = arrays_to_oracle(p.export())
    assert F.L == 4
    c = W.sphere_coefficients(Phi.shape[1])[:, 0]
    ref = Phi @ c
    assert np.linalg.norm(B.synthesize(F, c) - ref) / np.linalg.norm(ref) < 10 * eps
    g = W.gaussian(n, 3)
    refa = D.analyze(Phi, g, w)
    assert np.linalg.norm(B.analyze(F, g, w) - refa) / np.linalg.norm(refa) < 10 * eps


def test_host_build_torus_matches_nudft(mht_lib):
    n = m = 1024
    eps = 1e-10
    X = W.torus_points(n)
    K = W.torus_modes(m)
    Phi = H.torus_phi(X, K)
    p = _plan_cls().build(n=n, m=m, eigenvalues=W.torus_eigenvalues(K), evaluator="torus",
                          points=X, torus_modes=K, eps=eps, leaf_size=64, mode="fp64")
    d = p.export()
    assert d["complex"]
    F = arrays_to_oracle(d)
    c = W.gaussian(m, 1, True)
    ref = Phi @ c
    assert np.linalg.norm(B.synthesize(F, c) - ref) / np.linalg.norm(ref) < 10 * eps
    g = W.gaussian(n, 2, True)
    refa = Phi.conj().T @ g
    assert np.linalg.norm(B.analyze(F, g) - refa) / np.linalg.norm(refa) < 10 * eps


def test_rect_tree_and_frequency_tree_match_oracle(mht_lib):
    n = m = 1024
    X = W.torus_points(n, seed=4)
    K = W.torus_modes(m)
    lam = W.torus_eigenvalues(K)
    p = _plan_cls().build(n=n, m=m, eigenvalues=lam, evaluator="torus", points=X, torus_modes=K,
                          eps=1e-4, leaf_size=64, tree="rect")
    d = p.export()
    sp, so = B.space_tree(X, p.levels, "rect")
    mp, mo = B.frequency_tree(lam, p.levels)
    assert np.array_equal(d["mode_perm"], mp) and np.array_equal(d["mode_offsets"], mo)
    assert np.array_equal(d["space_offsets"], so)
    for t in range(len(so) - 1):
        assert set(d["space_perm"][so[t]:so[t + 1]]) == set(sp[so[t]:so[t + 1]])


def test_fiedler_tree_separates_clusters(mht_lib):
    rng = np.random.default_rng(3)
    X = np.vstack([rng.standard_normal((40, 3)) * 0.1, rng.standard_normal((40, 3)) * 0.1 + [5, 0, 0]])
    lam = np.arange(80.0)
    Phi = rng.standard_normal((80, 80))
    p = _plan_cls().build(n=80, m=80, eigenvalues=lam, evaluator="dense", dense=Phi, points=X,
                          eps=1e-8, levels=1, tree="fiedler")
    d = p.export()
    left = set(d["space_perm"][:d["space_offsets"][1]].tolist())
    assert left in (set(range(40)), set(range(40, 80)))


def test_library_evaluator_matches_the_oracle_harmonics(mht_lib):
    # the entries the build factors: real spherical harmonics up to degree 255 (every order, so
    # the order-to-order recurrences of the library's evaluator are all exercised) and complex
    # exponentials, against the oracle's independent closed forms (themselves pinned to scipy
    # and the FFT)
    from paper_2605_21828_gb300 import MhtError, phi_entries
    X = W.fibonacci_points(300, seed=4)
    P = H.sphere_phi(X, 255)
    Q = phi_entries(np.arange(300), np.arange(65536), n=300, m=65536, evaluator="sphere", points=X)
    assert np.abs(Q - P).max() < 1e-12
    rng = np.random.default_rng(1)
    rows, cols = rng.permutation(300)[:200], rng.choice(65536, 5000, replace=False)  # gaps, any order
    Q2 = phi_entries(rows, cols, n=300, m=65536, evaluator="sphere", points=X)
    assert np.abs(Q2 - P[np.ix_(rows, cols)]).max() < 1e-12
    Xt, K = W.torus_points(500), W.torus_modes(4096)
    Qt = phi_entries(np.arange(500), np.arange(4096), n=500, m=4096, evaluator="torus", points=Xt, torus_modes=K)
    assert Qt.dtype == np.complex128 and np.abs(Qt - H.torus_phi(Xt, K)).max() < 1e-12
    with pytest.raises(MhtError, match="INVALID_ARG"):
        phi_entries([300], [0], n=300, m=65536, evaluator="sphere", points=X)
    with pytest.raises(MhtError, match="INVALID_ARG"):
        phi_entries([0], [65536], n=300, m=65536, evaluator="sphere", points=X)


def test_import_export_roundtrip(mht_lib):
    n = 256
    X, Phi, lam = _sphere(n, 15)
    F = B.build(B.dense_evaluator(Phi), n, 256, lam, X, 1e-6, 32)
    arr = oracle_to_arrays(F)
    p = _plan_cls().from_factors(arr, mode="fp64")
    back = p.export()
    for key in ("space_perm", "space_offsets", "mode_perm", "mode_offsets", "ranks", "local_perm"):
        assert np.array_equal(np.asarray(back[key]), np.asarray(arr[key])), key
    assert np.array_equal(back["transfer"], arr["transfer"])
    assert np.array_equal(back["column_bases"], arr["column_bases"])
    info = p.info()
    assert info["stored_entries"] == F.stored_entries()
    assert sum(p.level_info(l)["transfer_entries"] for l in range(p.levels + 2)) == F.stored_entries()


def test_import_rejects_inconsistent_factors(mht_lib):
    from paper_2605_21828_gb300 import MhtError
    n = 128
    X, Phi, lam = _sphere(n, 11)
    F = B.build(B.dense_evaluator(Phi), n, 144, lam, X, 1e-6, 32)
    arr = oracle_to_arrays(F)
    bad = dict(arr)
    bad["local_perm"] = arr["local_perm"].copy()
    bad["local_perm"][0] = bad["local_perm"][1]  # not a permutation
    with pytest.raises(MhtError, match="FORMAT"):
        _plan_cls().from_factors(bad)
    bad = dict(arr)
    bad["space_perm"] = arr["space_perm"].copy()
    bad["space_perm"][0] = bad["space_perm"][1]
    with pytest.raises(MhtError, match="FORMAT"):
        _plan_cls().from_factors(bad)


def test_save_load_roundtrip_and_corruption(mht_lib, tmp_path):
    from paper_2605_21828_gb300 import MhtError
    n = 512
    X, Phi, lam = _sphere(n, 21)
    m = 484
    p = _plan_cls().build(n=n, m=m, eigenvalues=lam[:m], evaluator="dense", dense=Phi[:, :m],
                          points=X, eps=1e-7, leaf_size=64, weights=np.full(n, 2.0))
    path = str(tmp_path / "plan.bin")
    p.save(path)
    q = _plan_cls().load(path, mode="fp64")
    a, b = p.export(), q.export()
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(a[k], b[k]), k
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    bad = str(tmp_path / "bad.bin")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(MhtError, match="FORMAT"):
        _plan_cls().load(bad)
    open(bad, "wb").write(bytes(raw[:50]))
    with pytest.raises(MhtError, match="FORMAT"):
        _plan_cls().load(bad)
    open(bad, "wb").write(b"not a plan file at all........")
    with pytest.raises(MhtError, match="FORMAT"):
        _plan_cls().load(bad)


def test_callback_evaluator_equals_dense_and_propagates_errors(mht_lib):
    from paper_2605_21828_gb300 import MhtError
    n = 256
    X, Phi, lam = _sphere(n, 15)
    kw = dict(n=n, m=256, eigenvalues=lam, points=X, eps=1e-6, leaf_size=32, oversample=0)
    a = _plan_cls().build(evaluator="dense", dense=Phi, **kw).export()
    b = _plan_cls().build(evaluator="callback", callback=lambda r, c: Phi[np.ix_(r, c)], **kw).export()
    assert np.array_equal(a["ranks"], b["ranks"]) and np.array_equal(a["transfer"], b["transfer"])

    def broken(r, c):
        raise RuntimeError("evaluator failure")

    with pytest.raises(MhtError, match="CALLBACK"):
        _plan_cls().build(evaluator="callback", callback=broken, **kw)


def test_invalid_arguments_and_unbound_apply(mht_lib):
    from paper_2605_21828_gb300 import MhtError, _lib
    n = 64
    X, Phi, lam = _sphere(n, 7)
    with pytest.raises(MhtError, match="INVALID_ARG"):
        _plan_cls().build(n=n, m=64, eigenvalues=lam, evaluator="sphere", points=X, eps=2.0)
    with pytest.raises(MhtError, match="INVALID_ARG"):
        _plan_cls().build(n=n, m=64, eigenvalues=lam, evaluator="torus", points=X, eps=1e-6)
    bad = lam.copy()
    bad[3] = np.nan
    with pytest.raises(MhtError, match="NUMERIC"):
        _plan_cls().build(n=n, m=64, eigenvalues=bad, evaluator="sphere", points=X, eps=1e-6)
    p = _plan_cls().build(n=n, m=64, eigenvalues=lam, evaluator="sphere", points=X, eps=1e-6, leaf_size=16)
    lib = _lib.load()
    dummy = C.c_void_p(256)
    st = lib.mht_synthesize(p._h, dummy, 64, dummy, 64, 1, None)
    assert st == 9 and b"bound" in lib.mht_last_error()
    st = lib.mht_plan_bind_device(p._h, C.c_void_p(0), 0, C.c_void_p(0), 0, 1, None)
    assert st == 1
    st = lib.mht_plan_bind_device(p._h, C.c_void_p(256), 16, C.c_void_p(512), 16, 1, None)
    assert st == 2  # buffers too small: rejected before any device call


def test_fem_dense_build_and_analysis_inverts_synthesis(mht_lib):
    V, F_ = W.deformed_icosphere(3)
    lam, Phi, Md, K = fem.laplace_beltrami_basis(V, F_, 160)
    n = len(V)
    eps = 1e-8
    p = _plan_cls().build(n=n, m=160, eigenvalues=lam, evaluator="dense", dense=Phi, points=V,
                          eps=eps, leaf_size=64, weights=Md)
    F = arrays_to_oracle(p.export())
    c = W.gaussian(160, 5)
    f = B.synthesize(F, c)
    assert np.linalg.norm(f - Phi @ c) / np.linalg.norm(Phi @ c) < 10 * eps
    # Phi^T M Phi = I, so analysis (weights = lumped mass) undoes synthesis
    c2 = B.analyze(F, f, Md)
    assert np.linalg.norm(c2 - c) / np.linalg.norm(c) < 1e-6


def test_blocked_randomized_pivoting_id_matches_dense(mht_lib):
    # the block-pivoted ID (HQRRP) must keep the paper's accuracy: error about eps
    n, eps = 4096, 1e-6
    X, Phi, lam = _sphere(n, 63)
    errs = {}
    for meth in ("blocked", "classical"):
        p = _plan_cls().build(n=n, m=Phi.shape[1], eigenvalues=lam, evaluator="sphere", points=X, eps=eps,
                              leaf_size=128, id_method=meth)
        F = arrays_to_oracle(p.export())
        c = W.sphere_coefficients(Phi.shape[1])[:, 0]
        ref = Phi @ c
        errs[meth] = np.linalg.norm(B.synthesize(F, c) - ref) / np.linalg.norm(ref)
        g = W.gaussian(n, 3)
        refa = Phi.T @ g
        assert np.linalg.norm(B.analyze(F, g) - refa) / np.linalg.norm(refa) < 10 * eps
    assert errs["blocked"] < 10 * eps and errs["classical"] < 10 * eps


def test_blocked_complex_id_matches_dense(mht_lib):
    # complex Phi (flat torus): the block-pivoted complex ID and the Gram full-rank certificate
    # (leaf blocks with M >= 16 K) keep the accuracy and the ranks of the classical QRCP
    n, eps = 2304, 1e-6
    K, X = W.torus_modes(n), W.torus_points(n)
    Phi = H.torus_phi(X, K)
    ranks = {}
    for meth in ("blocked", "classical"):
        p = _plan_cls().build(n=n, m=n, eigenvalues=W.torus_eigenvalues(K), evaluator="torus", points=X,
                              torus_modes=K, eps=eps, leaf_size=32, id_method=meth)
        F = arrays_to_oracle(p.export())
        ranks[meth] = int(np.sum(p.export()["ranks"]))
        c = W.gaussian(n, 3, complex_=True)
        ref = Phi @ c
        assert np.linalg.norm(B.synthesize(F, c) - ref) / np.linalg.norm(ref) < 10 * eps, meth
        g = W.gaussian(n, 4, complex_=True)
        refa = Phi.conj().T @ g
        assert np.linalg.norm(B.analyze(F, g) - refa) / np.linalg.norm(refa) < 10 * eps, meth
    assert abs(ranks["blocked"] - ranks["classical"]) <= 0.01 * ranks["classical"]


def test_ranks_match_the_oracle_build_on_the_same_trees(mht_lib):
    # the library's build against the oracle's independent build (scipy pivoted QR) of the
    # same blocks: same space tree (handed in), same frequency order, same rank rule
    X = W.fibonacci_points(1024)
    Phi = H.sphere_phi(X, 31)
    lam = W.sphere_eigenvalues(1024)
    F = B.build(B.dense_evaluator(Phi), 1024, 1024, lam, X, 1e-6, 64)
    p = _plan_cls().build(n=1024, m=1024, eigenvalues=lam, evaluator="sphere", points=X, eps=1e-6, leaf_size=64,
                          space=(F.space_perm, F.space_off), id_method="classical")
    e = p.export()
    assert np.array_equal(e["mode_perm"], F.mode_perm)
    lib = np.asarray(e["ranks"]).reshape(F.L + 1, -1)
    assert np.array_equal(lib, np.array([np.asarray(r) for r in F.ranks]))  # block by block
    # complex exponentials all have the same column norm, so the first pivot of every block is
    # a tie that rounding decides; ranks may then differ by a column or two per block
    Xt, K = W.torus_points(1024), W.torus_modes(1024)
    lt = W.torus_eigenvalues(K)
    Ft = B.build(B.dense_evaluator(H.torus_phi(Xt, K)), 1024, 1024, lt, Xt, 1e-8, 64, "rect", complex_=True)
    for meth in ("classical", "blocked"):
        pt = _plan_cls().build(n=1024, m=1024, eigenvalues=lt, evaluator="torus", points=Xt, torus_modes=K, eps=1e-8,
                               leaf_size=64, space=(Ft.space_perm, Ft.space_off), id_method=meth)
        lib = np.asarray(pt.export()["ranks"]).reshape(Ft.L + 1, -1)
        ora = np.array([np.asarray(r) for r in Ft.ranks])
        assert np.abs(lib - ora).max() <= 2, meth
        assert np.all(np.abs(lib.sum(axis=1) - ora.sum(axis=1)) <= 0.005 * ora.sum(axis=1)), meth


def test_library_level_structure_matches_the_papers_figure(mht_lib):
    # Fig. BF-levels (Sec. 2, tests/golden/bf_levels_L3.txt): at level l the library factors the
    # block of the space node at depth l and the frequency node at height l; with a Gaussian
    # Phi and unequal leaf sizes every block's ID rank is min(|tau|, |nu|)
    from tests.test_oracle_butterfly import _expected_rank_for, _figure_blocks
    G = _figure_blocks()
    sx, sw, L = 32, 8, 3
    n, m = 8 * sx, 8 * sw
    Phi = np.random.default_rng(7).standard_normal((n, m))
    p = _plan_cls().build(n=n, m=m, eigenvalues=np.arange(m, dtype=float), evaluator="dense", dense=Phi,
                          eps=1e-12, leaf_size=sx, space=(np.arange(n), np.arange(0, n + 1, sx)))
    ranks = np.asarray(p.export()["ranks"]).reshape(L + 1, 8)
    for l in range(L + 1):
        nb = 1 << (L - l)
        for b in range(8):
            assert ranks[l, b] == _expected_rank_for(G[l], L, l, b // nb, b % nb, sx, sw)


@pytest.mark.parametrize("n", [64, 100])
def test_library_fiedler_tree_bisects_a_segment(mht_lib, n):
    from tests.test_oracle_butterfly import _assert_quarters, _segment_points
    x, X = _segment_points(n)
    Phi = np.random.default_rng(1).standard_normal((n, 16))
    e = _plan_cls().build(n=n, m=16, eigenvalues=np.arange(16.0), evaluator="dense", dense=Phi, points=X,
                          eps=1e-6, levels=2, tree="fiedler").export()
    _assert_quarters(x, e["space_perm"], e["space_offsets"])


def test_clone_and_set_mode(mht_lib):
    from paper_2605_21828_gb300 import MhtError
    n = 256
    X, Phi, lam = _sphere(n, 15)
    p = _plan_cls().build(n=n, m=256, eigenvalues=lam, evaluator="sphere", points=X, eps=1e-6, leaf_size=32)
    q = p.clone("fp64")
    assert q.mode == "fp64" and q.info()["mode"] == 0
    a, b = p.export(), q.export()
    for k in a:
        if isinstance(a[k], np.ndarray):
            assert np.array_equal(a[k], b[k]), k
    p.set_mode("3xtf32")
    assert p.info()["mode"] == 2
    p.set_mode("fp32")
    with pytest.raises(MhtError, match="INVALID_ARG"):
        q.set_mode("fp32")  # storage precision differs
    with pytest.raises(MhtError, match="INVALID_ARG"):
        p.set_mode("fp64")


def test_batch_create_validates_and_counts_items(mht_lib):
    import ctypes as C
    from paper_2605_21828_gb300 import Batch, MhtError, _lib
    X, Phi, lam = _sphere(512, 21)
    a = _plan_cls().build(n=512, m=484, eigenvalues=lam[:484], evaluator="sphere", points=X, eps=1e-6, leaf_size=64)
    Xt = W.torus_points(256)
    K = W.torus_modes(256)
    b = _plan_cls().build(n=256, m=256, eigenvalues=W.torus_eigenvalues(K), evaluator="torus", points=Xt,
                          torus_modes=K, eps=1e-6, leaf_size=32)
    bt = Batch([a, b], [3, 1])
    ib, wb = bt.device_bytes()
    assert ib > sum(p.device_bytes(1)[0] for p in (a, b)) // 2 and wb > 0
    lib = _lib.load()
    n0, n1 = C.c_int64(), C.c_int64()
    _lib.check(lib.mht_batch_info(bt._h, C.byref(n0), C.byref(n1), None))
    items = sum(sum(p.level_info(s)["items"] for s in range(p.levels + 2)) for p in (a, b)) \
        if "items" in a.level_info(0) else None
    assert n0.value > 0 and n1.value > 0
    if items is not None:
        assert n0.value == items
    with pytest.raises(MhtError, match="INVALID_ARG"):
        Batch([a, a.clone("fp64")], [1, 1])
    with pytest.raises(MhtError, match="INVALID_ARG"):
        Batch([a], [0])
    st = lib.mht_batch_synthesize(bt._h, None)
    assert st == 9  # not bound
    bt.close()


def test_new_entry_points_reject_bad_arguments_without_a_gpu(mht_lib):
    import ctypes as C
    from paper_2605_21828_gb300 import _lib
    lib = _lib.load()
    X, Phi, lam = _sphere(256, 15)
    p = _plan_cls().build(n=256, m=256, eigenvalues=lam, evaluator="sphere", points=X, eps=1e-6, leaf_size=32)
    dummy = C.c_void_p(256)
    # unbound plans: every device entry point refuses before touching the GPU
    assert lib.mht_plan_autotune(p._h, 1, None) == 9
    assert lib.mht_filter(p._h, dummy, 256, C.c_void_p(512), 256, 1, dummy, 1, None) == 9
    assert lib.mht_synthesize_scaled(p._h, dummy, 256, dummy, C.c_void_p(512), 256, 1, None) == 9
    it, rr = C.c_int32(), C.c_double()
    assert lib.mht_inverse_lsqr(p._h, dummy, 256, C.c_void_p(512), 256, 1, dummy, 1 << 20, 10, 1e-6, None,
                                C.byref(it), C.byref(rr)) == 9
    nb = C.c_size_t()
    assert lib.mht_lsqr_scratch_bytes(p._h, 2, C.byref(nb)) == 0 and nb.value > 2 * 256 * 4
    assert lib.mht_lsqr_scratch_bytes(p._h, 0, C.byref(nb)) == 1
    cfg = (C.c_int32 * 5)()
    assert lib.mht_plan_tune_info(p._h, 0, 0, cfg, None) == 1  # not tuned
    assert lib.mht_plan_set_path(p._h, 3) == 1
    # batches: mode and graph switches, unbound launches
    h = C.c_void_p()
    arr = (C.c_void_p * 1)(p._h)
    ks = (C.c_int64 * 1)(2)
    assert lib.mht_batch_create(arr, 1, ks, C.byref(h)) == 0
    assert lib.mht_batch_set_mode(h, 0) == 1  # FP64 is not a batch mode
    assert lib.mht_batch_set_mode(h, 2) == 0
    assert lib.mht_batch_analyze(h, 1, None) == 9
    assert lib.mht_batch_autotune(h, None, None) == 9
    assert lib.mht_batch_debug_hold(h, 0, 0, 1, None) == 9
    assert lib.mht_batch_destroy(h) == 0


def _full_rank_factors(L, cplx=False):
    """A structurally valid butterfly with one point and one mode per leaf and full-rank IDs
    (r = K at every level): no transfer entries, but level vectors that double per level, so
    2^L (2^(L+1) - 1) butterfly-vector entries in all."""
    nb = 1 << L
    ranks, lp, r = [], [], 1
    for lev in range(L + 1):
        K = 1 if lev == 0 else 2 * r
        r = K
        ranks += [r] * nb
        lp += list(range(K)) * nb
    dt = np.complex128 if cplx else np.float64
    return {"n": nb, "m": nb, "levels": L, "complex": cplx, "space_perm": np.arange(nb),
            "space_offsets": np.arange(nb + 1), "mode_perm": np.arange(nb), "mode_offsets": np.arange(nb + 1),
            "ranks": np.array(ranks, np.int32), "local_perm": np.array(lp, np.int32),
            "transfer": np.zeros(0, dt), "column_bases": np.ones(nb * r, dt)}


def test_noalloc_synthesis_rejects_what_its_fixed_scratch_cannot_serve(mht_lib):
    """The allocation-free synthesis checks, before any CUDA call: plans whose scratch exceeds
    the fixed array (message with both sizes), FP64 and complex plans, and plans whose fused
    kernel does not fit in shared memory.  None of these touch a GPU."""
    from paper_2605_21828_gb300 import Plan, _lib
    lib = _lib.load()
    fake = C.c_void_p(256)  # never dereferenced: every rejection happens on the host
    assert "(16u << 20)" in open(os.path.join(ROOT, "include", "mht.h")).read()
    big = Plan.from_factors(_full_rank_factors(11), mode="fp32")  # 2048 * 4095 vector entries
    rc = lib.mht_synthesize_noalloc(big._h, fake, fake, fake, None)
    msg = lib.mht_last_error().decode()
    assert rc == 8, msg  # UNSUPPORTED
    sizes = [int(x) for x in re.findall(r"\d+", msg)]
    assert 16 << 20 in sizes and any(s > 16 << 20 for s in sizes), msg
    for F, mode in ((_full_rank_factors(3), "fp64"), (_full_rank_factors(3, cplx=True), "fp32")):
        p = Plan.from_factors(F, mode=mode)
        assert lib.mht_synthesize_noalloc(p._h, fake, fake, fake, None) == 8
        assert "real FP32" in lib.mht_last_error().decode()
        assert lib.mht_noalloc_debug_hold(p._h, fake, 1, None) == 8
    # one block whose single row is 60000 entries wide: no fused ring slot fits in shared memory
    K = 60001
    wide = {"n": 1, "m": K, "levels": 0, "complex": False, "space_perm": np.arange(1), "space_offsets": [0, 1],
            "mode_perm": np.arange(K), "mode_offsets": [0, K], "ranks": np.array([1], np.int32),
            "local_perm": np.arange(K, dtype=np.int32), "transfer": np.ones(K - 1), "column_bases": np.ones(1)}
    p = Plan.from_factors(wide, mode="fp32")
    assert lib.mht_synthesize_noalloc(p._h, fake, fake, fake, None) == 8
    assert "shared memory" in lib.mht_last_error().decode()
    # misaligned factors and NULL arguments
    small = Plan.from_factors(_full_rank_factors(3), mode="fp32")
    assert lib.mht_synthesize_noalloc(small._h, C.c_void_p(260), fake, fake, None) == 1
    assert lib.mht_synthesize_noalloc(small._h, fake, None, fake, None) == 1
    assert lib.mht_noalloc_check(None, None) == 1


def test_host_allocation_failure_is_reported_as_oom(mht_lib):
    """An injected host allocation failure (the packed image over a test limit) surfaces as
    MHT_ERR_OOM from mht_plan_import, creates no plan, and the next import succeeds."""
    from paper_2605_21828_gb300 import MhtError, Plan, _lib
    lib = _lib.load()
    F = _full_rank_factors(4)
    assert lib.mht_debug_host_alloc_limit(1024) == 0
    try:
        with pytest.raises(MhtError, match="OOM"):
            Plan.from_factors(F, mode="fp32")
        assert "allocation" in lib.mht_last_error().decode()
    finally:
        lib.mht_debug_host_alloc_limit(0)
    p = Plan.from_factors(F, mode="fp32")
    assert p.info()["n"] == 16
