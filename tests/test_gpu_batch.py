"""Batched ragged apply (one persistent launch per direction for many plans) on the GPU.

Instances of different n, m, depth, field and RHS count -- sphere harmonics, complex torus
exponentials, FEM eigenvectors of a deformed sphere, an L = 0 plan and a tree with empty
leaves -- are applied in one batch and compared, per instance and element by element, with
the FP64 oracle apply of the same factors (relative l2 per RHS <= 1e-6), and with the
per-plan apply through mht_synthesize / mht_analyze (identical arithmetic, so equal bit for
bit).
"""
import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from oracle import fem
from oracle import harmonics as H
from tests._bridge import oracle_to_arrays

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a).reshape(len(a), -1)
    b = np.asarray(b).reshape(len(b), -1)
    return float((np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300)).max())


def _instances():
    out = []
    X = W.fibonacci_points(1000)
    Phi = H.sphere_phi(X, 15)  # m = 256
    out.append((B.build(B.dense_evaluator(Phi), 1000, 256, W.sphere_eigenvalues(256), X, 1e-6, 64), None, 3))
    Xt = W.torus_points(1024, seed=3)
    K = W.torus_modes(256)
    Pt = H.torus_phi(Xt, K)
    out.append((B.build(B.dense_evaluator(Pt), 1024, 256, W.torus_eigenvalues(K), Xt, 1e-6, 64, "rect",
                        complex_=True), None, 5))
    V, Fc = W.deformed_icosphere(3)
    lam, Pf, Md, _ = fem.laplace_beltrami_basis(V, Fc, 160)
    out.append((B.build(B.dense_evaluator(Pf), len(V), 160, lam, V, 1e-6, 64), Md, 1))
    X4 = W.fibonacci_points(4096, seed=2)
    P4 = H.sphere_phi(X4, 31)  # m = 1024
    out.append((B.build(B.dense_evaluator(P4), 4096, 1024, W.sphere_eigenvalues(1024), X4, 1e-6, 128), None, 12))
    X0 = W.fibonacci_points(60, seed=4)
    P0 = H.sphere_phi(X0, 6)
    out.append((B.build(B.dense_evaluator(P0), 60, 49, W.sphere_eigenvalues(49), X0, 1e-8, 64), None, 2))
    Xe = W.fibonacci_points(96, seed=5)
    Pe = H.sphere_phi(Xe, 9)
    perm = np.arange(96)
    off = np.array([0, 30, 60, 60, 96, 96, 96, 96, 96])
    out.append((B.build(B.dense_evaluator(Pe), 96, 100, W.sphere_eigenvalues(100), Xe, 1e-7, 12, space=(perm, off)),
                None, 1))
    return out


_INST = None


def _inst():
    global _INST
    if _INST is None:
        _INST = _instances()
    return _INST


@pytest.fixture(scope="module")
def torch_cuda(mht_lib):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_oracle_and_per_plan_apply(torch_cuda, graph):
    from paper_2605_21828_gb300 import Batch, Plan
    torch = torch_cuda
    inst = _inst()
    assert inst[4][0].L == 0 and min(inst[5][0].ranks[3]) == 0
    rng = np.random.default_rng(9)
    weights = [w if w is not None else rng.uniform(0.5, 1.5, F.n) for F, w, _ in inst]
    plans = [Plan.from_factors(oracle_to_arrays(F), mode="fp32", weights=w) for (F, _, _), w in zip(inst, weights)]
    bt = Batch(plans, [k for _, _, k in inst]).bind()
    bt.set_graph(graph)
    info = bt.info()
    assert info["items_synthesis"] > 0 and info["grid"] >= 1
    Cs, Gs = [], []
    for i, (F, _, k) in enumerate(inst):
        C_ = W.gaussian_columns(F.m, k, 20 + i, complex_=F.complex_)
        G = W.gaussian_columns(F.n, k, 40 + i, complex_=F.complex_)
        Cs.append(C_)
        Gs.append(G)
        bt.c[i].copy_(torch.from_numpy(C_).to(bt.c[i].dtype))
    fs = [f.cpu().numpy() for f in bt.synthesize()]
    assert bt.check() == 0
    for i, (F, _, k) in enumerate(inst):
        assert _rel(fs[i], B.synthesize(F, Cs[i])) <= 1e-6, i
    for i in range(len(inst)):
        bt.f[i].copy_(torch.from_numpy(Gs[i]).to(bt.f[i].dtype))
    for weighted in (True, False):
        cs = [c.cpu().numpy() for c in bt.analyze(weighted=weighted)]
        assert bt.check() == 0
        for i, (F, _, k) in enumerate(inst):
            ref = B.analyze(F, Gs[i], weights[i] if weighted else None)
            assert _rel(cs[i], ref) <= 1e-6, (i, weighted)
    # the per-plan apply runs the same row arithmetic: equal bit for bit
    for i, (F, _, k) in enumerate(inst):
        p = plans[i].bind(max_nrhs=k).set_path("staged")
        dt = bt.c[i].dtype
        fi = p.synthesize_raw(torch.from_numpy(Cs[i]).to(dt).cuda())
        assert torch.equal(fi.reshape(bt.f[i].shape[0], -1), torch.from_numpy(fs[i]).cuda().reshape(fi.shape[0], -1)), i
    # replays of the captured launch give identical results (analysis overwrote c: restore it)
    for i in range(len(inst)):
        bt.c[i].copy_(torch.from_numpy(Cs[i]).to(bt.c[i].dtype))
    f_again = [f.clone() for f in bt.synthesize()]
    f3 = bt.synthesize()
    for i, (a, b) in enumerate(zip(f_again, f3)):
        assert torch.equal(a, b)
        assert torch.equal(a.cpu(), torch.from_numpy(fs[i]))


def test_batch_autotune_keeps_results(torch_cuda):
    from paper_2605_21828_gb300 import Batch, Plan
    torch = torch_cuda
    inst = _inst()
    plans = [Plan.from_factors(oracle_to_arrays(F), mode="fp32") for F, _, _ in inst]
    bt = Batch(plans, [k for _, _, k in inst]).bind()
    Cs = [W.gaussian_columns(F.m, k, 90 + i, complex_=F.complex_) for i, (F, _, k) in enumerate(inst)]

    def run():
        for i in range(len(inst)):
            bt.c[i].copy_(torch.from_numpy(Cs[i]).to(bt.c[i].dtype))
        return [f.clone() for f in bt.synthesize()]

    before = run()
    ms = bt.autotune()
    assert ms > 0 and bt.check() == 0
    after = run()
    for i, (F, _, k) in enumerate(inst):
        assert torch.equal(before[i], after[i])  # launch shape does not change the arithmetic
        assert _rel(after[i].cpu().numpy(), B.synthesize(F, Cs[i])) <= 1e-6


@pytest.mark.parametrize("mode", ["6xbf16", "3xtf32"])
def test_batch_tensor_core_form_matches_per_plan_apply(torch_cuda, mode):
    # split tensor-core form: each instance's own apply (tensor cores from 16 real / 8 complex
    # RHS) on forked streams inside one CUDA graph; equal bit for bit to the per-plan apply
    from paper_2605_21828_gb300 import Batch, Plan
    torch = torch_cuda
    inst = _inst()
    ks = [20, 9, 1, 17, 2, 16]  # wide tiles on the tensor cores, narrow ones on SIMT
    rng = np.random.default_rng(12)
    weights = [w if w is not None else rng.uniform(0.5, 1.5, F.n) for F, w, _ in inst]
    plans = [Plan.from_factors(oracle_to_arrays(F), mode=mode, weights=w)
             for (F, _, _), w in zip(inst, weights)]
    bt = Batch(plans, ks).bind().set_mode(mode)
    Cs = [W.gaussian_columns(F.m, k, 130 + i, complex_=F.complex_) for i, ((F, _, _), k) in enumerate(zip(inst, ks))]
    Gs = [W.gaussian_columns(F.n, k, 150 + i, complex_=F.complex_) for i, ((F, _, _), k) in enumerate(zip(inst, ks))]
    for i in range(len(inst)):
        bt.c[i].copy_(torch.from_numpy(Cs[i]).to(bt.c[i].dtype))
        bt.f[i].copy_(torch.from_numpy(Gs[i]).to(bt.f[i].dtype))
    cs = [c.clone() for c in bt.analyze(weighted=True)]
    for i in range(len(inst)):
        bt.c[i].copy_(torch.from_numpy(Cs[i]).to(bt.c[i].dtype))
    fs = [f.clone() for f in bt.synthesize()]
    assert bt.check() == 0
    for i, ((F, _, _), k) in enumerate(zip(inst, ks)):
        assert _rel(fs[i].cpu().numpy(), B.synthesize(F, Cs[i])) <= 1e-6, i
        assert _rel(cs[i].cpu().numpy(), B.analyze(F, Gs[i], weights[i])) <= 1e-6, i
        p = plans[i].bind(max_nrhs=k).set_path("staged")
        dt = bt.c[i].dtype
        assert torch.equal(p.synthesize_raw(torch.from_numpy(Cs[i]).to(dt).cuda()), fs[i]), i
        assert torch.equal(p.analyze_raw(torch.from_numpy(Gs[i]).to(dt).cuda(), weighted=True), cs[i]), i
    # the graph replays: a second synthesis gives the same vectors
    f2 = bt.synthesize()
    for a, b in zip(fs, f2):
        assert torch.equal(a, b)


def test_batch_dependency_timeout_is_reported_and_the_context_recovers(torch_cuda):
    # failure path without a fault: one phase's dependency is made unsatisfiable on the device;
    # the persistent kernel gives up its bounded wait (2 s), stops every CTA and reports
    # TIMEOUT; after the records are restored the same batch computes correct results again
    import ctypes as C
    from paper_2605_21828_gb300 import Batch, MhtError, Plan, _lib
    torch = torch_cuda
    inst = _inst()[:2]
    plans = [Plan.from_factors(oracle_to_arrays(F), mode="fp32") for F, _, _ in inst]
    bt = Batch(plans, [k for _, _, k in inst]).bind()
    Cs = [W.gaussian_columns(F.m, k, 170 + i, complex_=F.complex_) for i, (F, _, k) in enumerate(inst)]
    for i in range(len(inst)):
        bt.c[i].copy_(torch.from_numpy(Cs[i]).to(bt.c[i].dtype))
    lib = _lib.load()
    _lib.check(lib.mht_batch_debug_hold(bt._h, 0, 0, 2, C.c_void_p(torch.cuda.current_stream().cuda_stream)))
    bt.synthesize()
    with pytest.raises(MhtError, match="TIMEOUT"):
        bt.check()
    bt.reset_io()
    f = [x.clone() for x in bt.synthesize()]
    assert bt.check() == 0
    for i, (F, _, k) in enumerate(inst):
        assert _rel(f[i].cpu().numpy(), B.synthesize(F, Cs[i])) <= 1e-6
