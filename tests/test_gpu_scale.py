"""Kernel parity at the benchmark's scale against the oracle's FP64 apply of the SAME plan.

The library builds the 16384-point sphere plan (eps = 1e-6, leaf 128, L = 7: the benchmark's
workload at a quarter of its size, with blocks of up to a thousand columns and per-stage work
items of hundreds of rows); its FP64 factors are exported and applied by the oracle
(`oracle.butterfly`, Sec. 2 stage by stage), and every GPU apply path is compared with that,
element by element, per right-hand side:
  * single RHS: autotuned per-stage launches (ring slot sizes, CTAs per SM), the persistent
    all-stage kernel;
  * several RHS: SIMT RHS tiles of 2, 4 and 8;
  * 64 RHS on the tensor cores (6xBF16 and 3xTF32), autotuned.
Tolerances: relative l2 per RHS <= 1e-6 for the FP32 kernels and 6xBF16 (max element error
<= 1e-5 of the largest entry); 3xTF32 keeps each operand to 22 of FP32's 24 bits, which costs
about twice FP32's rounding error, and is held to 2e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from tests._bridge import arrays_to_oracle

pytestmark = pytest.mark.gpu

N, LMAX, LEAF, EPS = 16384, 127, 128, 1e-6
TOL = {"fp32": 1e-6, "6xbf16": 1e-6, "3xtf32": 2e-6}


@pytest.fixture(scope="module")
def sphere(mht_lib):
    import torch
    from paper_2605_21828_gb300 import Plan
    assert torch.cuda.is_available(), "GPU test"
    m = (LMAX + 1) ** 2
    X = W.fibonacci_points(N)
    w = np.full(N, 4 * np.pi / N)
    plan = Plan.build(n=N, m=m, eigenvalues=W.sphere_eigenvalues(m), evaluator="sphere", points=X, eps=EPS,
                      leaf_size=LEAF, mode="fp32", weights=w)
    F = arrays_to_oracle(plan.export())
    return plan, F, w


def _check(got, ref, tol):
    got = np.asarray(got, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref).reshape(len(ref), -1)
    per = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    elem = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert per.max() <= tol, f"relative l2 error {per.max():.3e} > {tol:.1e}"
    assert elem <= 10 * tol, f"max element error {elem:.3e} > {10 * tol:.1e}"


def _apply_both(plan, F, w, k, seed):
    import torch
    C = W.gaussian_columns(F.m, k, seed)
    G = W.gaussian_columns(F.n, k, seed + 1)
    cd = torch.from_numpy(np.ascontiguousarray(C if k > 1 else C[:, 0])).float().cuda()
    gd = torch.from_numpy(np.ascontiguousarray(G if k > 1 else G[:, 0])).float().cuda()
    f = plan.synthesize_raw(cd).cpu().numpy()
    a = plan.analyze_raw(gd, weighted=True).cpu().numpy()
    assert plan.check() == 0
    return f, B.synthesize(F, C if k > 1 else C[:, 0]), a, B.analyze(F, G if k > 1 else G[:, 0], w)


@pytest.mark.parametrize("path,k", [("auto", 1), ("fused", 1), ("auto", 3), ("auto", 8)])
def test_fp32_kernels_match_the_oracle_apply_of_the_same_plan(sphere, path, k):
    plan, F, w = sphere
    plan.bind(max_nrhs=k).set_mode("fp32").set_path(path)
    if path == "auto":
        plan.autotune(k)  # the launch shapes the benchmark times
    f, fr, a, ar = _apply_both(plan, F, w, k, 300 + k)
    _check(f, fr, TOL["fp32"])
    _check(a, ar, TOL["fp32"])


@pytest.mark.parametrize("mode", ["6xbf16", "3xtf32"])
def test_tensor_core_split_products_match_the_oracle_apply_at_64_rhs(sphere, mode):
    plan, F, w = sphere
    plan.bind(max_nrhs=64).set_path("auto").set_mode(mode)
    tuned = plan.autotune(64)
    assert any(t["tensor"] for t in tuned)  # the large stages run on the tensor cores
    f, fr, a, ar = _apply_both(plan, F, w, 64, 400)
    _check(f, fr, TOL[mode])
    _check(a, ar, TOL[mode])
