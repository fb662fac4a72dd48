"""Deformed-sphere FEM configuration at its stated size (icosphere level 6: 40962 vertices,
81920 triangles, radius 1 + 0.2 h / max|h|; P1 cotangent stiffness and lumped mass; the 4096
lowest generalized eigenpairs; eps = 1e-6, leaf 128).

The eigenpairs take about half an hour of host time (the oracle's spectral slicing, Sec. 7.1,
by shift-invert Lanczos); the plan is built from them once by ``tests/c3_plan.py`` (the
library's host build with Algorithm 2's patch rule on the mesh) and saved, and this test reads
the saved plan from the path in the environment variable MHT_C3_PLAN (skipped when unset).

Checks, for the plan's FP32 image and its tensor-core forms:
  * the kernels against the oracle's FP64 apply (Sec. 2, stage by stage) of the same plan's
    exported factors, element by element per right-hand side: relative l2 <= 1e-6 for FP32 and
    6xBF16, 2e-6 for 3xTF32 (which keeps 22 of FP32's 24 bits per operand);
  * the discrete orthonormality Phi^T M Phi = I of the eigenvectors (Eq. eigenproblem with the
    lumped mass M as quadrature weights): the weighted analysis of a synthesis returns the
    coefficients to a few eps.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from tests._bridge import arrays_to_oracle

pytestmark = pytest.mark.gpu

PLAN = os.environ.get("MHT_C3_PLAN", "")
TOL = {"fp32": 1e-6, "6xbf16": 1e-6, "3xtf32": 2e-6}


@pytest.fixture(scope="module")
def c3(mht_lib):
    if not PLAN or not os.path.exists(PLAN):
        pytest.skip("MHT_C3_PLAN names no saved plan of the deformed-sphere configuration")
    import torch
    from paper_2605_21828_gb300 import Plan
    assert torch.cuda.is_available(), "GPU test"
    plan = Plan.load(PLAN, mode="fp32")
    E = plan.export()
    w = np.asarray(E["weights"], dtype=np.float64)
    assert plan.n == 40962 and plan.m == 4096 and len(w) == plan.n
    return plan, arrays_to_oracle(E), w


def _rel(got, ref):
    got = np.asarray(got, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref).reshape(len(ref), -1)
    return (np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max()


@pytest.mark.parametrize("mode,k", [("fp32", 1), ("fp32", 8), ("6xbf16", 64), ("3xtf32", 64)])
def test_c3_kernels_match_the_oracle_apply_of_the_same_plan(c3, mode, k):
    import torch
    plan, F, w = c3
    plan.bind(max_nrhs=k).set_path("auto").set_mode(mode)
    plan.autotune(k)
    C = W.gaussian_columns(F.m, k, 500 + k)
    G = W.gaussian_columns(F.n, k, 600 + k)
    cd = torch.from_numpy(np.ascontiguousarray(C if k > 1 else C[:, 0])).float().cuda()
    gd = torch.from_numpy(np.ascontiguousarray(G if k > 1 else G[:, 0])).float().cuda()
    f = plan.synthesize_raw(cd).cpu().numpy()
    a = plan.analyze_raw(gd, weighted=True).cpu().numpy()
    assert plan.check() == 0
    assert _rel(f, B.synthesize(F, C if k > 1 else C[:, 0])) <= TOL[mode]
    assert _rel(a, B.analyze(F, G if k > 1 else G[:, 0], w)) <= TOL[mode]


def test_c3_weighted_analysis_inverts_synthesis(c3):
    import torch
    plan, F, w = c3
    plan.bind(max_nrhs=8).set_path("auto").set_mode("fp32")
    C = W.gaussian_columns(F.m, 8, 700)
    f = plan.synthesize_raw(torch.from_numpy(C).float().cuda())
    c2 = plan.analyze_raw(f, weighted=True).cpu().numpy()
    assert plan.check() == 0
    assert _rel(c2, C) <= 1e-4
