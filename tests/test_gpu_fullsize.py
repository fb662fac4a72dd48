"""Parity at the full benchmark size (unit sphere, n = m = 65536, eps = 1e-6, leaf 128, FP32),
in the launch configuration the benchmark times (per-stage kernels, autotuned shapes).

The oracle cannot hold this Phi (34 GB in FP64), so it checks what it can compute one by one
and properties that hold at any size:
  * sampled rows of f = Phi c against the exact rows of Phi (normalized Legendre recurrence):
    the butterfly error is about eps (Sec. 6), so within 20 eps in relative l2 over the sample;
  * the adjoint identity <Phi c, W g> = <c, Phi^T W g> for the library's own apply pair;
and, element by element, the kernels against the oracle's FP64 apply (Sec. 2, stage by stage)
of the same plan's exported factors (15 GB of FP64 on the host): relative l2 <= 1e-6, the
FP32 kernel tolerance, for synthesis and weighted analysis.
"""
import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from oracle import harmonics as H
from tests._bridge import arrays_to_oracle

pytestmark = pytest.mark.gpu


def test_full_size_sphere_sampled_rows_and_adjoint_identity(mht_lib):
    import torch
    from paper_2605_21828_gb300 import Plan
    n, lmax, leaf, eps = 65536, 255, 128, 1e-6
    m = (lmax + 1) ** 2
    X = W.fibonacci_points(n)
    w = np.full(n, 4 * np.pi / n)
    plan = Plan.build(n=n, m=m, eigenvalues=W.sphere_eigenvalues(m), evaluator="sphere", points=X, eps=eps,
                      leaf_size=leaf, mode="fp32", weights=w).bind(max_nrhs=1)
    plan.autotune(1)
    c = W.sphere_coefficients(m)[:, 0]
    f = plan.synthesize_raw(torch.from_numpy(c).float().cuda()).double().cpu().numpy()
    assert plan.check() == 0
    rows = np.random.default_rng(17).choice(n, 48, replace=False)
    exact = H.sphere_phi(X[rows], lmax) @ c
    assert np.linalg.norm(f[rows] - exact) / np.linalg.norm(exact) <= 20 * eps
    g = W.gaussian(n, 23)
    a = plan.analyze_raw(torch.from_numpy(g).float().cuda(), weighted=True).double().cpu().numpy()
    lhs = float(np.dot(f, w * g))
    rhs = float(np.dot(c, a))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(f) * np.linalg.norm(w * g)
    # the kernels' rounding against the oracle's FP64 apply of the same factors
    F = arrays_to_oracle(plan.export())
    for got, ref in ((f, B.synthesize(F, c)), (a, B.analyze(F, g, w))):
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
