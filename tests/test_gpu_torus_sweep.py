"""The flat-torus scaling sweep's plans (Sec. 6.1 memory experiment: uniform points in
[-pi, pi]^2, the m = ceil(n / 25) lowest modes of Eq. 2D-DFT, leaf 64, eps in {1e-3, 1e-6}),
built by the library exactly as ``bench.py --workload torus_sweep`` builds them, applied on the
GPU in complex FP32 (single RHS, the autotuned launch shapes the sweep times), and checked
  * against the dense NUDFT f = Phi c, Phi_jk = exp(i k_k . x_j) (``oracle.harmonics``, the
    definition of the transform): relative l2 within 5 eps (the host build measures 0.4-0.7 eps),
    and the unweighted adjoint against Phi^H g likewise;
  * element by element against the oracle's FP64 apply (Sec. 2, stage by stage) of the same
    plan's factors: relative l2 <= 1e-6 (the FP32 kernel tolerance).
"""
import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from oracle import harmonics as H
from tests._bridge import arrays_to_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps", [1e-3, 1e-6])
@pytest.mark.parametrize("n", [4096, 16384])
def test_torus_sweep_plan_matches_nudft_and_oracle_apply(mht_lib, n, eps):
    import torch
    from paper_2605_21828_gb300 import Plan
    assert torch.cuda.is_available(), "GPU test"
    m = -(-n // 25)
    K = W.torus_modes_lowest(m)
    X = W.torus_points(n)
    plan = Plan.build(n=n, m=m, eigenvalues=W.torus_eigenvalues(K), evaluator="torus", points=X, torus_modes=K,
                      eps=eps, leaf_size=64, mode="fp32")
    plan.bind(max_nrhs=1)
    plan.autotune(1)
    c = W.gaussian(m, 1, True)
    g = W.gaussian(n, 2, True)
    f = plan.synthesize_raw(torch.from_numpy(c).to(torch.complex64).cuda()).cpu().numpy().astype(np.complex128)
    a = plan.analyze_raw(torch.from_numpy(g).to(torch.complex64).cuda(), weighted=False).cpu().numpy()
    a = a.astype(np.complex128)
    assert plan.check() == 0
    Phi = H.torus_phi(X, K)
    for got, exact in ((f, Phi @ c), (a, Phi.conj().T @ g)):
        assert np.linalg.norm(got - exact) / np.linalg.norm(exact) <= 5 * eps
    F = arrays_to_oracle(plan.export())
    for got, ref in ((f, B.synthesize(F, c)), (a, B.analyze(F, g))):
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
