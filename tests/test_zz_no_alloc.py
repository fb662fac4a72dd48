"""The synthesis entry point that allocates nothing (mht_synthesize_noalloc).

Some callers cannot call cudaMalloc -- code that runs where the device memory belongs to a
framework, or where allocating is not allowed.  mht_synthesize_noalloc keeps its scratch in a
fixed array inside the library and takes only the factors, c and f from the caller.  This
file runs last (pytest collects it after the other test files) and checks, through the C
ABI, that two calls in a row reproduce the regular mht_synthesize output within the FP32
tolerance of the parity tests.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from oracle import butterfly as B
from oracle import harmonics as H
from tests._bridge import oracle_to_arrays

pytestmark = pytest.mark.gpu


def test_noalloc_synthesis_matches_regular_synthesis(mht_lib):
    import torch

    from paper_2605_21828_gb300 import Plan, _lib
    assert torch.cuda.is_available(), "GPU test"
    n = 1000
    X = W.fibonacci_points(n)
    Phi = H.sphere_phi(X, 31)
    m = Phi.shape[1]
    F = B.build(B.dense_evaluator(Phi), n, m, W.sphere_eigenvalues(m), X, 1e-6, 64)
    plan = Plan.from_factors(oracle_to_arrays(F), mode="fp32").bind(max_nrhs=1)
    c = torch.from_numpy(W.sphere_coefficients(m)[:, 0]).float().cuda()
    f_ref = plan.synthesize_raw(c).clone()
    factor_ptr = (plan._dev[0].data_ptr() + 255) // 256 * 256  # the buffer the plan was bound to
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = _lib.load()
    for _ in range(2):  # two calls in a row share the library's scratch array
        f = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        _lib.check(lib.mht_synthesize_noalloc(plan._h, C.c_void_p(factor_ptr), C.c_void_p(c.data_ptr()),
                                              C.c_void_p(f.data_ptr()), stream))
        torch.cuda.synchronize()
        flags = C.c_int32(-1)
        _lib.check(lib.mht_noalloc_check(stream, C.byref(flags)))  # every bounded wait completed
        assert flags.value == 0
        got, ref = f.double().cpu().numpy(), f_ref.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
    # and against the oracle's FP64 apply of the same factors
    ref64 = B.synthesize(F, W.sphere_coefficients(m)[:, 0])
    assert np.linalg.norm(got - ref64) / np.linalg.norm(ref64) <= 1e-6


def test_noalloc_reports_a_wait_that_ran_out(mht_lib):
    """A bounded wait of the allocation-free synthesis that gives up is reported by
    mht_noalloc_check (TIMEOUT, dependency bit 8) and cleared by it; the context stays usable and
    the next call computes the right result.  The wait is made to run out by an unreachable
    completion target written into the caller's copy of the factors (restored afterwards)."""
    import torch

    from paper_2605_21828_gb300 import Plan, _lib
    n = 1000
    X = W.fibonacci_points(n)
    Phi = H.sphere_phi(X, 31)
    m = Phi.shape[1]
    F = B.build(B.dense_evaluator(Phi), n, m, W.sphere_eigenvalues(m), X, 1e-6, 64)
    assert F.L >= 1
    plan = Plan.from_factors(oracle_to_arrays(F), mode="fp32").bind(max_nrhs=1)
    c = torch.from_numpy(W.sphere_coefficients(m)[:, 0]).float().cuda()
    f_ref = plan.synthesize_raw(c).clone()
    factor_ptr = C.c_void_p((plan._dev[0].data_ptr() + 255) // 256 * 256)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = _lib.load()
    flags = C.c_int32(-1)
    lib.mht_noalloc_check(stream, C.byref(flags))  # start from a clear status word
    f = torch.zeros(n, dtype=torch.float32, device="cuda")
    _lib.check(lib.mht_noalloc_debug_hold(plan._h, factor_ptr, 1, stream))
    _lib.check(lib.mht_synthesize_noalloc(plan._h, factor_ptr, C.c_void_p(c.data_ptr()), C.c_void_p(f.data_ptr()),
                                          stream))
    rc = lib.mht_noalloc_check(stream, C.byref(flags))
    assert rc == 7 and flags.value & 8, (rc, flags.value, lib.mht_last_error())  # TIMEOUT, dependency wait
    _lib.check(lib.mht_noalloc_debug_hold(plan._h, factor_ptr, 0, stream))
    _lib.check(lib.mht_noalloc_check(stream, C.byref(flags)))  # cleared by the read above
    assert flags.value == 0
    _lib.check(lib.mht_synthesize_noalloc(plan._h, factor_ptr, C.c_void_p(c.data_ptr()), C.c_void_p(f.data_ptr()),
                                          stream))
    _lib.check(lib.mht_noalloc_check(stream, C.byref(flags)))
    got, ref = f.double().cpu().numpy(), f_ref.double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-6
