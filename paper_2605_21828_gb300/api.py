"""Python interface to libmht: plans, device binding, transforms and autograd.

Thin marshalling over the C ABI (include/mht.h): every transform runs in the library's CUDA
kernels; PyTorch supplies device memory, the current stream and autograd.  There is no CPU
fallback: without the built library or a CUDA device the calls raise.

    plan = Plan.build(n=n, m=m, eigenvalues=lam, evaluator="sphere", points=X,
                      eps=1e-6, leaf_size=128, mode="fp32", weights=w)
    plan.bind(max_nrhs=64)
    f = synthesize(plan, c)            # f = Phi c          (differentiable)
    c2 = analyze(plan, f)              # c = Phi^H diag(w) f (differentiable)
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

_MODES = {"fp64": L.APPLY_FP64, "fp32": L.APPLY_FP32, "3xtf32": L.APPLY_3XTF32, "6xbf16": L.APPLY_6XBF16}
_TREES = {"auto": L.TREE_AUTO, "fiedler": L.TREE_FIEDLER, "rect": L.TREE_RECT,
          "pca": L.TREE_PCA_MEDIAN, "given": L.TREE_GIVEN, "mesh": L.TREE_FIEDLER_MESH}
_EVALS = {"torus": L.EVAL_TORUS, "sphere": L.EVAL_SPHERE, "dense": L.EVAL_DENSE}


def _dptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


_IDS = {"auto": 0, "classical": 1, "blocked": 2}


def _options(eps=1e-6, leaf_size=128, levels=-1, mode="fp32", tree="auto", seed=0,
             num_threads=0, oversample=0.0, id_method="auto"):
    return L.Options(eps, leaf_size, levels, _MODES[mode], _TREES[tree], seed, num_threads,
                     oversample, _IDS[id_method])


def _problem(*, n, m, evaluator, points=None, torus_modes=None, dense=None, callback=None, complex_=None):
    """An mht_problem with the evaluator fields set; returns (problem, arrays to keep alive, complex)."""
    prob = L.Problem()
    keep = []
    if complex_ is None:
        complex_ = evaluator == "torus" or (dense is not None and np.iscomplexobj(dense))
    prob.n, prob.m = n, m
    prob.field = L.COMPLEX if complex_ else L.REAL
    if points is not None:
        pts = np.ascontiguousarray(points, dtype=np.float64)
        keep.append(pts)
        prob.points = _dptr(pts, C.c_double)
        prob.dim = pts.shape[1]
    if evaluator == "callback":
        prob.eval_kind = L.EVAL_CALLBACK

        def _cb(ctx, rows, nr, cols, nc, out):
            try:
                r = np.ctypeslib.as_array(rows, (nr,)).copy()
                cc = np.ctypeslib.as_array(cols, (nc,)).copy()
                blk = np.asarray(callback(r, cc))
                o = np.ctypeslib.as_array(out, (nr * nc * (2 if complex_ else 1),))
                if complex_:  # column-major, interleaved (re, im)
                    o[:] = np.ascontiguousarray(blk.astype(np.complex128).T).view(np.float64).reshape(-1)
                else:
                    o[:] = np.asarray(blk, dtype=np.float64).T.reshape(-1)
                return 0
            except Exception:  # noqa: BLE001 - reported to the library as a failure
                return 1

        fn = L.EVAL_FN(_cb)
        keep.append(fn)
        prob.eval = fn
    else:
        prob.eval_kind = _EVALS[evaluator]
    if torus_modes is not None:
        km = np.ascontiguousarray(torus_modes, dtype=np.int64)
        keep.append(km)
        prob.torus_modes = _dptr(km, C.c_int64)
    if dense is not None:
        if complex_:
            D = np.asfortranarray(dense, dtype=np.complex128)
            flat = D.reshape(-1, order="F").view(np.float64)
        else:
            D = np.asfortranarray(dense, dtype=np.float64)
            flat = D.reshape(-1, order="F")
        keep += [D, flat]
        prob.dense = _dptr(flat, C.c_double)
        prob.ld_dense = n
    return prob, keep, complex_


def phi_entries(rows, cols, *, n, m, evaluator="sphere", points=None, torus_modes=None, dense=None,
                callback=None, complex_=None) -> np.ndarray:
    """Phi(rows, cols) from the library's evaluator (``mht_problem_eval``): the FP64 values a
    build factors, as a (len(rows), len(cols)) float64 or complex128 array."""
    lib = L.load()
    prob, keep, cplx = _problem(n=n, m=m, evaluator=evaluator, points=points, torus_modes=torus_modes,
                                dense=dense, callback=callback, complex_=complex_)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.zeros(len(r) * len(c) * (2 if cplx else 1), dtype=np.float64)
    L.check(lib.mht_problem_eval(C.byref(prob), _dptr(r, C.c_int64), len(r), _dptr(c, C.c_int64), len(c),
                                 _dptr(out, C.c_double)))
    del keep
    if cplx:
        return out.view(np.complex128).reshape(len(c), len(r)).T
    return out.reshape(len(c), len(r)).T


class Plan:
    """A built (or imported) butterfly factorization and, once bound, its device copy."""

    def __init__(self, handle: C.c_void_p, mode: str, keep=()):
        self.grouping = {}
        self._h = handle
        self.mode = mode
        self._keep = list(keep)
        self._dev = None
        info = self.info()
        self.n, self.m, self.levels = info["n"], info["m"], info["levels"]
        self.complex = bool(info["field"] == L.COMPLEX)

    # ---------------------------------------------------------------- construction
    @staticmethod
    def build(*, n, m, eigenvalues, evaluator="sphere", points=None, torus_modes=None,
              dense=None, callback=None, complex_=None, weights=None, space=None, tris=None,
              **opts) -> "Plan":
        """Builds the factorization on the host (FP64) through ``mht_build_plan``.

        evaluator: "sphere" | "torus" | "dense" | "callback" (then ``callback(rows, cols)``
        returns Phi(rows, cols) as a float64/complex128 array).  ``space`` = (perm, offsets)
        selects tree="given".  ``tris`` (ntris x 3 vertex indices; the points are the mesh
        vertices) makes tree="auto" use Algorithm 2's patch rule ("mesh").
        """
        lib = L.load()
        prob, keep, _ = _problem(n=n, m=m, evaluator=evaluator, points=points, torus_modes=torus_modes,
                                 dense=dense, callback=callback, complex_=complex_)
        lam = np.ascontiguousarray(eigenvalues, dtype=np.float64)
        keep.append(lam)
        prob.eigenvalues = _dptr(lam, C.c_double)
        if weights is not None:
            w = np.ascontiguousarray(weights, dtype=np.float64)
            keep.append(w)
            prob.weights = _dptr(w, C.c_double)
        if tris is not None:
            tr = np.ascontiguousarray(tris, dtype=np.int64).reshape(-1, 3)
            keep.append(tr)
            prob.tris = _dptr(tr, C.c_int64)
            prob.ntris = len(tr)
        if space is not None:
            sp = np.ascontiguousarray(space[0], dtype=np.int64)
            so = np.ascontiguousarray(space[1], dtype=np.int64)
            keep += [sp, so]
            prob.space_perm = _dptr(sp, C.c_int64)
            prob.space_offsets = _dptr(so, C.c_int64)
            opts["tree"] = "given"
        o = _options(**opts)
        h = C.c_void_p()
        L.check(lib.mht_build_plan(C.byref(prob), C.byref(o), C.byref(h)))
        return Plan(h, opts.get("mode", "fp32"))

    @staticmethod
    def from_factors(F: dict, mode: str = "fp32", weights=None) -> "Plan":
        """Imports explicit factors (dict with the mht_factors arrays) via ``mht_plan_import``."""
        lib = L.load()
        cplx = bool(F["complex"])
        arr = {
            "space_perm": np.ascontiguousarray(F["space_perm"], dtype=np.int64),
            "space_offsets": np.ascontiguousarray(F["space_offsets"], dtype=np.int64),
            "mode_perm": np.ascontiguousarray(F["mode_perm"], dtype=np.int64),
            "mode_offsets": np.ascontiguousarray(F["mode_offsets"], dtype=np.int64),
            "ranks": np.ascontiguousarray(F["ranks"], dtype=np.int32),
            "local_perm": np.ascontiguousarray(F["local_perm"], dtype=np.int32),
        }
        for key in ("transfer", "column_bases"):
            v = np.asarray(F[key])
            v = np.ascontiguousarray(v, dtype=np.complex128).view(np.float64) if cplx else \
                np.ascontiguousarray(v, dtype=np.float64)
            arr[key] = v if v.size else np.zeros(1)
        fa = L.Factors()
        fa.n, fa.m, fa.levels = int(F["n"]), int(F["m"]), int(F["levels"])
        fa.field = L.COMPLEX if cplx else L.REAL
        for k in ("space_perm", "space_offsets", "mode_perm", "mode_offsets"):
            setattr(fa, k, _dptr(arr[k], C.c_int64))
        fa.ranks = _dptr(arr["ranks"], C.c_int32)
        fa.local_perm = _dptr(arr["local_perm"], C.c_int32) if arr["local_perm"].size else \
            _dptr(np.zeros(1, np.int32), C.c_int32)
        fa.transfer = _dptr(arr["transfer"], C.c_double)
        fa.column_bases = _dptr(arr["column_bases"], C.c_double)
        if weights is not None:
            arr["weights"] = np.ascontiguousarray(weights, dtype=np.float64)
            fa.weights = _dptr(arr["weights"], C.c_double)
        h = C.c_void_p()
        L.check(lib.mht_plan_import(C.byref(fa), C.byref(_options(mode=mode)), C.byref(h)))
        return Plan(h, mode)

    @staticmethod
    def load(path: str, mode: str = "fp32") -> "Plan":
        h = C.c_void_p()
        L.check(L.load().mht_plan_load(path.encode(), C.byref(_options(mode=mode)), C.byref(h)))
        return Plan(h, mode)

    def clone(self, mode: str = "fp64") -> "Plan":
        """An unbound copy of the same factors, packed for another apply mode."""
        h = C.c_void_p()
        L.check(L.load().mht_plan_clone(self._h, C.byref(_options(mode=mode)), C.byref(h)))
        return Plan(h, mode)

    def save(self, path: str):
        L.check(L.load().mht_plan_save(self._h, path.encode()))

    def export(self) -> dict:
        """FP64 factors as numpy arrays (the mht_factors content)."""
        info = self.info()
        nb = info["blocks_per_level"]
        cplx = info["field"] == L.COMPLEX
        W = 2 if cplx else 1
        out = {
            "n": info["n"], "m": info["m"], "levels": info["levels"], "complex": cplx,
            "space_perm": np.zeros(info["n"], np.int64), "space_offsets": np.zeros(nb + 1, np.int64),
            "mode_perm": np.zeros(info["m"], np.int64), "mode_offsets": np.zeros(nb + 1, np.int64),
            "ranks": np.zeros((info["levels"] + 1) * nb, np.int32),
            "local_perm": np.zeros(max(info["local_perm_entries"], 1), np.int32),
            "transfer": np.zeros(max(info["transfer_entries"] * W, 1)),
            "column_bases": np.zeros(max(info["column_basis_entries"] * W, 1)),
        }
        fa = L.Factors()
        for k in ("space_perm", "space_offsets", "mode_perm", "mode_offsets"):
            setattr(fa, k, _dptr(out[k], C.c_int64))
        fa.ranks = _dptr(out["ranks"], C.c_int32)
        fa.local_perm = _dptr(out["local_perm"], C.c_int32)
        fa.transfer = _dptr(out["transfer"], C.c_double)
        fa.column_bases = _dptr(out["column_bases"], C.c_double)
        w = np.full(info["n"], np.nan)
        fa.weights = _dptr(w, C.c_double)
        L.check(L.load().mht_plan_export(self._h, C.byref(fa)))
        out["weights"] = None if np.isnan(w).all() else w  # the analysis weights, if the plan has them
        out["local_perm"] = out["local_perm"][:info["local_perm_entries"]]
        t = out["transfer"][:info["transfer_entries"] * W]
        u = out["column_bases"][:info["column_basis_entries"] * W]
        out["transfer"] = t.view(np.complex128) if cplx else t
        out["column_bases"] = u.view(np.complex128) if cplx else u
        return out

    def info(self) -> dict:
        i = L.PlanInfo()
        L.check(L.load().mht_plan_info(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in L.PlanInfo._fields_}

    def level_info(self, level: int) -> dict:
        i = L.LevelInfo()
        L.check(L.load().mht_plan_level_info(self._h, level, C.byref(i)))
        return {k: getattr(i, k) for k, _ in L.LevelInfo._fields_}

    def launch_count(self, nrhs: int = 1) -> int:
        v = C.c_int64()
        L.check(L.load().mht_apply_launch_count(self._h, nrhs, C.byref(v)))
        return int(v.value)

    def check(self):
        """Raises MhtError(TIMEOUT) if a kernel gave up a bounded wait since the last check."""
        import torch
        f = C.c_int32()
        s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        L.check(L.load().mht_plan_check(self._h, s, C.byref(f)))
        return int(f.value)

    def set_path(self, path: str = "auto"):
        """'auto', 'staged' (one launch per stage) or 'fused' (one persistent launch)."""
        L.check(L.load().mht_plan_set_path(self._h, {"auto": 0, "staged": 1, "fused": 2}[path]))
        return self

    def set_mode(self, mode: str):
        """'fp32', '3xtf32' or '6xbf16' on a float plan (same packed factors, no rebinding)."""
        L.check(L.load().mht_plan_set_mode(self._h, _MODES[mode]))
        self.mode = mode
        return self

    def autotune(self, nrhs: int = 1):
        """Times each stage's candidate launch configurations for ``nrhs`` RHS and keeps the
        fastest (used by later applies with exactly ``nrhs`` RHS); returns the choices."""
        import torch
        s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        L.check(L.load().mht_plan_autotune(self._h, int(nrhs), s))
        out = []
        cfg = (C.c_int32 * 5)()
        ms = C.c_double()
        for d in (0, 1):
            for st in range(self.levels + 2):
                if L.load().mht_plan_tune_info(self._h, d, st, cfg, C.byref(ms)) == 0:
                    out.append({"direction": d, "stage": st, "tensor": cfg[0], "rhs_tile": cfg[1],
                                "slots": cfg[2], "ctas_per_sm": cfg[3], "slot_kb": cfg[4], "ms": ms.value})
        self.grouping = {}
        for d in (0, 1):  # stages grouped into one persistent launch at each end of a direction
            if L.load().mht_plan_tune_info(self._h, d, -1, cfg, C.byref(ms)) == 0:
                self.grouping[d] = {"head": cfg[1], "tail": cfg[2], "ms": ms.value}
        return out

    def profile(self, enable: bool = True):
        L.check(L.load().mht_plan_profile(self._h, 1 if enable else 0))

    def stage_times(self, direction: int):
        """(ms[L+3], launches[L+3]) summed since the last read (direction 0 synth, 1 analyze)."""
        ns = self.levels + 3
        ms = (C.c_double * ns)()
        ln = (C.c_int64 * ns)()
        L.check(L.load().mht_plan_stage_times(self._h, direction, ms, ln))
        return np.array(ms[:]), np.array(ln[:])

    def close(self):
        if self._h:
            L.load().mht_destroy(self._h)
            self._h = None
        self._dev = None  # releases the device buffers this plan allocated

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    # ---------------------------------------------------------------- device
    @property
    def dtype(self):
        import torch
        if self.mode == "fp64":
            return torch.complex128 if self.complex else torch.float64
        return torch.complex64 if self.complex else torch.float32

    def device_bytes(self, max_nrhs: int = 1):
        fb, wb = C.c_size_t(), C.c_size_t()
        L.check(L.load().mht_plan_device_bytes(self._h, max_nrhs, C.byref(fb), C.byref(wb)))
        return int(fb.value), int(wb.value)

    def bind(self, device="cuda", max_nrhs: int = 1, factor_buffer=None, workspace_buffer=None):
        """Allocates (or takes) device buffers and uploads the packed factors."""
        import torch
        fb, wb = self.device_bytes(max_nrhs)
        fac = factor_buffer if factor_buffer is not None else torch.empty(fb + 256, dtype=torch.uint8, device=device)
        ws = workspace_buffer if workspace_buffer is not None else torch.empty(wb + 256, dtype=torch.uint8, device=device)
        fp = (fac.data_ptr() + 255) // 256 * 256
        wp = (ws.data_ptr() + 255) // 256 * 256
        stream = torch.cuda.current_stream(fac.device).cuda_stream
        L.check(L.load().mht_plan_bind_device(self._h, C.c_void_p(fp), fb, C.c_void_p(wp), wb, max_nrhs,
                                              C.c_void_p(stream)))
        self._dev = (fac, ws, max_nrhs)
        return self

    @property
    def max_nrhs(self):
        return self._dev[2] if self._dev else 0

    def _colmajor(self, x, rows):
        import torch
        if x.dtype != self.dtype:
            raise TypeError(f"expected {self.dtype}, got {x.dtype}")
        if not x.is_cuda:
            raise ValueError("device transforms need CUDA tensors (use *_host for host arrays)")
        if x.shape[0] != rows:
            raise ValueError(f"expected {rows} rows, got {x.shape[0]}")
        if x.dim() == 1:
            return x.contiguous(), 1, True
        return x.t().contiguous(), x.shape[1], False  # (k, rows) C-order = column-major

    def _apply(self, x, synth: bool, weighted: bool):
        import torch
        lib = L.load()
        nin, nout = (self.m, self.n) if synth else (self.n, self.m)
        buf, k, vec = self._colmajor(x, nin)
        out = torch.empty((k, nout), dtype=self.dtype, device=x.device)
        stream = C.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
        if synth:
            fn = lib.mht_synthesize_weighted if weighted else lib.mht_synthesize
            L.check(fn(self._h, C.c_void_p(buf.data_ptr()), nin, C.c_void_p(out.data_ptr()), nout, k, stream))
        else:
            L.check(lib.mht_analyze(self._h, C.c_void_p(buf.data_ptr()), nin, C.c_void_p(out.data_ptr()), nout, k,
                                    1 if weighted else 0, stream))
        return out[0] if vec else out.t()

    def _real_vector(self, v, length, name):
        import torch
        rdt = torch.float64 if self.mode == "fp64" else torch.float32
        if v.dtype != rdt or not v.is_cuda or v.numel() != length:
            raise ValueError(f"{name} must be a CUDA {rdt} vector of {length} entries")
        return v.contiguous()

    def synthesize_scaled(self, c, scale):
        """f = Phi diag(scale) c, the scale fused into the leaf stage (GRF sampling, filters)."""
        import torch
        lib = L.load()
        buf, k, vec = self._colmajor(c, self.m)
        s = self._real_vector(scale, self.m, "scale")
        out = torch.empty((k, self.n), dtype=self.dtype, device=c.device)
        st = C.c_void_p(torch.cuda.current_stream(c.device).cuda_stream)
        L.check(lib.mht_synthesize_scaled(self._h, C.c_void_p(buf.data_ptr()), self.m, C.c_void_p(s.data_ptr()),
                                          C.c_void_p(out.data_ptr()), self.n, k, st))
        return out[0] if vec else out.t()

    def filter(self, f, filt, weighted: bool = True):
        """Phi diag(filt) Phi^H W f as one CUDA graph (analysis, fused diagonal, synthesis)."""
        import torch
        lib = L.load()
        buf, k, vec = self._colmajor(f, self.n)
        s = self._real_vector(filt, self.m, "filter")
        out = torch.empty((k, self.n), dtype=self.dtype, device=f.device)
        st = C.c_void_p(torch.cuda.current_stream(f.device).cuda_stream)
        L.check(lib.mht_filter(self._h, C.c_void_p(buf.data_ptr()), self.n, C.c_void_p(out.data_ptr()), self.n, k,
                               C.c_void_p(s.data_ptr()), 1 if weighted else 0, st))
        return out[0] if vec else out.t()

    def inverse(self, f, max_iter: int = 100, tol: float = 1e-6):
        """c = argmin ||Phi c - f||_2 by LSQR on the fast transform; returns (c, iterations,
        largest relative residual estimate)."""
        import torch
        lib = L.load()
        buf, k, vec = self._colmajor(f, self.n)
        nb = C.c_size_t()
        L.check(lib.mht_lsqr_scratch_bytes(self._h, k, C.byref(nb)))
        scratch = torch.empty(nb.value + 256, dtype=torch.uint8, device=f.device)
        sp = (scratch.data_ptr() + 255) // 256 * 256
        out = torch.empty((k, self.m), dtype=self.dtype, device=f.device)
        it, rr = C.c_int32(), C.c_double()
        st = C.c_void_p(torch.cuda.current_stream(f.device).cuda_stream)
        L.check(lib.mht_inverse_lsqr(self._h, C.c_void_p(buf.data_ptr()), self.n, C.c_void_p(out.data_ptr()), self.m,
                                     k, C.c_void_p(sp), nb.value, int(max_iter), float(tol), st, C.byref(it),
                                     C.byref(rr)))
        return (out[0] if vec else out.t()), int(it.value), float(rr.value)

    def synthesize_raw(self, c, weighted: bool = False):
        return self._apply(c, True, weighted)

    def analyze_raw(self, f, weighted: bool = True):
        return self._apply(f, False, weighted)

    # ---------------------------------------------------------------- host arrays
    def _host(self, x: np.ndarray, synth: bool, weighted: bool, stream=None):
        lib = L.load()
        npdt = {("fp64", False): np.float64, ("fp64", True): np.complex128}.get(
            (self.mode, self.complex), np.complex64 if self.complex else np.float32)
        nin, nout = (self.m, self.n) if synth else (self.n, self.m)
        vec = x.ndim == 1
        xin = np.asfortranarray(x.reshape(nin, -1), dtype=npdt)
        k = xin.shape[1]
        out = np.zeros((nout, k), dtype=npdt, order="F")
        s = C.c_void_p(stream or 0)
        if synth:
            L.check(lib.mht_synthesize_host(self._h, xin.ctypes.data_as(C.c_void_p), nin,
                                            out.ctypes.data_as(C.c_void_p), nout, k, s))
        else:
            L.check(lib.mht_analyze_host(self._h, xin.ctypes.data_as(C.c_void_p), nin,
                                         out.ctypes.data_as(C.c_void_p), nout, k, 1 if weighted else 0, s))
        return out[:, 0] if vec else out

    def synthesize_host(self, c: np.ndarray, stream=None) -> np.ndarray:
        return self._host(c, True, False, stream)

    def analyze_host(self, f: np.ndarray, weighted: bool = True, stream=None) -> np.ndarray:
        return self._host(f, False, weighted, stream)


def _autograd():
    import torch

    class Synthesize(torch.autograd.Function):
        """f = Phi c; the gradient is the unweighted adjoint sweep grad_c = Phi^H grad_f."""

        @staticmethod
        def forward(ctx, c, plan):
            ctx.plan = plan
            return plan.synthesize_raw(c)

        @staticmethod
        def backward(ctx, g):
            return ctx.plan.analyze_raw(g.contiguous() if g.dim() == 1 else g, weighted=False), None

    class Analyze(torch.autograd.Function):
        """c = Phi^H diag(w) f; the gradient is grad_f = diag(w) Phi grad_c."""

        @staticmethod
        def forward(ctx, f, plan, weighted):
            ctx.plan, ctx.weighted = plan, weighted
            return plan.analyze_raw(f, weighted)

        @staticmethod
        def backward(ctx, g):
            return ctx.plan.synthesize_raw(g, weighted=ctx.weighted), None, None

    return Synthesize, Analyze


_AG = None


class Batch:
    """Many FP32 plans applied together: one persistent launch per direction (CUDA graph).

    ``c[i]`` (m_i x k_i) and ``f[i]`` (n_i x k_i) are device tensors owned by the batch
    (column-major views); fill ``c`` and call :meth:`synthesize`, or fill ``f`` and call
    :meth:`analyze`.  The plans must stay alive until :meth:`bind` returns.
    """

    def __init__(self, plans, nrhs):
        lib = L.load()
        n = len(plans)
        if n == 0 or len(nrhs) != n:
            raise ValueError("need one RHS count per plan")
        hs = (C.c_void_p * n)(*[p._h for p in plans])
        ks = (C.c_int64 * n)(*[int(k) for k in nrhs])
        h = C.c_void_p()
        L.check(lib.mht_batch_create(hs, n, ks, C.byref(h)))
        self._h = h
        self._plans = list(plans)
        self.nrhs = [int(k) for k in nrhs]
        self.shapes = [(p.n, p.m, p.complex) for p in plans]
        self._dev = None
        self.c = self.f = None

    def device_bytes(self):
        ib, wb = C.c_size_t(), C.c_size_t()
        L.check(L.load().mht_batch_device_bytes(self._h, C.byref(ib), C.byref(wb)))
        return int(ib.value), int(wb.value)

    def bind(self, device="cuda"):
        import torch
        lib = L.load()
        ib, wb = self.device_bytes()
        img = torch.empty(ib + 256, dtype=torch.uint8, device=device)
        ws = torch.empty(wb + 256, dtype=torch.uint8, device=device)
        ip = (img.data_ptr() + 255) // 256 * 256
        wp = (ws.data_ptr() + 255) // 256 * 256
        stream = C.c_void_p(torch.cuda.current_stream(img.device).cuda_stream)
        L.check(lib.mht_batch_bind_device(self._h, C.c_void_p(ip), ib, C.c_void_p(wp), wb, stream))
        self._plans = None  # factors are on the device now
        cs, fs = [], []
        for (n, m, cplx), k in zip(self.shapes, self.nrhs):
            dt = torch.complex64 if cplx else torch.float32
            cs.append(torch.zeros((k, m), dtype=dt, device=img.device))
            fs.append(torch.zeros((k, n), dtype=dt, device=img.device))
        nb = len(cs)
        cp = (C.c_void_p * nb)(*[t.data_ptr() for t in cs])
        fp = (C.c_void_p * nb)(*[t.data_ptr() for t in fs])
        ldc = (C.c_int64 * nb)(*[m for (_, m, _) in self.shapes])
        ldf = (C.c_int64 * nb)(*[n for (n, _, _) in self.shapes])
        L.check(lib.mht_batch_set_io(self._h, cp, ldc, fp, ldf, stream))
        self._io = (cp, ldc, fp, ldf)
        self._dev = (img, ws, cs, fs)
        self.c = [t.t() for t in cs]  # m x k views of the column-major buffers
        self.f = [t.t() for t in fs]
        return self

    def reset_io(self):
        """Rewrites the device records of the batch's vectors (undoes a debug hold)."""
        cp, ldc, fp, ldf = self._io
        L.check(L.load().mht_batch_set_io(self._h, cp, ldc, fp, ldf, self._stream()))
        return self

    def _stream(self):
        import torch
        return C.c_void_p(torch.cuda.current_stream(self._dev[0].device).cuda_stream)

    def synthesize(self):
        """f[i] = Phi_i c[i] for every instance (one launch); returns the list f."""
        L.check(L.load().mht_batch_synthesize(self._h, self._stream()))
        return self.f

    def analyze(self, weighted: bool = True):
        """c[i] = Phi_i^H W_i f[i] (or without W) for every instance; returns the list c."""
        L.check(L.load().mht_batch_analyze(self._h, 1 if weighted else 0, self._stream()))
        return self.c

    def autotune(self):
        """Picks the fastest (ring slots, CTAs per SM) for this batch; overwrites f and c."""
        ms = C.c_double()
        L.check(L.load().mht_batch_autotune(self._h, self._stream(), C.byref(ms)))
        return ms.value

    def set_mode(self, mode: str = "fp32"):
        """'fp32': one persistent FP32 launch per direction; '3xtf32' / '6xbf16': a CUDA graph of
        each instance's own apply with tensor-core block products for wide RHS counts."""
        L.check(L.load().mht_batch_set_mode(self._h, _MODES[mode]))
        return self

    def set_graph(self, use_graph: bool = True):
        L.check(L.load().mht_batch_set_graph(self._h, 1 if use_graph else 0))
        return self

    def info(self):
        a, b, g = C.c_int64(), C.c_int64(), C.c_int32()
        L.check(L.load().mht_batch_info(self._h, C.byref(a), C.byref(b), C.byref(g)))
        return {"items_synthesis": int(a.value), "items_analysis": int(b.value), "grid": int(g.value)}

    def check(self):
        f = C.c_int32()
        L.check(L.load().mht_batch_check(self._h, self._stream(), C.byref(f)))
        return int(f.value)

    def close(self):
        if self._h:
            L.load().mht_batch_destroy(self._h)
            self._h = None
        self._dev = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def synthesize(plan: Plan, c):
    """Differentiable f = Phi c on the plan's device."""
    global _AG
    if _AG is None:
        _AG = _autograd()
    return _AG[0].apply(c, plan)


def analyze(plan: Plan, f, weighted: bool = True):
    """Differentiable c = Phi^H diag(w) f (w = the plan's weights; ones if none)."""
    global _AG
    if _AG is None:
        _AG = _autograd()
    return _AG[1].apply(f, plan, weighted)
