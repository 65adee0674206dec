"""Thin Python binding of the C ABI in include/feti.h (argument marshalling only).

Every numeric step runs in the CUDA library libfeti_gb300.so; this module only
converts NumPy inputs to the C structs, passes torch device pointers and the
current CUDA stream, and routes device allocations through torch's caching
allocator.  There is no CPU fallback: if the library is missing, loading
raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libfeti_gb300.so")

FETI_OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_ALLOC", 3: "ERR_NOT_SPD", 4: "ERR_NOT_CONVERGED",
          5: "ERR_CUDA", 6: "ERR_STATE", 7: "ERR_TIMEOUT"}
PREC = {"fp64": 0, "tf32": 1, "split_bf16": 2}

_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)


class FetiSubdomain(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("K_rowptr", _i64p), ("K_col", _i32p),
                ("K_val", _f64p), ("m", C.c_int32), ("B_rowptr", _i64p), ("B_col", _i32p),
                ("B_val", _f64p), ("B_lambda", _i32p), ("d", C.c_int32), ("R", _f64p), ("f", _f64p),
                ("nfix", C.c_int32), ("fix_dofs", _i32p), ("coords", _f64p), ("nelem", C.c_int32),
                ("edofs", C.c_int32), ("elem_dofs", _i32p), ("dKe", _f64p), ("dKe_ref", _f64p),
                ("dKe_scale", _f64p)]


class FetiProblem(C.Structure):
    _fields_ = [("nsub", C.c_int32), ("sub", C.POINTER(FetiSubdomain)), ("n_lambda", C.c_int32),
                ("c", _f64p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class FetiOptions(C.Structure):
    _fields_ = [("prec", C.c_int), ("refine_every", C.c_int32), ("tol", C.c_double), ("maxit", C.c_int32),
                ("recompute_X", C.c_int32), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("stream", C.c_void_p), ("leaf_dofs", C.c_int32),
                ("use_coords", C.c_int32), ("refine_drop", C.c_double), ("refine_restart", C.c_int32),
                ("precond", C.c_int32), ("adjoint_work_bytes", C.c_int64), ("assembly_route", C.c_int32),
                ("chol_split", C.c_int32), ("syrk_kernel", C.c_int32), ("chol_tc", C.c_int32), ("chol_tc_front", C.c_int32)]


class FetiSolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("refinements", C.c_int32), ("rel_residual", C.c_double),
                ("converged", C.c_int32), ("initial_residual", C.c_double)]


class FetiStats(C.Structure):
    _fields_ = [("nsub", C.c_int32), ("n_lambda", C.c_int32), ("npatterns", C.c_int32), ("nbplans", C.c_int32),
                ("sum_n", C.c_int64), ("sum_m", C.c_int64), ("L_doubles", C.c_int64), ("X_elems", C.c_int64),
                ("F_elems", C.c_int64), ("workspace_bytes", C.c_int64), ("device_bytes", C.c_int64),
                ("chol_flops", C.c_double), ("trsm_flops", C.c_double), ("syrk_flops", C.c_double),
                ("syrk_exec_flops", C.c_double), ("apply_bytes", C.c_double), ("implicit_bytes", C.c_double),
                ("t_chol_ms", C.c_double), ("t_trsm_ms", C.c_double), ("t_syrk_ms", C.c_double),
                ("t_coarse_ms", C.c_double), ("t_assemble_ms", C.c_double), ("t_chol_tc_ms", C.c_double),
                ("t_symbolic_ms", C.c_double),
                ("launches", C.c_int64), ("apply_calls", C.c_int64), ("apply_ms", C.c_double),
                ("apply_tiles_ms", C.c_double), ("implicit_calls", C.c_int64), ("implicit_ms", C.c_double),
                ("apply_variant", C.c_int32), ("apply_grid", C.c_int32), ("trsm_cols", C.c_int32),
                ("trsm_grid", C.c_int32), ("chol_tasks", C.c_int32), ("syrk_variant", C.c_int32), ("assembly_route", C.c_int32),
                ("route_ms", C.c_double * 3)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["route_ms"] = list(self.route_ms)
        return d



EXPORTS = ["feti_create", "feti_update_values", "feti_assemble", "feti_apply", "feti_apply_implicit",
           "feti_solve", "feti_solve_warm", "feti_adjoint", "feti_get_F", "feti_get_stats", "feti_last_error", "feti_destroy",
           "feti_analyse", "feti_analyse_lumped", "feti_version", "feti_apply_one_static", "feti_set_profiling",
           "feti_weighted_trace"]

_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libfeti_gb300.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.feti_create.argtypes = [C.POINTER(FetiProblem), C.POINTER(FetiOptions), C.POINTER(vp)]
    lib.feti_update_values.argtypes = [vp, C.c_int32, _f64p]
    lib.feti_assemble.argtypes = [vp]
    lib.feti_apply.argtypes = [vp, vp, vp]
    lib.feti_apply_implicit.argtypes = [vp, vp, vp]
    lib.feti_solve.argtypes = [vp, vp, vp, vp, C.POINTER(FetiSolveInfo)]
    lib.feti_solve_warm.argtypes = [vp, vp, vp, vp, C.POINTER(FetiSolveInfo)]
    lib.feti_adjoint.argtypes = [vp, vp, vp]
    lib.feti_weighted_trace.argtypes = [vp, vp, vp]
    lib.feti_get_F.argtypes = [vp, C.c_int32, _f64p]
    lib.feti_get_stats.argtypes = [vp, C.POINTER(FetiStats)]
    lib.feti_last_error.argtypes = [vp]
    lib.feti_last_error.restype = C.c_char_p
    lib.feti_destroy.argtypes = [vp]
    lib.feti_destroy.restype = None
    lib.feti_analyse.argtypes = [C.POINTER(FetiSubdomain), C.POINTER(FetiOptions), _f64p, _i32p, _i32p]
    lib.feti_analyse_lumped.argtypes = [C.POINTER(FetiProblem), vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.feti_version.restype = C.c_char_p
    lib.feti_apply_one_static.argtypes = [C.c_int32, C.c_int32, vp, vp, vp, vp, vp]
    lib.feti_set_profiling.argtypes = [vp, C.c_int32]
    for name in EXPORTS:
        if name not in ("feti_last_error", "feti_destroy", "feti_version"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class FetiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


class _Marshal:
    """Keeps the NumPy arrays behind a FetiProblem alive during feti_create."""

    def __init__(self, problem, with_elements=False, unit_scale=False, per_element=False):
        self.keep = []
        subs = (FetiSubdomain * problem.nsub)()
        for i, s in enumerate(problem.subs):
            sub = subs[i]
            a = lambda x, dt: self._k(np.ascontiguousarray(x, dtype=dt))
            sub.n = s.n
            sub.nnz = s.K_col.shape[0]
            sub.K_rowptr = _ptr(a(s.K_rowptr, np.int64), C.c_int64)
            sub.K_col = _ptr(a(s.K_col, np.int32), C.c_int32)
            sub.K_val = _ptr(a(s.K_val, np.float64), C.c_double)
            sub.m = s.m
            sub.B_rowptr = _ptr(a(np.arange(s.m + 1), np.int64), C.c_int64)
            sub.B_col = _ptr(a(s.B_dof, np.int32), C.c_int32)
            sub.B_val = _ptr(a(s.B_sign, np.float64), C.c_double)
            sub.B_lambda = _ptr(a(s.B_lambda, np.int32), C.c_int32)
            sub.d = s.R.shape[1]
            sub.R = _ptr(a(np.asfortranarray(s.R).ravel(order="F"), np.float64), C.c_double)
            sub.f = _ptr(a(s.f, np.float64), C.c_double)
            sub.nfix = len(s.fix_dofs)
            sub.fix_dofs = _ptr(a(s.fix_dofs, np.int32), C.c_int32)
            sub.coords = _ptr(a(s.coords, np.float64), C.c_double) if s.coords is not None else None
            if with_elements:
                sub.nelem = s.elem_dofs.shape[0]
                sub.edofs = s.elem_dofs.shape[1]
                sub.elem_dofs = _ptr(a(s.elem_dofs, np.int32), C.c_int32)
                scale = np.ones(s.elem_dofs.shape[0]) if unit_scale else s.elem_dcoef
                if per_element:
                    # one d K_e / d theta_e matrix per element (the general form of the ABI)
                    dke = scale[:, None, None] * np.asarray(problem.K_ref)[None]
                    sub.dKe = _ptr(a(dke, np.float64), C.c_double)
                else:
                    sub.dKe_ref = _ptr(a(problem.K_ref, np.float64), C.c_double)
                    sub.dKe_scale = _ptr(a(scale, np.float64), C.c_double)
        self.subs = subs
        self.c = self._k(np.ascontiguousarray(problem.c, dtype=np.float64))
        self.prob = FetiProblem(problem.nsub, subs, problem.n_lambda, _ptr(self.c, C.c_double))

    def _k(self, x):
        self.keep.append(x)
        return x


def subdomain_struct(s, keep):
    """FetiSubdomain for one problems.Subdomain (used by feti_analyse)."""
    class _P:
        pass
    p = _P()
    p.subs = [s]
    p.nsub = 1
    p.c = np.zeros(0)
    p.n_lambda = 0
    m = _Marshal(p)
    keep.append(m)
    return m.subs[0]


def analyse(sub, leaf_dofs=16, use_coords=True, route="syrk"):
    """Host-only symbolic analysis of one subdomain (no GPU): returns a dict
    of the plan's statistics, the permutation and the supernode partition."""
    lib = load_library()
    keep = []
    st = subdomain_struct(sub, keep)
    opt = FetiOptions()
    opt.leaf_dofs = leaf_dofs
    opt.use_coords = 1 if use_coords else 0
    opt.assembly_route = {"syrk": 0, "schur": 1}[route]
    info = np.zeros(16)
    perm = np.zeros(sub.n, dtype=np.int32)
    snb = np.zeros(4 * sub.n, dtype=np.int32)
    rc = lib.feti_analyse(C.byref(st), C.byref(opt), _ptr(info, C.c_double), _ptr(perm, C.c_int32),
                          _ptr(snb, C.c_int32))
    if rc != FETI_OK:
        raise FetiError(rc, "feti_analyse failed")
    keys = ["n", "nsn", "max_front", "max_width", "nnzL", "chol_flops", "Lsize", "m", "Xsize", "trsm_flops",
            "syrk_flops", "ntile_contrib", "chol_stack", "rhs_stack", "nroots", "nlast"]
    out = {k: info[i] for i, k in enumerate(keys)}
    ns = int(out["nsn"])
    out["perm"] = perm
    out["sn_c0"] = snb[:ns].copy()
    out["sn_w"] = snb[ns:2 * ns].copy()
    out["sn_parent"] = snb[2 * ns:3 * ns].copy()
    out["sn_r"] = snb[3 * ns:4 * ns].copy()
    return out


class FetiOperator:
    """Explicit FETI dual operator on one GPU (wraps feti_create / feti_assemble /
    feti_apply / feti_apply_implicit / feti_solve / feti_solve_warm / feti_adjoint).

    prec: "fp64", "tf32" or "split_bf16" (tensor-core TRSM updates and SYRK,
    FP32 F tiles); route: "syrk" (pruned TRSM + SYRK on a nested-dissection
    ordering) or "schur" (the DOFs B touches ordered last, F_i from the
    factor of their Schur complement); refine_every / refine_drop / refine_restart: the FP64
    residual replacement of the mixed solve; precond: "none" (M = I) or
    "lumped" (M = (BB^T)^-1 sum_i B_i K_i B_i^T (BB^T)^-1) or "dirichlet"
    (the same with the Schur complements S_i of K_i onto the DOFs B touches in
    place of K_i; needs route="schur"); chol_split: "auto" (autotuned), "whole"
    (one subdomain per CTA) or "tasks" (heavy subtrees on CTAs of their own); syrk_kernel: -1 (autotuned)
    or the split-bf16 SYRK kernel 0, 1, 2 to use; chol_tc: the large fronts' updates on
    the tensor cores (exact bf16 slicing) or all of the Cholesky on the FP64 pipe."""

    def __init__(self, problem, prec: str = "fp64", tol: float = 1e-10, maxit: int = 2000,
                 refine_every: int = 0, refine_drop: float = 0.0, refine_restart: bool = False,
                 precond: str = "none", leaf_dofs: int = 16, use_coords: bool = True,
                 with_elements: bool = False, unit_scale: bool = False, per_element: bool = False,
                 recompute_X: bool = False, adjoint_work_bytes: int = 0, route: str = "syrk",
                 chol_split: str = "auto", syrk_kernel: int = -1, chol_tc: bool = True,
                 chol_tc_front: int = 0, torch_alloc: bool = True):
        import torch
        self.torch = torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("FetiOperator needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream(self.device)
        self.problem = problem
        self.n_lambda = problem.n_lambda
        self.dtot = sum(s.R.shape[1] for s in problem.subs)
        self.sum_n = sum(s.n for s in problem.subs)
        opt = FetiOptions()
        opt.prec = PREC[prec]
        opt.refine_every = refine_every
        opt.refine_drop = refine_drop
        opt.refine_restart = 1 if refine_restart else 0
        opt.precond = {"none": 0, "lumped": 1, "dirichlet": 2}[precond]
        opt.tol = tol
        opt.maxit = maxit
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        opt.leaf_dofs = leaf_dofs
        opt.use_coords = 1 if use_coords else 0
        opt.recompute_X = 1 if recompute_X else 0
        opt.adjoint_work_bytes = int(adjoint_work_bytes)
        opt.assembly_route = {"syrk": 0, "schur": 1, "trsm": 2, "auto": 3}[route]
        opt.chol_split = {"auto": 0, "whole": 1, "tasks": 2}[chol_split]
        opt.syrk_kernel = 0 if syrk_kernel < 0 else syrk_kernel + 1
        opt.chol_tc = 0 if chol_tc else 1
        opt.chol_tc_front = int(chol_tc_front)
        self._cb = None
        if torch_alloc:
            dev = self.device.index
            st = self.stream.cuda_stream

            def _alloc(nbytes, _ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:
                    return None

            def _free(ptr, _ctx):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            opt.dev_alloc, opt.dev_free = self._cb
        self.opt = opt
        m = _Marshal(problem, with_elements=with_elements, unit_scale=unit_scale, per_element=per_element)
        h = C.c_void_p()
        rc = self.lib.feti_create(C.byref(m.prob), C.byref(opt), C.byref(h))
        self.h = h
        if rc != FETI_OK:
            msg = self.lib.feti_last_error(h).decode() if h else ""
            if h:
                self.lib.feti_destroy(h)
                self.h = None
            raise FetiError(rc, msg)

    # -- helpers
    def _check(self, rc):
        if rc != FETI_OK:
            raise FetiError(rc, self.lib.feti_last_error(self.h).decode())

    def _dvec(self, n):
        return self.torch.empty(n, dtype=self.torch.float64, device=self.device)

    # -- API
    def assemble(self):
        self._check(self.lib.feti_assemble(self.h))

    def update_values(self, sub, K_val):
        K_val = np.ascontiguousarray(K_val, dtype=np.float64)
        self._check(self.lib.feti_update_values(self.h, sub, _ptr(K_val, C.c_double)))

    def apply(self, p, out=None):
        assert p.dtype == self.torch.float64 and p.is_cuda and p.numel() == self.n_lambda
        p = p.contiguous()
        q = out if out is not None else self._dvec(self.n_lambda)
        self._check(self.lib.feti_apply(self.h, C.c_void_p(p.data_ptr()), C.c_void_p(q.data_ptr())))
        return q

    def apply_implicit(self, p, out=None):
        p = p.contiguous()
        q = out if out is not None else self._dvec(self.n_lambda)
        self._check(self.lib.feti_apply_implicit(self.h, C.c_void_p(p.data_ptr()), C.c_void_p(q.data_ptr())))
        return q

    def solve(self, lambda_guess=None):
        """PCPG solve (feti_solve); with lambda_guess (n_lambda values) it starts
        from lambda_I + P lambda_guess (feti_solve_warm)."""
        lam = self._dvec(self.n_lambda)
        alpha = self._dvec(max(self.dtot, 1))
        u = self._dvec(self.sum_n)
        info = FetiSolveInfo()
        fn = self.lib.feti_solve
        if lambda_guess is not None:
            lam.copy_(self.torch.as_tensor(lambda_guess, dtype=self.torch.float64).reshape(-1))
            fn = self.lib.feti_solve_warm
        rc = fn(self.h, C.c_void_p(lam.data_ptr()), C.c_void_p(alpha.data_ptr()),
                C.c_void_p(u.data_ptr()), C.byref(info))
        if rc not in (FETI_OK, 4):
            self._check(rc)
        return lam, alpha[:self.dtot], u, dict(iterations=info.iterations, refinements=info.refinements,
                                                 rel_residual=info.rel_residual, converged=bool(info.converged),
                                                 initial_residual=info.initial_residual)

    def adjoint(self, W):
        """dL/dtheta_e for L = sum_i <W_i, F_i> (feti_adjoint).  W: list of
        m_i x m_i arrays/tensors in B-row order, or one concatenated FP64 CUDA
        tensor.  Returns a CUDA FP64 tensor over all elements (subdomain order)."""
        W = self._W_dev(W)
        nel = sum(s.elem_dofs.shape[0] for s in self.problem.subs)
        out = self._dvec(nel)
        self._check(self.lib.feti_adjoint(self.h, C.c_void_p(W.data_ptr()), C.c_void_p(out.data_ptr())))
        return out

    def _W_dev(self, W):
        torch = self.torch
        if isinstance(W, (list, tuple)):
            W = torch.cat([torch.as_tensor(w, dtype=torch.float64).reshape(-1) for w in W]).to(self.device)
        return W.contiguous()

    def weighted_trace(self, W):
        """L = sum_i <W_i, F_i> of the assembled F_i (feti_weighted_trace); W as in adjoint.
        Returns a one-element FP64 CUDA tensor."""
        W = self._W_dev(W)
        out = self._dvec(1)
        self._check(self.lib.feti_weighted_trace(self.h, C.c_void_p(W.data_ptr()), C.c_void_p(out.data_ptr())))
        return out

    def get_F(self, sub):
        m = self.problem.subs[sub].m
        out = np.zeros((m, m))
        self._check(self.lib.feti_get_F(self.h, sub, _ptr(out, C.c_double)))
        return out

    def set_profiling(self, enable=True):
        self._check(self.lib.feti_set_profiling(self.h, 1 if enable else 0))

    def stats(self):
        st = FetiStats()
        self._check(self.lib.feti_get_stats(self.h, C.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.torch.cuda.synchronize(self.device)
            self.lib.feti_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _feti_weighted_trace():
    import torch

    class FetiWeightedTrace(torch.autograd.Function):
        """L(coef) = sum_i <W_i, F_i(coef)>, K_e = coef_e K_ref per element.

        forward sets the CSR values of K_i from the element coefficients
        (finite-element assembly of the inputs), runs feti_assemble and forms
        L on the device (feti_weighted_trace); backward maps dL/dF_i = W_i to
        dL/dcoef_e with the FP64 adjoint kernel (feti_adjoint, X_i recomputed
        from L_i).  The operator must be created with with_elements=True and
        unit_scale=True (dK_e/dcoef_e = K_ref)."""

        @staticmethod
        def forward(ctx, coef, op, Ws):
            from .problems import subdomain_K_values
            c = coef.detach().cpu().numpy()
            off = 0
            for i, s in enumerate(op.problem.subs):
                ne = s.elem_dofs.shape[0]
                op.update_values(i, subdomain_K_values(op.problem, i, c[off:off + ne]))
                off += ne
            op.assemble()
            Wd = op._W_dev(Ws)
            L = op.weighted_trace(Wd)[0]
            ctx.op, ctx.Wd = op, Wd
            return L.to(coef.device)

        @staticmethod
        def backward(ctx, grad_out):
            g = ctx.op.adjoint(ctx.Wd)
            return grad_out * g.to(grad_out.device), None, None

    return FetiWeightedTrace


def weighted_trace(coef, op, Ws):
    """Differentiable L = sum_i <W_i, F_i(coef)> (see FetiWeightedTrace)."""
    return _feti_weighted_trace().apply(coef, op, Ws)


def lumped_plan(problem):
    """Host plan of the lumped preconditioner (feti_analyse_lumped): returns
    dict(w_off, w_col, w_val, m_off, m_col, c_off, c_kidx, c_sign) as NumPy
    arrays.  No device is needed."""
    lib = load_library()
    m = _Marshal(problem)
    sizes = np.zeros(3, dtype=np.int64)
    nul = C.c_void_p()
    rc = lib.feti_analyse_lumped(C.byref(m.prob), sizes.ctypes.data_as(C.c_void_p), *([nul] * 8))
    if rc != FETI_OK:
        raise FetiError(rc, "feti_analyse_lumped rejected the problem")
    n = problem.n_lambda
    out = dict(w_off=np.zeros(n + 1, np.int32), w_col=np.zeros(sizes[0], np.int32), w_val=np.zeros(sizes[0]),
               m_off=np.zeros(n + 1, np.int32), m_col=np.zeros(sizes[1], np.int32),
               c_off=np.zeros(sizes[1] + 1, np.int64), c_kidx=np.zeros(sizes[2], np.int64), c_sign=np.zeros(sizes[2]))
    ptr = [out[k].ctypes.data_as(C.c_void_p) for k in ("w_off", "w_col", "w_val", "m_off", "m_col", "c_off",
                                                        "c_kidx", "c_sign")]
    rc = lib.feti_analyse_lumped(C.byref(m.prob), sizes.ctypes.data_as(C.c_void_p), *ptr)
    if rc != FETI_OK:
        raise FetiError(rc, "feti_analyse_lumped rejected the problem")
    return out
