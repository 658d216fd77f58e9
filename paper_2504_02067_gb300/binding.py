"""Thin Python binding of the C ABI declared in include/eot.h.

Argument marshalling only: tensors become raw device pointers, the current torch
stream becomes the cudaStream_t, and every computation runs inside libeot.so.
There is no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import buildlib as _build

EOT_OK = 0
STATUS_NAMES = {0: "EOT_OK", 1: "EOT_ERR_INVALID_ARG", 2: "EOT_ERR_NONFINITE",
                3: "EOT_ERR_CG_MAXITER", 4: "EOT_ERR_LINESEARCH", 5: "EOT_ERR_MAXSTAGES",
                6: "EOT_ERR_MAXNEWTON", 7: "EOT_ERR_RANGE", 8: "EOT_ERR_CUDA",
                9: "EOT_ERR_UNSUPPORTED", 10: "EOT_ERR_DEVICE_TIMEOUT", 11: "EOT_ERR_TIME_LIMIT"}

COST_DENSE_F32, COST_DENSE_F64, COST_SQEUCLID_POINTS = 0, 1, 2
PRECISIONS = {"fp64": 0, "mixed": 1, "plain_fp32": 2}


class EotProblem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("d", ctypes.c_int64),
                ("ldc", ctypes.c_int64), ("C", ctypes.c_void_p), ("X", ctypes.c_void_p),
                ("Y", ctypes.c_void_p), ("cost_scale", ctypes.c_double),
                ("r", ctypes.c_void_p), ("c", ctypes.c_void_p)]


class EotParams(ctypes.Structure):
    _fields_ = [("gamma_i", ctypes.c_double), ("gamma_f", ctypes.c_double),
                ("p", ctypes.c_double), ("q1", ctypes.c_double), ("w_r", ctypes.c_double),
                ("tol_final", ctypes.c_double), ("max_stages", ctypes.c_int32),
                ("max_newton", ctypes.c_int32), ("max_cg", ctypes.c_int32),
                ("max_ls", ctypes.c_int32), ("projector", ctypes.c_int32),
                ("max_sinkhorn", ctypes.c_int32), ("newton_system", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("max_seconds", ctypes.c_double)]


PROJECT_NEWTON, PROJECT_SINKHORN = 0, 1
NEWTON_REDUCED, NEWTON_FULL = 0, 1


class EotStageRecord(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("eps", ctypes.c_double), ("delta_min", ctypes.c_double),
                ("q_next", ctypes.c_double), ("newton_steps", ctypes.c_int32),
                ("cg_iters", ctypes.c_int32), ("ls_trials", ctypes.c_int32),
                ("sinkhorn_iters", ctypes.c_int32), ("sweeps", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class EotStats(ctypes.Structure):
    _fields_ = [("sweeps_cg", ctypes.c_int64), ("sweeps_newton", ctypes.c_int64),
                ("sweeps_linesearch", ctypes.c_int64), ("sweeps_sinkhorn", ctypes.c_int64),
                ("sweeps_total", ctypes.c_int64), ("stages", ctypes.c_int32),
                ("newton_steps", ctypes.c_int32), ("cg_iters", ctypes.c_int32),
                ("cg_solves", ctypes.c_int32), ("ls_trials", ctypes.c_int32),
                ("sinkhorn_iters", ctypes.c_int32), ("curvature_stops", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("final_gamma", ctypes.c_double),
                ("final_rho", ctypes.c_double), ("grad_l1", ctypes.c_double),
                ("marg_err_l1", ctypes.c_double), ("seconds", ctypes.c_double),
                ("sweeps_stage", ctypes.c_int64), ("stage_records", ctypes.POINTER(EotStageRecord)),
                ("stage_records_cap", ctypes.c_int32), ("stage_records_len", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "stage_records"}
        if self.stage_records:
            d["stage_records"] = [self.stage_records[i].as_dict() for i in range(self.stage_records_len)]
        return d


EXPORTS = ["eot_create", "eot_destroy", "eot_last_error", "eot_status_string",
           "eot_params_default", "eot_marginals", "eot_hvp", "eot_newton_solve", "eot_solve",
           "eot_backward", "eot_sweep_bench", "eot_marginals_noalloc", "eot_kernel_launches",
           "eot_solve_batched", "eot_batch_last_config", "eot_round", "eot_value",
           "eot_plan_argmax", "eot_plan_support", "eot_newton_solve_full"]

_LIB = None


def load_library(path=None):
    """Load libeot.so (built by build.build()); raises if it is absent."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    path = path or _build.LIBPATH
    if not os.path.exists(path):
        raise RuntimeError("libeot.so is not built (expected at %s); run "
                           "paper_2504_02067_gb300.build.build() first" % path)
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    P = ctypes.POINTER(EotProblem)
    L.eot_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, i64, i64, i64]
    L.eot_destroy.argtypes = [vp]
    L.eot_last_error.argtypes = [vp]
    L.eot_last_error.restype = ctypes.c_char_p
    L.eot_status_string.argtypes = [ctypes.c_int]
    L.eot_status_string.restype = ctypes.c_char_p
    L.eot_params_default.restype = EotParams
    L.eot_marginals.argtypes = [vp, P, vp, vp, dbl, vp, vp, vp, vp, vp, vp]
    L.eot_hvp.argtypes = [vp, P, vp, vp, dbl, dbl, vp, vp, vp, vp, vp, vp, vp]
    L.eot_newton_solve.argtypes = [vp, P, vp, vp, dbl, vp, dbl, dbl, i32, vp, vp,
                                   ctypes.POINTER(dbl), ctypes.POINTER(i32), vp]
    L.eot_newton_solve_full.argtypes = L.eot_newton_solve.argtypes
    L.eot_solve.argtypes = [vp, P, ctypes.POINTER(EotParams), vp, vp, ctypes.POINTER(EotStats), vp]
    L.eot_backward.argtypes = [vp, P, vp, vp, dbl, dbl, vp, vp, vp, vp, vp, vp, vp]
    L.eot_value.argtypes = [vp, P, vp, vp, dbl, vp, vp]
    L.eot_plan_argmax.argtypes = [vp, P, vp, dbl, vp, vp]
    L.eot_plan_support.argtypes = [vp, P, vp, vp, dbl, dbl, vp, vp, vp]
    L.eot_sweep_bench.argtypes = [vp, P, vp, vp, dbl, i32, i32, vp, ctypes.c_size_t, ctypes.POINTER(dbl), vp]
    L.eot_marginals_noalloc.argtypes = [P, vp, vp, dbl, vp, vp, vp, vp]
    L.eot_marginals_noalloc.restype = ctypes.c_int
    L.eot_solve_batched.argtypes = [vp, i32, P, ctypes.POINTER(EotParams), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.POINTER(i32), ctypes.POINTER(EotStats),
                                    vp]
    L.eot_batch_last_config.argtypes = [vp, ctypes.POINTER(i32)]
    L.eot_batch_last_config.restype = ctypes.c_int
    L.eot_round.argtypes = [vp, P, vp, vp, dbl, vp, vp, vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp]
    L.eot_kernel_launches.argtypes = [vp]
    L.eot_kernel_launches.restype = i64
    for f in ("eot_create", "eot_destroy", "eot_marginals", "eot_hvp", "eot_newton_solve",
              "eot_solve", "eot_backward", "eot_sweep_bench", "eot_solve_batched", "eot_round",
              "eot_value", "eot_plan_argmax", "eot_plan_support", "eot_newton_solve_full"):
        getattr(L, f).restype = ctypes.c_int
    if path == _build.LIBPATH:
        _LIB = L
    return L


class EotError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Problem:
    """An eot_problem over torch tensors (kept alive by this object).

    Dense: C (float32 -> DENSE_F32 with precision "mixed" or "plain_fp32";
    float64 -> DENSE_F64, precision "fp64"), r, c float64 on the device.
    """

    def __init__(self, C=None, r=None, c=None, precision=None, X=None, Y=None, cost_scale=0.0):
        self.C, self.r, self.c, self.X, self.Y = C, r, c, X, Y
        s = EotProblem()
        if C is not None:
            assert C.dim() == 2 and C.stride(1) == 1, "C must be row-major with unit column stride"
            s.kind = COST_DENSE_F64 if C.dtype == torch.float64 else COST_DENSE_F32
            s.n, s.m = C.shape
            s.ldc = C.stride(0)
            s.C = C.data_ptr()
            if precision is None:
                precision = "fp64" if C.dtype == torch.float64 else "mixed"
        else:
            s.kind = COST_SQEUCLID_POINTS
            s.n, s.d = X.shape
            s.m = Y.shape[0]
            s.X, s.Y = X.data_ptr(), Y.data_ptr()
            precision = precision or "mixed"
        s.precision = PRECISIONS[precision]
        s.cost_scale = cost_scale
        s.r = r.data_ptr() if r is not None else None
        s.c = c.data_ptr() if c is not None else None
        self.struct = s
        self.n, self.m, self.d = int(s.n), int(s.m), int(s.d)
        self.precision = precision

    def ref(self):
        return ctypes.byref(self.struct)


class Handle:
    """Owns an eot_handle (device workspace)."""

    def __init__(self, device=0, max_n=1, max_m=1, max_d=0):
        self.lib = load_library()
        self.h = ctypes.c_void_p()
        self.device = device
        st = self.lib.eot_create(ctypes.byref(self.h), device, max_n, max_m, max_d)
        if st != EOT_OK:
            raise EotError(st, "eot_create failed")

    def close(self):
        if self.h:
            self.lib.eot_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        if st != EOT_OK:
            raise EotError(st, self.lib.eot_last_error(self.h).decode())

    def launches(self):
        return int(self.lib.eot_kernel_launches(self.h))

    # ---- same names as the C ABI; outputs are caller-provided tensors ----
    def eot_marginals(self, prob, u, v, gamma, r_out=None, c_out=None, log_r_out=None,
                      log_c_out=None, total_out=None, stream=None):
        self.check(self.lib.eot_marginals(self.h, prob.ref(), _p(u), _p(v), float(gamma),
                                          _p(r_out), _p(c_out), _p(log_r_out), _p(log_c_out),
                                          _p(total_out), _stream(stream)))

    def eot_round(self, prob, u, v, gamma, u_out=None, v_out=None, a_out=None, b_out=None,
                  stream=None):
        """Round of P(u, v; gamma) onto U(r, c) (eot_round of include/eot.h); returns
        (<Round(P), C>, ||a||_1) and fills the given implicit-plan outputs."""
        cost = ctypes.c_double(0.0)
        corr = ctypes.c_double(0.0)
        self.check(self.lib.eot_round(self.h, prob.ref(), _p(u), _p(v), float(gamma), _p(u_out),
                                      _p(v_out), _p(a_out), _p(b_out), ctypes.byref(cost),
                                      ctypes.byref(corr), _stream(stream)))
        return cost.value, corr.value

    def eot_hvp(self, prob, u, v, gamma, s, du, dv, out_u, out_v, r_out=None, c_out=None,
                stream=None):
        self.check(self.lib.eot_hvp(self.h, prob.ref(), _p(u), _p(v), float(gamma), float(s),
                                    _p(du), _p(dv), _p(out_u), _p(out_v), _p(r_out), _p(c_out),
                                    _stream(stream)))

    def eot_newton_solve(self, prob, u, v, gamma, r_target, eta, rho0, du_out, dv_out=None,
                         max_cg=0, stream=None, full=False):
        """NewtonSolve (Alg. 2); full=True: eot_newton_solve_full (the full discounted system)."""
        rho = ctypes.c_double(0.0)
        it = ctypes.c_int32(0)
        fn = self.lib.eot_newton_solve_full if full else self.lib.eot_newton_solve
        self.check(fn(self.h, prob.ref(), _p(u), _p(v), float(gamma), _p(r_target), float(eta),
                      float(rho0), int(max_cg), _p(du_out), _p(dv_out), ctypes.byref(rho),
                      ctypes.byref(it), _stream(stream)))
        return rho.value, it.value

    def eot_solve(self, prob, params, u, v, stream=None, stage_records=256):
        """Returns the call's EotStats; with stage_records > 0 it also carries up to
        that many per-stage records of Alg. 1 (stats.as_dict()["stage_records"])."""
        stats = EotStats()
        if stage_records > 0:
            stats._records = (EotStageRecord * stage_records)()  # kept alive with stats
            stats.stage_records = ctypes.cast(stats._records, ctypes.POINTER(EotStageRecord))
            stats.stage_records_cap = stage_records
        st = self.lib.eot_solve(self.h, prob.ref(), ctypes.byref(params), _p(u), _p(v),
                                ctypes.byref(stats), _stream(stream))
        if st != EOT_OK:
            err = EotError(st, self.lib.eot_last_error(self.h).decode())
            err.stats = stats.as_dict()  # the work done before the error (see include/eot.h)
            raise err
        return stats

    def eot_backward(self, prob, u, v, gamma, grad_scale=1.0, dC=None, dX=None, dY=None,
                     dr=None, dc=None, grad_scale_dev=None, stream=None):
        self.check(self.lib.eot_backward(self.h, prob.ref(), _p(u), _p(v), float(gamma),
                                         float(grad_scale), _p(grad_scale_dev), _p(dC), _p(dX),
                                         _p(dY), _p(dr), _p(dc), _stream(stream)))

    def eot_value(self, prob, u, v, gamma, value_out, stream=None):
        """The dual value (<r, u> + <c, v> - sum P + 1) / gamma into a device FP64 scalar."""
        self.check(self.lib.eot_value(self.h, prob.ref(), _p(u), _p(v), float(gamma), _p(value_out),
                                      _stream(stream)))

    def eot_plan_argmax(self, prob, v, gamma, idx_out, stream=None):
        """Row argmax of the plan (lowest index on ties) into a device int64 tensor [n]."""
        self.check(self.lib.eot_plan_argmax(self.h, prob.ref(), _p(v), float(gamma), _p(idx_out),
                                            _stream(stream)))

    def eot_plan_support(self, prob, u, v, gamma, log_tau, row_counts_out=None, total_out=None,
                         stream=None):
        """Counts of plan entries above exp(log_tau), per row and in total (device int64)."""
        self.check(self.lib.eot_plan_support(self.h, prob.ref(), _p(u), _p(v), float(gamma),
                                             float(log_tau), _p(row_counts_out), _p(total_out),
                                             _stream(stream)))

    def eot_sweep_bench(self, prob, u, v, gamma, kind, iters, flush=None, stream=None):
        """Milliseconds per launch of sweep kind `kind`; with `flush` (a device
        tensor larger than L2) every launch is timed alone after overwriting it."""
        ms = ctypes.c_double(0.0)
        nbytes = flush.numel() * flush.element_size() if flush is not None else 0
        self.check(self.lib.eot_sweep_bench(self.h, prob.ref(), _p(u), _p(v), float(gamma),
                                            int(kind), int(iters), _p(flush), nbytes,
                                            ctypes.byref(ms), _stream(stream)))
        return ms.value

    def eot_solve_batched(self, probs, params, us, vs, stream=None):
        """probs: list of point Problems; us, vs: lists of output tensors. Returns
        (per-problem status list, per-problem stats dicts); raises on a failed launch."""
        k = len(probs)
        arr = (EotProblem * k)(*[p.struct for p in probs])
        up = (ctypes.c_void_p * k)(*[u.data_ptr() for u in us])
        vq = (ctypes.c_void_p * k)(*[v.data_ptr() for v in vs])
        st = (ctypes.c_int32 * k)(*([-1] * k))
        stats = (EotStats * k)()
        rc = self.lib.eot_solve_batched(self.h, k, arr, ctypes.byref(params), up, vq, st, stats,
                                        _stream(stream))
        if rc != EOT_OK and (rc == 8 or all(x == -1 for x in st)):
            self.check(rc)  # the batch did not run (bad arguments) or its launch failed
        return [int(x) for x in st], [s.as_dict() for s in stats]

    def batch_last_config(self):
        out = (ctypes.c_int32 * 3)()
        self.check(self.lib.eot_batch_last_config(self.h, out))
        return tuple(int(x) for x in out)

    # ---- conveniences that allocate the outputs ----
    def marginals(self, prob, u, v, gamma):
        dev = u.device
        r = torch.empty(prob.n, dtype=torch.float64, device=dev)
        c = torch.empty(prob.m, dtype=torch.float64, device=dev)
        lr = torch.empty_like(r)
        lc = torch.empty_like(c)
        tot = torch.empty(1, dtype=torch.float64, device=dev)
        self.eot_marginals(prob, u, v, gamma, r, c, lr, lc, tot)
        return r, c, lr, lc, tot

    def hvp(self, prob, u, v, gamma, s, du, dv):
        ou, ov = torch.empty_like(du), torch.empty_like(dv)
        r, c = torch.empty_like(du), torch.empty_like(dv)
        self.eot_hvp(prob, u, v, gamma, s, du, dv, ou, ov, r, c)
        return ou, ov, r, c

    def newton_solve(self, prob, u, v, gamma, r_target, eta, rho0=0.0, max_cg=0, full=False):
        du, dv = torch.empty_like(u), torch.empty_like(v)
        rho, it = self.eot_newton_solve(prob, u, v, gamma, r_target, eta, rho0, du, dv, max_cg, full=full)
        return du, dv, rho, it

    def solve(self, prob, params=None, **overrides):
        p = params or default_params()
        for k, val in overrides.items():
            setattr(p, k, val)
        dev = prob.r.device
        u = torch.empty(prob.n, dtype=torch.float64, device=dev)
        v = torch.empty(prob.m, dtype=torch.float64, device=dev)
        stats = self.eot_solve(prob, p, u, v)
        return u, v, stats.as_dict()


def solve_batched(handle, probs, params=None, **overrides):
    """Solve a list of point Problems in one launch; returns (us, vs, statuses, stats)."""
    p = params or default_params()
    for k, val in overrides.items():
        setattr(p, k, val)
    us = [torch.empty(q.n, dtype=torch.float64, device=q.r.device) for q in probs]
    vs = [torch.empty(q.m, dtype=torch.float64, device=q.r.device) for q in probs]
    st, stats = handle.eot_solve_batched(probs, p, us, vs)
    return us, vs, st, stats


def default_params(**overrides):
    p = load_library().eot_params_default()
    for k, val in overrides.items():
        setattr(p, k, val)
    return p


def eot_marginals_noalloc(prob, u, v, gamma, r_out, c_out, status_out=None, stream=None):
    """eot_marginals_noalloc of include/eot.h: marginals into caller-provided
    tensors, no handle, no device allocation by the library."""
    st = load_library().eot_marginals_noalloc(prob.ref(), _p(u), _p(v), float(gamma), _p(r_out),
                                              _p(c_out), _p(status_out), _stream(stream))
    if st != EOT_OK:
        raise EotError(st, "eot_marginals_noalloc failed")
