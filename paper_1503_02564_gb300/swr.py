"""Thin ctypes binding of libswr (the C ABI declared in include/swr.h).

Argument marshalling only: every step of the SWR path runs in the library's CUDA
kernels.  Arrays are torch tensors on the CUDA device (complex128 for complex
arrays, float64 for potentials); their ``data_ptr()`` is passed straight through,
together with the current torch CUDA stream.  There is no CPU fallback: if the
library is missing or the device is not a GPU, the call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libswr.so")

SWR_OK, SWR_ERR_ARG, SWR_ERR_SINGULAR, SWR_ERR_NOT_CONVERGED = 0, 1, 2, 3
SWR_ERR_NONFINITE, SWR_ERR_TIMEOUT, SWR_ERR_NOMEM, SWR_ERR_CUDA = 4, 5, 6, 7
SWR_ERR_STATE, SWR_ERR_UNSUPPORTED = 8, 9
SWR_V_STATIC, SWR_V_TIME, SWR_V_NONLINEAR = 0, 1, 2
SWR_TC_ROBIN, SWR_TC_S02, SWR_TC_S03, SWR_TC_S04, SWR_TC_S12, SWR_TC_S14 = 0, 1, 2, 3, 4, 5
SWR_SOLVER_GMRES, SWR_SOLVER_FIXED_POINT, SWR_SOLVER_CLASSICAL, SWR_SOLVER_CAUSAL = 0, 1, 2, 3
SWR_SOLVER_BICGSTAB = 4
SWR_PC_NONE, SWR_PC_ZERO_POTENTIAL, SWR_PC_CAUSAL, SWR_PC_MEAN_POTENTIAL = 0, 1, 2, 3
# swr_stats.march_variant
MARCH_CONSTANT, MARCH_TDEP_REFACTOR, MARCH_NONLINEAR, MARCH_TDEP_STREAMED = 0, 1, 2, 3


class swr_desc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("a0", ctypes.c_double), ("b0", ctypes.c_double),
        ("nt", ctypes.c_int32), ("dt", ctypes.c_double), ("nsub", ctypes.c_int32),
        ("node_off", ctypes.POINTER(ctypes.c_int32)), ("vkind", ctypes.c_int32),
        ("tc", ctypes.c_int32), ("tc_re", ctypes.c_double), ("tc_im", ctypes.c_double),
        ("solver", ctypes.c_int32), ("restart", ctypes.c_int32), ("maxit", ctypes.c_int32),
        ("tol_abs", ctypes.c_double), ("precond", ctypes.c_int32), ("nl_maxit", ctypes.c_int32),
        ("nl_tol", ctypes.c_double), ("nl_coef", ctypes.c_double),
        ("pc_sweeps", ctypes.c_int32),
    ]


class swr_tuning(ctypes.Structure):
    """Execution choices of a plan (include/swr.h); zero-filled means the defaults."""
    _fields_ = [
        ("chunk_L", ctypes.c_int32), ("autotune", ctypes.c_int32),
        ("toeplitz_fft", ctypes.c_int32), ("superpose", ctypes.c_int32),
        ("long_march", ctypes.c_int32), ("graph", ctypes.c_int32),
        ("tdep_precomp", ctypes.c_int32), ("two_level", ctypes.c_int32),
        ("debug", ctypes.c_int32), ("history_fft", ctypes.c_int32),
    ]


def make_tuning(tuning):
    """A swr_tuning from a dict of field -> int (None: NULL, the library defaults)."""
    if tuning is None:
        return None
    t = swr_tuning()
    for k, v in tuning.items():
        if k not in dict(swr_tuning._fields_):
            raise KeyError(f"unknown tuning field {k}")
        setattr(t, k, int(v))
    return t


class swr_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32),
        ("residual", ctypes.c_double), ("residual0", ctypes.c_double),
        ("interface_jump", ctypes.c_double), ("t_build_ms", ctypes.c_double),
        ("t_solve_ms", ctypes.c_double), ("t_final_ms", ctypes.c_double),
        ("march_point_steps", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class swr_stats(ctypes.Structure):
    _fields_ = [
        ("march_launches", ctypes.c_int64), ("march_point_steps", ctypes.c_int64),
        ("march_ms", ctypes.c_double), ("toeplitz_launches", ctypes.c_int64),
        ("toeplitz_ms", ctypes.c_double), ("precond_calls", ctypes.c_int64),
        ("precond_ms", ctypes.c_double), ("march_variant", ctypes.c_int32),
        ("march_factor_bytes_per_step", ctypes.c_int64),
        ("march_point_iterations", ctypes.c_int64),
        ("nl_march_launches", ctypes.c_int64), ("nl_march_ms", ctypes.c_double),
        ("superposed", ctypes.c_int32), ("toeplitz_fft_length", ctypes.c_int32),
        ("causal_sweeps", ctypes.c_int32), ("causal_window", ctypes.c_int32),
        ("two_level_launches", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SWRError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {swr_status_string(status)}")


_lib = None


def lib():
    """Load libswr.so (built by paper_1503_02564_gb300.build_ext); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libswr.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp = ctypes.c_void_p, ctypes.c_void_p
        L.swr_plan.argtypes = [ctypes.POINTER(swr_desc), ctypes.POINTER(vp), vp]
        L.swr_plan_batch.argtypes = [ctypes.POINTER(swr_desc), ctypes.c_int32,
                                     ctypes.POINTER(vp), vp]
        L.swr_plan_ex.argtypes = [ctypes.POINTER(swr_desc), ctypes.POINTER(swr_tuning),
                                  ctypes.POINTER(vp), vp]
        L.swr_plan_batch_ex.argtypes = [ctypes.POINTER(swr_desc), ctypes.c_int32,
                                        ctypes.POINTER(swr_tuning), ctypes.POINTER(vp), vp]
        L.swr_tuning_defaults.argtypes = [ctypes.POINTER(swr_tuning)]
        L.swr_tuning_defaults.restype = None
        L.swr_build_interface.argtypes = [vp, dp, dp]
        L.swr_solve.argtypes = [vp, dp, ctypes.c_int32, dp, ctypes.POINTER(swr_info)]
        L.swr_apply_R.argtypes = [vp, dp, dp]
        L.swr_apply_interface.argtypes = [vp, dp, dp]
        L.swr_get_interface.argtypes = [vp, dp, dp]
        L.swr_apply_precond.argtypes = [vp, dp, dp]
        L.swr_adjoint.argtypes = [vp, dp, dp, ctypes.c_int32]
        L.swr_misfit.argtypes = [vp, dp, dp, dp, ctypes.POINTER(ctypes.c_double)]
        L.swr_get_stats.argtypes = [vp, ctypes.POINTER(swr_stats), ctypes.c_int32]
        L.swr_causal_solve_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               dp, dp, dp, vp]
        L.swr_fp64_peak.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_int32, dp, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_float), vp]
        L.swr_test_wait_hook.argtypes = [ctypes.c_int64, ctypes.c_int32]
        L.swr_destroy.argtypes = [vp]
        L.swr_destroy.restype = None
        L.swr_kernel_launch_count.argtypes = []
        L.swr_kernel_launch_count.restype = ctypes.c_int64
        L.swr_status_string.argtypes = [ctypes.c_int]
        L.swr_status_string.restype = ctypes.c_char_p
        for f in ("swr_plan", "swr_plan_batch", "swr_plan_ex", "swr_plan_batch_ex",
                  "swr_build_interface", "swr_solve", "swr_apply_R",
                  "swr_apply_interface", "swr_get_interface", "swr_apply_precond", "swr_adjoint",
                  "swr_get_stats", "swr_causal_solve_noalloc", "swr_misfit", "swr_fp64_peak",
                  "swr_test_wait_hook"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def swr_status_string(status: int) -> str:
    return lib().swr_status_string(int(status)).decode()


def swr_kernel_launch_count() -> int:
    return int(lib().swr_kernel_launch_count())


def _ptr(t, dtype, n=None, name="array"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _check(st, where, allow=()):
    if st != SWR_OK and st not in allow:
        raise SWRError(st, where)
    return st


def swr_causal_solve_noalloc(nsub, nt, sweeps, cols, y, x, stream=None):
    """x = (I - L)^{-1} y (causal substitution) without any device allocation;
    for callers that cannot allocate device memory (see include/swr.h)."""
    n = (2 * nsub - 2) * nt
    if stream is None:
        stream = torch.cuda.current_stream()
    return lib().swr_causal_solve_noalloc(
        int(nsub), int(nt), int(sweeps), _ptr(cols, torch.complex128, 4 * nsub * nt, "cols"),
        _ptr(y, torch.complex128, n, "y"), _ptr(x, torch.complex128, n, "x"),
        ctypes.c_void_p(stream.cuda_stream))


def swr_test_wait_hook(max_polls=0, withhold=-1):
    """Test hook of the substitution's bounded waits on the current device (see
    include/swr.h); (0, -1) restores the defaults."""
    _check(lib().swr_test_wait_hook(int(max_polls), int(withhold)), "swr_test_wait_hook")


def swr_fp64_peak(kind, iters, blocks, threads, sink, stream=None):
    """One timed FP64 probe launch (kind 0: DFMA, 1: DMMA m8n8k4); returns
    (flops, ms).  sink: float64 CUDA tensor of blocks * threads entries."""
    if stream is None:
        stream = torch.cuda.current_stream()
    flops, ms = ctypes.c_double(), ctypes.c_float()
    _check(lib().swr_fp64_peak(int(kind), int(iters), int(blocks), int(threads),
                               _ptr(sink, torch.float64, blocks * threads, "sink"),
                               ctypes.byref(flops), ctypes.byref(ms),
                               ctypes.c_void_p(stream.cuda_stream)), "swr_fp64_peak")
    return flops.value, float(ms.value)


class Plan:
    """An SWR plan (C handle) with the entry points of include/swr.h as methods."""

    def __init__(self, *, nx, a0, b0, nt, dt, nsub, node_off=None, vkind=SWR_V_STATIC,
                 tc=SWR_TC_ROBIN, p=0j, solver=SWR_SOLVER_GMRES, restart=30, maxit=2000,
                 tol_abs=1e-10, precond=SWR_PC_NONE, nl_maxit=50, nl_tol=1e-13, nl_coef=1.0,
                 pc_sweeps=-1, stream=None, tuning=None):
        d = swr_desc()
        d.nx, d.a0, d.b0, d.nt, d.dt, d.nsub = nx, a0, b0, nt, dt, nsub
        self._off = None
        if node_off is not None:
            arr = (ctypes.c_int32 * (nsub + 1))(*[int(v) for v in node_off])
            self._off = arr
            d.node_off = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32))
        d.vkind, d.tc = vkind, tc
        d.tc_re, d.tc_im = complex(p).real, complex(p).imag
        d.solver, d.restart, d.maxit, d.tol_abs, d.precond = solver, restart, maxit, tol_abs, precond
        d.nl_maxit, d.nl_tol, d.nl_coef = nl_maxit, nl_tol, nl_coef
        d.pc_sweeps = pc_sweeps
        self.desc = d
        self.nx, self.nt, self.nsub, self.nblk, self.vkind = nx, nt, nsub, 2 * nsub - 2, vkind
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        tu = make_tuning(tuning)
        _check(lib().swr_plan_ex(ctypes.byref(d), ctypes.byref(tu) if tu is not None else None,
                                 ctypes.byref(h), ctypes.c_void_p(stream.cuda_stream)),
               "swr_plan")
        self.handle = h

    @property
    def n_interface(self):
        return self.nblk * self.nt

    @property
    def n_cols(self):
        return 4 * self.nsub * self.nt

    def build_interface(self, V, u0):
        nV = self.nx if self.vkind != SWR_V_TIME else (self.nt + 1) * self.nx
        _check(lib().swr_build_interface(self.handle, _ptr(V, torch.float64, nV, "V"),
                                         _ptr(u0, torch.complex128, self.nx, "u0")),
               "swr_build_interface")

    def solve(self, g=None, g_is_initial=False, uT=None, allow_not_converged=False):
        info = swr_info()
        st = lib().swr_solve(self.handle, _ptr(g, torch.complex128, self.n_interface, "g"),
                             int(bool(g_is_initial)), _ptr(uT, torch.complex128, self.nx, "uT"),
                             ctypes.byref(info))
        _check(st, "swr_solve", allow=(SWR_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        out = info.as_dict()
        out["status"] = st
        return out

    def apply_R(self, g_in, g_out):
        _check(lib().swr_apply_R(self.handle, _ptr(g_in, torch.complex128, self.n_interface, "g_in"),
                                 _ptr(g_out, torch.complex128, self.n_interface, "g_out")),
               "swr_apply_R")

    def apply_interface(self, x, y):
        _check(lib().swr_apply_interface(self.handle, _ptr(x, torch.complex128, self.n_interface, "x"),
                                         _ptr(y, torch.complex128, self.n_interface, "y")),
               "swr_apply_interface")

    def get_interface(self, d=None, cols=None):
        _check(lib().swr_get_interface(self.handle, _ptr(d, torch.complex128, self.n_interface, "d"),
                                       _ptr(cols, torch.complex128, self.n_cols, "cols")),
               "swr_get_interface")

    def apply_precond(self, y, x):
        _check(lib().swr_apply_precond(self.handle, _ptr(y, torch.complex128, self.n_interface, "y"),
                                       _ptr(x, torch.complex128, self.n_interface, "x")),
               "swr_apply_precond")

    def misfit(self, uT, u_target, ubar=None):
        """J = (uT - u_target)^H M (uT - u_target); ubar (optional) receives 2 (uT - u_target)."""
        J = ctypes.c_double()
        _check(lib().swr_misfit(self.handle, _ptr(uT, torch.complex128, self.nx, "uT"),
                                _ptr(u_target, torch.complex128, self.nx, "u_target"),
                                _ptr(ubar, torch.complex128, self.nx, "ubar"), ctypes.byref(J)),
               "swr_misfit")
        return J.value

    def adjoint(self, ubar, grad, ckpt_every=0):
        """grad <- dJ/dV for the M-weighted cotangent ubar of J at u(T) (after solve());
        grad has nx entries, or (nt + 1) nx for a time-dependent potential (the layout
        of V)."""
        ng = (self.nt + 1) * self.nx if self.vkind == SWR_V_TIME else self.nx
        _check(lib().swr_adjoint(self.handle, _ptr(ubar, torch.complex128, self.nx, "ubar"),
                                 _ptr(grad, torch.float64, ng, "grad"), int(ckpt_every)),
               "swr_adjoint")

    def get_stats(self, reset=False):
        st = swr_stats()
        _check(lib().swr_get_stats(self.handle, ctypes.byref(st), int(bool(reset))), "swr_get_stats")
        return st.as_dict()

    def destroy(self):
        if getattr(self, "handle", None):
            lib().swr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class SWRMisfit(torch.autograd.Function):
    """J(V) = ||u(T) - u_target||_M^2 with u the converged SWR solution for the
    static potential V (a CUDA float64 tensor of nx nodal values); the backward
    pass is swr_adjoint.  plan: a Plan with a static potential, Robin
    transmission and GMRES; u0, u_target: complex128 CUDA tensors."""

    @staticmethod
    def forward(ctx, V, plan, u0, u_target, ckpt_every=0):
        plan.build_interface(V, u0)
        uT = torch.empty(plan.nx, dtype=torch.complex128, device=V.device)
        plan.solve(None, False, uT)
        ubar = torch.empty_like(uT)
        J = plan.misfit(uT, u_target, ubar)
        ctx.plan, ctx.ckpt_every = plan, ckpt_every
        ctx.save_for_backward(ubar)
        return torch.tensor(J, dtype=torch.float64, device=V.device)

    @staticmethod
    def backward(ctx, gJ):
        (ubar,) = ctx.saved_tensors
        grad = torch.empty(ctx.plan.nx, dtype=torch.float64, device=ubar.device)
        ctx.plan.adjoint(ubar, grad, ctx.ckpt_every)
        return grad * gJ, None, None, None, None


class BatchPlan(Plan):
    """swr_plan_batch: independent instances in one plan.  `instances` is a list of
    dicts with the per-instance fields nx, a0, b0, nt, nsub and optionally
    node_off; the keyword arguments are shared.  Arrays (V, u0, uT, interface
    vectors, first columns) are the instances' arrays concatenated in order;
    `inst_nx`, `inst_nb` and `inst_ncols` give the per-instance lengths."""

    def __init__(self, instances, *, dt, tc=SWR_TC_ROBIN, p=0j, solver=SWR_SOLVER_GMRES,
                 restart=30, maxit=2000, tol_abs=1e-10, precond=SWR_PC_NONE, pc_sweeps=-1,
                 stream=None, tuning=None):
        count = len(instances)
        descs = (swr_desc * count)()
        self._offs = []
        for i, ins in enumerate(instances):
            d = descs[i]
            d.nx, d.a0, d.b0, d.nt, d.dt, d.nsub = (int(ins["nx"]), float(ins["a0"]),
                                                    float(ins["b0"]), int(ins["nt"]), dt,
                                                    int(ins["nsub"]))
            if ins.get("node_off") is not None:
                arr = (ctypes.c_int32 * (d.nsub + 1))(*[int(v) for v in ins["node_off"]])
                self._offs.append(arr)
                d.node_off = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int32))
            d.vkind, d.tc = SWR_V_STATIC, tc
            d.tc_re, d.tc_im = complex(p).real, complex(p).imag
            d.solver, d.restart, d.maxit, d.tol_abs, d.precond = (solver, restart, maxit,
                                                                  tol_abs, precond)
            d.nl_maxit, d.nl_tol, d.nl_coef, d.pc_sweeps = 50, 1e-13, 1.0, pc_sweeps
        self.descs = descs
        self.inst_nx = [int(i["nx"]) for i in instances]
        self.inst_nb = [(2 * int(i["nsub"]) - 2) * int(i["nt"]) for i in instances]
        self.inst_ncols = [4 * int(i["nsub"]) * int(i["nt"]) for i in instances]
        self.nx = sum(self.inst_nx)
        self.nt = max(int(i["nt"]) for i in instances)
        self.nsub = sum(int(i["nsub"]) for i in instances)
        self.nblk = 2 * self.nsub - 2 * count
        self.vkind = SWR_V_STATIC
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        tu = make_tuning(tuning)
        _check(lib().swr_plan_batch_ex(descs, count, ctypes.byref(tu) if tu is not None else None,
                                       ctypes.byref(h), ctypes.c_void_p(stream.cuda_stream)),
               "swr_plan_batch")
        self.handle = h

    @property
    def n_interface(self):
        return sum(self.inst_nb)

    @property
    def n_cols(self):
        return sum(self.inst_ncols)
