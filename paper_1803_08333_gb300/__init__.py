"""Python binding of librfcmp, the GB300 library for the RWG EFIE and the
refinement-free Calderon multiplicative preconditioner (arXiv 1803.08333).

Argument marshalling only: every step of assembly, preconditioning and the
solve runs in the library's CUDA kernels (include/rfcmp.h).  PyTorch provides
device memory and streams.  Vectors are torch.complex128 CUDA tensors of
shape (nrhs, N): row r is column r of the column-major N x nrhs block the C
ABI expects.  The library must be built (``build.build()``); importing the
binding without it raises at first use, there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librfcmp.so")

APPLY = {"T": 0, "T_A": 1, "T_PHI": 2, "T_ADJ": 3, "A": 4, "A_INNER": 5}
PREC = {"P_O": 0, "P_O_ADJ": 1, "P_M": 2, "P_SIGMA": 3, "P_LAMBDAH": 4, "P_GSIGMA": 5}
OUTER = {"sigma": 0, "gsigma": 1}
SCALING = {"power": 0, "k": 1, "fixed": 2}
PRECISION = {"mixed": 0, "ff": 1}
EXPORT = {"T_A": 0, "V": 1, "LPLUS": 2, "GLL_INV": 3, "GTP_INV": 4}
MAX_K_EXTENT = 1.0e5  # RFCMP_MAX_K_EXTENT: largest k x (bounding-box diagonal) an op accepts

# every symbol include/rfcmp.h declares
EXPORTED_SYMBOLS = [
    "rfcmp_ctx_create", "rfcmp_ctx_destroy", "rfcmp_ctx_clear_cache", "rfcmp_ctx_bytes_in_use",
    "rfcmp_op_create", "rfcmp_op_info_get", "rfcmp_op_destroy", "rfcmp_op_export", "rfcmp_op_edges",
    "rfcmp_rhs_planewave", "rfcmp_apply", "rfcmp_precondition", "rfcmp_solve", "rfcmp_solve_host",
    "rfcmp_farfield", "rfcmp_strerror", "rfcmp_last_error", "rfcmp_op_opts_default",
    "rfcmp_solve_opts_default", "rfcmp_profile_enable", "rfcmp_profile_read", "rfcmp_apply_ta_noalloc",
    "rfcmp_gemm_bf16x3", "rfcmp_plan_default", "rfcmp_ctx_set_plan", "rfcmp_op_set_plan", "rfcmp_op_get_plan",
    "rfcmp_op_trim", "rfcmp_launch_count", "rfcmp_set_solve_graphs", "rfcmp_rhs_voltage_gap",
    "rfcmp_pool_stats", "rfcmp_pool_reset_high", "rfcmp_pool_trim", "rfcmp_batch_create", "rfcmp_batch_destroy",
    "rfcmp_batch_admit", "rfcmp_batch_step", "rfcmp_batch_take", "rfcmp_batch_counts",
    "rfcmp_hm_opts_default", "rfcmp_hm_partition", "rfcmp_hm_create", "rfcmp_hm_apply", "rfcmp_hm_info_get",
    "rfcmp_hm_destroy",
]
HM = {"T_A": 0, "V": 1}


class C128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class OpOpts(ctypes.Structure):
    _fields_ = [
        ("scaling", ctypes.c_int32), ("power_steps", ctypes.c_int32),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
        ("factor_tol", ctypes.c_double), ("power_rtol", ctypes.c_double), ("scaling_start", ctypes.c_void_p),
        ("outer", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7),
    ]


class Plan(ctypes.Structure):
    """Launch shapes of one operator (zero fields: the library's built-in choices)."""

    _fields_ = [
        ("mrhs_min", ctypes.c_int32), ("gemm_bn", ctypes.c_int32), ("gemv_chunk", ctypes.c_int32),
        ("gemv_ctas_per_sm", ctypes.c_int32), ("far_min_blocks", ctypes.c_int32), ("exact_min", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 2),
    ]
    KEYS = ("mrhs_min", "gemm_bn", "gemv_chunk", "gemv_ctas_per_sm", "far_min_blocks", "exact_min")

    @classmethod
    def of(cls, d: "dict | None") -> "Plan":
        p = cls()
        for k_, v in (d or {}).items():
            if k_ not in cls.KEYS:
                raise KeyError("unknown plan field %r" % k_)
            setattr(p, k_, int(v))
        return p

    def as_dict(self) -> dict:
        return {k_: int(getattr(self, k_)) for k_ in self.KEYS}


class SolveOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("max_refine", ctypes.c_int32),
        ("inner_tol", ctypes.c_double), ("precision", ctypes.c_int32),
        ("fail_on_nonconvergence", ctypes.c_int32), ("reserved", ctypes.c_int32 * 8),
    ]


class SolveReport(ctypes.Structure):
    _fields_ = [
        ("converged", ctypes.c_int32), ("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("residual", ctypes.c_double),
    ]


class OpInfo(ctypes.Structure):
    _fields_ = [
        ("n_edges", ctypes.c_int64), ("n_vertices", ctypes.c_int64), ("n_cells", ctypes.c_int64),
        ("genus", ctypes.c_int32), ("boundaries", ctypes.c_int32),
        ("k", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("gamma", ctypes.c_double),
        ("device_bytes", ctypes.c_uint64), ("ms_assembly", ctypes.c_double), ("ms_factors", ctypes.c_double),
        ("ms_scaling", ctypes.c_double), ("factor_iterations_lplus", ctypes.c_int32),
        ("factor_iterations_gll", ctypes.c_int32),
    ]


class ProfileEntry(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 40), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
        ("bytes", ctypes.c_double), ("flops", ctypes.c_double),
    ]


class HmOpts(ctypes.Structure):
    _fields_ = [
        ("eps", ctypes.c_double), ("eta", ctypes.c_double), ("leaf", ctypes.c_int32), ("max_rank", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 6),
    ]


class HmInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64 * 2), ("lowrank_blocks", ctypes.c_int64 * 2), ("dense_blocks", ctypes.c_int64 * 2),
        ("capped_blocks", ctypes.c_int64 * 2), ("small_blocks", ctypes.c_int64 * 2), ("bytes", ctypes.c_int64 * 2),
        ("max_rank", ctypes.c_int32 * 2),
        ("reserved", ctypes.c_int32 * 6),
    ]


class RfcmpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("rfcmp status %d: %s" % (status, msg))
        self.status = status


_LIB = None


def lib():
    """The loaded shared library (raises if it was never built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "librfcmp.so is missing (%s): build it with paper_1803_08333_gb300.build.build()" % LIB_PATH
            )
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.rfcmp_ctx_create.argtypes = [i32, ctypes.c_uint64, ctypes.POINTER(vp)]
        L.rfcmp_ctx_destroy.argtypes = [vp]
        L.rfcmp_ctx_clear_cache.argtypes = [vp]
        L.rfcmp_ctx_bytes_in_use.argtypes = [vp]
        L.rfcmp_ctx_bytes_in_use.restype = ctypes.c_uint64
        L.rfcmp_op_create.argtypes = [vp, vp, i64, vp, i64, dbl, ctypes.POINTER(OpOpts), ctypes.POINTER(vp)]
        L.rfcmp_op_info_get.argtypes = [vp, ctypes.POINTER(OpInfo)]
        L.rfcmp_op_destroy.argtypes = [vp]
        L.rfcmp_op_trim.argtypes = [vp]
        L.rfcmp_op_export.argtypes = [vp, i32, vp, ctypes.c_uint64, vp]
        L.rfcmp_op_edges.argtypes = [vp, vp, vp]
        L.rfcmp_rhs_planewave.argtypes = [vp, vp, vp, i64, vp, vp]
        L.rfcmp_rhs_voltage_gap.argtypes = [vp, vp, vp, C128, vp, vp]
        L.rfcmp_apply.argtypes = [vp, i32, vp, vp, i64, vp]
        L.rfcmp_precondition.argtypes = [vp, i32, vp, vp, i64, vp]
        L.rfcmp_solve.argtypes = [vp, vp, vp, i64, ctypes.POINTER(SolveOpts), vp, vp]
        L.rfcmp_solve_host.argtypes = [vp, vp, vp, i64, ctypes.POINTER(SolveOpts), vp, vp]
        L.rfcmp_farfield.argtypes = [vp, vp, i64, vp, i64, vp, vp]
        L.rfcmp_strerror.argtypes = [i32]
        L.rfcmp_strerror.restype = ctypes.c_char_p
        L.rfcmp_last_error.restype = ctypes.c_char_p
        L.rfcmp_op_opts_default.argtypes = [ctypes.POINTER(OpOpts)]
        L.rfcmp_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts)]
        L.rfcmp_apply_ta_noalloc.argtypes = [vp, vp, vp, i64, vp]
        L.rfcmp_gemm_bf16x3.argtypes = [vp, i64, vp, i64, vp, i64, i64, i64, i64, i32, vp]
        L.rfcmp_plan_default.argtypes = [ctypes.POINTER(Plan)]
        L.rfcmp_plan_default.restype = None
        L.rfcmp_ctx_set_plan.argtypes = [vp, ctypes.POINTER(Plan)]
        L.rfcmp_op_set_plan.argtypes = [vp, ctypes.POINTER(Plan)]
        L.rfcmp_op_get_plan.argtypes = [vp, ctypes.POINTER(Plan)]
        L.rfcmp_profile_enable.argtypes = [i32]
        L.rfcmp_profile_read.argtypes = [ctypes.POINTER(ProfileEntry), i32, ctypes.POINTER(ctypes.c_int)]
        L.rfcmp_launch_count.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.rfcmp_set_solve_graphs.argtypes = [i32]
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.rfcmp_pool_stats.argtypes = [u64p, u64p, u64p, u64p]
        i32p = ctypes.POINTER(ctypes.c_int32)
        L.rfcmp_batch_create.argtypes = [vp, i32, ctypes.POINTER(SolveOpts), ctypes.POINTER(vp)]
        L.rfcmp_batch_destroy.argtypes = [vp]
        L.rfcmp_batch_admit.argtypes = [vp, vp, i32, i32p, vp]
        L.rfcmp_batch_step.argtypes = [vp, i32p, i32p, vp]
        L.rfcmp_batch_take.argtypes = [vp, i32p, i32, vp, ctypes.POINTER(SolveReport), vp]
        L.rfcmp_batch_counts.argtypes = [vp, i32p, i32p, i32p]
        L.rfcmp_hm_opts_default.argtypes = [ctypes.POINTER(HmOpts)]
        L.rfcmp_hm_opts_default.restype = None
        L.rfcmp_hm_partition.argtypes = [vp, vp, vp, i64, i32, dbl, vp, vp, i64, ctypes.POINTER(ctypes.c_int64)]
        L.rfcmp_hm_create.argtypes = [vp, ctypes.POINTER(HmOpts), ctypes.POINTER(vp)]
        L.rfcmp_hm_apply.argtypes = [vp, i32, vp, vp, i64, vp]
        L.rfcmp_hm_info_get.argtypes = [vp, ctypes.POINTER(HmInfo)]
        L.rfcmp_hm_destroy.argtypes = [vp]
        _LIB = L
    return _LIB


def _check(status: int):
    if status != 0:
        raise RfcmpError(status, lib().rfcmp_last_error().decode())


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def profile_enable(enable: bool = True):
    """Clears and (de)activates the per-kernel-family launch counters."""
    _check(lib().rfcmp_profile_enable(1 if enable else 0))


def profile_read() -> dict:
    """{family: {launches, total_ms, bytes, flops}}; synchronises the device."""
    n = ctypes.c_int()
    buf = (ProfileEntry * 64)()
    _check(lib().rfcmp_profile_read(buf, 64, ctypes.byref(n)))
    out = {}
    for i in range(min(n.value, 64)):
        e = buf[i]
        out[e.name.decode()] = {"launches": e.launches, "total_ms": e.total_ms, "bytes": e.bytes, "flops": e.flops}
    return out


def set_solve_graphs(enable: bool) -> bool:
    """Solve loops as one CUDA graph per op (True, the default) or launched kernel by kernel;
    returns the previous setting.  The arithmetic, and so every result, is the same."""
    return bool(lib().rfcmp_set_solve_graphs(1 if enable else 0))


def pool_stats() -> dict:
    """Bytes of the library's device pool: used, used_high, reserved, reserved_high."""
    v = [ctypes.c_uint64() for _ in range(4)]
    _check(lib().rfcmp_pool_stats(*[ctypes.byref(x) for x in v]))
    return dict(zip(("used", "used_high", "reserved", "reserved_high"), (int(x.value) for x in v)))


def pool_reset_high():
    _check(lib().rfcmp_pool_reset_high())


def pool_trim():
    """Returns the pool's unused device memory to the driver (synchronises the device)."""
    _check(lib().rfcmp_pool_trim())


def launch_count() -> int:
    """Kernel launches of the library so far (device counters; synchronises the device)."""
    v = ctypes.c_uint64()
    _check(lib().rfcmp_launch_count(ctypes.byref(v)))
    return int(v.value)


def gemm_bf16x3(A, B, D=None, accumulate=False):
    """D = A @ B.T (+ D) with float32 CUDA tensors through the split-BF16 tensor-core GEMM."""
    import torch

    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    if D is None:
        D = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    _check(lib().rfcmp_gemm_bf16x3(_ptr(A), K, _ptr(B), K, _ptr(D), N, M, N, K, 1 if accumulate else 0, _stream()))
    return D


class Context:
    """One CUDA device with an HBM budget and the cache of topology factors."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().rfcmp_ctx_create(int(device), int(hbm_budget_bytes), ctypes.byref(self._h)))
        self.device = device

    def clear_cache(self):
        _check(lib().rfcmp_ctx_clear_cache(self._h))

    def set_plan(self, plan: "dict | None" = None):
        """Plan that operators created from now on start with (fields of `Plan`; None: built-in)."""
        p = Plan.of(plan)
        _check(lib().rfcmp_ctx_set_plan(self._h, ctypes.byref(p)))

    def bytes_in_use(self) -> int:
        return int(lib().rfcmp_ctx_bytes_in_use(self._h))

    def close(self):
        if self._h:
            _check(lib().rfcmp_ctx_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h:
                lib().rfcmp_ctx_destroy(self._h)
        except Exception:
            pass


@dataclass
class Report:
    converged: bool
    iterations: int
    refinements: int
    residual: float


class Operator:
    """Mesh + wavenumber -> resident EFIE blocks, RF-CMP factors and scaling."""

    def __init__(self, ctx: Context, verts, tris, k: float, scaling: str = "power", power_steps: int = 30,
                 alpha: float = 1.0, beta: float = 1.0, gamma: float = 1.0, factor_tol: float = 1e-13,
                 power_rtol: float = 1e-3, scaling_start: "Operator | None" = None, outer: str = "sigma"):
        """outer: "sigma" (P_o with P_S, the numerical variant of Sec. 4) or "gsigma" (P_gS of Sec. 3)."""
        self.ctx = ctx
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        o = OpOpts()
        lib().rfcmp_op_opts_default(ctypes.byref(o))
        o.scaling = SCALING[scaling]
        o.power_steps = int(power_steps)
        o.alpha, o.beta, o.gamma = float(alpha), float(beta), float(gamma)
        o.factor_tol = float(factor_tol)
        o.power_rtol = float(power_rtol)
        o.outer = OUTER[outer]
        if scaling_start is not None:
            o.scaling_start = scaling_start._h
        self._h = ctypes.c_void_p()
        _check(
            lib().rfcmp_op_create(
                ctx._h, self.verts.ctypes.data_as(ctypes.c_void_p), self.verts.shape[0],
                self.tris.ctypes.data_as(ctypes.c_void_p), self.tris.shape[0], float(k), ctypes.byref(o),
                ctypes.byref(self._h),
            )
        )
        self.k = float(k)
        inf = self.info()
        self.N, self.nc, self.nv = int(inf.n_edges), int(inf.n_cells), int(inf.n_vertices)
        self.tuning = None  # an autotune.Table: solve() and apply("A_INNER") take its plans
        self._plan_set = None

    def info(self) -> OpInfo:
        out = OpInfo()
        _check(lib().rfcmp_op_info_get(self._h, ctypes.byref(out)))
        return out

    def trim(self):
        """Frees the planes, digits and workspace of wide products (rebuilt on the next wide call)."""
        _check(lib().rfcmp_op_trim(self._h))

    def plan(self) -> dict:
        p = Plan()
        _check(lib().rfcmp_op_get_plan(self._h, ctypes.byref(p)))
        return p.as_dict()

    def set_plan(self, plan: "dict | None" = None):
        """Launch shapes for this operator's later calls (fields of `Plan`; None: built-in)."""
        p = Plan.of(plan)
        _check(lib().rfcmp_op_set_plan(self._h, ctypes.byref(p)))

    @property
    def scaling(self):
        i = self.info()
        return i.alpha, i.beta, i.gamma

    def export(self, which: str):
        """T_A, V (complex64 n x n) or LPLUS, GLL_INV, GTP_INV (float64 n x n from the hi + lo planes) as CUDA tensors."""
        import torch

        n = {"T_A": self.N, "V": self.nc, "LPLUS": self.nc, "GLL_INV": self.nv, "GTP_INV": self.nc}[which]
        if which in ("T_A", "V"):
            t = torch.empty((n, n), dtype=torch.complex64, device="cuda")
            _check(lib().rfcmp_op_export(self._h, EXPORT[which], _ptr(t), n * n * 8, _stream()))
            return t
        t = torch.empty((2, n, n), dtype=torch.float32, device="cuda")
        _check(lib().rfcmp_op_export(self._h, EXPORT[which], _ptr(t), n * n * 8, _stream()))
        return t[0].double() + t[1].double()

    def edges(self):
        ev = np.empty((self.N, 2), np.int32)
        ec = np.empty((self.N, 2), np.int32)
        _check(lib().rfcmp_op_edges(self._h, ev.ctypes.data_as(ctypes.c_void_p), ec.ctypes.data_as(ctypes.c_void_p)))
        return ev, ec

    def rhs_planewave(self, khat, pol):
        import torch

        khat = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
        pol = np.ascontiguousarray(np.atleast_2d(pol), dtype=np.float64)
        nr = khat.shape[0]
        e = torch.empty((nr, self.N), dtype=torch.complex128, device="cuda")
        _check(lib().rfcmp_rhs_planewave(self._h, khat.ctypes.data_as(ctypes.c_void_p),
                                         pol.ctypes.data_as(ctypes.c_void_p), nr, _ptr(e), _stream()))
        return e

    def rhs_voltage_gap(self, origin, normal, voltage: complex = 1.0):
        """Delta-gap excitation across the mesh edges cut by the plane (origin, normal): (1, N)."""
        import torch

        o = np.ascontiguousarray(origin, dtype=np.float64).reshape(3)
        u = np.ascontiguousarray(normal, dtype=np.float64).reshape(3)
        e = torch.empty((1, self.N), dtype=torch.complex128, device="cuda")
        v = C128(float(np.real(voltage)), float(np.imag(voltage)))
        _check(lib().rfcmp_rhs_voltage_gap(self._h, o.ctypes.data_as(ctypes.c_void_p), u.ctypes.data_as(ctypes.c_void_p),
                                           v, _ptr(e), _stream()))
        return e

    def _vec(self, x):
        import torch

        x = x.to(device="cuda", dtype=torch.complex128)
        if x.dim() == 1:
            x = x[None]
        return x.contiguous()

    def apply(self, which: str, x, out=None):
        import torch

        x = self._vec(x)
        y = torch.empty_like(x) if out is None else out
        if which == "A_INNER":
            self._tuned(x.shape[0], "mixed")
        _check(lib().rfcmp_apply(self._h, APPLY[which], _ptr(x), _ptr(y), x.shape[0], _stream()))
        return y

    def _tuned(self, nrhs: int, precision: str):
        """Applies the tuning table's plan for this call's shape (if the operator carries a table)."""
        if self.tuning is None:
            return
        plan = self.tuning.lookup(self.N, nrhs, precision) or {}
        plan = {k_: v for k_, v in plan.items() if k_ != "far_min_blocks"}
        if plan != self._plan_set:
            self.set_plan(plan)
            self._plan_set = plan

    def apply_ta_noalloc(self, x, out=None):
        """y = T_A x through the allocation-free entry point; `out` may be preallocated."""
        import torch

        x = self._vec(x)
        y = torch.empty_like(x) if out is None else out
        _check(lib().rfcmp_apply_ta_noalloc(self._h, _ptr(x), _ptr(y), x.shape[0], _stream()))
        return y

    def precondition(self, which: str, x):
        import torch

        x = self._vec(x)
        y = torch.empty_like(x)
        _check(lib().rfcmp_precondition(self._h, PREC[which], _ptr(x), _ptr(y), x.shape[0], _stream()))
        return y

    @staticmethod
    def _solve_opts(tol, max_iter, max_refine, inner_tol, precision):
        o = SolveOpts()
        lib().rfcmp_solve_opts_default(ctypes.byref(o))
        o.tol, o.max_iter, o.max_refine, o.inner_tol = float(tol), int(max_iter), int(max_refine), float(inner_tol)
        o.precision = PRECISION[precision]
        return o

    def solve(self, e, tol: float = 1e-6, max_iter: int = 2000, max_refine: int = 24, inner_tol: float = 1e-4,
              precision: str = "mixed"):
        """j with T j = -e via RF-CMP + CG; returns (j, [Report per column])."""
        import torch

        e = self._vec(e)
        j = torch.empty_like(e)
        nr = e.shape[0]
        rep = (SolveReport * nr)()
        o = self._solve_opts(tol, max_iter, max_refine, inner_tol, precision)
        self._tuned(nr, precision)
        _check(lib().rfcmp_solve(self._h, _ptr(e), _ptr(j), nr, ctypes.byref(o), rep, _stream()))
        return j, [Report(bool(r.converged), r.iterations, r.refinements, r.residual) for r in rep]

    def solve_host(self, e: np.ndarray, tol: float = 1e-6, max_iter: int = 2000, max_refine: int = 24,
                   inner_tol: float = 1e-4, precision: str = "mixed", stream=None, out: "np.ndarray | None" = None):
        """Same solve with host arrays (nrhs, N) complex128; copies happen inside the C call.

        `out` (optional, C-contiguous complex128 of e's shape, e.g. a view of pinned memory)
        receives j; otherwise a new array is returned."""
        e = np.ascontiguousarray(np.atleast_2d(e), dtype=np.complex128)
        if out is not None:
            if out.shape != e.shape or out.dtype != np.complex128 or not out.flags.c_contiguous:
                raise ValueError("out must be a C-contiguous complex128 array of shape %s" % (e.shape,))
            j = out
        else:
            j = np.empty_like(e)
        nr = e.shape[0]
        rep = (SolveReport * nr)()
        o = self._solve_opts(tol, max_iter, max_refine, inner_tol, precision)
        self._tuned(nr, precision)
        _check(lib().rfcmp_solve_host(self._h, e.ctypes.data_as(ctypes.c_void_p), j.ctypes.data_as(ctypes.c_void_p),
                                      nr, ctypes.byref(o), rep, _stream(stream)))
        return j, [Report(bool(r.converged), r.iterations, r.refinements, r.residual) for r in rep]

    def batch(self, capacity: int, tol: float = 1e-6, max_iter: int = 2000, max_refine: int = 24,
              inner_tol: float = 1e-4, precision: str = "mixed") -> "Batch":
        """A batch session on this operator (continuous batching; see Batch)."""
        return Batch(self, capacity, self._solve_opts(tol, max_iter, max_refine, inner_tol, precision))

    def farfield(self, j, dirs) -> np.ndarray:
        """Bistatic RCS in dBsm, shape (nrhs, ndir)."""
        j = self._vec(j)
        dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
        out = np.empty((j.shape[0], dirs.shape[0]), np.float64)
        _check(lib().rfcmp_farfield(self._h, _ptr(j), j.shape[0], dirs.ctypes.data_as(ctypes.c_void_p),
                                    dirs.shape[0], out.ctypes.data_as(ctypes.c_void_p), _stream()))
        return out

    def close(self):
        if self._h:
            _check(lib().rfcmp_op_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h:
                lib().rfcmp_op_destroy(self._h)
        except Exception:
            pass


def hm_partition(centres, sup_lo, sup_hi, leaf: int = 32, eta: float = 1.0):
    """Cluster order (n,) and symmetric block list (B, 5: r0, r1, c0, c1, admissible) of n items
    with centres and support boxes (n x 3 each), computed by the library on the host."""
    c = np.ascontiguousarray(centres, dtype=np.float64)
    lo = np.ascontiguousarray(sup_lo, dtype=np.float64)
    hi = np.ascontiguousarray(sup_hi, dtype=np.float64)
    n = c.shape[0]
    if lo.shape != c.shape or hi.shape != c.shape or (n and c.shape[1] != 3):
        raise ValueError("centres, sup_lo and sup_hi must all be n x 3")
    perm = np.empty(n, dtype=np.int32)
    nb = ctypes.c_int64()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().rfcmp_hm_partition(vp(c), vp(lo), vp(hi), n, int(leaf), float(eta), vp(perm), None, 0,
                                    ctypes.byref(nb)))
    blocks = np.empty((nb.value, 5), dtype=np.int32)
    _check(lib().rfcmp_hm_partition(vp(c), vp(lo), vp(hi), n, int(leaf), float(eta), vp(perm), vp(blocks),
                                    nb.value, ctypes.byref(nb)))
    return perm, blocks


class Compressed:
    """T_A and V of an operator compressed apart (rfcmp_hm_*): symmetric hierarchical matrices
    with ACA crosses on the admissible blocks (Sec. 4)."""

    def __init__(self, op: "Operator", eps: float = 1e-4, eta: float = 1.0, leaf: int = 32, max_rank: int = 64):
        self.op = op
        o = HmOpts()
        lib().rfcmp_hm_opts_default(ctypes.byref(o))
        o.eps, o.eta, o.leaf, o.max_rank = float(eps), float(eta), int(leaf), int(max_rank)
        self._h = ctypes.c_void_p()
        _check(lib().rfcmp_hm_create(op._h, ctypes.byref(o), ctypes.byref(self._h)))

    def apply(self, which: str, x, out=None, stream=None):
        """y = H x for H the compressed "T_A" or "V"; x (nrhs, n) or (n,) on the device."""
        import torch

        x = x.to(device="cuda", dtype=torch.complex128)
        if x.dim() == 1:
            x = x[None]
        x = x.contiguous()
        n = self.op.N if which == "T_A" else self.op.nc
        if x.shape[1] != n:
            raise ValueError("x has %d rows, the compressed %s has %d" % (x.shape[1], which, n))
        y = torch.empty_like(x) if out is None else out
        _check(lib().rfcmp_hm_apply(self._h, HM[which], _ptr(x), _ptr(y), x.shape[0], _stream(stream)))
        return y

    def info(self) -> dict:
        i = HmInfo()
        _check(lib().rfcmp_hm_info_get(self._h, ctypes.byref(i)))
        out = {}
        for w, name in enumerate(("T_A", "V")):
            out[name] = {
                "n": i.n[w], "lowrank_blocks": i.lowrank_blocks[w], "dense_blocks": i.dense_blocks[w],
                "capped_blocks": i.capped_blocks[w], "small_blocks": i.small_blocks[w], "bytes": i.bytes[w],
                "max_rank": i.max_rank[w],
            }
        return out

    def close(self):
        if self._h:
            _check(lib().rfcmp_hm_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h:
                lib().rfcmp_hm_destroy(self._h)
        except Exception:
            pass


class Batch:
    """Continuous batching of one operator's solves (rfcmp_batch_*): excitations join free slots
    between refinement sweeps, step() runs one sweep over all running columns, take() returns a
    finished column's current and frees its slot."""

    def __init__(self, op: Operator, capacity: int, opts: SolveOpts):
        self.op = op
        self.capacity = int(capacity)
        self._h = ctypes.c_void_p()
        _check(lib().rfcmp_batch_create(op._h, self.capacity, ctypes.byref(opts), ctypes.byref(self._h)))

    def admit(self, e, stream=None) -> list:
        e = self.op._vec(e)
        n = e.shape[0]
        slots = (ctypes.c_int32 * n)()
        _check(lib().rfcmp_batch_admit(self._h, _ptr(e), n, slots, _stream(stream)))
        return list(slots)

    def step(self, stream=None) -> list:
        fin = (ctypes.c_int32 * self.capacity)()
        nf = ctypes.c_int32()
        _check(lib().rfcmp_batch_step(self._h, fin, ctypes.byref(nf), _stream(stream)))
        return list(fin[: nf.value])

    def take(self, slots, stream=None):
        """Currents (len(slots) x N) and reports of finished slots, which become free."""
        import torch

        slots = [int(s) for s in np.atleast_1d(slots)]
        n = len(slots)
        sl = (ctypes.c_int32 * n)(*slots)
        j = torch.empty((n, self.op.N), dtype=torch.complex128, device="cuda")
        r = (SolveReport * n)()
        _check(lib().rfcmp_batch_take(self._h, sl, n, _ptr(j), r, _stream(stream)))
        return j, [Report(bool(x.converged), x.iterations, x.refinements, x.residual) for x in r]

    def counts(self) -> tuple:
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().rfcmp_batch_counts(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def close(self):
        if self._h:
            _check(lib().rfcmp_batch_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h:
                lib().rfcmp_batch_destroy(self._h)
        except Exception:
            pass
