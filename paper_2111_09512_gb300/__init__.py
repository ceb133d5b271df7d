"""silu: scaled-ILU Richardson smoothers on GB300 (sm_103a).

Thin ctypes binding of libsilu.so, the C ABI declared in include/silu.h.  The
functions keep the C names (silu_ctx_create, silu_mat_create, ilu_setup,
ilu_refactor, ilu_smooth, direct_trisolve, fgmres_solve, ...) and only
marshal arguments: host CSR arrays as numpy, device vectors as torch CUDA
tensors (or raw pointers), the stream as a torch stream.  Every step of the
smoother runs in the library's CUDA kernels.  There is no fallback: if
libsilu.so is missing or fails to load, every call raises.

The method is that of Thomas, Carr, Mullowney, Swirydowicz and Day, "Scaled
ILU Smoothers for Navier-Stokes Pressure Projection" (arXiv 2111.09512):
incomplete LU factors with the upper factor row-scaled to unit diagonal
(Eq. extractD, Eq. newD), triangular solves replaced by Richardson sweeps
(Alg. ILUJac, Eq. richard), inside flexible GMRES (Sec. 6).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsilu.so")

# silu_status
OK, ERR_INVALID_ARG, ERR_ZERO_PIVOT, ERR_NOT_CONVERGED, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, WARN_DIVERGED, \
    ERR_NO_DEVICE, ERR_TOO_LARGE, ERR_BUSY, ERR_CANCELLED = range(12)
# silu_kind
ILU0, ILUK, ILUT, GS, SGS = 0, 1, 2, 3, 4
# silu_scale
SCALE_NONE, SCALE_ROW, SCALE_NONE_RICH, SCALE_ROWCOL = 0, 1, 2, 3
# silu_prec
FP64, FP32 = 0, 1
# silu_precond
PRECOND_SWEEPS, PRECOND_DIRECT, PRECOND_NONE, PRECOND_AMG, PRECOND_AMG_DIRECT, PRECOND_SCHUR = 0, 1, 2, 3, 4, 5
PRECOND_AMG_SCHUR = 6
# silu_schur_iface
SCHUR_IFACE_NONE, SCHUR_IFACE_DIAG = 0, 1
# silu_kclass
K_RESIDUAL, K_SWEEP_L, K_SWEEP_U, K_LEVEL, K_KRYLOV, K_ELEMENTWISE = range(6)
K_NAMES = ["residual", "sweep_L", "sweep_U", "level", "krylov", "elementwise", "fused"]

KINDS = {"ilu0": ILU0, "iluk": ILUK, "ilut": ILUT, "gs": GS, "sgs": SGS}

_lib = None


class RequestParams(ctypes.Structure):
    """silu_request_params"""
    _fields_ = [("kind", ctypes.c_int), ("tau", ctypes.c_double), ("fill", ctypes.c_int), ("prec", ctypes.c_int),
                ("tol", ctypes.c_double), ("restart", ctypes.c_int), ("maxit", ctypes.c_int),
                ("sweeps_L", ctypes.c_int), ("sweeps_U", ctypes.c_int), ("precond", ctypes.c_int)]


class Result(ctypes.Structure):
    """silu_result"""
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("relres", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_setup_done", ctypes.c_double),
                ("t_done", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


class SiluError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"silu status {status}: {message}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile libsilu.so for sm_103a (nvcc must be on the machine)."""
    from . import _build
    return _build.build(force=force)


def load():
    """Load libsilu.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise SiluError(-1, f"{LIB_PATH} is not built: call paper_2111_09512_gb300.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    pvp = ctypes.POINTER(vp)
    sigs = {
        "silu_version": (ctypes.c_char_p, []),
        "silu_ctx_create": (i32, [i32, vp, pvp]),
        "silu_ctx_destroy": (None, [vp]),
        "silu_last_error": (ctypes.c_char_p, [vp]),
        "silu_mat_create": (i32, [vp, i64, i64, vp, vp, vp, pvp]),
        "silu_mat_destroy": (None, [vp]),
        "silu_mat_residual": (i32, [vp, vp, vp, vp, i32]),
        "silu_mat_set_shape": (i32, [vp, i32, i32, i32]),
        "ilu_setup": (i32, [vp, vp, i32, dbl, i32, i32, i32, pvp]),
        "ilu_refactor": (i32, [vp, vp]),
        "silu_ilu_save": (i32, [vp, ctypes.c_char_p]),
        "silu_ilu_load": (i32, [vp, vp, ctypes.c_char_p, pvp]),
        "ilu_smooth": (i32, [vp, vp, vp, i32, i32, i32]),
        "direct_trisolve": (i32, [vp, vp, vp, i32]),
        "fgmres_solve": (i32, [vp, vp, vp, dbl, i32, i32, i32, i32, i32, ctypes.POINTER(i32),
                               ctypes.POINTER(dbl)]),
        "silu_ilu_reserve": (i32, [vp, i32, i32]),
        "silu_ilu_stats": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "silu_ilu_export": (i32, [vp] * 13),
        "silu_ilu_export_sizes": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "silu_ilu_export_colscale": (i32, [vp, vp, ctypes.POINTER(ctypes.c_int32)]),
        "silu_ilu_power_norms": (i32, [vp, i32, i32, i32, vp, vp]),
        "silu_ilu_dep": (i32, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "silu_amg_setup": (i32, [vp, vp]),
        "silu_amg_vcycle": (i32, [vp, vp, vp, i32, i32]),
        "silu_amg_vcycle_schur": (i32, [vp, vp, vp, i32, i32]),
        "silu_amg_level_ilu": (i32, [vp, i32, vp]),
        "silu_amg_stats": (i32, [vp, i32, ctypes.POINTER(i32), vp, vp, vp]),
        "silu_amg_export_level": (i32, [vp, i32] + [vp] * 7),
        "silu_schur_setup": (i32, [vp, i32, dbl, i32]),
        "silu_schur_smooth": (i32, [vp, vp, vp, i32, i32]),
        "silu_schur_stats": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), vp]),
        "silu_schur_set_interface_prec": (i32, [vp, i32]),
        "silu_ilu_destroy": (None, [vp]),
        "silu_ilu_set_lanes": (i32, [vp, i32, i32, i32]),
        "silu_ctx_profile": (i32, [vp, i32]),
        "silu_ctx_profile_read": (i32, [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(dbl)]),
        "silu_ctx_launch_count": (i32, [vp, ctypes.POINTER(i64)]),
        "silu_ctx_check": (i32, [vp]),
        "silu_ctx_selftest_timeout": (i32, [vp, i32]),
        "silu_ilu_set_kernel": (i32, [vp, i32]),
        "silu_ilu_set_direct": (i32, [vp, i32]),
        "silu_ilu_set_fused": (i32, [vp, i32]),
        "silu_ilu_layout": (i32, [vp, vp, vp, vp]),
        "silu_ctx_set_overlap": (i32, [vp, i32]),
        "silu_ctx_set_l2_reuse": (i32, [vp, i32]),
        "silu_mat_autotune": (i32, [vp, vp, vp, vp, vp]),
        "silu_ilu_tune_table": (i32, [vp, i32, vp, vp, vp]),
        "silu_smooth_noalloc": (i32, [i32, vp, i64] + [vp] * 12 + [i32, i32]),
        "silu_batch_setup": (i32, [vp, i32, vp, vp, vp, vp, i32, dbl, i32, i32, i32, pvp]),
        "silu_batch_info": (i32, [vp, ctypes.POINTER(i32), vp, pvp]),
        "silu_batch_smooth": (i32, [vp, vp, vp, i32, i32]),
        "silu_batch_fgmres": (i32, [vp, vp, vp, dbl, i32, i32, i32, i32, i32, vp, vp]),
        "silu_batch_destroy": (None, [vp]),
        "silu_ilu_autotune": (i32, [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl)]),
        "silu_server_create": (i32, [i32, i64, i32, i32, pvp]),
        "silu_server_submit": (i32, [vp, i64, vp, vp, vp, vp, ctypes.POINTER(RequestParams),
                                     ctypes.POINTER(ctypes.c_uint64)]),
        "silu_server_cancel": (i32, [vp, ctypes.c_uint64]),
        "silu_server_poll": (i32, [vp, ctypes.c_uint64, i32, ctypes.POINTER(i32), ctypes.POINTER(Result), vp]),
        "silu_server_stats": (i32, [vp] + [ctypes.POINTER(i64)] * 5),
        "silu_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the binding declares (all must be exported by libsilu.so)."""
    return ["silu_version", "silu_ctx_create", "silu_ctx_destroy", "silu_last_error", "silu_mat_create",
            "silu_mat_destroy", "silu_mat_residual", "silu_mat_set_shape", "silu_mat_autotune", "ilu_setup", "ilu_refactor", "silu_ilu_save", "silu_ilu_load", "ilu_smooth", "direct_trisolve", "fgmres_solve",
            "silu_ilu_reserve", "silu_ilu_stats", "silu_ilu_export", "silu_ilu_export_sizes",
            "silu_ilu_export_colscale", "silu_ilu_power_norms", "silu_ilu_dep", "silu_amg_setup", "silu_amg_vcycle", "silu_amg_vcycle_schur",
            "silu_amg_level_ilu", "silu_amg_stats", "silu_amg_export_level", "silu_schur_setup", "silu_schur_smooth",
            "silu_schur_stats", "silu_schur_set_interface_prec",
            "silu_ilu_destroy", "silu_ilu_set_lanes", "silu_ctx_profile", "silu_ctx_profile_read",
            "silu_ctx_launch_count", "silu_ctx_check", "silu_ctx_selftest_timeout", "silu_ilu_set_kernel", "silu_ilu_set_direct", "silu_ilu_set_fused", "silu_ilu_layout", "silu_ilu_tune_table", "silu_ctx_set_overlap",
            "silu_ctx_set_l2_reuse",
            "silu_smooth_noalloc",
            "silu_batch_setup", "silu_batch_info", "silu_batch_smooth", "silu_batch_fgmres", "silu_batch_destroy",
            "silu_ilu_autotune", "silu_server_create", "silu_server_submit", "silu_server_cancel",
            "silu_server_poll", "silu_server_stats", "silu_server_destroy"]


def _ptr(t) -> int:
    """Device (or host) address of a torch tensor / numpy array / int."""
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t.data_ptr())


def _check(ctx_handle, status: int, what: str):
    if status != OK:
        msg = load().silu_last_error(ctx_handle) if ctx_handle else b""
        raise SiluError(status, f"{what}: {msg.decode() if msg else ''}")


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ----------------------------------------------------------------- handles

class Context:
    """silu_ctx: a device (or -1 for host-only setup) and a CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        lib = load()
        h = ctypes.c_void_p()
        st = lib.silu_ctx_create(device, _stream_handle(stream), ctypes.byref(h))
        if st != OK:
            raise SiluError(st, f"silu_ctx_create(device={device})")
        self.handle = h.value
        self.device = device
        self.stream = stream

    def close(self):
        if getattr(self, "handle", None):
            load().silu_ctx_destroy(self.handle)
            self.handle = None

    def set_overlap(self, enable: bool):
        """Launch each staged sweep as a programmatic dependent of the kernel before it (default on)."""
        _check(self.handle, load().silu_ctx_set_overlap(self.handle, 1 if enable else 0), "silu_ctx_set_overlap")

    def set_l2_reuse(self, flags: int):
        """L2 reuse flags of staged sweeps: 1 alternate direction, 2 factor at normal priority, 4 vectors at
        normal priority (results are the same bits for every setting)."""
        _check(self.handle, load().silu_ctx_set_l2_reuse(self.handle, int(flags)), "silu_ctx_set_l2_reuse")

    def profile(self, enable: bool):
        """Start (clearing earlier records) or stop event timing of the library's launches."""
        _check(self.handle, load().silu_ctx_profile(self.handle, 1 if enable else 0), "silu_ctx_profile")

    def profile_read(self):
        """{class name: (launches, total ms)} of the recorded launches (blocks on the stream)."""
        out = {}
        for k, name in enumerate(K_NAMES):
            cnt, ms = ctypes.c_int64(), ctypes.c_double()
            _check(self.handle, load().silu_ctx_profile_read(self.handle, k, ctypes.byref(cnt), ctypes.byref(ms)),
                   "silu_ctx_profile_read")
            out[name] = (cnt.value, ms.value)
        return out

    def check(self):
        """Synchronise and raise if a kernel's bounded wait gave up (SILU_ERR_TIMEOUT)."""
        _check(self.handle, load().silu_ctx_check(self.handle), "silu_ctx_check")

    def selftest_timeout(self, timeout_ms: int = 50):
        """Run a bounded GPU wait on a flag nothing sets (the next check() reports ERR_TIMEOUT)."""
        _check(self.handle, load().silu_ctx_selftest_timeout(self.handle, timeout_ms), "silu_ctx_selftest_timeout")

    def launch_count(self) -> int:
        """Kernels this context has launched since it was created."""
        c = ctypes.c_int64()
        _check(self.handle, load().silu_ctx_launch_count(self.handle, ctypes.byref(c)), "silu_ctx_launch_count")
        return c.value

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


AMG_L1_JACOBI, AMG_POLY_GS = 0, 1


class AmgParams(ctypes.Structure):
    """silu_amg_params."""
    _fields_ = [("theta", ctypes.c_double), ("max_levels", ctypes.c_int), ("coarse_size", ctypes.c_int),
                ("jacobi_sweeps", ctypes.c_int), ("coarse_smoother", ctypes.c_int), ("gs_terms", ctypes.c_int),
                ("ilu_levels", ctypes.c_int)]


class Matrix:
    """silu_mat: a CSR matrix copied into the library (and onto the device)."""

    def __init__(self, ctx: Context, row_ptr, col_idx, val):
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        va = np.ascontiguousarray(val, dtype=np.float64)
        n = len(rp) - 1
        h = ctypes.c_void_p()
        st = load().silu_mat_create(ctx.handle, n, int(rp[-1]), _ptr(rp), _ptr(ci), _ptr(va), ctypes.byref(h))
        _check(ctx.handle, st, "silu_mat_create")
        self.handle = h.value
        self.ctx = ctx
        self.n = n
        self.nnz = int(rp[-1])

    def set_shape(self, lanes: int = 0, passes: int = 0, chunk: int = 16):
        """Launch shape of the staged kernel on this matrix (residual and FGMRES products)."""
        _check(self.ctx.handle, load().silu_mat_set_shape(self.handle, int(lanes), int(passes), int(chunk)),
               "silu_mat_set_shape")

    def autotune(self):
        """Time the launch shapes of the staged kernel on this matrix, keep the fastest;
        ((lanes, passes, chunk), ms per product)."""
        g, p, c, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
        _check(self.ctx.handle, load().silu_mat_autotune(self.handle, ctypes.byref(g), ctypes.byref(p),
                                                         ctypes.byref(c), ctypes.byref(ms)), "silu_mat_autotune")
        return (g.value, p.value, c.value), ms.value

    def residual(self, r, x, b):
        """r = b - A x on the device (torch tensors n x nrhs or length n, FP64)."""
        nrhs = 1 if b.dim() == 1 else int(b.shape[1])
        _check(self.ctx.handle, load().silu_mat_residual(self.handle, _ptr(r), _ptr(x), _ptr(b), nrhs),
               "silu_mat_residual")
        return r

    def close(self):
        if getattr(self, "handle", None):
            load().silu_mat_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ILU:
    """silu_ilu: factors of a Matrix, row-scaled and packed on the device."""

    def __init__(self, A: Matrix, kind="ilu0", tau: float = 0.0, fill: int = 0, scale: int = SCALE_ROW,
                 prec: int = FP64):
        kind = KINDS[kind] if isinstance(kind, str) else kind
        h = ctypes.c_void_p()
        st = load().ilu_setup(A.ctx.handle, A.handle, kind, float(tau), int(fill), scale, prec, ctypes.byref(h))
        _check(A.ctx.handle, st, "ilu_setup")
        self.handle = h.value
        self.A = A          # keeps the matrix alive as long as the factors
        self.ctx = A.ctx
        self.n = A.n
        self.prec = prec
        self.scale = scale

    @classmethod
    def load_file(cls, A: Matrix, path: str) -> "ILU":
        """Factors of A read from a file written by save() (no factorisation)."""
        h = ctypes.c_void_p()
        _check(A.ctx.handle, load().silu_ilu_load(A.ctx.handle, A.handle, os.fsencode(path), ctypes.byref(h)),
               "silu_ilu_load")
        F = cls.__new__(cls)
        F.handle = h.value
        F.A = A
        F.ctx = A.ctx
        F.n = A.n
        F.prec = None
        F.scale = None
        return F

    def save(self, path: str):
        """Write L_s and U with their kind, scaling and precision to a file."""
        _check(self.ctx.handle, load().silu_ilu_save(self.handle, os.fsencode(path)), "silu_ilu_save")

    def close(self):
        if getattr(self, "handle", None) and not getattr(self, "_borrowed", False):
            load().silu_ilu_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- queries
    def stats(self):
        n, nl, nu = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ll, lu = ctypes.c_int32(), ctypes.c_int32()
        _check(self.ctx.handle, load().silu_ilu_stats(self.handle, ctypes.byref(n), ctypes.byref(nl),
                                                      ctypes.byref(nu), ctypes.byref(ll), ctypes.byref(lu)),
               "silu_ilu_stats")
        return {"n": n.value, "nnz_L": nl.value, "nnz_U": nu.value, "levels_L": ll.value, "levels_U": lu.value}

    def export(self):
        """Host copies: L_s, U (diagonal first), Utilde_s, dinv, level of each row."""
        lib = load()
        nl, nf, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self.ctx.handle, lib.silu_ilu_export_sizes(self.handle, ctypes.byref(nl), ctypes.byref(nf),
                                                          ctypes.byref(ns)), "silu_ilu_export_sizes")
        n = self.n
        Lp, Up, Sp = (np.empty(n + 1, np.int64) for _ in range(3))
        Lc, Lv = np.empty(max(nl.value, 1), np.int32), np.empty(max(nl.value, 1), np.float64)
        Uc, Uv = np.empty(max(nf.value, 1), np.int32), np.empty(max(nf.value, 1), np.float64)
        Sc, Sv = np.empty(max(ns.value, 1), np.int32), np.empty(max(ns.value, 1), np.float64)
        dinv = np.empty(max(n, 1), np.float64)
        levL, levU = np.empty(max(n, 1), np.int32), np.empty(max(n, 1), np.int32)
        st = lib.silu_ilu_export(self.handle, *[_ptr(a) for a in (Lp, Lc, Lv, Up, Uc, Uv, Sp, Sc, Sv, dinv,
                                                                   levL, levU)])
        _check(self.ctx.handle, st, "silu_ilu_export")
        return {"L": (Lp, Lc[:nl.value], Lv[:nl.value]), "U": (Up, Uc[:nf.value], Uv[:nf.value]),
                "Us": (Sp, Sc[:ns.value], Sv[:ns.value]), "dinv": dinv[:n], "levL": levL[:n],
                "levU": levU[:n]}

    def colscale(self):
        """Row/column scaling only: (D_c, number of Ruiz steps)."""
        dc = np.empty(max(self.n, 1), np.float64)
        steps = ctypes.c_int32()
        _check(self.ctx.handle, load().silu_ilu_export_colscale(self.handle, _ptr(dc), ctypes.byref(steps)),
               "silu_ilu_export_colscale")
        return dc[:self.n], steps.value

    def dep(self):
        """Departure from normality (Eq. depB): {"L": dep(L), "U": dep(U), "scaled": dep of the sweep factor}."""
        a, b_, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self.ctx.handle, load().silu_ilu_dep(self.handle, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)),
               "silu_ilu_dep")
        return {"L": a.value, "U": b_.value, "scaled": c.value}

    def power_norms(self, which: str, pmax: int, iters: int, v0) -> np.ndarray:
        """Estimates of ||T^p||_2, p = 1..pmax, for T = L_s ("L") or the scaled strict upper factor ("U")."""
        v0 = np.ascontiguousarray(v0, np.float64).reshape(self.n)
        out = np.empty(max(pmax, 1), np.float64)
        st = load().silu_ilu_power_norms(self.handle, 0 if which == "L" else 1, int(pmax), int(iters), _ptr(v0),
                                         _ptr(out))
        _check(self.ctx.handle, st, "silu_ilu_power_norms")
        return out[:pmax]

    def amg_setup(self, theta: float = 0.25, max_levels: int = 25, coarse_size: int = 400, jacobi_sweeps: int = 1,
                  coarse_smoother: int = AMG_L1_JACOBI, gs_terms: int = 2, ilu_levels: int = 1):
        """Build and attach the AMG hierarchy of A (Sec. 3); this factor object smooths its finest level,
        l1-Jacobi or polynomial Gauss-Seidel (gs_terms Neumann terms) the coarser ones; with ilu_levels > 1
        the next ilu_levels - 1 levels get ILU smoothers of their own (same kind, tau and fill)."""
        p = AmgParams(float(theta), int(max_levels), int(coarse_size), int(jacobi_sweeps), int(coarse_smoother),
                      int(gs_terms), int(ilu_levels))
        _check(self.ctx.handle, load().silu_amg_setup(self.handle, ctypes.byref(p)), "silu_amg_setup")

    def amg_vcycle(self, x, b, sweeps_L: int, sweeps_U: int):
        """One V-cycle on A x = b (device tensors of length n), x in/out."""
        _check(self.ctx.handle, load().silu_amg_vcycle(self.handle, _ptr(x), _ptr(b), int(sweeps_L),
                                                       int(sweeps_U)), "silu_amg_vcycle")

    def amg_vcycle_schur(self, x, b, sweeps_L: int, sweeps_U: int):
        """One V-cycle whose finest level is smoothed by the Schur complement smoother (schur_setup),
        x in/out."""
        _check(self.ctx.handle, load().silu_amg_vcycle_schur(self.handle, _ptr(x), _ptr(b), int(sweeps_L),
                                                             int(sweeps_U)), "silu_amg_vcycle_schur")

    def amg_stats(self):
        """Per level: rows, entries of A_l, entries of P_l."""
        lev = ctypes.c_int()
        rows, nza, nzp = (np.zeros(64, np.int64) for _ in range(3))
        _check(self.ctx.handle, load().silu_amg_stats(self.handle, 64, ctypes.byref(lev), _ptr(rows), _ptr(nza),
                                                      _ptr(nzp)), "silu_amg_stats")
        k = lev.value
        return {"levels": k, "rows": rows[:k].tolist(), "nnz_A": nza[:k].tolist(), "nnz_P": nzp[:k].tolist()}

    def amg_level_ilu(self, level: int) -> "ILU":
        """The (borrowed) factor object that smooths AMG level `level` with the ILU smoother: self for
        level 0, the row-scaled factors of A_l for levels below it that amg_setup(ilu_levels=...)
        gave one; valid while this hierarchy lives."""
        h = ctypes.c_void_p()
        _check(self.ctx.handle, load().silu_amg_level_ilu(self.handle, int(level), ctypes.byref(h)),
               "silu_amg_level_ilu")
        if level == 0:
            return self
        G = ILU.__new__(ILU)
        G.handle = h.value
        G._borrowed = True
        G._owner = self
        G.A = None
        G.ctx = self.ctx
        G.n = int(self.amg_stats()["rows"][level])
        G.prec = self.prec
        G.scale = SCALE_ROW
        return G

    def amg_level(self, level: int):
        """Host copies of level `level`: A_l, P_l (None on the coarsest level), coarse-point marks."""
        st = self.amg_stats()
        n, nza, nzp = st["rows"][level], st["nnz_A"][level], st["nnz_P"][level]
        Ap = np.empty(n + 1, np.int64)
        Ac, Av = np.empty(max(nza, 1), np.int32), np.empty(max(nza, 1), np.float64)
        last = level == st["levels"] - 1
        Pp = np.empty(n + 1, np.int64)
        Pc, Pv = np.empty(max(nzp, 1), np.int32), np.empty(max(nzp, 1), np.float64)
        cf = np.empty(max(n, 1), np.int32)
        _check(self.ctx.handle, load().silu_amg_export_level(self.handle, int(level), _ptr(Ap), _ptr(Ac), _ptr(Av),
                                                             None if last else _ptr(Pp), None if last else _ptr(Pc),
                                                             None if last else _ptr(Pv),
                                                             None if last else _ptr(cf)), "silu_amg_export_level")
        return {"A": (Ap, Ac[:nza], Av[:nza]), "P": None if last else (Pp, Pc[:nzp], Pv[:nzp]),
                "cf": None if last else cf[:n]}

    def schur_setup(self, parts: int, tau: float, fill: int):
        """Attach the ILUT Schur complement smoother (Sec. 3.1) over `parts` contiguous row blocks."""
        _check(self.ctx.handle, load().silu_schur_setup(self.handle, int(parts), float(tau), int(fill)),
               "silu_schur_setup")

    def schur_smooth(self, x, b, sweeps_L: int, sweeps_U: int):
        """x <- x + M^{-1}(b - A x) with the Schur complement smoother (device tensors of length n)."""
        _check(self.ctx.handle, load().silu_schur_smooth(self.handle, _ptr(x), _ptr(b), int(sweeps_L),
                                                         int(sweeps_U)), "silu_schur_smooth")

    def schur_set_interface_prec(self, mode: int):
        """Right preconditioner of the Schur complement smoother's interface GMRES iteration:
        SCHUR_IFACE_NONE (the paper's) or SCHUR_IFACE_DIAG (diag(C))."""
        _check(self.ctx.handle, load().silu_schur_set_interface_prec(self.handle, int(mode)),
               "silu_schur_set_interface_prec")

    def schur_stats(self):
        ni, ng = ctypes.c_int64(), ctypes.c_int64()
        marks = np.empty(max(self.n, 1), np.int32)
        _check(self.ctx.handle, load().silu_schur_stats(self.handle, ctypes.byref(ni), ctypes.byref(ng),
                                                        _ptr(marks)), "silu_schur_stats")
        return {"interior": ni.value, "interface": ng.value, "marks": marks[:self.n]}

    def reserve(self, nrhs: int = 1, restart: int = 0):
        _check(self.ctx.handle, load().silu_ilu_reserve(self.handle, nrhs, restart), "silu_ilu_reserve")

    def set_kernel(self, variant: int):
        """0 automatic, 1 lanes-per-row kernel, 2 staged (bulk-copy) kernel where it applies (natural
        row order), 3 staged kernel on the length-sorted copies where they exist."""
        _check(self.ctx.handle, load().silu_ilu_set_kernel(self.handle, variant), "silu_ilu_set_kernel")

    def set_direct(self, mode: int):
        """Schedule of the exact triangular solves: 0 automatic (default; the faster of the two, timed
        once per column count), 1 one launch per level (captured graph), 2 one persistent launch."""
        _check(self.ctx.handle, load().silu_ilu_set_direct(self.handle, mode), "silu_ilu_set_direct")

    def set_fused(self, mode: int):
        """Whole smoother application in one cooperative launch: 0 for small systems (default), 1 never,
        2 always."""
        _check(self.ctx.handle, load().silu_ilu_set_fused(self.handle, mode), "silu_ilu_set_fused")

    def layout(self):
        """FMA slots per entry of one-lane-per-row tiles, natural and length-sorted rows, for
        (L_s, upper factor), and whether the current variant sweeps a sorted copy."""
        nat, srt = np.zeros(2), np.zeros(2)
        use = np.zeros(2, np.int32)
        _check(self.ctx.handle, load().silu_ilu_layout(self.handle, _ptr(nat), _ptr(srt), _ptr(use)),
               "silu_ilu_layout")
        return {"pad_natural": nat, "pad_sorted": srt, "in_use": use.astype(bool)}

    def autotune(self, sweeps_L: int = 3, sweeps_U: int = 3):
        """Time the candidate launch shapes of the sweep kernels, keep the fastest; (choice, ms)."""
        ch, ms = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(self.ctx.handle, load().silu_ilu_autotune(self.handle, sweeps_L, sweeps_U, ctypes.byref(ch),
                                                         ctypes.byref(ms)), "silu_ilu_autotune")
        return ch.value, ms.value

    def tune_table(self):
        """[(variant, lanes, passes, chunk, ms)] of the last autotune (ms -1: candidate not run)."""
        cnt = ctypes.c_int(0)
        _check(self.ctx.handle, load().silu_ilu_tune_table(self.handle, 0, 0, 0, ctypes.byref(cnt)),
               "silu_ilu_tune_table")
        shape = np.zeros(4 * cnt.value, np.int32)
        ms = np.zeros(cnt.value)
        _check(self.ctx.handle, load().silu_ilu_tune_table(self.handle, cnt.value, _ptr(shape), _ptr(ms),
                                                           ctypes.byref(cnt)), "silu_ilu_tune_table")
        return [tuple(int(v) for v in shape[4 * k:4 * k + 4]) + (float(ms[k]),) for k in range(cnt.value)]

    def set_lanes(self, lanes_L: int = 0, lanes_U: int = 0, lanes_A: int = 0):
        _check(self.ctx.handle, load().silu_ilu_set_lanes(self.handle, lanes_L, lanes_U, lanes_A),
               "silu_ilu_set_lanes")


class Batch:
    """silu_batch: independent systems factored in parallel, packed block-diagonally."""

    def __init__(self, ctx: Context, systems, kind="ilu0", tau: float = 0.0, fill: int = 0,
                 scale: int = SCALE_ROW, prec: int = FP64):
        kind = KINDS[kind] if isinstance(kind, str) else kind
        arrs = []
        for rp, ci, va in systems:
            arrs.append((np.ascontiguousarray(rp, dtype=np.int64), np.ascontiguousarray(ci, dtype=np.int32),
                         np.ascontiguousarray(va, dtype=np.float64)))
        cnt = len(arrs)
        n = np.array([len(a[0]) - 1 for a in arrs], dtype=np.int64)
        P = ctypes.c_void_p * cnt
        rps = P(*[a[0].ctypes.data for a in arrs])
        cis = P(*[a[1].ctypes.data for a in arrs])
        vas = P(*[a[2].ctypes.data for a in arrs])
        h = ctypes.c_void_p()
        st = load().silu_batch_setup(ctx.handle, cnt, n.ctypes.data, ctypes.addressof(rps), ctypes.addressof(cis),
                                     ctypes.addressof(vas), kind, float(tau), int(fill), scale, prec, ctypes.byref(h))
        _check(ctx.handle, st, "silu_batch_setup")
        self.handle = h.value
        self.ctx = ctx
        self.count = cnt
        self.offsets = np.empty(cnt + 1, dtype=np.int64)
        fh = ctypes.c_void_p()
        c = ctypes.c_int(0)
        _check(ctx.handle, load().silu_batch_info(self.handle, ctypes.byref(c), self.offsets.ctypes.data,
                                                  ctypes.byref(fh)), "silu_batch_info")
        self.n = int(self.offsets[-1])
        # a non-owning view of the concatenated factors (owned by the batch)
        self.factors = ILU.__new__(ILU)
        self.factors.handle = fh.value
        self.factors.ctx = ctx
        self.factors.n = self.n
        self.factors.prec = prec
        self.factors.scale = scale
        self.factors.A = None
        self.factors._borrowed = True

    def close(self):
        if getattr(self, "handle", None):
            self.factors.handle = None
            load().silu_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def silu_batch_smooth(B: Batch, x, b, sweeps_L: int, sweeps_U: int) -> None:
    _check_vec(x, B.n, 1)
    _check_vec(b, B.n, 1)
    _check(B.ctx.handle, load().silu_batch_smooth(B.handle, _ptr(x), _ptr(b), sweeps_L, sweeps_U),
           "silu_batch_smooth")


def silu_batch_fgmres(B: Batch, x, b, tol: float = 1e-8, restart: int = 20, maxit: int = 1000, sweeps_L: int = 3,
                      sweeps_U: int = 3, precond: int = PRECOND_SWEEPS):
    """Per-system FGMRES on the whole batch; returns (status, iterations[count], relres[count])."""
    _check_vec(x, B.n, 1)
    _check_vec(b, B.n, 1)
    its = np.zeros(B.count, dtype=np.int32)
    rel = np.zeros(B.count, dtype=np.float64)
    st = load().silu_batch_fgmres(B.handle, _ptr(x), _ptr(b), float(tol), int(restart), int(maxit), int(sweeps_L),
                                  int(sweeps_U), int(precond), its.ctypes.data, rel.ctypes.data)
    if st not in (OK, ERR_NOT_CONVERGED):
        _check(B.ctx.handle, st, "silu_batch_fgmres")
    return st, its, rel


class Server:
    """silu_server: continuous batching of FGMRES solves under an HBM budget."""

    def __init__(self, device: int = 0, hbm_budget: int = 120 << 30, workers: int = 4, max_queue: int = 64):
        h = ctypes.c_void_p()
        st = load().silu_server_create(device, int(hbm_budget), workers, max_queue, ctypes.byref(h))
        if st != OK:
            raise SiluError(st, "silu_server_create")
        self.handle = h.value
        self._keep = {}

    def submit(self, A, b, kind="ilu0", tau=0.0, fill=0, prec=FP32, tol=1e-8, restart=30, maxit=5000,
               sweeps_L=3, sweeps_U=3, precond=PRECOND_SWEEPS):
        """Returns (status, ticket); status ERR_OOM / ERR_BUSY when refused."""
        rp = np.ascontiguousarray(A[0], dtype=np.int64)
        ci = np.ascontiguousarray(A[1], dtype=np.int32)
        va = np.ascontiguousarray(A[2], dtype=np.float64)
        bb = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        n = len(rp) - 1
        p = RequestParams(KINDS[kind] if isinstance(kind, str) else kind, float(tau), int(fill), int(prec),
                          float(tol), int(restart), int(maxit), int(sweeps_L), int(sweeps_U), int(precond))
        t = ctypes.c_uint64(0)
        st = load().silu_server_submit(self.handle, n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(bb), ctypes.byref(p),
                                       ctypes.byref(t))
        if st == OK:
            self._keep[t.value] = n
        return st, t.value

    def poll(self, ticket: int, wait: bool = False, want_x: bool = True):
        """(done, Result, x or None); a finished ticket is released."""
        n = self._keep.get(ticket, 0)
        x = np.empty(max(n, 1), dtype=np.float64) if want_x else None
        done = ctypes.c_int(0)
        res = Result()
        st = load().silu_server_poll(self.handle, ticket, 1 if wait else 0, ctypes.byref(done), ctypes.byref(res),
                                     _ptr(x) if x is not None else 0)
        if st != OK:
            raise SiluError(st, "silu_server_poll")
        if done.value:
            self._keep.pop(ticket, None)
            return True, res, (x[:n] if x is not None else None)
        return False, None, None

    def cancel(self, ticket: int) -> int:
        return load().silu_server_cancel(self.handle, ticket)

    def stats(self):
        vals = [ctypes.c_int64() for _ in range(5)]
        load().silu_server_stats(self.handle, *[ctypes.byref(v) for v in vals])
        return dict(zip(["queued", "running", "completed", "refused", "bytes_in_use"], [v.value for v in vals]))

    def close(self):
        if getattr(self, "handle", None):
            load().silu_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- C-named functions

def silu_version() -> str:
    return load().silu_version().decode()


def silu_ctx_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def silu_mat_create(ctx: Context, row_ptr, col_idx, val) -> Matrix:
    return Matrix(ctx, row_ptr, col_idx, val)


def ilu_setup(ctx: Context, A: Matrix, kind="ilu0", tau: float = 0.0, fill: int = 0, scale: int = SCALE_ROW,
              prec: int = FP64) -> ILU:
    if A.ctx is not ctx:
        raise SiluError(ERR_INVALID_ARG, "matrix belongs to another context")
    return ILU(A, kind, tau, fill, scale, prec)


def ilu_refactor(F: ILU, new_val) -> None:
    v = np.ascontiguousarray(new_val, dtype=np.float64)
    if v.size != F.A.nnz:
        raise SiluError(ERR_INVALID_ARG, "new values must match the matrix's entry count")
    _check(F.ctx.handle, load().ilu_refactor(F.handle, _ptr(v)), "ilu_refactor")


def _nrhs_of(x, n):
    shape = tuple(x.shape)
    if len(shape) == 1:
        return 1
    if shape[0] != n:
        raise SiluError(ERR_INVALID_ARG, "vectors must be n x nrhs")
    return int(shape[1])


def _check_vec(t, n, nrhs):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise SiluError(ERR_INVALID_ARG, "vectors must be contiguous float64 CUDA tensors")
    if t.numel() != n * nrhs:
        raise SiluError(ERR_INVALID_ARG, "vector size mismatch")


def ilu_smooth(F: ILU, x, b, sweeps_L: int, sweeps_U: int) -> None:
    """x <- x + M^{-1}(b - A x) with sweeps_L / sweeps_U Richardson sweeps (in place)."""
    nrhs = _nrhs_of(x, F.n)
    _check_vec(x, F.n, nrhs)
    _check_vec(b, F.n, nrhs)
    _check(F.ctx.handle, load().ilu_smooth(F.handle, _ptr(x), _ptr(b), nrhs, sweeps_L, sweeps_U), "ilu_smooth")


def direct_trisolve(F: ILU, x, b) -> None:
    """x <- x + Utilde^{-1} D^{-1} L^{-1} (b - A x) by level-scheduled substitution."""
    nrhs = _nrhs_of(x, F.n)
    _check_vec(x, F.n, nrhs)
    _check_vec(b, F.n, nrhs)
    _check(F.ctx.handle, load().direct_trisolve(F.handle, _ptr(x), _ptr(b), nrhs), "direct_trisolve")


def silu_smooth_noalloc(device: int, stream, n: int, A, L, Us, dinv, x, b, sweeps_L: int, sweeps_U: int) -> int:
    """Allocation-free smoother application on caller-owned device arrays.

    A, L and Us are (row_ptr int32, col int32, val float64) device tensors;
    dinv, x (in/out) and b are float64 device vectors of length n.  Returns
    the status (ERR_TOO_LARGE above the fixed capacity); nothing is allocated
    by the library during the call.
    """
    args = [_ptr(t) for t in (*A, *L, *Us, dinv, x, b)]
    return load().silu_smooth_noalloc(device, _stream_handle(stream), n, *args, sweeps_L, sweeps_U)


def fgmres_solve(F: ILU, x, b, tol: float = 1e-8, restart: int = 30, maxit: int = 1000, sweeps_L: int = 3,
                 sweeps_U: int = 3, precond: int = PRECOND_SWEEPS, raise_on_nonconvergence: bool = False):
    """FGMRES(restart) on A x = b; returns (status, iterations, true relative residual)."""
    _check_vec(x, F.n, 1)
    _check_vec(b, F.n, 1)
    its = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = load().fgmres_solve(F.handle, _ptr(x), _ptr(b), float(tol), int(restart), int(maxit), int(sweeps_L),
                             int(sweeps_U), int(precond), ctypes.byref(its), ctypes.byref(rel))
    if st not in (OK, ERR_NOT_CONVERGED) or (st == ERR_NOT_CONVERGED and raise_on_nonconvergence):
        _check(F.ctx.handle, st, "fgmres_solve")
    return st, its.value, rel.value
