"""CPU oracle for the scaled-ILU Richardson smoother (TEST INFRASTRUCTURE).

Plain, slow, single-threaded FP64 code (oracle.c, compiled with
-ffp-contract=off) that states what the smoother computes, step by step from
Thomas et al., "Scaled ILU Smoothers for Navier-Stokes Pressure Projection"
(arXiv 2111.09512): ILU(0) / ILU(k) / ILUT factorisation (Sec. 4.2, Sec. 5.1), row
scaling (Eq. extractD, Eq. newD), the Richardson sweeps of Alg. ILUJac and
Eq. richard, the direct triangular solves with level sets (Sec. 4), FGMRES
with modified Gram-Schmidt (Sec. 6) and the diagnostics dep (Eq. depB) and
NRBE (Eq. nbre), the polynomial Gauss-Seidel smoother of Sec. 3.1 and the
row/column (Ruiz) scaling of Eq. rowcolScale, and the power-iteration
estimates of ||T_s^p||_2 behind the paper's numerical nilpotence (Fig. Up),
and algebraic multigrid (Sec. 3: Ruge-Stueben coarsening, direct
interpolation, Galerkin coarse operators, the V-cycle of Alg. mgcycle with
the ILU smoother on the finest level), and the ILUT Schur complement
smoother of Sec. 3.1 (Eq. schur).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.  Each wrapper
below returns numpy arrays; vectors with R right-hand sides are (n, R)
row-major.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

OK, BADARG, ZERO_PIVOT, NOT_CONVERGED, NOMEM = 0, 1, 2, 3, 4

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (no FMA contraction, so each operation rounds as written)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "orc_ilu0": (vp, [i64, vp, vp, vp, ip]),
        "orc_iluk": (vp, [i64, vp, vp, vp, i32, ip]),
        "orc_ilut": (vp, [i64, vp, vp, vp, dbl, i32, ip]),
        "orc_lu_nnz": (None, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "orc_lu_copy": (None, [vp, vp, vp, vp, vp, vp, vp]),
        "orc_lu_free": (None, [vp]),
        "orc_iluk_pattern": (i32, [i64, vp, vp, i32, ctypes.POINTER(i64), ctypes.POINTER(vp),
                                   ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "orc_free": (None, [vp]),
        "orc_row_scale": (i32, [i64, vp, vp, vp, vp, vp, vp, vp]),
        "orc_spmv": (None, [i64, i32, vp, vp, vp, vp, vp]),
        "orc_residual": (None, [i64, i32, vp, vp, vp, vp, vp, vp]),
        "orc_richardson_lower": (i32, [i64, i32, vp, vp, vp, vp, i32, vp]),
        "orc_richardson_upper": (i32, [i64, i32, vp, vp, vp, vp, vp, i32, vp]),
        "orc_smooth": (i32, [i64, i32] + [vp] * 12 + [i32, i32]),
        "orc_upper_unscaled_richardson": (i32, [i64, i32, vp, vp, vp, vp, i32, vp]),
        "orc_upper_jacobi": (i32, [i64, i32, vp, vp, vp, vp, i32, vp]),
        "orc_forward_subst": (None, [i64, i32, vp, vp, vp, vp, vp]),
        "orc_backward_subst_unit": (None, [i64, i32, vp, vp, vp, vp, vp]),
        "orc_direct_apply": (i32, [i64, i32] + [vp] * 12),
        "orc_levels_lower": (i64, [i64, vp, vp, vp]),
        "orc_levels_upper": (i64, [i64, vp, vp, vp]),
        "orc_fgmres": (i32, [i64] + [vp] * 12 + [dbl, i32, i32, i32, i32, i32,
                                                   ctypes.POINTER(ctypes.c_int),
                                                   ctypes.POINTER(dbl)]),
        "orc_dep_triangular": (dbl, [i64, vp, vp, vp, i32]),
        "orc_norm2_est": (dbl, [i64, vp, vp, vp, i32]),
        "orc_nrbe": (dbl, [i64, vp, vp, vp, dbl, vp, vp]),
        "orc_poly_gs_lower": (i32, [i64, i32, vp, vp, vp, vp, i32, vp]),
        "orc_poly_gs_upper_unit": (i32, [i64, i32, vp, vp, vp, vp, i32, vp]),
        "orc_poly_gs_smooth": (i32, [i64, i32, vp, vp, vp, vp, vp, i32, i32, i32]),
        "orc_ruiz_rowcol": (i32, [i64, vp, vp, vp, i32, dbl, vp, vp, vp, vp, vp]),
        "orc_smooth_rowcol": (i32, [i64, i32] + [vp] * 13 + [i32, i32]),
        "orc_power_norms": (i32, [i64, vp, vp, vp, i32, i32, vp, vp]),
        "orc_amg_setup": (vp, [i64, vp, vp, vp, dbl, i32, i64, ip]),
        "orc_amg_free": (None, [vp]),
        "orc_amg_nlev": (i32, [vp]),
        "orc_amg_level_sizes": (None, [vp, i32] + [ctypes.POINTER(i64)] * 4),
        "orc_amg_level_copy": (None, [vp, i32] + [vp] * 7),
        "orc_amg_vcycle": (i32, [vp] + [vp] * 7 + [i32, i32, i32, i32, i32, vp, vp]),
        "orc_schur_interface": (i64, [i64, vp, vp, i32, vp]),
        "orc_schur_apply": (i32, [i64, vp, vp, vp, i32, dbl, i32, i32, i32, vp, vp]),
        "orc_schur_apply_prec": (i32, [i64, vp, vp, vp, i32, dbl, i32, i32, i32, i32, vp, vp]),
        "orc_amg_vcycle_schur": (i32, [vp, i32, dbl, i32, i32, i32, i32, i32, i32, i32, vp, vp]),
        "orc_amg_vcycle_ilu": (i32, [vp, i32] + [vp] * 9 + [i32, i32, i32, i32, dbl, i32, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _csr(A):
    rp, ci, va = A
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    va = np.ascontiguousarray(va, dtype=np.float64)
    return rp, ci, va


def _vec(x, n):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x.reshape(n, 1)
    return x


@dataclass
class Factors:
    """ILU factors: L_s strict lower CSR, U with diagonal first in each row."""
    n: int
    L: tuple
    U: tuple


@dataclass
class Scaled:
    """Row-scaled factors: L_s, Utilde_s = strict part of D^{-1} U, dinv = 1/diag(U)."""
    n: int
    L: tuple
    Us: tuple
    dinv: np.ndarray


def _take(h, n, what):
    lib = _load()
    nl, nu = ctypes.c_int64(), ctypes.c_int64()
    lib.orc_lu_nnz(h, ctypes.byref(nl), ctypes.byref(nu))
    lp = np.empty(n + 1, np.int64)
    up = np.empty(n + 1, np.int64)
    lc = np.empty(max(nl.value, 1), np.int32)
    lv = np.empty(max(nl.value, 1), np.float64)
    uc = np.empty(max(nu.value, 1), np.int32)
    uv = np.empty(max(nu.value, 1), np.float64)
    lib.orc_lu_copy(h, _p(lp), _p(lc), _p(lv), _p(up), _p(uc), _p(uv))
    lib.orc_lu_free(h)
    return Factors(n, (lp, lc[:nl.value], lv[:nl.value]), (up, uc[:nu.value], uv[:nu.value]))


def ilu0(A) -> Factors:
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    st = ctypes.c_int(0)
    h = _load().orc_ilu0(n, _p(rp), _p(ci), _p(va), ctypes.byref(st))
    if not h:
        raise OracleError(st.value, "ilu0")
    return _take(h, n, "ilu0")


def iluk(A, k: int) -> Factors:
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    st = ctypes.c_int(0)
    h = _load().orc_iluk(n, _p(rp), _p(ci), _p(va), k, ctypes.byref(st))
    if not h:
        raise OracleError(st.value, "iluk")
    return _take(h, n, "iluk")


def iluk_pattern(A, k: int):
    """(row_ptr, col, level) of the ILU(k) fill pattern, L and U parts together."""
    rp, ci, _ = _csr(A)
    n = len(rp) - 1
    lib = _load()
    nnz = ctypes.c_int64()
    pp, pc, pl = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    st = lib.orc_iluk_pattern(n, _p(rp), _p(ci), k, ctypes.byref(nnz), ctypes.byref(pp),
                              ctypes.byref(pc), ctypes.byref(pl))
    if st:
        raise OracleError(st, "iluk_pattern")
    m = nnz.value
    out_p = np.ctypeslib.as_array((ctypes.c_int64 * (n + 1)).from_address(pp.value)).copy()
    out_c = np.ctypeslib.as_array((ctypes.c_int32 * max(m, 1)).from_address(pc.value))[:m].copy()
    out_l = np.ctypeslib.as_array((ctypes.c_int32 * max(m, 1)).from_address(pl.value))[:m].copy()
    for q in (pp, pc, pl):
        lib.orc_free(q)
    return out_p, out_c, out_l


def ilut(A, tau: float, p: int) -> Factors:
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    st = ctypes.c_int(0)
    h = _load().orc_ilut(n, _p(rp), _p(ci), _p(va), float(tau), int(p), ctypes.byref(st))
    if not h:
        raise OracleError(st.value, "ilut")
    return _take(h, n, "ilut")


def factor(A, kind: str = "ilu0", tau: float = 0.0, fill: int = 0) -> Factors:
    if kind == "ilu0":
        return ilu0(A)
    if kind == "iluk":
        return iluk(A, fill)
    if kind == "ilut":
        return ilut(A, tau, fill)
    raise ValueError(kind)


def row_scale(F: Factors) -> Scaled:
    up, uc, uv = F.U
    n = F.n
    m = max(len(uc) - n, 1)
    dinv = np.empty(n, np.float64)
    sp = np.empty(n + 1, np.int64)
    sc = np.empty(m, np.int32)
    sv = np.empty(m, np.float64)
    st = _load().orc_row_scale(n, _p(up), _p(uc), _p(uv), _p(dinv), _p(sp), _p(sc), _p(sv))
    if st:
        raise OracleError(st, "row_scale")
    k = len(uc) - n
    return Scaled(n, F.L, (sp, sc[:k], sv[:k]), dinv)


def spmv(A, x):
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    x = _vec(x, n)
    y = np.empty_like(x)
    _load().orc_spmv(n, x.shape[1], _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def residual(A, x, b):
    rp, ci, va = _csr(A)
    n = len(rp) - 1
    x, b = _vec(x, n), _vec(b, n)
    r = np.empty_like(b)
    _load().orc_residual(n, b.shape[1], _p(rp), _p(ci), _p(va), _p(x), _p(b), _p(r))
    return r


def richardson_lower(L, r, m: int):
    lp, lc, lv = _csr(L)
    n = len(lp) - 1
    r = _vec(r, n)
    y = np.empty_like(r)
    st = _load().orc_richardson_lower(n, r.shape[1], _p(lp), _p(lc), _p(lv), _p(r), m, _p(y))
    if st:
        raise OracleError(st, "richardson_lower")
    return y


def richardson_upper(Us, dinv, y, m: int):
    sp, sc, sv = _csr(Us)
    n = len(sp) - 1
    y = _vec(y, n)
    dinv = np.ascontiguousarray(dinv, np.float64)
    v = np.empty_like(y)
    st = _load().orc_richardson_upper(n, y.shape[1], _p(sp), _p(sc), _p(sv), _p(dinv), _p(y), m, _p(v))
    if st:
        raise OracleError(st, "richardson_upper")
    return v


def smooth(A, S: Scaled, x, b, mL: int, mU: int):
    """x + M^{-1}(b - A x) by m_L + m_U Richardson sweeps (returns a new array)."""
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    x = _vec(x, n).copy()
    b = _vec(b, n)
    lp, lc, lv = _csr(S.L)
    sp, sc, sv = _csr(S.Us)
    st = _load().orc_smooth(n, b.shape[1], _p(ap), _p(ac), _p(av), _p(lp), _p(lc), _p(lv), _p(sp),
                            _p(sc), _p(sv), _p(S.dinv), _p(x), _p(b), mL, mU)
    if st:
        raise OracleError(st, "smooth")
    return x


def direct_apply(A, S: Scaled, x, b):
    """x + Utilde^{-1} D^{-1} L^{-1} (b - A x) by substitution (returns a new array)."""
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    x = _vec(x, n).copy()
    b = _vec(b, n)
    lp, lc, lv = _csr(S.L)
    sp, sc, sv = _csr(S.Us)
    st = _load().orc_direct_apply(n, b.shape[1], _p(ap), _p(ac), _p(av), _p(lp), _p(lc), _p(lv),
                                  _p(sp), _p(sc), _p(sv), _p(S.dinv), _p(x), _p(b))
    if st:
        raise OracleError(st, "direct_apply")
    return x


def upper_unscaled_richardson(U, y, m: int):
    up, uc, uv = _csr(U)
    n = len(up) - 1
    y = _vec(y, n)
    v = np.empty_like(y)
    st = _load().orc_upper_unscaled_richardson(n, y.shape[1], _p(up), _p(uc), _p(uv), _p(y), m, _p(v))
    if st:
        raise OracleError(st, "upper_unscaled_richardson")
    return v


def upper_jacobi(U, y, m: int):
    up, uc, uv = _csr(U)
    n = len(up) - 1
    y = _vec(y, n)
    v = np.empty_like(y)
    st = _load().orc_upper_jacobi(n, y.shape[1], _p(up), _p(uc), _p(uv), _p(y), m, _p(v))
    if st:
        raise OracleError(st, "upper_jacobi")
    return v


def forward_subst(L, r):
    lp, lc, lv = _csr(L)
    n = len(lp) - 1
    r = _vec(r, n)
    y = np.empty_like(r)
    _load().orc_forward_subst(n, r.shape[1], _p(lp), _p(lc), _p(lv), _p(r), _p(y))
    return y


def backward_subst_unit(Us, c):
    sp, sc, sv = _csr(Us)
    n = len(sp) - 1
    c = _vec(c, n)
    v = np.empty_like(c)
    _load().orc_backward_subst_unit(n, c.shape[1], _p(sp), _p(sc), _p(sv), _p(c), _p(v))
    return v


def levels_lower(L):
    lp, lc, _ = _csr(L)
    n = len(lp) - 1
    lev = np.empty(max(n, 1), np.int32)
    nl = _load().orc_levels_lower(n, _p(lp), _p(lc), _p(lev))
    return int(nl), lev[:n]


def levels_upper(Us):
    sp, sc, _ = _csr(Us)
    n = len(sp) - 1
    lev = np.empty(max(n, 1), np.int32)
    nl = _load().orc_levels_upper(n, _p(sp), _p(sc), _p(lev))
    return int(nl), lev[:n]


def fgmres(A, S: Scaled | None, b, x0=None, tol: float = 1e-8, restart: int = 30, maxit: int = 1000,
           mL: int = 3, mU: int = 3, precond: int = 0):
    """FGMRES(restart) for one RHS.  Returns (x, status, iterations, true relres)."""
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    b = np.ascontiguousarray(b, np.float64).reshape(n)
    x = np.zeros(n) if x0 is None else np.ascontiguousarray(x0, np.float64).reshape(n).copy()
    if S is None:
        if precond != 2:
            raise ValueError("a preconditioner needs factors")
        z64 = np.zeros(1, np.int64)
        z32 = np.zeros(1, np.int32)
        zf = np.zeros(max(n, 1))
        lp = np.zeros(n + 1, np.int64)
        L = (lp, z32, zf)
        Us = (lp, z32, zf)
        dinv = zf
        del z64
    else:
        L, Us, dinv = _csr(S.L), _csr(S.Us), S.dinv
    its = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _load().orc_fgmres(n, _p(ap), _p(ac), _p(av), _p(L[0]), _p(L[1]), _p(L[2]), _p(Us[0]),
                            _p(Us[1]), _p(Us[2]), _p(dinv), _p(x), _p(b), float(tol), int(restart),
                            int(maxit), int(mL), int(mU), int(precond), ctypes.byref(its),
                            ctypes.byref(rel))
    if st not in (OK, NOT_CONVERGED):
        raise OracleError(st, "fgmres")
    return x, st, its.value, rel.value


def dep_triangular(T, unit_diag: bool = False) -> float:
    tp, tc, tv = _csr(T)
    n = len(tp) - 1
    return float(_load().orc_dep_triangular(n, _p(tp), _p(tc), _p(tv), 1 if unit_diag else 0))


def norm2_est(A, iters: int = 100) -> float:
    ap, ac, av = _csr(A)
    return float(_load().orc_norm2_est(len(ap) - 1, _p(ap), _p(ac), _p(av), iters))


def nrbe(A, x, b, norm2A: float) -> float:
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    x = np.ascontiguousarray(x, np.float64).reshape(n)
    b = np.ascontiguousarray(b, np.float64).reshape(n)
    return float(_load().orc_nrbe(n, _p(ap), _p(ac), _p(av), float(norm2A), _p(x), _p(b)))


def poly_gs_lower(A, r, p: int):
    """sum_{j=0}^{p} (-D^{-1} L)^j D^{-1} r, term by term (Sec. 3.1, polynomial Gauss-Seidel)."""
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    r = _vec(r, n)
    z = np.empty_like(r)
    st = _load().orc_poly_gs_lower(n, r.shape[1], _p(ap), _p(ac), _p(av), _p(r), int(p), _p(z))
    if st:
        raise OracleError(st, "poly_gs_lower")
    return z


def poly_gs_upper_unit(A, z, q: int):
    """sum_{j=0}^{q} (-D^{-1} U)^j z, term by term (backward half of symmetric Gauss-Seidel)."""
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    z = _vec(z, n)
    w = np.empty_like(z)
    st = _load().orc_poly_gs_upper_unit(n, z.shape[1], _p(ap), _p(ac), _p(av), _p(z), int(q), _p(w))
    if st:
        raise OracleError(st, "poly_gs_upper_unit")
    return w


def poly_gs_smooth(A, x, b, pL: int, pU: int = 0, symmetric: bool = False):
    """x + M^{-1}(b - A x) with M^{-1} the truncated Gauss-Seidel polynomial (returns a new array)."""
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    x = _vec(x, n).copy()
    b = _vec(b, n)
    st = _load().orc_poly_gs_smooth(n, b.shape[1], _p(ap), _p(ac), _p(av), _p(x), _p(b), int(pL), int(pU),
                                    1 if symmetric else 0)
    if st:
        raise OracleError(st, "poly_gs_smooth")
    return x


@dataclass
class RowCol:
    """Row/column-scaled factors: L_s, Uhat_s = strict part of D_r U D_c (unit
    diagonal), dr, dc, and the number of Ruiz steps taken."""
    n: int
    L: tuple
    Us: tuple
    dr: np.ndarray
    dc: np.ndarray
    steps: int


def ruiz_rowcol(F: Factors, maxit: int = 20, tol: float = 1e-2) -> RowCol:
    up, uc, uv = F.U
    n = F.n
    k = len(uc) - n
    dr = np.empty(max(n, 1), np.float64)
    dc = np.empty(max(n, 1), np.float64)
    sp = np.empty(n + 1, np.int64)
    sc = np.empty(max(k, 1), np.int32)
    sv = np.empty(max(k, 1), np.float64)
    st = _load().orc_ruiz_rowcol(n, _p(up), _p(uc), _p(uv), int(maxit), float(tol), _p(dr), _p(dc), _p(sp),
                                 _p(sc), _p(sv))
    if st < 0:
        raise OracleError(-st, "ruiz_rowcol")
    return RowCol(n, F.L, (sp, sc[:k], sv[:k]), dr[:n], dc[:n], int(st))


def smooth_rowcol(A, S: RowCol, x, b, mL: int, mU: int):
    """x + D_c Uhat^{-1} D_r L^{-1} (b - A x), each inverse by Richardson sweeps (new array)."""
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    x = _vec(x, n).copy()
    b = _vec(b, n)
    lp, lc, lv = _csr(S.L)
    sp, sc, sv = _csr(S.Us)
    dr = np.ascontiguousarray(S.dr, np.float64)
    dc = np.ascontiguousarray(S.dc, np.float64)
    st = _load().orc_smooth_rowcol(n, b.shape[1], _p(ap), _p(ac), _p(av), _p(lp), _p(lc), _p(lv), _p(sp),
                                   _p(sc), _p(sv), _p(dr), _p(dc), _p(x), _p(b), int(mL), int(mU))
    if st:
        raise OracleError(st, "smooth_rowcol")
    return x


def power_norms(T, pmax: int, iters: int, v0) -> np.ndarray:
    """Power-iteration estimates of ||T^p||_2 for p = 1..pmax from start vector v0 (Sec. 5.2, Fig. Up)."""
    tp, tc, tv = _csr(T)
    n = len(tp) - 1
    v0 = np.ascontiguousarray(v0, np.float64).reshape(n)
    out = np.empty(max(pmax, 1), np.float64)
    st = _load().orc_power_norms(n, _p(tp), _p(tc), _p(tv), int(pmax), int(iters), _p(v0), _p(out))
    if st:
        raise OracleError(st, "power_norms")
    return out[:pmax]


@dataclass
class AMGLevel:
    """One level: A_l (CSR), and below the coarsest P_l (CSR, n_l x n_{l+1}) and the C/F marks."""
    n: int
    A: tuple
    P: tuple | None
    cf: np.ndarray | None


class AMG:
    """AMG hierarchy built by the oracle (Sec. 3).  levels[l] holds copies of A_l, P_l, cf."""

    def __init__(self, A, theta: float = 0.25, max_levels: int = 25, coarse_size: int = 400):
        ap, ac, av = _csr(A)
        n = len(ap) - 1
        st = ctypes.c_int(0)
        lib = _load()
        self._h = lib.orc_amg_setup(n, _p(ap), _p(ac), _p(av), float(theta), int(max_levels), int(coarse_size),
                                    ctypes.byref(st))
        if st.value:
            raise OracleError(st.value, "amg_setup")
        self.levels = []
        for l in range(lib.orc_amg_nlev(self._h)):
            nn, nz, nc, pz = (ctypes.c_int64() for _ in range(4))
            lib.orc_amg_level_sizes(self._h, l, ctypes.byref(nn), ctypes.byref(nz), ctypes.byref(nc),
                                    ctypes.byref(pz))
            m = nn.value
            lap = np.empty(m + 1, np.int64)
            lac = np.empty(max(nz.value, 1), np.int32)
            lav = np.empty(max(nz.value, 1), np.float64)
            if pz.value or nc.value:
                pp = np.empty(m + 1, np.int64)
                pc = np.empty(max(pz.value, 1), np.int32)
                pv = np.empty(max(pz.value, 1), np.float64)
                cf = np.empty(max(m, 1), np.int32)
                lib.orc_amg_level_copy(self._h, l, _p(lap), _p(lac), _p(lav), _p(pp), _p(pc), _p(pv), _p(cf))
                P = (pp, pc[:pz.value], pv[:pz.value])
                cf = cf[:m]
            else:
                lib.orc_amg_level_copy(self._h, l, _p(lap), _p(lac), _p(lav), None, None, None, None)
                P, cf = None, None
            self.levels.append(AMGLevel(m, (lap, lac[:nz.value], lav[:nz.value]), P, cf))

    def vcycle(self, S: Scaled, x, b, mL: int, mU: int, nu: int = 1, coarse: str = "jacobi", terms: int = 2):
        """One V-cycle (Alg. mgcycle) from x: ILU smoother (m_L + m_U sweeps on S) on the finest
        level, nu steps of l1-Jacobi (coarse="jacobi") or of polynomial Gauss-Seidel with `terms`
        terms (coarse="gs") below, direct solve on the coarsest.  Returns a new array."""
        n = self.levels[0].n
        x = np.ascontiguousarray(x, np.float64).reshape(n).copy()
        b = np.ascontiguousarray(b, np.float64).reshape(n)
        lp, lc, lv = _csr(S.L)
        sp, sc, sv = _csr(S.Us)
        st = _load().orc_amg_vcycle(self._h, _p(lp), _p(lc), _p(lv), _p(sp), _p(sc), _p(sv), _p(S.dinv), int(mL),
                                    int(mU), int(nu), 1 if coarse == "gs" else 0, int(terms), _p(x), _p(b))
        if st:
            raise OracleError(st, "amg_vcycle")
        return x

    def level_factors(self, kind: str = "ilu0", tau: float = 0.0, fill: int = 0, count: int | None = None):
        """Row-scaled incomplete factors of A_l for the first `count` levels (default: every level
        above the coarsest), for vcycle_ilu."""
        top = max(len(self.levels) - 1, 1)
        k = top if count is None else max(1, min(int(count), top))
        return [row_scale(factor(self.levels[l].A, kind, tau, fill)) for l in range(k)]

    def vcycle_ilu(self, factors, x, b, mL, mU, nu: int = 1, coarse: str = "jacobi", terms: int = 2,
                   schur=None):
        """One V-cycle as vcycle with the ILU smoother on the first len(factors) levels: level l
        is smoothed by m_L + m_U sweeps on factors[l] (the row-scaled factors of A_l; mL, mU an
        int or one count per level), the levels below by the coarse smoother.  schur = (parts,
        tau, fill[, iface_prec]) smooths the finest level by the ILUT Schur complement smoother
        instead (factors[0] is then not read).  Returns a new array."""
        k = len(factors)
        n = self.levels[0].n
        x = np.ascontiguousarray(x, np.float64).reshape(n).copy()
        b = np.ascontiguousarray(b, np.float64).reshape(n)
        mLs = np.ascontiguousarray(np.broadcast_to(np.asarray(mL, np.int32), (k,)), np.int32)
        mUs = np.ascontiguousarray(np.broadcast_to(np.asarray(mU, np.int32), (k,)), np.int32)
        keep = []

        def ptrs(arrays):
            arrs = [np.ascontiguousarray(a) for a in arrays]
            keep.extend(arrs)
            return (ctypes.c_void_p * k)(*[a.ctypes.data for a in arrs])

        Ls = [_csr(S.L) for S in factors]
        Us = [_csr(S.Us) for S in factors]
        st = _load().orc_amg_vcycle_ilu(self._h, k, ptrs([t[0] for t in Ls]), ptrs([t[1] for t in Ls]),
                                        ptrs([t[2] for t in Ls]), ptrs([t[0] for t in Us]), ptrs([t[1] for t in Us]),
                                        ptrs([t[2] for t in Us]), ptrs([S.dinv for S in factors]), _p(mLs), _p(mUs),
                                        int(nu), 1 if coarse == "gs" else 0, int(terms),
                                        int(schur[0]) if schur else 0, float(schur[1]) if schur else 0.0,
                                        int(schur[2]) if schur else 0,
                                        int(schur[3]) if schur and len(schur) > 3 else 0, _p(x), _p(b))
        if st:
            raise OracleError(st, "amg_vcycle_ilu")
        return x

    def vcycle_schur(self, x, b, parts: int, tau: float, fill: int, mL: int, mU: int, nu: int = 1,
                     coarse: str = "jacobi", terms: int = 2, iface_prec: int = 0):
        """One V-cycle as vcycle, the finest level smoothed (before and after the coarse-grid
        correction) by one application of the ILUT Schur complement smoother (schur_apply over
        `parts` row blocks, iface_prec as there) instead of the ILU smoother.  Returns a new array."""
        n = self.levels[0].n
        x = np.ascontiguousarray(x, np.float64).reshape(n).copy()
        b = np.ascontiguousarray(b, np.float64).reshape(n)
        st = _load().orc_amg_vcycle_schur(self._h, int(parts), float(tau), int(fill), int(iface_prec), int(mL),
                                          int(mU), int(nu), 1 if coarse == "gs" else 0, int(terms), _p(x), _p(b))
        if st:
            raise OracleError(st, "amg_vcycle_schur")
        return x

    def __del__(self):
        try:
            if self._h:
                _load().orc_amg_free(self._h)
                self._h = None
        except Exception:
            pass


def schur_interface(A, parts: int):
    """Interface rows (1) of a parts-way contiguous block-row partition; returns (count, marks)."""
    ap, ac, _ = _csr(A)
    n = len(ap) - 1
    marks = np.empty(max(n, 1), np.int32)
    k = _load().orc_schur_interface(n, _p(ap), _p(ac), int(parts), _p(marks))
    return int(k), marks[:n]


def schur_apply(A, r, parts: int, tau: float, fill: int, mL: int, mU: int, iface_prec: int = 0):
    """z = M^{-1} r of the ILUT Schur complement smoother (Sec. 3.1, Eq. schur), one right-hand side;
    iface_prec = 1 right-preconditions the interface GMRES iteration by diag(C) (not in the paper)."""
    ap, ac, av = _csr(A)
    n = len(ap) - 1
    r = np.ascontiguousarray(r, np.float64).reshape(n)
    z = np.empty(max(n, 1), np.float64)
    st = _load().orc_schur_apply_prec(n, _p(ap), _p(ac), _p(av), int(parts), float(tau), int(fill), int(mL),
                                      int(mU), int(iface_prec), _p(r), _p(z))
    if st:
        raise OracleError(st, "schur_apply")
    return z[:n]
