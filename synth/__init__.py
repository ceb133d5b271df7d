"""Seeded synthetic inputs for the scaled-ILU smoother: matrices and vectors.

This module holds none of the smoother's arithmetic.  It builds the CSR
matrices A (pressure-Poisson operators standing in for the paper's PeleLM and
Nalu-Wind matrices, Sec. 1 and Sec. 6) and the right-hand sides b that the CUDA
library, the CPU oracle, the tests and the benchmark all consume.  The C side
(synth.c) uses a counter-based generator, so every value is reproducible from
(seed, stream, index) on any host.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_SO = os.path.join(_HERE, "libsynth.so")

POISSON7 = 0
CUTCELL7 = 1
HEX27 = 2

_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (skipped when up to date)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                   check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    i64, i32, u64, dbl, vp = (ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                              ctypes.c_double, ctypes.c_void_p)
    lib.synth_nnz.restype = i64
    lib.synth_nnz.argtypes = [i32, i32, i32, i32]
    lib.synth_fill.restype = i32
    lib.synth_fill.argtypes = [i32, i32, i32, i32, u64, dbl, dbl, vp, vp, vp]
    lib.synth_hex27_nodes.restype = i32
    lib.synth_hex27_nodes.argtypes = [i32, i32, i32, u64, dbl, vp, vp]
    lib.synth_rowptr27.restype = i32
    lib.synth_rowptr27.argtypes = [i32, i32, i32, vp]
    lib.synth_fill27_range.restype = i32
    lib.synth_fill27_range.argtypes = [i32, i32, i32, vp, vp, i64, i64, vp, vp, vp]
    lib.synth_rowptr7.restype = i32
    lib.synth_rowptr7.argtypes = [i32, i32, i32, vp]
    lib.synth_fill7_range.restype = i32
    lib.synth_fill7_range.argtypes = [i32, i32, i32, i32, u64, dbl, dbl, i64, i64, vp, vp, vp]
    lib.synth_uniform.restype = None
    lib.synth_uniform.argtypes = [u64, u64, i64, dbl, dbl, vp]
    lib.synth_randint.restype = None
    lib.synth_randint.argtypes = [u64, u64, i64, i32, i32, vp]
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def matrix(kind: int, nx: int, ny: int, nz: int, seed: int = 0, sigma: float = 0.0,
           frac_cut: float = 0.0, threads: int | None = None):
    """CSR (row_ptr int64[n+1], col int32[nnz], val float64[nnz]) of `kind`.

    Columns are sorted within each row and the diagonal is always stored.
    """
    lib = _load()
    n = nx * ny * nz
    nnz = lib.synth_nnz(kind, nx, ny, nz)
    if nnz < 0 or n >= 2**31 - 1:
        raise ValueError("bad grid")
    rp = np.empty(n + 1, dtype=np.int64)
    ci = np.empty(nnz, dtype=np.int32)
    va = np.empty(nnz, dtype=np.float64)
    if kind == HEX27 and n > 200_000:
        ne = (nx + 2) * (ny + 2) * (nz + 2)
        xyz = np.empty(3 * ne, dtype=np.float64)
        coef = np.empty(ne, dtype=np.float64)
        if lib.synth_hex27_nodes(nx, ny, nz, seed, sigma, _ptr(xyz), _ptr(coef)):
            raise RuntimeError("synth_hex27_nodes failed")
        lib.synth_rowptr27(nx, ny, nz, _ptr(rp))
        nt = threads or max(1, min(32, os.cpu_count() or 1))
        bounds = np.linspace(0, n, nt + 1).astype(np.int64)

        def work(t):
            return lib.synth_fill27_range(nx, ny, nz, _ptr(xyz), _ptr(coef), int(bounds[t]),
                                          int(bounds[t + 1]), _ptr(rp), _ptr(ci), _ptr(va))

        with ThreadPoolExecutor(nt) as ex:
            if any(ex.map(work, range(nt))):
                raise RuntimeError("synth_fill27_range failed")
    elif kind in (POISSON7, CUTCELL7) and n > 200_000:
        lib.synth_rowptr7(nx, ny, nz, _ptr(rp))
        nt = threads or max(1, min(32, os.cpu_count() or 1))
        bounds = np.linspace(0, n, nt + 1).astype(np.int64)

        def work7(t):
            return lib.synth_fill7_range(kind, nx, ny, nz, seed, sigma, frac_cut, int(bounds[t]),
                                         int(bounds[t + 1]), _ptr(rp), _ptr(ci), _ptr(va))

        with ThreadPoolExecutor(nt) as ex:
            if any(ex.map(work7, range(nt))):
                raise RuntimeError("synth_fill7_range failed")
    else:
        rc = lib.synth_fill(kind, nx, ny, nz, seed, sigma, frac_cut, _ptr(rp), _ptr(ci), _ptr(va))
        if rc:
            raise RuntimeError(f"synth_fill failed ({rc})")
    return rp, ci, va


def poisson7(nx: int, ny: int | None = None, nz: int | None = None):
    """7-point constant-coefficient Poisson (diagonal 6, neighbours -1), Dirichlet."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return matrix(POISSON7, nx, ny, nz)


def cutcell7(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 1,
             sigma: float = 2.0, frac_cut: float = 0.1):
    """Cut-cell-like variable-coefficient 7-point pressure Poisson operator."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return matrix(CUTCELL7, nx, ny, nz, seed=seed, sigma=sigma, frac_cut=frac_cut)


def hex27(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 2,
          sigma: float = 1.5, threads: int | None = None):
    """27-point weighted graph Laplacian on a randomly perturbed hex lattice."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return matrix(HEX27, nx, ny, nz, seed=seed, sigma=sigma, threads=threads)


def uniform(seed: int, stream: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """`count` doubles uniform on [lo, hi) from the counter-based generator."""
    lib = _load()
    out = np.empty(count, dtype=np.float64)
    lib.synth_uniform(seed, stream, count, lo, hi, _ptr(out))
    return out


def randint(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """`count` int32 uniform on [lo, hi] from the counter-based generator."""
    lib = _load()
    out = np.empty(count, dtype=np.int32)
    lib.synth_randint(seed, stream, count, lo, hi, _ptr(out))
    return out


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Right-hand sides uniform on [-1, 1), shape (n, nrhs), RHS interleaved (row-major)."""
    return uniform(seed, 0, n * nrhs).reshape(n, nrhs)


def banded(n: int, max_lower: int, bandwidth: int, seed: int, long_rows: dict | None = None, min_lower: int = 0):
    """A structurally symmetric, strictly diagonally dominant CSR matrix with
    uneven rows, for edge cases of the row tiles: row i couples to a seeded
    random set of c_i earlier rows within `bandwidth` (c_i uniform on
    [min_lower, max_lower], or long_rows[i] for the rows listed there), and every
    coupling is mirrored, so the ILU(0) factors have exactly these patterns
    (a row listed in long_rows may reach back to row 0: long_rows={n-1: n-1}
    gives a dense last row and column)
    (L_s row i: c_i entries; some rows end up with a diagonal only).
    Off-diagonal values are -U(0.1, 1); the diagonal is 1 + the row's
    absolute off-diagonal sum.  Returns (row_ptr int64, col int32, val)."""
    long_rows = long_rows or {}
    counts = randint(seed, 1, n, min_lower, max_lower)
    lower = []
    for i in range(n):
        c = int(long_rows.get(i, counts[i]))
        width = i if i in long_rows else min(i, bandwidth)
        c = min(c, width)
        if c == 0:
            lower.append(np.zeros(0, dtype=np.int64))
            continue
        # c distinct offsets in [1, width], chosen by a seeded partial shuffle
        keys = uniform(seed, 2 + i, width, 0.0, 1.0)
        offs = np.argsort(keys, kind="stable")[:c] + 1
        lower.append(np.sort(i - offs))
    rows = [[] for _ in range(n)]
    for i in range(n):
        for j in lower[i]:
            rows[i].append(int(j))
            rows[int(j)].append(i)
    rp = np.zeros(n + 1, dtype=np.int64)
    ci_parts, va_parts = [], []
    for i in range(n):
        off = np.array(sorted(rows[i]), dtype=np.int64)
        vals = -uniform(seed, 3_000_000 + i, off.size, 0.1, 1.0)
        cols = np.concatenate([off[off < i], [i], off[off > i]]).astype(np.int32)
        d = 1.0 + np.abs(vals).sum()
        k = int((off < i).sum())
        ci_parts.append(cols)
        va_parts.append(np.concatenate([vals[:k], [d], vals[k:]]))
        rp[i + 1] = rp[i] + cols.size
    return rp, np.concatenate(ci_parts), np.concatenate(va_parts)
