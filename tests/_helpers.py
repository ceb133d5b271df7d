"""Small dense brute-force utilities for the tests (independent of the oracle)."""
import numpy as np


def dense(A, n=None):
    rp, ci, va = A
    n = len(rp) - 1 if n is None else n
    M = np.zeros((n, n))
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            M[i, ci[p]] += va[p]
    return M


def dense_unit_lower(L):
    n = len(L[0]) - 1
    return np.eye(n) + dense(L, n)


def dense_unit_upper(Us):
    n = len(Us[0]) - 1
    return np.eye(n) + dense(Us, n)


def doolittle(M):
    """Textbook dense LU without pivoting: M = L U, L unit lower."""
    n = M.shape[0]
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            U[i, j] = M[i, j] - L[i, :i] @ U[:i, j]
        for j in range(i + 1, n):
            L[j, i] = (M[j, i] - L[j, :i] @ U[:i, i]) / U[i, i]
    return L, U


def grid_index(i, j, k, nx, ny):
    return (k * ny + j) * nx + i


def csr_from_dense(M, tol=0.0):
    n = M.shape[0]
    rp = [0]
    ci, va = [], []
    for i in range(n):
        for j in range(n):
            if abs(M[i, j]) > tol or i == j:
                ci.append(j)
                va.append(M[i, j])
        rp.append(len(ci))
    return (np.array(rp, np.int64), np.array(ci, np.int32), np.array(va, np.float64))


def relerr(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def maxabs_err(a, b):
    """max_i |a_i - b_i| / max_i |b_i|: a wrong value in a few rows of a long
    vector, which the 2-norm ratio can hide, shows here."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.max(np.abs(b)) if b.size else 0.0
    return float(np.max(np.abs(a - b))) / (nb if nb > 0 else 1.0) if b.size else 0.0
