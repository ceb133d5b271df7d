"""Pins of the oracle's polynomial Gauss-Seidel smoother (Sec. 3.1: the
Gauss-Seidel splitting M = D + L, (D + L)^{-1} = (I + D^{-1} L)^{-1} D^{-1},
the inverse replaced by a truncated Neumann series).  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth
from _helpers import csr_from_dense, dense, relerr


def scipy_csr(A):
    rp, ci, va = A
    n = len(rp) - 1
    return sp.csr_matrix((va, ci, rp), shape=(n, n))


def gs_sweep_textbook(M, x, b, backward=False):
    """One classical Gauss-Seidel sweep, row by row, newest values used."""
    n = M.shape[0]
    x = x.copy()
    order = range(n - 1, -1, -1) if backward else range(n)
    for i in order:
        s = b[i] - sum(M[i, j] * x[j] for j in range(n) if j != i)
        x[i] = s / M[i, i]
    return x


def lower_levels(A):
    """Longest dependency chain of the strictly lower part (brute force)."""
    M = dense(A)
    n = M.shape[0]
    lev = [0] * n
    for i in range(n):
        lev[i] = max([lev[j] + 1 for j in range(i) if M[i, j] != 0.0], default=0)
    return max(lev) + 1 if n else 0


def test_p0_is_jacobi():
    """With p = 0 only the j = 0 term D^{-1} r remains (Jacobi, Eq. compact)."""
    A = synth.cutcell7(5, 4, 3, seed=2)
    n = len(A[0]) - 1
    r = synth.rhs(n, 2, seed=3)
    d = np.diag(dense(A))
    z = oracle.poly_gs_lower(A, r, 0)
    assert np.array_equal(z, r / d[:, None])


def test_terms_are_dense_matrix_powers():
    """z = sum_{j<=p} (-D^{-1} L)^j D^{-1} r by explicit dense powers, and the
    backward half sum_{j<=q} (-D^{-1} U)^j z likewise."""
    A = synth.hex27(4, 3, 3, seed=5)
    n = len(A[0]) - 1
    M = dense(A)
    D = np.diag(np.diag(M))
    Dinv = np.diag(1.0 / np.diag(M))
    L = np.tril(M, -1)
    U = np.triu(M, 1)
    r = synth.rhs(n, 3, seed=7)
    for p in (1, 2, 4, 7):
        want = sum(np.linalg.matrix_power(-Dinv @ L, j) @ (Dinv @ r) for j in range(p + 1))
        assert relerr(oracle.poly_gs_lower(A, r, p), want) < 1e-13
        wantu = sum(np.linalg.matrix_power(-Dinv @ U, j) @ want for j in range(p + 1))
        assert relerr(oracle.poly_gs_upper_unit(A, want, p), wantu) < 1e-13
    del D


def test_enough_terms_give_the_exact_forward_solve():
    """(-D^{-1} L) is nilpotent: with p + 1 >= #levels of L the series is
    (D + L)^{-1} r exactly (up to rounding), checked against scipy."""
    A = synth.cutcell7(6, 5, 4, seed=3)
    n = len(A[0]) - 1
    nlev = lower_levels(A)
    assert nlev == 6 + 5 + 4 - 2
    r = synth.rhs(n, 2, seed=4)
    S = scipy_csr(A)
    DL = sp.tril(S, 0, format="csr")
    want = spla.spsolve_triangular(DL, r, lower=True)
    assert relerr(oracle.poly_gs_lower(A, r, nlev - 1), want) < 1e-13
    # a dense 8 x 8 matrix with O(1) off-diagonals: 8 levels, p = 7 is exact,
    # p = 6 misses the last term (a chain of 7 products, far above rounding)
    rng = np.random.default_rng(11)
    Md = rng.uniform(-1.0, 1.0, (8, 8))
    np.fill_diagonal(Md, rng.uniform(0.5, 1.5, 8))
    B = csr_from_dense(Md)
    rb = rng.uniform(-1.0, 1.0, (8, 1))
    wantb = np.linalg.solve(np.tril(Md), rb)
    assert relerr(oracle.poly_gs_lower(B, rb, 7), wantb) < 1e-12
    assert relerr(oracle.poly_gs_lower(B, rb, 6), wantb) > 1e-6


@pytest.mark.parametrize("gen", ["poisson", "cutcell", "hex27"])
def test_smoother_equals_textbook_gauss_seidel(gen):
    """x + (D + L)^{-1}(b - A x) with all terms is one classical forward
    Gauss-Seidel sweep; the symmetric form with both halves is a forward
    sweep followed by a backward sweep (M = (D + L) D^{-1} (D + U))."""
    A = {"poisson": lambda: synth.poisson7(4, 3, 3),
         "cutcell": lambda: synth.cutcell7(4, 3, 3, seed=6),
         "hex27": lambda: synth.hex27(3, 3, 3, seed=2)}[gen]()
    n = len(A[0]) - 1
    M = dense(A)
    b = synth.rhs(n, 1, seed=8)[:, 0]
    x0 = synth.rhs(n, 1, seed=9)[:, 0]
    x1 = oracle.poly_gs_smooth(A, x0, b, n, 0, symmetric=False)[:, 0]
    assert relerr(x1, gs_sweep_textbook(M, x0, b)) < 1e-12
    x2 = oracle.poly_gs_smooth(A, x0, b, n, n, symmetric=True)[:, 0]
    want = gs_sweep_textbook(M, gs_sweep_textbook(M, x0, b), b, backward=True)
    assert relerr(x2, want) < 1e-12


def test_truncated_smoother_converges_on_poisson():
    """Repeated truncated polynomial GS on the diagonally dominant Poisson
    matrix reduces the residual monotonically (||D^{-1} L||_inf = 1/2 there)."""
    A = synth.poisson7(6, 5, 4)
    n = len(A[0]) - 1
    b = synth.rhs(n, 1, seed=1)[:, 0]
    x = np.zeros(n)
    prev = np.linalg.norm(b)
    for _ in range(6):
        x = oracle.poly_gs_smooth(A, x, b, 2, 0)[:, 0]
        res = np.linalg.norm(b - scipy_csr(A) @ x)
        assert res < prev
        prev = res


def test_zero_diagonal_is_reported():
    M = np.array([[4.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 4.0]])
    A = csr_from_dense(M)
    with pytest.raises(oracle.OracleError) as e:
        oracle.poly_gs_lower(A, np.ones(3), 2)
    assert e.value.status == oracle.ZERO_PIVOT
