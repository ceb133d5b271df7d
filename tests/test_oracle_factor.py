"""Pins of the oracle's factorisations and row scaling (CPU only).

Each test ties the oracle to something other than itself: a textbook dense LU,
the defining property of ILU(0), a closed-form pivot recurrence, a brute-force
level-of-fill computation, a hand-worked ILUT example (tests/golden/), the
eigenvalue definition of the departure from normality, or a library routine.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from _helpers import dense, dense_unit_lower, dense_unit_upper, doolittle, grid_index, csr_from_dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lu_dense(F):
    n = F.n
    return dense_unit_lower(F.L), dense(F.U, n)


# ---------------------------------------------------------------- ILU(0)

def test_ilu0_tridiagonal_is_exact_lu():
    """ILU(0) of a tridiagonal matrix has no fill to drop, so it is the exact LU."""
    A = synth.poisson7(17, 1, 1)          # tridiagonal: 6 on the diagonal, -1 off
    M = dense(A)
    L, U = lu_dense(oracle.ilu0(A))
    Lr, Ur = doolittle(M)
    assert np.max(np.abs(L - Lr)) < 1e-15
    assert np.max(np.abs(U - Ur)) < 1e-14
    # scipy's partial pivoting swaps nothing on this diagonally dominant matrix
    P, Ls, Us = scipy.linalg.lu(M)
    assert np.array_equal(P, np.eye(17))
    assert np.max(np.abs(L - Ls)) < 1e-15 and np.max(np.abs(U - Us)) < 1e-14


@pytest.mark.parametrize("gen", ["cutcell", "hex27", "poisson"])
def test_ilu0_matches_a_on_its_pattern(gen):
    """Defining property of ILU(0): (LU)_ij = a_ij for every (i, j) in pattern(A)."""
    if gen == "cutcell":
        A = synth.cutcell7(4, 3, 5, seed=11)
    elif gen == "hex27":
        A = synth.hex27(4, 3, 3, seed=12)
    else:
        A = synth.poisson7(5, 4, 3)
    F = oracle.ilu0(A)
    L, U = lu_dense(F)
    M = dense(A)
    LU = L @ U
    absprod = np.abs(L) @ np.abs(U)
    rp, ci, _ = A
    for i in range(len(rp) - 1):
        for p in range(rp[i], rp[i + 1]):
            j = ci[p]
            assert abs(LU[i, j] - M[i, j]) <= 1e-14 * absprod[i, j]
    # the factors have exactly the pattern of A
    assert np.array_equal((L - np.eye(len(M)) != 0) | (U != 0), M != 0)


def test_ilu0_poisson7_pivot_recurrence_and_fixed_point():
    """7-point constant coefficients: u_ii = 6 - sum over lower neighbours k of 1/u_kk.

    Deep-interior pivots approach the fixed point d = 6 - 3/d, d = 3 + sqrt(6).
    """
    nx = ny = nz = 14
    A = synth.poisson7(nx, ny, nz)
    F = oracle.ilu0(A)
    up, uc, uv = F.U
    piv = uv[up[:-1]]
    assert np.all(uc[up[:-1]] == np.arange(nx * ny * nz))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = grid_index(i, j, k, nx, ny)
                s = 6.0
                if i > 0:
                    s -= 1.0 / piv[r - 1]
                if j > 0:
                    s -= 1.0 / piv[r - nx]
                if k > 0:
                    s -= 1.0 / piv[r - nx * ny]
                assert abs(piv[r] - s) <= 1e-15 * s
    d = 3.0 + math.sqrt(6.0)
    assert abs(piv[-1] - d) < 1e-6
    assert np.all(piv >= d - 1e-12)


# ---------------------------------------------------------------- ILU(k)

def brute_level_of_fill(M, K):
    """Level of fill by the KIJ form on a dense boolean pattern (brute force)."""
    n = M.shape[0]
    INF = 10 ** 9
    lev = np.where(M != 0, 0, INF).astype(np.int64)
    for k in range(n):
        rows = np.nonzero(lev[k + 1:, k] <= K)[0] + k + 1
        cols = np.nonzero(lev[k, k + 1:] <= K)[0] + k + 1
        if len(rows) == 0 or len(cols) == 0:
            continue
        cand = lev[rows, k][:, None] + lev[k, cols][None, :] + 1
        sub = lev[np.ix_(rows, cols)]
        lev[np.ix_(rows, cols)] = np.minimum(sub, cand)
    return lev


@pytest.mark.parametrize("K", [0, 1, 2, 3])
@pytest.mark.parametrize("grid", [(5, 4, 1), (3, 3, 3), (4, 3, 2)])
def test_iluk_pattern_matches_brute_force(K, grid):
    A = synth.cutcell7(*grid, seed=5)
    M = dense(A)
    lev = brute_level_of_fill(M, K)
    pp, pc, pl = oracle.iluk_pattern(A, K)
    n = M.shape[0]
    got = np.full((n, n), -1)
    for i in range(n):
        for p in range(pp[i], pp[i + 1]):
            got[i, pc[p]] = pl[p]
    want = np.where(lev <= K, lev, -1)
    assert np.array_equal(got, want)


def test_iluk_27pt_pattern_matches_brute_force():
    A = synth.hex27(3, 3, 3, seed=3)
    M = dense(A)
    for K in (1, 2):
        lev = brute_level_of_fill(M, K)
        pp, pc, pl = oracle.iluk_pattern(A, K)
        n = M.shape[0]
        got = np.full((n, n), -1)
        for i in range(n):
            got[i, pc[pp[i]:pp[i + 1]]] = pl[pp[i]:pp[i + 1]]
        assert np.array_equal(got, np.where(lev <= K, lev, -1))


def test_iluk_5pt_level1_adds_the_known_diagonals():
    """ILU(1) of the 5-point 2-D Laplacian (natural order) fills exactly the
    diagonals at offsets +-(nx - 1) inside the grid."""
    nx, ny = 6, 5
    A = synth.poisson7(nx, ny, 1)
    pp, pc, pl = oracle.iluk_pattern(A, 1)
    M = dense(A)
    n = nx * ny
    fill = set()
    for i in range(n):
        for p in range(pp[i], pp[i + 1]):
            if M[i, pc[p]] == 0:
                assert pl[p] == 1
                fill.add((i, int(pc[p])))
    want = set()
    for j in range(ny):
        for i in range(nx):
            r = grid_index(i, j, 0, nx, ny)
            if j > 0 and i < nx - 1:
                want.add((r, r - nx + 1))     # lower: (i+1, j-1)
            if j < ny - 1 and i > 0:
                want.add((r, r + nx - 1))     # upper: (i-1, j+1)
    assert fill == want


def test_iluk_full_fill_is_exact_lu():
    A = synth.cutcell7(3, 3, 2, seed=8)
    M = dense(A)
    n = M.shape[0]
    L, U = lu_dense(oracle.iluk(A, n))
    Lr, Ur = doolittle(M)
    assert np.max(np.abs(L - Lr)) < 1e-13
    assert np.max(np.abs(U - Ur)) < 1e-13 * np.max(np.abs(Ur))
    # ILU(0) through the ILU(k) path equals the direct ILU(0)
    F0, Fk = oracle.ilu0(A), oracle.iluk(A, 0)
    for a, b in zip(F0.L + F0.U, Fk.L + Fk.U):
        assert np.array_equal(a, b)


# ---------------------------------------------------------------- ILUT

def test_ilut_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "ilut_hand_3x3.json")))
    A = (np.array(g["A"]["row_ptr"]), np.array(g["A"]["col"]), np.array(g["A"]["val"]))
    for case in g["cases"]:
        F = oracle.ilut(A, g["tau"], case["p"])
        for part, got in (("L", F.L), ("U", F.U)):
            want = case[part]
            assert np.array_equal(got[0], want["row_ptr"]), part
            assert np.array_equal(got[1], want["col"]), part
            assert np.allclose(got[2], want["val"], rtol=1e-15, atol=0), part


def test_ilut_no_drop_is_exact_lu():
    A = synth.hex27(3, 3, 2, seed=4)
    M = dense(A)
    n = M.shape[0]
    L, U = lu_dense(oracle.ilut(A, 0.0, n))
    Lr, Ur = doolittle(M)
    assert np.max(np.abs(L - Lr)) < 1e-13
    assert np.max(np.abs(U - Ur)) < 1e-13 * np.max(np.abs(Ur))


def test_ilut_infinite_threshold_keeps_the_diagonal_only():
    """tau = inf drops everything off the diagonal: U = diag(A), L = I, so
    Utilde_s = 0 and dep(Utilde) = 0 (Eq. diagDep)."""
    A = synth.cutcell7(5, 4, 3, seed=2)
    F = oracle.ilut(A, np.inf, 10)
    assert len(F.L[1]) == 0
    M = dense(A)
    assert np.array_equal(dense(F.U, F.n), np.diag(np.diag(M)))
    S = oracle.row_scale(F)
    assert len(S.Us[1]) == 0
    assert oracle.dep_triangular(S.Us, unit_diag=True) == 0.0


def test_ilut_invariants_on_cut_cell_matrix():
    """Stored off-diagonals pass the threshold, each part holds at most p
    entries per row, the diagonal is always present."""
    A = synth.cutcell7(10, 9, 8, seed=21)
    tau, p = 1e-3, 4
    F = oracle.ilut(A, tau, p)
    rp, ci, va = A
    n = len(rp) - 1
    lp, lc, lv = F.L
    up, uc, uv = F.U
    for i in range(n):
        tau_i = tau * math.sqrt(np.sum(va[rp[i]:rp[i + 1]] ** 2))
        assert lp[i + 1] - lp[i] <= p
        assert up[i + 1] - up[i] <= p + 1
        assert uc[up[i]] == i
        assert np.all(np.abs(lv[lp[i]:lp[i + 1]]) >= tau_i)
        assert np.all(np.abs(uv[up[i] + 1:up[i + 1]]) >= tau_i)
        assert np.all(lc[lp[i]:lp[i + 1]] < i) and np.all(uc[up[i] + 1:up[i + 1]] > i)
        assert np.all(np.diff(lc[lp[i]:lp[i + 1]]) > 0) and np.all(np.diff(uc[up[i]:up[i + 1]]) > 0)
    # ILUT with a generous fill limit approximates A better than ILU(0)
    M = dense(A)
    F0 = oracle.ilu0(A)
    Ft = oracle.ilut(A, 1e-4, 30)
    e0 = np.linalg.norm(dense_unit_lower(F0.L) @ dense(F0.U, n) - M)
    et = np.linalg.norm(dense_unit_lower(Ft.L) @ dense(Ft.U, n) - M)
    assert et < e0


def test_zero_pivot_is_reported():
    M = np.array([[0.0, 1.0], [1.0, 2.0]])
    A = csr_from_dense(M)
    for f in (oracle.ilu0, lambda a: oracle.ilut(a, 0.0, 2), lambda a: oracle.iluk(a, 1)):
        with pytest.raises(oracle.OracleError) as e:
            f(A)
        assert e.value.status == oracle.ZERO_PIVOT


# ---------------------------------------------------------------- scaling, dep

def test_row_scaling_is_d_inverse_u():
    """Utilde = D^{-1} U with D = diag(U) (Eq. extractD, Eq. newD) has a unit
    diagonal, and for symmetric A under ILU(0) it equals L^T."""
    for A in (synth.cutcell7(5, 4, 3, seed=9), synth.hex27(4, 3, 3, seed=1)):
        F = oracle.ilu0(A)
        S = oracle.row_scale(F)
        n = F.n
        U = dense(F.U, n)
        d = np.diag(U)
        assert np.array_equal(S.dinv, 1.0 / d)
        Ut = dense_unit_upper(S.Us)
        assert np.max(np.abs(Ut - U / d[:, None])) <= 1e-15 * np.max(np.abs(U / d[:, None]))
        L = dense_unit_lower(F.L)
        assert np.max(np.abs(Ut - L.T)) < 1e-14
        # Table dep: dep(L) equals dep(D^{-1} U) for every matrix listed
        dl = oracle.dep_triangular(F.L, unit_diag=True)
        du = oracle.dep_triangular(S.Us, unit_diag=True)
        assert abs(dl - du) <= 1e-13 * dl


def test_dep_matches_eigenvalue_definition():
    """dep(T) = sqrt(||T||_F^2 - ||Lambda||_F^2) with Lambda from an eigensolver."""
    rng = np.random.default_rng(7)
    for trial in range(5):
        n = 6
        T = np.triu(rng.standard_normal((n, n)))
        T[np.abs(T) < 0.3] = 0.0
        np.fill_diagonal(T, rng.uniform(1, 3, n))
        lam = np.linalg.eigvals(T)
        want = math.sqrt(max(np.linalg.norm(T, "fro") ** 2 - np.sum(np.abs(lam) ** 2), 0.0))
        got = oracle.dep_triangular(csr_from_dense(T))
        assert abs(got - want) <= 1e-10 * max(want, 1.0)
        Ts = np.triu(T, 1)
        got_unit = oracle.dep_triangular(csr_from_dense(Ts), unit_diag=True)
        assert abs(got_unit - np.linalg.norm(Ts, "fro")) <= 1e-14 * np.linalg.norm(Ts, "fro")
        # unit-diagonal triangular: dep = sqrt(||I + T_s||_F^2 - n) (Eq. diagDep)
        assert abs(got_unit - math.sqrt(np.linalg.norm(np.eye(n) + Ts, "fro") ** 2 - n)) < 1e-12
