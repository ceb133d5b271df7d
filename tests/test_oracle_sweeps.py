"""Pins of the oracle's residual, Richardson sweeps, direct solves, level sets
and FGMRES (CPU only)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth
from _helpers import dense, dense_unit_lower, dense_unit_upper, grid_index, relerr


def scipy_csr(A):
    rp, ci, va = A
    n = len(rp) - 1
    return sp.csr_matrix((va, ci, rp), shape=(n, n))


def scaled(A, kind="ilu0", tau=0.0, fill=0):
    return oracle.row_scale(oracle.factor(A, kind, tau, fill))


# ---------------------------------------------------------------- residual

def test_residual_matches_scipy():
    A = synth.hex27(5, 4, 3, seed=3)
    n = len(A[0]) - 1
    x = synth.rhs(n, 3, seed=5)
    b = synth.rhs(n, 3, seed=6)
    r = oracle.residual(A, x, b)
    want = b - scipy_csr(A) @ x
    assert relerr(r, want) < 1e-15
    assert relerr(oracle.spmv(A, x), scipy_csr(A) @ x) < 1e-15


# ---------------------------------------------------------------- sweeps

@pytest.mark.parametrize("gen", ["poisson", "cutcell_ilut"])
def test_sweeps_are_neumann_partial_sums(gen):
    """y^m = sum_{j<m} (-L_s)^j r and v^m = sum_{j<m} (-U_s)^j D^{-1} y
    (Eq. Neumann), by explicit dense matrix powers."""
    if gen == "poisson":
        A = synth.poisson7(4, 3, 3)
        S = scaled(A)
    else:
        A = synth.cutcell7(4, 4, 3, seed=4)
        S = scaled(A, "ilut", 1e-3, 5)
    n = S.n
    Ls = dense(S.L, n)
    Us = dense(S.Us, n)
    r = synth.rhs(n, 2, seed=1)
    for m in (1, 2, 3, 5, 8):
        want_y = sum(np.linalg.matrix_power(-Ls, j) @ r for j in range(m))
        y = oracle.richardson_lower(S.L, r, m)
        assert relerr(y, want_y) < 1e-13
        c = S.dinv[:, None] * y
        want_v = sum(np.linalg.matrix_power(-Us, j) @ c for j in range(m))
        v = oracle.richardson_upper(S.Us, S.dinv, y, m)
        assert relerr(v, want_v) < 1e-13
    assert np.all(oracle.richardson_lower(S.L, r, 0) == 0)


def test_sweeps_are_exact_after_levels_and_after_n():
    """L_s is nilpotent (Sec. 5.2): after #levels sweeps, and so after n, the
    iterate equals forward substitution, which matches scipy's triangular solve."""
    A = synth.cutcell7(5, 4, 3, seed=3)
    S = scaled(A)
    n = S.n
    r = synth.rhs(n, 2, seed=2)
    y_star = oracle.forward_subst(S.L, r)
    Lsp = sp.csr_matrix(dense_unit_lower(S.L))
    assert relerr(y_star, spla.spsolve_triangular(Lsp, r, lower=True)) < 1e-14
    nlev, _ = oracle.levels_lower(S.L)
    assert nlev == 5 + 4 + 3 - 2
    for m in (nlev, n):
        assert relerr(oracle.richardson_lower(S.L, r, m), y_star) < 1e-14
    # one sweep short of the level count is not yet exact
    assert relerr(oracle.richardson_lower(S.L, r, nlev - 1), y_star) > 1e-8
    c = S.dinv[:, None] * y_star
    v_star = oracle.backward_subst_unit(S.Us, c)
    Usp = sp.csr_matrix(dense_unit_upper(S.Us))
    assert relerr(v_star, spla.spsolve_triangular(Usp, c, lower=False)) < 1e-14
    nlu, _ = oracle.levels_upper(S.Us)
    for m in (nlu, n):
        assert relerr(oracle.richardson_upper(S.Us, S.dinv, y_star, m), v_star) < 1e-14


def test_poisson32_sweep_error_bound():
    """32^3 Poisson ILU(0): ||L_s||_inf = ||Utilde_s||_inf <= 3/(3+sqrt(6)) and the
    Richardson error obeys ||y^m - y*||_inf <= rho^m ||y*||_inf."""
    A = synth.poisson7(32)
    S = scaled(A)
    n = S.n
    bound = 3.0 / (3.0 + math.sqrt(6.0))
    lp, _, lv = S.L
    rowsum = np.add.reduceat(np.abs(lv), lp[:-1]) if len(lv) else np.zeros(n)
    rowsum[lp[:-1] == lp[1:]] = 0.0
    rho = rowsum.max()
    assert rho <= bound + 1e-12 and rho > bound - 1e-3
    r = synth.rhs(n, 4, seed=0)
    y_star = oracle.forward_subst(S.L, r)
    for m in (1, 3, 5):
        y = oracle.richardson_lower(S.L, r, m)
        assert np.max(np.abs(y - y_star)) <= rho ** m * np.max(np.abs(y_star)) * (1 + 1e-12)


def test_unscaled_variants():
    """Jacobi on raw U (Eq. LUiterMat) equals scaled Richardson up to rounding;
    plain Richardson on raw U diverges on the cut-cell matrix (Sec. 6.1)."""
    A = synth.cutcell7(8, 8, 8, seed=1)
    F = oracle.ilu0(A)
    S = oracle.row_scale(F)
    n = F.n
    y = synth.rhs(n, 1, seed=3)
    for m in (1, 4, 10):
        v = oracle.richardson_upper(S.Us, S.dinv, y, m)
        vj = oracle.upper_jacobi(F.U, y, m)
        assert relerr(vj, v) < 1e-12
    v1 = oracle.upper_unscaled_richardson(F.U, y, 1)
    assert np.array_equal(v1, y)
    grow = [np.linalg.norm(oracle.upper_unscaled_richardson(F.U, y, m)) for m in (2, 4, 8)]
    assert grow[2] > 1e3 * grow[0]


@pytest.mark.parametrize("gen", ["cutcell_ilu0", "cutcell_ilut", "hex27_ilu0"])
def test_unscaled_iterations_are_dense_partial_sums(gen):
    """Plain Richardson on the raw upper factor, v <- y - (U - I) v from
    v = 0, gives v^m = sum_{j<m} (I - U)^j y; Jacobi on raw U (Eq. LUiterMat,
    G_U = I - D_U^{-1} U) gives sum_{j<m} G_U^j D_U^{-1} y.  Both by explicit
    dense matrix powers of U with its true (non-unit) diagonal, so taking
    y - U v for the Richardson step, or dropping D_U^{-1}, fails here."""
    if gen == "cutcell_ilu0":
        A = synth.cutcell7(4, 4, 3, seed=4)
        F = oracle.factor(A, "ilu0", 0.0, 0)
    elif gen == "cutcell_ilut":
        A = synth.cutcell7(4, 3, 3, seed=5)
        F = oracle.factor(A, "ilut", 1e-3, 5)
    else:
        A = synth.hex27(3, 3, 3, seed=6)
        F = oracle.factor(A, "ilu0", 0.0, 0)
    n = F.n
    U = dense(F.U, n)
    assert np.max(np.abs(np.diag(U) - 1.0)) > 0.5  # a diagonal far from one
    I = np.eye(n)
    Dinv = np.diag(1.0 / np.diag(U))
    y = synth.rhs(n, 2, seed=1)
    for m in (1, 2, 3, 4, 5):
        want = sum(np.linalg.matrix_power(I - U, j) @ y for j in range(m))
        got = oracle.upper_unscaled_richardson(F.U, y, m)
        assert relerr(got, want) < 1e-13, m
        want_j = sum(np.linalg.matrix_power(I - Dinv @ U, j) @ (Dinv @ y) for j in range(m))
        assert relerr(oracle.upper_jacobi(F.U, y, m), want_j) < 1e-13, m
    assert np.all(oracle.upper_unscaled_richardson(F.U, y, 0) == 0)


def test_smooth_composes_the_sweeps():
    """x + M^{-1}(b - A x) (Eq. ILUsplit): residual, m_L lower sweeps, D^{-1},
    m_U upper sweeps, update; with enough sweeps it equals the direct solves,
    and the direct solves equal a dense solve with M = L D Utilde."""
    A = synth.cutcell7(6, 5, 4, seed=7)
    S = scaled(A, "ilut", 1e-3, 6)
    n = S.n
    x0 = synth.rhs(n, 2, seed=8)
    b = synth.rhs(n, 2, seed=9)
    got = oracle.smooth(A, S, x0, b, 3, 4)
    r = oracle.residual(A, x0, b)
    y = oracle.richardson_lower(S.L, r, 3)
    v = oracle.richardson_upper(S.Us, S.dinv, y, 4)
    assert np.array_equal(got, x0 + v)
    M = dense_unit_lower(S.L) @ np.diag(1.0 / S.dinv) @ dense_unit_upper(S.Us)
    want = x0 + np.linalg.solve(M, b - dense(A) @ x0)
    direct = oracle.direct_apply(A, S, x0, b)
    assert relerr(direct, want) < 1e-12
    nl, _ = oracle.levels_lower(S.L)
    nu, _ = oracle.levels_upper(S.Us)
    assert relerr(oracle.smooth(A, S, x0, b, nl, nu), direct) < 1e-13
    # zero sweeps skip a factor
    assert np.array_equal(oracle.smooth(A, S, x0, b, 0, 0), x0 + r)


# ---------------------------------------------------------------- level sets

def brute_longest_path_levels(T, lower=True):
    """Relax lev(i) = max(lev(i), lev(j) + 1) over all edges until nothing
    changes (Bellman-Ford style), independent of the row order."""
    tp, tc, _ = T
    n = len(tp) - 1
    rows = np.repeat(np.arange(n), np.diff(tp))
    lev = np.zeros(n, np.int64)
    for _ in range(n + 1):
        new = lev.copy()
        np.maximum.at(new, rows, lev[tc] + 1)
        if np.array_equal(new, lev):
            break
        lev = new
    return lev


def test_levels_7pt_closed_form():
    nx, ny, nz = 6, 5, 4
    S = scaled(synth.poisson7(nx, ny, nz))
    nl, lev = oracle.levels_lower(S.L)
    nu, levu = oracle.levels_upper(S.Us)
    assert nl == nu == nx + ny + nz - 2
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = grid_index(i, j, k, nx, ny)
                assert lev[r] == i + j + k
                assert levu[r] == (nx - 1 - i) + (ny - 1 - j) + (nz - 1 - k)
    assert np.array_equal(lev, brute_longest_path_levels(S.L))


def test_levels_27pt_closed_form():
    nx, ny, nz = 5, 4, 4
    S = scaled(synth.hex27(nx, ny, nz, seed=6))
    nl, lev = oracle.levels_lower(S.L)
    assert nl == (nx - 1) + 2 * (ny - 1) + 4 * (nz - 1) + 1
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                assert lev[grid_index(i, j, k, nx, ny)] == i + 2 * j + 4 * k
    assert np.array_equal(lev, brute_longest_path_levels(S.L))
    nu, levu = oracle.levels_upper(S.Us)
    assert nu == nl


def test_levels_ilut_brute_force():
    S = scaled(synth.cutcell7(6, 6, 5, seed=2), "ilut", 1e-3, 8)
    _, lev = oracle.levels_lower(S.L)
    assert np.array_equal(lev, brute_longest_path_levels(S.L))


# ---------------------------------------------------------------- FGMRES

def test_fgmres_unpreconditioned_full_restart_is_exact():
    # well conditioned (no cut cells): GMRES(n) is exact after at most n steps
    A = synth.cutcell7(3, 3, 3, seed=2, sigma=0.5, frac_cut=0.0)
    n = len(A[0]) - 1
    b = synth.rhs(n, 1, seed=4)[:, 0]
    x, st, its, rel = oracle.fgmres(A, None, b, tol=1e-13, restart=n, maxit=n, precond=2)
    assert st == oracle.OK and rel <= 1e-13 and its <= n
    assert relerr(x, np.linalg.solve(dense(A), b)) < 1e-10


def test_fgmres_with_exact_factors_converges_in_one_iteration():
    """With ILU(k >= n), M = A; both the direct and the converged-sweep
    preconditioners then solve the system in one FGMRES iteration."""
    A = synth.cutcell7(4, 3, 2, seed=3)
    n = len(A[0]) - 1
    S = scaled(A, "iluk", fill=n)
    b = synth.rhs(n, 1, seed=5)[:, 0]
    want = np.linalg.solve(dense(A), b)
    x, st, its, rel = oracle.fgmres(A, S, b, tol=1e-10, restart=10, precond=1)
    assert st == oracle.OK and its == 1 and relerr(x, want) < 1e-12
    x, st, its, rel = oracle.fgmres(A, S, b, tol=1e-10, restart=10, mL=n, mU=n, precond=0)
    assert st == oracle.OK and its == 1 and relerr(x, want) < 1e-12


def test_fgmres_smoothed_cut_cell_reaches_tolerance():
    A = synth.cutcell7(12, 12, 12, seed=1)
    n = len(A[0]) - 1
    S = scaled(A)
    b = synth.rhs(n, 1, seed=1)[:, 0]
    x, st, its, rel = oracle.fgmres(A, S, b, tol=1e-10, restart=30, maxit=500, mL=3, mU=3)
    assert st == oracle.OK and rel <= 1e-10
    true = np.linalg.norm(b - scipy_csr(A) @ x) / np.linalg.norm(b)
    assert abs(true - rel) <= 1e-3 * rel
    # a smaller restart still converges (restarts recompute the true residual)
    x5, st5, its5, rel5 = oracle.fgmres(A, S, b, tol=1e-10, restart=5, maxit=2000, mL=3, mU=3)
    assert st5 == oracle.OK and rel5 <= 1e-10 and its5 >= its
    # too few iterations: reported as not converged, best iterate returned
    _, st1, its1, rel1 = oracle.fgmres(A, S, b, tol=1e-10, restart=30, maxit=3, mL=3, mU=3)
    assert st1 == oracle.NOT_CONVERGED and its1 == 3 and rel1 > 1e-10


def test_norm2_and_nrbe():
    A = synth.cutcell7(5, 5, 4, seed=3, sigma=1.0)
    M = dense(A)
    nrm = oracle.norm2_est(A, iters=2000)
    assert abs(nrm - np.linalg.norm(M, 2)) <= 1e-6 * nrm
    n = M.shape[0]
    b = synth.rhs(n, 1, seed=2)[:, 0]
    x = synth.rhs(n, 1, seed=3)[:, 0]
    want = np.linalg.norm(b - M @ x) / (np.linalg.norm(b) + nrm * np.linalg.norm(x))
    assert abs(oracle.nrbe(A, x, b, nrm) - want) <= 1e-14 * want
