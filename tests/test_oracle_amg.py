"""Pins of the oracle's algebraic multigrid (Sec. 3: strength threshold,
Ruge-Stueben coarsening, Galerkin coarse operators A_{l+1} = P^T A_l P, and
the V-cycle of Alg. mgcycle with the ILU smoother on the finest level, or on
the first few levels).
CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
from _helpers import csr_from_dense, dense, relerr


def laplace1d(n):
    M = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return csr_from_dense(M)


def aniso2d(nx, ny, ay):
    """5-point operator with x couplings -1 and y couplings -ay (Dirichlet)."""
    n = nx * ny
    M = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            M[r, r] = 2.0 + 2.0 * ay
            if i > 0:
                M[r, r - 1] = -1.0
            if i < nx - 1:
                M[r, r + 1] = -1.0
            if j > 0:
                M[r, r - nx] = -ay
            if j < ny - 1:
                M[r, r + nx] = -ay
    return csr_from_dense(M)


def test_1d_laplacian_closed_forms():
    """tridiag(-1, 2, -1): the first pass takes every other point (the odd
    ones: equal measures, smallest index first), direct interpolation is
    linear interpolation (1/2, 1/2), and the Galerkin operator is
    tridiag(-1/2, 1, -1/2), all exact in binary."""
    n = 9
    H = oracle.AMG(laplace1d(n), theta=0.25, max_levels=2, coarse_size=1)
    L0 = H.levels[0]
    assert list(L0.cf) == [0, 1, 0, 1, 0, 1, 0, 1, 0]
    P = np.zeros((n, 4))
    pp, pc, pv = L0.P
    for i in range(n):
        for q in range(pp[i], pp[i + 1]):
            P[i, pc[q]] = pv[q]
    want = np.zeros((n, 4))
    for c in range(4):
        want[2 * c + 1, c] = 1.0
        want[2 * c, c] = 0.5
        want[2 * c + 2, c] = 0.5
    assert np.array_equal(P, want)
    Ac = dense(H.levels[1].A, 4)
    assert np.array_equal(Ac, np.eye(4) - 0.5 * np.eye(4, k=1) - 0.5 * np.eye(4, k=-1))


def test_strength_threshold_gives_semicoarsening():
    """Strong x couplings (-1) and weak y couplings (-0.01): with theta = 0.25
    only the x couplings are strong, so every x-line is coarsened like the 1-D
    Laplacian (odd i coarse); with theta = 0.005 every coupling is strong and
    the first pass gives the red-black coarsening of the 5-point stencil
    (C where i + j is even, starting from the corner of largest measure)."""
    nx, ny = 9, 5
    A = aniso2d(nx, ny, 0.01)
    cf = oracle.AMG(A, theta=0.25, max_levels=2, coarse_size=1).levels[0].cf.reshape(ny, nx)
    assert np.array_equal(cf, np.tile([0, 1, 0, 1, 0, 1, 0, 1, 0], (ny, 1)))
    cf2 = oracle.AMG(A, theta=0.005, max_levels=2, coarse_size=1).levels[0].cf.reshape(ny, nx)
    jj, ii = np.mgrid[0:ny, 0:nx]
    assert np.array_equal(cf2, ((ii + jj) % 2 == 0).astype(np.int32))


def strong(Arow_cols, Arow_vals, i, theta):
    off = [(j, abs(v)) for j, v in zip(Arow_cols, Arow_vals) if j != i]
    mx = max([a for _, a in off], default=0.0)
    return {j for j, a in off if mx > 0 and a >= theta * mx}


@pytest.mark.parametrize("gen", ["cutcell", "hex27"])
def test_split_and_interpolation_invariants(gen):
    """Every F point that some undecided-or-C point strongly influences has a
    strong C neighbour (first-pass property); P is the identity on C points;
    F rows interpolate only from strong C neighbours; rows of A with zero row
    sum and negative couplings interpolate constants exactly (sum w = 1)."""
    A = synth.cutcell7(7, 6, 5, seed=3) if gen == "cutcell" else synth.hex27(6, 5, 5, seed=4)
    n = len(A[0]) - 1
    H = oracle.AMG(A, theta=0.25, max_levels=2, coarse_size=1)
    L0 = H.levels[0]
    ap, ac, av = A
    pp, pc, pv = L0.P
    cidx = np.cumsum(L0.cf) - 1
    for i in range(n):
        cols, vals = ac[ap[i]:ap[i + 1]], av[ap[i]:ap[i + 1]]
        S = strong(cols, vals, i, 0.25)
        row = dict(zip(pc[pp[i]:pp[i + 1]], pv[pp[i]:pp[i + 1]]))
        if L0.cf[i]:
            assert row == {cidx[i]: 1.0}
            continue
        SC = {j for j in S if L0.cf[j]}
        assert set(row) == {cidx[j] for j in SC}
        if S and not SC:
            assert all(L0.cf[j] == 0 for j in S)
        rowsum = vals.sum()
        if SC and abs(rowsum) < 1e-12 * abs(vals).max() and np.all(vals[cols != i] <= 0):
            assert abs(sum(row.values()) - 1.0) < 1e-14


def test_galerkin_matches_dense_triple_product():
    A = synth.cutcell7(9, 8, 7, seed=5)
    H = oracle.AMG(A, theta=0.25, max_levels=6, coarse_size=10)
    assert len(H.levels) >= 3
    for l in range(len(H.levels) - 1):
        L, C = H.levels[l], H.levels[l + 1]
        Ad = dense(L.A, L.n)
        P = np.zeros((L.n, C.n))
        pp, pc, pv = L.P
        for i in range(L.n):
            for q in range(pp[i], pp[i + 1]):
                P[i, pc[q]] = pv[q]
        assert relerr(dense(C.A, C.n), P.T @ Ad @ P) < 1e-14


def scipy_csr(A):
    rp, ci, va = A
    n = len(rp) - 1
    return sp.csr_matrix((va, ci, rp), shape=(n, n))


def test_two_level_cycle_is_the_two_grid_operator():
    """A two-level V-cycle = pre-smoothing, exact coarse correction
    x + P A_c^{-1} P^T (b - A x), post-smoothing (Alg. mgcycle), with the
    coarse correction formed densely here."""
    A = synth.cutcell7(8, 7, 6, seed=6)
    n = len(A[0]) - 1
    S = oracle.row_scale(oracle.ilu0(A))
    H = oracle.AMG(A, theta=0.25, max_levels=2, coarse_size=1)
    assert len(H.levels) == 2
    L0, C = H.levels
    P = np.zeros((n, C.n))
    pp, pc, pv = L0.P
    for i in range(n):
        for q in range(pp[i], pp[i + 1]):
            P[i, pc[q]] = pv[q]
    Ad = dense(A, n)
    b = synth.rhs(n, 1, seed=2)[:, 0]
    x0 = synth.rhs(n, 1, seed=3)[:, 0]
    x1 = oracle.smooth(A, S, x0, b, 3, 2)[:, 0]
    x2 = x1 + P @ np.linalg.solve(P.T @ Ad @ P, P.T @ (b - Ad @ x1))
    x3 = oracle.smooth(A, S, x2, b, 3, 2)[:, 0]
    got = H.vcycle(S, x0, b, 3, 2)
    assert relerr(got, x3) < 1e-12


@pytest.mark.parametrize("iface_prec", [0, 1])
def test_two_level_cycle_with_the_schur_smoother_is_the_two_grid_composition(iface_prec):
    """The V-cycle with the ILUT Schur complement smoother on the finest level
    (Sec. 3.1: the smoother of one level of the V-cycle) = one application of
    schur_apply to the residual before and after the exact coarse correction
    x + P A_c^{-1} P^T (b - A x), composed here from schur_apply and a dense
    coarse solve (the smoother is not linear in r, so the composition applies
    it to each residual)."""
    A = synth.cutcell7(9, 8, 7, seed=6)
    n = len(A[0]) - 1
    H = oracle.AMG(A, theta=0.25, max_levels=2, coarse_size=1)
    assert len(H.levels) == 2
    L0, C = H.levels
    P = np.zeros((n, C.n))
    pp, pc, pv = L0.P
    for i in range(n):
        for q in range(pp[i], pp[i + 1]):
            P[i, pc[q]] = pv[q]
    Ad = dense(A, n)
    b = synth.rhs(n, 1, seed=2)[:, 0]
    x0 = synth.rhs(n, 1, seed=3)[:, 0]
    parts, tau, fill, mL, mU = 3, 1e-3, 6, 3, 2
    x1 = x0 + oracle.schur_apply(A, b - Ad @ x0, parts, tau, fill, mL, mU, iface_prec)
    x2 = x1 + P @ np.linalg.solve(P.T @ Ad @ P, P.T @ (b - Ad @ x1))
    x3 = x2 + oracle.schur_apply(A, b - Ad @ x2, parts, tau, fill, mL, mU, iface_prec)
    got = H.vcycle_schur(x0, b, parts, tau, fill, mL, mU, iface_prec=iface_prec)
    assert relerr(got, x3) < 1e-12
    assert oracle.schur_interface(A, parts)[0] > 0


def test_schur_smoothed_cycle_with_one_part_is_the_ilut_cycle():
    """One part has no interface rows, and the Schur complement smoother is
    then the ILUT smoother of the whole matrix: the cycle equals the ILU-smoothed
    V-cycle with the row-scaled ILUT(tau, fill) factors, on three levels with
    l1-Jacobi below."""
    A = synth.cutcell7(10, 9, 8, seed=8)
    n = len(A[0]) - 1
    H = oracle.AMG(A, theta=0.25, max_levels=3, coarse_size=1)
    assert len(H.levels) == 3
    S = oracle.row_scale(oracle.factor(A, "ilut", 1e-3, 6))
    b = synth.rhs(n, 1, seed=4)[:, 0]
    x0 = synth.rhs(n, 1, seed=5)[:, 0]
    want = H.vcycle(S, x0, b, 4, 3)
    got = H.vcycle_schur(x0, b, 1, 1e-3, 6, 4, 3)
    assert relerr(got, want) < 1e-12


def test_single_level_is_a_direct_solve():
    A = synth.cutcell7(5, 4, 4, seed=7)
    n = len(A[0]) - 1
    H = oracle.AMG(A, coarse_size=1000)
    assert len(H.levels) == 1
    S = oracle.row_scale(oracle.ilu0(A))
    b = synth.rhs(n, 1, seed=4)[:, 0]
    assert relerr(H.vcycle(S, np.zeros(n), b, 2, 2), np.linalg.solve(dense(A, n), b)) < 1e-13


def test_vcycle_convergence_on_poisson():
    """Textbook AMG behaviour: as a stationary iteration on the 7-point
    Poisson matrix the V-cycle reduces the residual by at least 3x per cycle,
    on a hierarchy of more than two levels."""
    A = synth.poisson7(12)
    n = len(A[0]) - 1
    H = oracle.AMG(A, theta=0.25, coarse_size=20)
    assert len(H.levels) >= 4
    S = oracle.row_scale(oracle.ilu0(A))
    M = scipy_csr(A)
    b = synth.rhs(n, 1, seed=1)[:, 0]
    x = np.zeros(n)
    prev = np.linalg.norm(b)
    for _ in range(6):
        x = H.vcycle(S, x, b, 2, 2)
        res = np.linalg.norm(b - M @ x)
        assert res < prev / 3.0
        prev = res


def test_three_level_cycle_with_l1_jacobi_matches_dense_recursion():
    """Alg. mgcycle on three levels, written densely: ILU smoothing on level 0,
    nu sweeps of l1-Jacobi x <- x + (b - A x) / d (d_i = sum_j |a_ij|) before
    and after the correction on level 1, direct solve on level 2."""
    A = synth.cutcell7(9, 8, 7, seed=8)
    n = len(A[0]) - 1
    S = oracle.row_scale(oracle.ilu0(A))
    H = oracle.AMG(A, theta=0.25, max_levels=3, coarse_size=1)
    assert len(H.levels) == 3

    def Pmat(L, nc):
        P = np.zeros((L.n, nc))
        pp, pc, pv = L.P
        for i in range(L.n):
            for q in range(pp[i], pp[i + 1]):
                P[i, pc[q]] = pv[q]
        return P

    L0, L1, L2 = H.levels
    P0, P1 = Pmat(L0, L1.n), Pmat(L1, L2.n)
    A1, A2 = dense(L1.A, L1.n), dense(L2.A, L2.n)
    d1 = np.abs(A1).sum(axis=1)
    nu = 2

    def level1(b1):
        x = np.zeros(L1.n)
        for _ in range(nu):
            x = x + (b1 - A1 @ x) / d1
        x = x + P1 @ np.linalg.solve(A2, P1.T @ (b1 - A1 @ x))
        for _ in range(nu):
            x = x + (b1 - A1 @ x) / d1
        return x

    Ad = dense(A, n)
    b = synth.rhs(n, 1, seed=5)[:, 0]
    x0 = np.zeros(n)
    x1 = oracle.smooth(A, S, x0, b, 2, 2)[:, 0]
    x2 = x1 + P0 @ level1(P0.T @ (b - Ad @ x1))
    x3 = oracle.smooth(A, S, x2, b, 2, 2)[:, 0]
    assert relerr(H.vcycle(S, x0, b, 2, 2, nu=nu), x3) < 1e-12


def test_three_level_cycle_with_polynomial_gs_matches_dense_recursion():
    """The mixed V-cycle of Sec. 6.3: ILU on the finest level, polynomial
    Gauss-Seidel below, x <- x + sum_{j<terms} (-D^{-1} L)^j D^{-1} (b - A x)
    with dense matrix powers here."""
    A = synth.cutcell7(9, 8, 7, seed=9)
    n = len(A[0]) - 1
    S = oracle.row_scale(oracle.ilu0(A))
    H = oracle.AMG(A, theta=0.25, max_levels=3, coarse_size=1)
    assert len(H.levels) == 3

    def Pmat(L, nc):
        P = np.zeros((L.n, nc))
        pp, pc, pv = L.P
        for i in range(L.n):
            for q in range(pp[i], pp[i + 1]):
                P[i, pc[q]] = pv[q]
        return P

    L0, L1, L2 = H.levels
    P0, P1 = Pmat(L0, L1.n), Pmat(L1, L2.n)
    A1, A2 = dense(L1.A, L1.n), dense(L2.A, L2.n)
    Dinv = np.diag(1.0 / np.diag(A1))
    G = -Dinv @ np.tril(A1, -1)
    terms, nu = 3, 2
    poly = sum(np.linalg.matrix_power(G, j) for j in range(terms)) @ Dinv

    def level1(b1):
        x = np.zeros(L1.n)
        for _ in range(nu):
            x = x + poly @ (b1 - A1 @ x)
        x = x + P1 @ np.linalg.solve(A2, P1.T @ (b1 - A1 @ x))
        for _ in range(nu):
            x = x + poly @ (b1 - A1 @ x)
        return x

    Ad = dense(A, n)
    b = synth.rhs(n, 1, seed=6)[:, 0]
    x1 = oracle.smooth(A, S, np.zeros(n), b, 2, 2)[:, 0]
    x2 = x1 + P0 @ level1(P0.T @ (b - Ad @ x1))
    x3 = oracle.smooth(A, S, x2, b, 2, 2)[:, 0]
    got = H.vcycle(S, np.zeros(n), b, 2, 2, nu=nu, coarse="gs", terms=terms)
    assert relerr(got, x3) < 1e-12


def dense_smoother(S, n, mL, mU):
    """M^{-1} of the row-scaled ILU smoother with m_L + m_U sweeps (Eq. LUiterMat),
    written as the dense truncated Neumann series (sum_{j<m_U} (-Utilde_s)^j)
    D^{-1} (sum_{j<m_L} (-L_s)^j)."""
    Ls, Us = dense(S.L, n), dense(S.Us, n)
    left = sum(np.linalg.matrix_power(-Us, j) for j in range(mU))
    right = sum(np.linalg.matrix_power(-Ls, j) for j in range(mL))
    return left @ np.diag(S.dinv) @ right


def test_ilu_on_the_finest_level_only_is_the_mixed_cycle():
    """vcycle_ilu with one level of factors is vcycle, bit for bit."""
    A = synth.cutcell7(9, 8, 7, seed=8)
    n = len(A[0]) - 1
    H = oracle.AMG(A, theta=0.25, max_levels=4, coarse_size=1)
    fac = H.level_factors("ilu0")
    assert len(fac) == len(H.levels) - 1 == 3
    b = synth.rhs(n, 1, seed=5)[:, 0]
    x0 = synth.rhs(n, 1, seed=6)[:, 0]
    for coarse in ("jacobi", "gs"):
        want = H.vcycle(fac[0], x0, b, 3, 2, nu=2, coarse=coarse, terms=3)
        assert np.array_equal(H.vcycle_ilu(fac[:1], x0, b, 3, 2, nu=2, coarse=coarse, terms=3), want)


def test_three_level_cycle_with_ilu_on_two_levels_matches_dense_recursion():
    """Alg. mgcycle on three levels with the ILU smoother on levels 0 and 1
    (Sec. 6: ILU smoothing from the finest level down), each level with its
    own sweep counts, written densely: x <- x + M_l^{-1} (b - A_l x) with M_l^{-1}
    the dense Neumann series of level l's row-scaled ILU(0) factors, before
    and after the correction, direct solve on level 2."""
    A = synth.cutcell7(9, 8, 7, seed=8)
    n = len(A[0]) - 1
    H = oracle.AMG(A, theta=0.25, max_levels=3, coarse_size=1)
    assert len(H.levels) == 3
    L0, L1, L2 = H.levels

    def Pmat(L, nc):
        P = np.zeros((L.n, nc))
        pp, pc, pv = L.P
        for i in range(L.n):
            for q in range(pp[i], pp[i + 1]):
                P[i, pc[q]] = pv[q]
        return P

    P0, P1 = Pmat(L0, L1.n), Pmat(L1, L2.n)
    A0, A1, A2 = dense(A, n), dense(L1.A, L1.n), dense(L2.A, L2.n)
    S0 = oracle.row_scale(oracle.ilu0(A))
    S1 = oracle.row_scale(oracle.ilu0(L1.A))
    mL, mU = (3, 2), (2, 4)
    M0 = dense_smoother(S0, n, mL[0], mU[0])
    M1 = dense_smoother(S1, L1.n, mL[1], mU[1])

    def level1(b1):
        x = M1 @ b1
        x = x + P1 @ np.linalg.solve(A2, P1.T @ (b1 - A1 @ x))
        return x + M1 @ (b1 - A1 @ x)

    b = synth.rhs(n, 1, seed=5)[:, 0]
    x0 = synth.rhs(n, 1, seed=7)[:, 0]
    x1 = x0 + M0 @ (b - A0 @ x0)
    x2 = x1 + P0 @ level1(P0.T @ (b - A0 @ x1))
    x3 = x2 + M0 @ (b - A0 @ x2)
    got = H.vcycle_ilu([S0, S1], x0, b, list(mL), list(mU), nu=3, coarse="gs", terms=2)
    assert relerr(got, x3) < 1e-12
    # the coarse smoother's settings no longer reach level 1
    assert np.array_equal(got, H.vcycle_ilu([S0, S1], x0, b, list(mL), list(mU), nu=1, coarse="jacobi"))
    # and level 1 is not smoothed by it: l1-Jacobi there gives another iterate (far outside the
    # 1e-12 agreement above; the coarse correction is a small part of this iterate)
    assert relerr(H.vcycle(S0, x0, b, mL[0], mU[0], nu=1), x3) > 1e-9


def test_exact_ilu_on_level_one_gives_the_two_grid_cycle():
    """On the 1-D Laplacian every level is tridiagonal, ILU(0) is its exact LU
    and n_l + n_l sweeps reach the exact solve (nilpotence): with that
    smoother on level 1 the coarse-grid correction is exact, so the cycle is
    the two-grid cycle x + P A_1^{-1} P^T (b - A x) between two finest-level
    smoothings, whatever the levels below do."""
    n = 63
    A = laplace1d(n)
    H = oracle.AMG(A, theta=0.25, max_levels=6, coarse_size=2)
    assert len(H.levels) >= 4
    fac = H.level_factors("ilu0", count=2)
    n1 = H.levels[1].n
    L0 = H.levels[0]
    P = np.zeros((n, n1))
    pp, pc, pv = L0.P
    for i in range(n):
        for q in range(pp[i], pp[i + 1]):
            P[i, pc[q]] = pv[q]
    A0 = dense(A, n)
    M0 = dense_smoother(fac[0], n, 1, 1)  # one sweep each: D^{-1}, a weak smoother
    b = synth.rhs(n, 1, seed=3)[:, 0]
    x0 = np.zeros(n)
    x1 = x0 + M0 @ (b - A0 @ x0)
    x2 = x1 + P @ np.linalg.solve(P.T @ A0 @ P, P.T @ (b - A0 @ x1))
    x3 = x2 + M0 @ (b - A0 @ x2)
    got = H.vcycle_ilu(fac, x0, b, [1, n1], [1, n1], nu=1)
    assert relerr(got, x3) < 1e-13
    # with too few sweeps on level 1 the correction is no longer exact
    assert relerr(H.vcycle_ilu(fac, x0, b, [1, 2], [1, 2], nu=1), x3) > 1e-6


def test_schur_on_the_finest_level_with_ilu_below_matches_dense_recursion():
    """The Schur-smoothed cycle with the ILU smoother on level 1 as well:
    schur_apply to the residual on level 0 (before and after), the dense
    Neumann series of level 1's row-scaled ILU(0) factors there, direct solve
    on level 2; and with one level of factors it is vcycle_schur bit for bit."""
    A = synth.cutcell7(10, 9, 8, seed=8)
    n = len(A[0]) - 1
    H = oracle.AMG(A, theta=0.25, max_levels=3, coarse_size=1)
    assert len(H.levels) == 3
    L0, L1, L2 = H.levels

    def Pmat(L, nc):
        P = np.zeros((L.n, nc))
        pp, pc, pv = L.P
        for i in range(L.n):
            for q in range(pp[i], pp[i + 1]):
                P[i, pc[q]] = pv[q]
        return P

    P0, P1 = Pmat(L0, L1.n), Pmat(L1, L2.n)
    A0, A1, A2 = dense(A, n), dense(L1.A, L1.n), dense(L2.A, L2.n)
    fac = H.level_factors("ilu0", count=2)
    parts, tau, fill = 3, 1e-3, 6
    mL, mU = [3, 2], [2, 3]
    M1 = dense_smoother(fac[1], L1.n, mL[1], mU[1])

    def level1(b1):
        x = M1 @ b1
        x = x + P1 @ np.linalg.solve(A2, P1.T @ (b1 - A1 @ x))
        return x + M1 @ (b1 - A1 @ x)

    b = synth.rhs(n, 1, seed=4)[:, 0]
    x0 = synth.rhs(n, 1, seed=5)[:, 0]
    x1 = x0 + oracle.schur_apply(A, b - A0 @ x0, parts, tau, fill, mL[0], mU[0])
    x2 = x1 + P0 @ level1(P0.T @ (b - A0 @ x1))
    x3 = x2 + oracle.schur_apply(A, b - A0 @ x2, parts, tau, fill, mL[0], mU[0])
    got = H.vcycle_ilu(fac, x0, b, mL, mU, schur=(parts, tau, fill))
    assert relerr(got, x3) < 1e-12
    one = H.vcycle_ilu(fac[:1], x0, b, mL[0], mU[0], nu=2, schur=(parts, tau, fill))
    assert np.array_equal(one, H.vcycle_schur(x0, b, parts, tau, fill, mL[0], mU[0], nu=2))
