"""Pins of the oracle's row/column (Ruiz) scaling of U (Sec. 5.1,
Eq. rowcolScale) and of the smoother that iterates on D_r U D_c.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth
from _helpers import dense, relerr


def lu_of(M):
    """Factors object for a dense upper triangular U (diagonal first per row) and L = I."""
    n = M.shape[0]
    up, uc, uv = [0], [], []
    for i in range(n):
        uc.append(i)
        uv.append(M[i, i])
        for j in range(i + 1, n):
            if M[i, j] != 0.0:
                uc.append(j)
                uv.append(M[i, j])
        up.append(len(uc))
    U = (np.array(up, np.int64), np.array(uc, np.int32), np.array(uv, np.float64))
    L = (np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    return oracle.Factors(n, L, U)


def test_hand_worked_2x2():
    """U = [[4, 16], [0, 1]].  Step 1 divides rows by sqrt(16), sqrt(1) and
    columns by sqrt(4), sqrt(16): column scale (1/2, 1/4); the unit diagonal
    then needs dr = (1/(4/2), 1/(1/4)) = (1/2, 4), and uhat_01 = 1/2 * 16 * 1/4 = 2.
    Step 2 works on [[1/2, 1], [0, 1/4]]: columns divided by sqrt(1/2) and 1,
    so dc = (sqrt(1/2), 1/4), dr_0 = 1/(4 sqrt(1/2)) and uhat_01 = sqrt(2)."""
    F = lu_of(np.array([[4.0, 16.0], [0.0, 1.0]]))
    S = oracle.ruiz_rowcol(F, maxit=1, tol=0.0)
    assert S.steps == 1
    assert list(S.dc) == [0.5, 0.25] and list(S.dr) == [0.5, 4.0]
    assert list(S.Us[2]) == [2.0]
    S2 = oracle.ruiz_rowcol(F, maxit=2, tol=0.0)
    assert S2.steps == 2
    assert abs(S2.dc[0] - math.sqrt(0.5)) < 3e-16 and S2.dc[1] == 0.25
    assert abs(S2.dr[0] - 1.0 / (4.0 * math.sqrt(0.5))) < 3e-16 and S2.dr[1] == 4.0
    assert abs(S2.Us[2][0] - math.sqrt(2.0)) < 4e-16


def test_diagonal_u_converges_in_one_step():
    """A diagonal U (ILUT with an infinite drop tolerance) is equilibrated by
    one step, dc = 1/sqrt|d|; the unit diagonal leaves no strict part."""
    A = synth.cutcell7(5, 4, 3, seed=2)
    F = oracle.ilut(A, math.inf, 4)
    d = F.U[2]
    S = oracle.ruiz_rowcol(F, maxit=20, tol=1e-12)
    assert S.steps == 1
    assert np.allclose(S.dc, 1.0 / np.sqrt(np.abs(d)), rtol=1e-15, atol=0)
    assert len(S.Us[1]) == 0
    assert np.allclose(S.dr * d * S.dc, 1.0, rtol=1e-15, atol=0)


def test_equilibrated_rows_and_columns():
    """After enough steps every row and column maximum of the Ruiz-scaled
    D_r' U D_c (before the unit-diagonal row fix) is 1 within tol; the row
    fix rescales rows only, so D_c alone must already equilibrate the columns
    to within that tol of the row factors it implies."""
    A = synth.cutcell7(8, 7, 6, seed=3)
    F = oracle.ilu0(A)
    tol = 1e-6
    S = oracle.ruiz_rowcol(F, maxit=200, tol=tol)
    assert 1 < S.steps < 200
    n = F.n
    U = dense(F.U, n)
    # recover the Ruiz row factors: each row's maximum after column scaling is 1/rs
    B = np.abs(U) * S.dc[None, :]
    rs = 1.0 / B.max(axis=1)
    E = rs[:, None] * B
    assert np.all(np.abs(E.max(axis=1) - 1.0) <= tol * 1.01)
    assert np.all(np.abs(E.max(axis=0) - 1.0) <= 2 * tol)


@pytest.mark.parametrize("gen", ["cutcell_ilu0", "cutcell_ilut", "hex27"])
def test_rowcol_smoother_equals_row_scaled(gen):
    """D_r U D_c = D_c^{-1} (D^{-1} U) D_c when its diagonal is one, so the
    Richardson iterates on it, mapped back by D_c, are the row-scaled
    iterates: the two smoothers agree for every sweep count (to rounding)."""
    if gen == "cutcell_ilu0":
        A = synth.cutcell7(9, 8, 7, seed=4)
        F = oracle.ilu0(A)
    elif gen == "cutcell_ilut":
        A = synth.cutcell7(9, 8, 7, seed=5)
        F = oracle.ilut(A, 1e-3, 6)
    else:
        A = synth.hex27(6, 5, 5, seed=6)
        F = oracle.ilu0(A)
    n = F.n
    S = oracle.row_scale(F)
    RC = oracle.ruiz_rowcol(F)
    U = dense(F.U, n)
    Uhat = np.eye(n) + dense(RC.Us, n)
    assert relerr(Uhat, RC.dr[:, None] * U * RC.dc[None, :]) < 1e-15
    b = synth.rhs(n, 2, seed=7)
    x0 = synth.rhs(n, 2, seed=8)
    for mL, mU in [(1, 1), (3, 3), (5, 2), (0, 4), (4, 0), (n, n)]:
        want = oracle.smooth(A, S, x0, b, mL, mU)
        got = oracle.smooth_rowcol(A, RC, x0, b, mL, mU)
        assert relerr(got, want) < 1e-12, (mL, mU)


def test_rowcol_zero_pivot():
    F = lu_of(np.array([[0.0, 1.0], [0.0, 2.0]]))
    with pytest.raises(oracle.OracleError) as e:
        oracle.ruiz_rowcol(F)
    assert e.value.status == oracle.ZERO_PIVOT
