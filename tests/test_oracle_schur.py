"""Pins of the oracle's ILUT Schur complement smoother (Sec. 3.1, Eq. schur:
interior / interface partition, S = C - F B^{-1} E, one GMRES iteration on
S y = g - F B^{-1} f, back-substitution x = B^{-1}(f - E y)).  CPU only."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import csr_from_dense, dense, relerr


def brute_interface(A, parts):
    rp, ci, _ = A
    n = len(rp) - 1
    bounds = [k * n // parts for k in range(parts + 1)]

    def block(i):
        return max(k for k in range(parts) if bounds[k] <= i)

    return np.array([int(any(block(j) != block(i) for j in ci[rp[i]:rp[i + 1]])) for i in range(n)], np.int32)


@pytest.mark.parametrize("parts", [1, 2, 3, 5])
def test_interface_detection(parts):
    A = synth.cutcell7(7, 6, 5, seed=2)
    k, marks = oracle.schur_interface(A, parts)
    want = brute_interface(A, parts)
    assert np.array_equal(marks, want) and k == want.sum()
    if parts == 1:
        assert k == 0


def test_one_part_is_the_ilut_smoother():
    """No interface: M^{-1} r is B^{-1} r with B = A, the ILUT smoother from zero."""
    A = synth.cutcell7(6, 5, 5, seed=3)
    n = len(A[0]) - 1
    r = synth.rhs(n, 1, seed=4)[:, 0]
    S = oracle.row_scale(oracle.ilut(A, 1e-3, 8))
    want = oracle.smooth(A, S, np.zeros((n, 1)), r, 3, 2)[:, 0]
    assert np.array_equal(oracle.schur_apply(A, r, 1, 1e-3, 8, 3, 2), want)


def dense_schur(A, r, parts, iface_prec=0):
    """The smoother with exact B^{-1}, written densely: the one GMRES step from
    zero is the minimal-residual step y = (s.Sq / Sq.Sq) q with q = s, or, with
    the interface iteration right-preconditioned by M = diag(C), q = M^{-1} s
    (the step minimises ||s - S y|| over y in span{M^{-1} s})."""
    n = len(A[0]) - 1
    M = dense(A, n)
    _, g = oracle.schur_interface(A, parts)
    I = np.flatnonzero(g == 0)
    G = np.flatnonzero(g == 1)
    B, E, F, C = M[np.ix_(I, I)], M[np.ix_(I, G)], M[np.ix_(G, I)], M[np.ix_(G, G)]
    Binv = np.linalg.inv(B)
    f, gg = r[I], r[G]
    s = gg - F @ Binv @ f
    Sm = C - F @ Binv @ E
    q = s / np.diag(C) if iface_prec else s
    Sq = Sm @ q
    y = (s @ Sq) / (Sq @ Sq) * q if np.linalg.norm(s) > 0 else np.zeros_like(s)
    z = np.zeros(n)
    z[I] = Binv @ (f - E @ y)
    z[G] = y
    return z, np.linalg.norm(s - Sm @ y) / np.linalg.norm(s)


@pytest.mark.parametrize("iface_prec", [0, 1])
@pytest.mark.parametrize("gen,parts", [("poisson", 2), ("cutcell", 3), ("hex27", 2)])
def test_exact_b_matches_dense_composition(gen, parts, iface_prec):
    """With ILUT keeping everything (tau = 0, fill = n: exact LU of B) and
    as many sweeps as rows (nilpotence: exact triangular solves) every step is
    exact, so the smoother equals its dense statement, with or without the
    diag(C) preconditioner on the interface iteration; the GMRES step reduces
    the interface residual."""
    A = {"poisson": lambda: synth.poisson7(6, 5, 6), "cutcell": lambda: synth.cutcell7(6, 6, 6, seed=5),
         "hex27": lambda: synth.hex27(5, 4, 6, seed=6)}[gen]()
    n = len(A[0]) - 1
    r = synth.rhs(n, 1, seed=7)[:, 0]
    got = oracle.schur_apply(A, r, parts, 0.0, n, n, n, iface_prec=iface_prec)
    want, red = dense_schur(A, r, parts, iface_prec)
    assert relerr(got, want) < 1e-11
    assert red < 1.0
    if gen == "cutcell":  # the two steps differ where diag(C) varies
        assert relerr(got, dense_schur(A, r, parts, 1 - iface_prec)[0]) > 1e-6


def test_interface_prec_is_inert_for_a_constant_diagonal():
    """On the Poisson matrix every c_kk is 6, and a constant M changes no
    minimal-residual step: q = s / 6 and the coefficient scales by 6."""
    A = synth.poisson7(8, 7, 6)
    n = len(A[0]) - 1
    r = synth.rhs(n, 1, seed=2)[:, 0]
    a = oracle.schur_apply(A, r, 3, 1e-3, 10, 3, 2, iface_prec=0)
    b = oracle.schur_apply(A, r, 3, 1e-3, 10, 3, 2, iface_prec=1)
    assert relerr(b, a) < 1e-13


def test_interface_prec_zero_diagonal_is_reported():
    """A zero c_kk cannot precondition: ORC_ZERO_PIVOT, and the plain step still runs."""
    M = np.array([[2.0, 1.0], [1.0, 0.0]])  # rows 0 and 1 in separate parts: both interface, C = M
    A = csr_from_dense(M)
    r = np.array([1.0, -1.0])
    with pytest.raises(oracle.OracleError):
        oracle.schur_apply(A, r, 2, 0.0, 2, 2, 2, iface_prec=1)
    z = oracle.schur_apply(A, r, 2, 0.0, 2, 2, 2, iface_prec=0)
    assert np.all(np.isfinite(z))


def test_single_interface_row_gives_the_exact_solve():
    """Two blocks coupled only through one entry of row m (nonsymmetric): the
    interface is that one row, S is 1 x 1, one GMRES iteration solves it
    exactly, and with exact B the smoother returns A^{-1} r."""
    rng = np.random.default_rng(3)
    m = 6
    n = 2 * m
    M = np.zeros((n, n))
    for blk in range(2):
        o = blk * m
        for i in range(m):
            M[o + i, o + i] = 4.0 + rng.uniform()
            if i > 0:
                M[o + i, o + i - 1] = -1.0 - rng.uniform()
            if i < m - 1:
                M[o + i, o + i + 1] = -1.0 - rng.uniform()
    M[m, m - 1] = -0.7
    A = csr_from_dense(M)
    k, marks = oracle.schur_interface(A, 2)
    assert k == 1 and marks[m] == 1
    r = rng.uniform(-1.0, 1.0, n)
    for iface_prec in (0, 1):  # a 1 x 1 S is solved by any nonzero scaling
        z = oracle.schur_apply(A, r, 2, 0.0, n, n, n, iface_prec=iface_prec)
        assert relerr(z, np.linalg.solve(M, r)) < 1e-13
