"""Pins of the oracle's power-iteration estimate of ||T_s^p||_2 (Sec. 5.2:
numerical nilpotence of the strictly triangular part, Fig. Up).  CPU only."""
import numpy as np

import oracle
import synth
from _helpers import dense


def test_two_by_two_closed_form():
    """T = [[0, a], [0, 0]]: ||T||_2 = |a|, T^2 = 0.  From v0 = (0.6, 0.8) the
    first iteration sees ||T v|| = 0.8|a|; the second starts from v = (0, 1)."""
    a = -3.25
    T = (np.array([0, 1, 1], np.int64), np.array([1], np.int32), np.array([a]))
    v0 = np.array([0.6, 0.8])
    assert oracle.power_norms(T, 1, 1, v0)[0] == 0.8 * abs(a)
    out = oracle.power_norms(T, 3, 2, v0)
    assert out[0] == abs(a) and out[1] == 0.0 and out[2] == 0.0


def test_matches_dense_spectral_norm():
    """Against numpy's exact 2-norm of the dense matrix power."""
    A = synth.cutcell7(4, 3, 3, seed=2)
    S = oracle.row_scale(oracle.ilut(A, 1e-4, 8))
    n = S.n
    T = dense(S.Us, n)
    v0 = synth.rhs(n, 1, seed=3)[:, 0]
    est = oracle.power_norms(S.Us, 8, 400, v0)
    for p in range(1, 9):
        exact = np.linalg.norm(np.linalg.matrix_power(T, p), 2)
        if exact == 0.0:
            assert est[p - 1] == 0.0
        else:
            assert abs(est[p - 1] - exact) / exact < 1e-6, (p, est[p - 1], exact)
    L = dense(S.L, n)
    estL = oracle.power_norms(S.L, 4, 400, v0)
    for p in range(1, 5):
        exact = np.linalg.norm(np.linalg.matrix_power(L, p), 2)
        assert abs(estL[p - 1] - exact) / exact < 1e-6


def test_exactly_zero_beyond_the_levels():
    """A strictly triangular T is nilpotent of index <= #levels: T^p v has no
    nonzero term once p reaches the longest dependency chain (Sec. 5.2)."""
    A = synth.poisson7(5, 4, 3)
    S = oracle.row_scale(oracle.ilu0(A))
    nlev, _ = oracle.levels_upper(S.Us)
    assert nlev == 5 + 4 + 3 - 2
    v0 = synth.rhs(S.n, 1, seed=1)[:, 0]
    est = oracle.power_norms(S.Us, nlev + 2, 5, v0)
    assert np.all(est[:nlev - 1] > 0.0)
    assert np.all(est[nlev - 1:] == 0.0)
