"""The uneven-row generator synth.banded (inputs of the row-shape edge cases):
structurally symmetric, strictly diagonally dominant, columns sorted, the
requested lower counts exactly (long rows included), reproducible from the
seed, and ILU(0) of it keeps A's pattern (no fill), so the factor's rows have
the lengths the edge cases are built for."""
import numpy as np

import oracle
import synth


def dense(A):
    rp, ci, va = A
    n = len(rp) - 1
    D = np.zeros((n, n))
    for i in range(n):
        D[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    return D


def test_banded_structure_and_counts():
    A = synth.banded(700, 10, 40, seed=3, min_lower=5, long_rows={350: 11, 699: 699})
    rp, ci, va = A
    n = len(rp) - 1
    D = dense(A)
    assert np.array_equal(D != 0, (D != 0).T)
    off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    assert np.all(np.diag(D) > off) and np.allclose(np.diag(D), 1.0 + off, rtol=1e-14, atol=0)
    for i in range(n):
        cols = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0)
        lower = int((cols < i).sum())
        if i == 350:
            assert lower == 11
        elif i == 699:
            assert lower == 699  # a dense last row
        else:
            assert min(i, 5) <= lower <= 10 and np.all(i - cols[cols < i] <= 40)
    B = synth.banded(700, 10, 40, seed=3, min_lower=5, long_rows={350: 11, 699: 699})
    assert all(np.array_equal(a, b) for a, b in zip(A, B))


def test_banded_ilu0_has_no_fill():
    A = synth.banded(300, 6, 25, seed=4)
    S = oracle.row_scale(oracle.factor(A, "ilu0", 0.0, 0))
    rp, ci, _ = A
    Lrp, Lci = np.asarray(S.L[0]), np.asarray(S.L[1])
    Urp, Uci = np.asarray(S.Us[0]), np.asarray(S.Us[1])
    for i in range(len(rp) - 1):
        cols = ci[rp[i]:rp[i + 1]]
        assert np.array_equal(np.sort(Lci[Lrp[i]:Lrp[i + 1]]), cols[cols < i])
        assert np.array_equal(np.sort(Uci[Urp[i]:Urp[i + 1]]), cols[cols > i])
