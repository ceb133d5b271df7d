"""The algorithmic-byte accounting that bench.py's GB/s and roofline figures
rest on, checked on the CPU against hand-counted cases: one Richardson sweep
reads every stored entry of the strict factor (value + int32 column), the
row pointers, the iterate and c, and writes the new iterate; the residual does
the same with A in FP64; one application adds the D^{-1} read and the
read-modify-write of x."""
import bench


def test_sweep_and_residual_bytes_by_hand():
    # 3 rows, 2 strict entries, one right-hand side, FP64: 2 * (8 + 4) + 4 * 4 + 3 * 3 * 8
    assert bench.sweep_bytes(3, 2, 1, 8) == 24 + 16 + 72
    # FP32 values and vectors: 2 * (4 + 4) + 4 * 4 + 3 * 3 * 4
    assert bench.sweep_bytes(3, 2, 1, 4) == 16 + 16 + 36
    # four interleaved right-hand sides multiply only the vector traffic
    assert bench.sweep_bytes(3, 2, 4, 8) == 24 + 16 + 3 * 3 * 4 * 8
    # the residual always reads A in FP64: 7 entries, x and b read, r written
    assert bench.resid_bytes(3, 7, 1) == 7 * 12 + 16 + 3 * 3 * 8


def test_application_bytes_count_free_first_sweeps():
    n, nnzA, nnzL, nnzU = 5, 13, 4, 4
    # m_L = m_U = 1: the first sweep of each factor costs no SpMV
    one = bench.apply_bytes(n, nnzA, nnzL, nnzU, 1, 8, 1, 1)
    assert one == bench.resid_bytes(n, nnzA, 1) + 8 * n + 8 * n
    # each further sweep adds exactly one sweep's bytes
    assert bench.apply_bytes(n, nnzA, nnzL, nnzU, 1, 8, 3, 1) - one == 2 * bench.sweep_bytes(n, nnzL, 1, 8)
    assert bench.apply_bytes(n, nnzA, nnzL, nnzU, 1, 8, 1, 4) - one == 3 * bench.sweep_bytes(n, nnzU, 1, 8)
    # m = 0 adds no sweep (the count never goes negative)
    assert bench.apply_bytes(n, nnzA, nnzL, nnzU, 1, 8, 0, 0) == one


def test_headline_workload_bytes():
    """The 128^3 cut-cell ILUT(1e-3,10) application with 10+10 sweeps: the
    step bytes the benchmark reports, and the per-launch sweep bytes quoted
    beside the ncu traffic (256.3 MB per L sweep, 301.4 MB per U sweep)."""
    n, nnzA, nnzL, nnzU = 2097152, 14581760, 16463399, 20224407
    assert bench.apply_bytes(n, nnzA, nnzL, nnzU, 1, 8, 10, 10) == 5286503540
    assert round(bench.sweep_bytes(n, nnzL, 1, 8) / 1e6, 1) == 256.3
    assert round(bench.sweep_bytes(n, nnzU, 1, 8) / 1e6, 1) == 301.4


def test_vcycle_bytes_by_hand():
    """The V-cycle model (Sec. 6.3 in kind) on a three-level hierarchy with
    hand-picked sizes: finest level 10 rows (A 28 entries, P 12), level 1 4
    rows (A 10, P 5), coarsest 2 rows; L_s / Utilde_s 9 entries each, 2 + 2
    sweeps, one l1-Jacobi step."""
    st = {"levels": 3, "rows": [10, 4, 2], "nnz_A": [28, 10, 3], "nnz_P": [12, 5, 0]}
    n0, n1, n2 = 10, 4, 2
    post = bench.apply_bytes(n0, 28, 9, 9, 1, 8, 2, 2)
    pre = post - bench.resid_bytes(n0, 28, 1) - 8 * n0      # from x = 0: no residual, no read of x
    lev0 = (bench.resid_bytes(n0, 28, 1)                     # r = b - A x
            + (12 * 12 + 4 * (n1 + 1) + 8 * n0 + 8 * n1)     # R r: P's entries, n1 rows, reads r, writes b_1
            + (12 * 12 + 4 * (n0 + 1) + 8 * n1 + 8 * n0) + 8 * n0)  # x += P v (x read and written)
    jac1 = 3 * 8 * n1 + (10 * 12 + 4 * (n1 + 1) + 8 * n1 + 8 * n1 + 3 * 8 * n1)  # x = D^-1 b, then one sweep
    lev1 = (jac1 + bench.resid_bytes(n1, 10, 1)
            + (5 * 12 + 4 * (n2 + 1) + 8 * n1 + 8 * n2)
            + (5 * 12 + 4 * (n1 + 1) + 8 * n2 + 8 * n1) + 8 * n1)
    coarsest = 8 * n2 * n2 + 16 * n2
    assert bench.vcycle_bytes(st, 9, 9, 2, 2, 1) == pre + post + lev0 + lev1 + coarsest
    # no smoothing steps below the finest level: the level's x is only cleared (one write)
    assert (bench.vcycle_bytes(st, 9, 9, 2, 2, 1) - bench.vcycle_bytes(st, 9, 9, 2, 2, 0)
            == jac1 - 8 * n1)
