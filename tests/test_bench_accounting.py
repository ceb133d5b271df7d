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
