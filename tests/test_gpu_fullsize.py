"""Parity at the benchmark's full size and launch configuration: the 128^3
cut-cell pressure matrix (2,097,152 rows), ILUT(1e-3, 10), FP64, one
smoother application with 10 + 10 sweeps, one right-hand side -- compared
element by element with the oracle over the whole vector."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_cutcell128_ilut_smooth_full_vector():
    import paper_2111_09512_gb300 as silu
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    silu.build()
    A = synth.cutcell7(128, seed=1)
    n = len(A[0]) - 1
    ctx = silu.Context(0, torch.cuda.current_stream())
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", 1e-3, 10)
    OF = oracle.ilut(A, 1e-3, 10)
    S = oracle.row_scale(OF)
    ex = F.export()
    assert np.array_equal(ex["L"][0], OF.L[0]) and np.array_equal(ex["L"][1], OF.L[1])
    assert np.array_equal(ex["U"][0], OF.U[0]) and np.array_equal(ex["U"][1], OF.U[1])
    b = synth.rhs(n, 1, seed=1)
    x0 = np.zeros((n, 1))
    want = oracle.smooth(A, S, x0, b, 10, 10)
    x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    silu.ilu_smooth(F, x, torch.from_numpy(b).cuda(), 10, 10)
    torch.cuda.synchronize()
    got = x.cpu().numpy()
    assert relerr(got, want) < 1e-12
    # a second application from the first iterate (x != 0 exercises the residual)
    want2 = oracle.smooth(A, S, want, b, 10, 10)
    silu.ilu_smooth(F, x, torch.from_numpy(b).cuda(), 10, 10)
    torch.cuda.synchronize()
    assert relerr(x.cpu().numpy(), want2) < 1e-12
