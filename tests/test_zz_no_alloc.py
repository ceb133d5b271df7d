"""The allocation-free smoother entry point, silu_smooth_noalloc.

Callers that cannot allocate device memory when they apply the smoother --
an application whose device memory is owned up front by its own pool or by
another framework's allocator, or a latency-critical time-stepping loop that
must not pay cudaMalloc's implicit synchronisation -- pass their own device
arrays and get their working vectors from a fixed array inside the library.
This test checks, through the C ABI, that two calls in a row give what
ilu_smooth gives on the same inputs (FP64 tolerance 1e-12 relative), that the
second call is not disturbed by what the first left in the shared array, and
that a problem above the fixed capacity is refused before any work.
"""
import numpy as np
import pytest

import synth
from _helpers import relerr

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_matches_ilu_smooth_on_two_calls():
    import paper_2111_09512_gb300 as silu
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    silu.build()
    stream = torch.cuda.current_stream()
    ctx = silu.Context(0, stream)
    A = synth.cutcell7(40, 36, 30, seed=3)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", 1e-3, 10)
    ex = F.export()

    def dev_csr(rp, ci, va):
        return (torch.from_numpy(np.asarray(rp, np.int32)).cuda(),
                torch.from_numpy(np.asarray(ci, np.int32)).cuda(),
                torch.from_numpy(np.asarray(va, np.float64)).cuda())

    dA = dev_csr(*A)
    dL = dev_csr(*ex["L"])
    dU = dev_csr(*ex["Us"])
    dinv = torch.from_numpy(ex["dinv"].copy()).cuda()

    calls = [(synth.rhs(n, 1, seed=5)[:, 0], synth.rhs(n, 1, seed=6)[:, 0], 4, 5),
             (synth.rhs(n, 1, seed=7)[:, 0] * 0.0, synth.rhs(n, 1, seed=8)[:, 0], 6, 3)]
    for x0, b, mL, mU in calls:
        b_d = torch.from_numpy(b.copy()).cuda()
        x_ref = torch.from_numpy(x0.copy()).cuda().reshape(n, 1)
        silu.ilu_smooth(F, x_ref, b_d.reshape(n, 1), mL, mU)
        x_new = torch.from_numpy(x0.copy()).cuda()
        st = silu.silu_smooth_noalloc(0, stream, n, dA, dL, dU, dinv, x_new, b_d, mL, mU)
        assert st == silu.OK
        torch.cuda.synchronize()
        assert relerr(x_new.cpu().numpy(), x_ref.cpu().numpy().reshape(n)) < 1e-12

    # above the fixed capacity: refused, nothing written
    big = 524288 + 1
    x_untouched = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = silu.silu_smooth_noalloc(0, stream, big, dA, dL, dU, dinv, x_untouched, x_untouched, 1, 1)
    assert st == silu.ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert torch.count_nonzero(x_untouched).item() == 0
