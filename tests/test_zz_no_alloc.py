"""The allocation-free smoother entry point, silu_smooth_noalloc.

Callers that cannot allocate device memory when they apply the smoother --
an application whose device memory is owned up front by its own pool or by
another framework's allocator, or a latency-critical time-stepping loop that
must not pay cudaMalloc's implicit synchronisation -- pass their own device
arrays and get their working vectors from a fixed array inside the library.
These tests check, through the C ABI, that calls in a row give what
ilu_smooth gives on the same inputs (FP64 tolerance 1e-12 relative) for
every branch of the application (no L sweep, one, several; no U factor, one
U step, several), that a call is not disturbed by what the one before left
in the shared array, that the very first call of a fresh process (the one
that looks the array up on the device) and the calls after it succeed, and
that a problem above the fixed capacity is refused before any work.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
from _helpers import maxabs_err, relerr

torch = pytest.importorskip("torch")

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _inputs(silu, ctx, A):
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", 1e-3, 10)
    ex = F.export()

    def dev_csr(rp, ci, va):
        return (torch.from_numpy(np.asarray(rp, np.int32)).cuda(),
                torch.from_numpy(np.asarray(ci, np.int32)).cuda(),
                torch.from_numpy(np.asarray(va, np.float64)).cuda())

    return F, dev_csr(*A), dev_csr(*ex["L"]), dev_csr(*ex["Us"]), torch.from_numpy(ex["dinv"].copy()).cuda()


@pytest.mark.gpu
def test_noalloc_matches_ilu_smooth_on_calls_in_a_row():
    import paper_2111_09512_gb300 as silu
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    silu.build()
    stream = torch.cuda.current_stream()
    ctx = silu.Context(0, stream)
    A = synth.cutcell7(40, 36, 30, seed=3)
    n = len(A[0]) - 1
    F, dA, dL, dU, dinv = _inputs(silu, ctx, A)

    # (x0 seed or None for zero, b seed, sweeps_L, sweeps_U); the pairs cover
    # every branch: no / one / several L sweeps, no U factor, one U step
    # (D^{-1} y only), several U sweeps
    calls = [(5, 6, 4, 5), (None, 8, 6, 3), (9, 10, 0, 0), (11, 12, 1, 0), (13, 14, 1, 1), (15, 16, 0, 2),
             (17, 18, 3, 1), (19, 20, 2, 0), (None, 21, 0, 1)]
    for xs, bs, mL, mU in calls:
        x0 = synth.rhs(n, 1, seed=xs)[:, 0] if xs is not None else np.zeros(n)
        b = synth.rhs(n, 1, seed=bs)[:, 0]
        b_d = torch.from_numpy(b.copy()).cuda()
        x_ref = torch.from_numpy(x0.copy()).cuda().reshape(n, 1)
        silu.ilu_smooth(F, x_ref, b_d.reshape(n, 1), mL, mU)
        x_new = torch.from_numpy(x0.copy()).cuda()
        st = silu.silu_smooth_noalloc(0, stream, n, dA, dL, dU, dinv, x_new, b_d, mL, mU)
        assert st == silu.OK, (mL, mU)
        torch.cuda.synchronize()
        got, want = x_new.cpu().numpy(), x_ref.cpu().numpy().reshape(n)
        assert relerr(got, want) < 1e-12, (mL, mU)
        assert maxabs_err(got, want) < 1e-12, (mL, mU)

    # above the fixed capacity: refused, nothing written
    big = 524288 + 1
    x_untouched = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = silu.silu_smooth_noalloc(0, stream, big, dA, dL, dU, dinv, x_untouched, x_untouched, 1, 1)
    assert st == silu.ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert torch.count_nonzero(x_untouched).item() == 0


_FRESH = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import numpy as np, torch
import paper_2111_09512_gb300 as silu, synth
from _helpers import relerr
A = synth.cutcell7(23, 19, 17, seed=4)
n = len(A[0]) - 1
# the caller's own arrays, made before the first call of the entry point
from oracle import factor, row_scale
d32 = lambda a: torch.from_numpy(np.asarray(a, np.int32)).cuda()
d64 = lambda a: torch.from_numpy(np.asarray(a, np.float64)).cuda()
S = row_scale(factor(A, "ilut", 1e-3, 10))
dA = (d32(A[0]), d32(A[1]), d64(A[2]))
dL = (d32(S.L[0]), d32(S.L[1]), d64(S.L[2]))
dU = (d32(S.Us[0]), d32(S.Us[1]), d64(S.Us[2]))
dinv = d64(S.dinv)
b = d64(synth.rhs(n, 1, seed=2)[:, 0])
stream = torch.cuda.current_stream()
outs = []
for k in range(2):
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = silu.silu_smooth_noalloc(0, stream, n, dA, dL, dU, dinv, x, b, 3, 4)
    assert st == silu.OK, ("call", k, st)
    torch.cuda.synchronize()
    outs.append(x.cpu().numpy())
ctx = silu.Context(0, stream)
F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", 1e-3, 10)
xr = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
silu.ilu_smooth(F, xr, b.reshape(n, 1), 3, 4)
torch.cuda.synchronize()
want = xr.cpu().numpy().reshape(n)
for k in range(2):
    assert relerr(outs[k], want) < 1e-12, ("call", k, relerr(outs[k], want))
print("fresh-process noalloc ok")
"""


@pytest.mark.gpu
def test_noalloc_first_call_in_a_fresh_process():
    """The first call of a process looks the scratch array up on the device
    (and, with lazy module loading, loads it there); it and the call after it
    succeed and agree with ilu_smooth.  The factors here come from the
    caller's own arrays (the oracle's, as a user's own setup would be), so
    the library has done nothing on the device before that first call."""
    import paper_2111_09512_gb300 as silu
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    silu.build()
    code = _FRESH.format(root=_ROOT, tests=os.path.join(_ROOT, "tests"))
    res = subprocess.run([sys.executable, "-c", code], cwd=_ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-4000:]
    assert "fresh-process noalloc ok" in res.stdout
