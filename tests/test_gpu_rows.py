"""Row-shape edge cases of the sweep kernels, against the CPU oracle.

The staged sweep cuts a factor into 32-row tiles of at most 416 entries
(352 in the narrow configuration, chosen when no row has more than 10
entries and rows hold 9 on average at most); a row too long for any tile
sends the whole factor to the lanes-per-row kernel.  These seeded
structurally symmetric matrices (synth.banded) put the shapes at those
edges: rows of up to 10 lower entries (narrow tiles), one row of 11 (not
narrow), a row of 400 entries that nearly fills a tile of its own, a dense
last row and column (an arrow: too long for a tile, in L and in A), rows
holding only a diagonal, and sizes below and just above one tile.  Each is
smoothed (ILU(0), row-scaled) with every kernel choice, FP64 to 1e-12 of
the oracle (relative 2-norm and max-abs) and FP32 to single precision,
and solved by FGMRES to 1e-10."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import maxabs_err, relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def silu():
    import paper_2111_09512_gb300 as s
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s.build()
    return s


@pytest.fixture(scope="module")
def ctx(silu):
    return silu.Context(0, torch.cuda.current_stream())


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


CASES = [
    ("rows of 5 to 10 (narrow)", lambda: synth.banded(5003, 10, 48, seed=7, min_lower=5)),
    ("one row of 11", lambda: synth.banded(5003, 10, 48, seed=7, min_lower=5, long_rows={2500: 11})),
    ("rows of 9 or 10 (mean above 9)", lambda: synth.banded(4099, 10, 40, seed=13, min_lower=9)),
    ("rows of 0 to 5 (two rows per lane)", lambda: synth.banded(5003, 5, 48, seed=14)),
    ("a row of 400", lambda: synth.banded(6007, 6, 600, seed=8, long_rows={3001: 400})),
    ("arrow (dense last row and column)", lambda: synth.banded(1300, 4, 32, seed=9, long_rows={1299: 1299})),
    ("33 rows", lambda: synth.banded(33, 3, 8, seed=10)),
    ("31 rows", lambda: synth.banded(31, 5, 31, seed=11)),
    ("1 row", lambda: synth.banded(1, 0, 1, seed=12)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_row_shapes_match_oracle(silu, ctx, case):
    name, gen = case
    A = gen()
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    Fo = oracle.factor(A, "ilu0", 0.0, 0)
    S = oracle.row_scale(Fo)
    b = synth.rhs(n, 1, seed=21)
    x0 = synth.rhs(n, 1, seed=22) * 0.5
    r = torch.empty(n, 1, dtype=torch.float64, device="cuda")
    M.residual(r, dev(x0), dev(b))
    want_r = oracle.residual(A, x0, b)
    assert relerr(host(r)[:, 0], want_r[:, 0]) < 1e-13
    for variant in (0, 1, 2):
        F = silu.ilu_setup(ctx, M, "ilu0")
        F.set_kernel(variant)
        for mL, mU in [(1, 1), (2, 3), (5, 5), (10, 10)]:
            for start in (x0, np.zeros_like(x0)):
                x = dev(start.copy())
                silu.ilu_smooth(F, x, dev(b), mL, mU)
                ctx.check()
                got = host(x)[:, 0]
                want = oracle.smooth(A, S, start, b, mL, mU)[:, 0]
                assert relerr(got, want) < 1e-12, (name, variant, mL, mU)
                assert maxabs_err(got, want) < 1e-12, (name, variant, mL, mU)
    F32 = silu.ilu_setup(ctx, M, "ilu0", prec=silu.FP32)
    x = dev(x0.copy())
    silu.ilu_smooth(F32, x, dev(b), 4, 4)
    ctx.check()
    assert relerr(host(x)[:, 0], oracle.smooth(A, S, x0, b, 4, 4)[:, 0]) < 1e-5, name
    F = silu.ilu_setup(ctx, M, "ilu0")
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, xs, dev(b[:, 0].copy()), tol=1e-10, restart=30, maxit=400, sweeps_L=4,
                                     sweeps_U=4)
    assert st == silu.OK and rel <= 1e-10, (name, st, its, rel)
    res = oracle.residual(A, host(xs).reshape(n, 1), b)
    assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(b), name
