"""The fused smoother application (one cooperative launch with grid-wide
barriers between the steps of Alg. ILUJac) against the CPU oracle and
against the launch-per-sweep path: FP64 results equal the oracle to 1e-12
and, with one right-hand side, the launch-per-sweep path bit for bit (same
steps, same per-row summation order as its staged kernels); FP32 factors stay within single-precision rounding of the
launch-per-sweep path.  Sizes are ragged (rows not a multiple of the 256-row
blocks) and span many blocks; every branch of the step sequence (no lower
sweep, one, several; no upper factor, one upper term, several; row and
row/column scaling; zero and non-zero initial guess) is exercised."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import maxabs_err, relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SWEEPS = [(5, 5), (0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 3), (3, 1), (1, 4), (7, 2)]


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
    ("poisson32 ilu0 R4", lambda: synth.poisson7(32), "ilu0", 0.0, 0, 4),
    ("cutcell 29x23x17 ilut R1", lambda: synth.cutcell7(29, 23, 17, seed=2), "ilut", 1e-3, 10, 1),
    ("hex27 17x15x13 ilu0 R2", lambda: synth.hex27(17, 15, 13, seed=3), "ilu0", 0.0, 0, 2),
    ("cutcell 21x19x17 iluk1 R3", lambda: synth.cutcell7(21, 19, 17, seed=4), "iluk", 0.0, 1, 3),
]


@pytest.mark.parametrize("scale", ["row", "rowcol"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fused_fp64_matches_oracle_and_unfused_bits(silu, ctx, case, scale):
    name, gen, kind, tau, fill, nrhs = case
    A = gen()
    n = len(A[0]) - 1
    sc = silu.SCALE_ROW if scale == "row" else silu.SCALE_ROWCOL
    M = silu.Matrix(ctx, *A)
    Ff = silu.ilu_setup(ctx, M, kind, tau, fill, scale=sc)
    Fu = silu.ilu_setup(ctx, M, kind, tau, fill, scale=sc)
    Ff.set_fused(2)
    Fu.set_fused(1)
    Fo = oracle.factor(A, kind, tau, fill)
    S = oracle.row_scale(Fo) if scale == "row" else oracle.ruiz_rowcol(Fo)
    smooth = oracle.smooth if scale == "row" else oracle.smooth_rowcol
    b = synth.rhs(n, nrhs, seed=31)
    x0 = synth.rhs(n, nrhs, seed=32) * 0.25
    for mL, mU in SWEEPS:
        xf = dev(x0.copy())
        xu = dev(x0.copy())
        silu.ilu_smooth(Ff, xf, dev(b), mL, mU)
        silu.ilu_smooth(Fu, xu, dev(b), mL, mU)
        ctx.check()
        gf, gu = host(xf), host(xu)
        if nrhs == 1:
            # the unfused path runs the staged kernels, whose rows sum in the same order
            assert np.array_equal(gf, gu), (mL, mU)
        want = smooth(A, S, x0, b, mL, mU)
        for k in range(nrhs):
            assert relerr(gf[:, k], gu[:, k]) < 1e-14, (mL, mU, k)
            assert relerr(gf[:, k], want[:, k]) < 1e-12, (mL, mU, k)
            assert maxabs_err(gf[:, k], want[:, k]) < 1e-12, (mL, mU, k)


def test_fused_fp32_and_inside_fgmres(silu, ctx):
    """FP32 factors: the fused application stays within FP32 rounding of the
    launch-per-sweep one; FGMRES with the fused smoother (captured in its
    iteration graphs, from a zero guess) equals the unfused FGMRES in FP64
    bit for bit and converges with FP32 factors."""
    A = synth.cutcell7(33, 31, 19, seed=5)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    b = synth.rhs(n, 2, seed=7)
    Ff = silu.ilu_setup(ctx, M, "ilu0", prec=silu.FP32)
    Fu = silu.ilu_setup(ctx, M, "ilu0", prec=silu.FP32)
    Ff.set_fused(2)
    Fu.set_fused(1)
    for mL, mU in [(3, 3), (5, 5), (1, 2), (2, 1)]:
        xf = torch.zeros(n, 2, dtype=torch.float64, device="cuda")
        xu = torch.zeros_like(xf)
        silu.ilu_smooth(Ff, xf, dev(b), mL, mU)
        silu.ilu_smooth(Fu, xu, dev(b), mL, mU)
        ctx.check()
        assert relerr(host(xf), host(xu)) < 1e-6, (mL, mU)
    bv = dev(b[:, 0].copy())
    for prec in (silu.FP64, silu.FP32):
        res = []
        for mode in (2, 1):
            F = silu.ilu_setup(ctx, M, "ilu0", prec=prec)
            F.set_fused(mode)
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            st, its, rel = silu.fgmres_solve(F, x, bv, tol=1e-9, restart=30, maxit=3000, sweeps_L=4, sweeps_U=4)
            ctx.check()
            assert st == silu.OK and rel <= 1e-9, (prec, mode, st, its, rel)
            res.append((its, host(x)))
        if prec == silu.FP64:
            assert res[0][0] == res[1][0] and np.array_equal(res[0][1], res[1][1])
        else:
            assert abs(res[0][0] - res[1][0]) <= 2


def test_fused_large_grid_matches_unfused(silu, ctx):
    """Forced onto a system larger than the automatic bound (several rows per
    thread in the grid-stride loops), the fused application still equals the
    launch-per-sweep one bit for bit."""
    A = synth.cutcell7(97, 89, 31, seed=9)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    Ff = silu.ilu_setup(ctx, M, "ilut", 1e-3, 10)
    Fu = silu.ilu_setup(ctx, M, "ilut", 1e-3, 10)
    Ff.set_fused(2)
    Fu.set_fused(1)
    b = dev(synth.rhs(n, 1, seed=3))
    xf = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    xu = torch.zeros_like(xf)
    for _ in range(2):
        silu.ilu_smooth(Ff, xf, b, 6, 6)
        silu.ilu_smooth(Fu, xu, b, 6, 6)
    ctx.check()
    assert np.array_equal(host(xf), host(xu))
