"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

FP64 results must agree to 1e-12 relative (||delta||_2 / ||ref||_2, per
right-hand side); FP32 factors / sweeps report their error against the FP64
oracle and are held to a bound derived from single-precision rounding.
Sizes span many thread blocks and ragged tails (row counts not multiples of
the launch tile)."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import maxabs_err, relerr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


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


def percol_relerr(got, want):
    """Per right-hand side, the larger of the relative 2-norm error and the
    max-abs error over max |ref|; the worst column."""
    got = got.reshape(want.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    return max(max(relerr(got[:, k], want[:, k]), maxabs_err(got[:, k], want[:, k])) for k in range(want.shape[1]))


def oracle_scaled(A, kind, tau, fill):
    F = oracle.factor(A, kind, tau, fill)
    return F, oracle.row_scale(F)


# --------------------------------------------------------------- smoother

SMOOTH_CASES = [
    # name, generator, kind, tau, fill, nrhs, (mL, mU) list
    ("poisson32 ilu0 R4", lambda: synth.poisson7(32), "ilu0", 0.0, 0, 4, [(5, 5), (1, 1), (2, 3), (0, 4), (3, 0)]),
    ("cutcell 37x29x23 ilu0 R1", lambda: synth.cutcell7(37, 29, 23, seed=1), "ilu0", 0.0, 0, 1,
     [(5, 5), (1, 2), (2, 1), (7, 9)]),
    ("cutcell 33x31x17 ilut R3", lambda: synth.cutcell7(33, 31, 17, seed=2), "ilut", 1e-3, 10, 3,
     [(10, 10), (1, 1), (4, 6)]),
    ("hex27 21x19x17 ilu0 R2", lambda: synth.hex27(21, 19, 17, seed=3), "ilu0", 0.0, 0, 2, [(3, 3), (6, 2)]),
    ("cutcell 19x17x13 iluk2 R1", lambda: synth.cutcell7(19, 17, 13, seed=4), "iluk", 0.0, 2, 1, [(4, 4)]),
    ("hex27 13x11x9 ilut R5", lambda: synth.hex27(13, 11, 9, seed=5), "ilut", 1e-3, 12, 5, [(3, 4)]),
]


@pytest.mark.parametrize("variant", [1, 2, 3], ids=["lanes", "staged", "sorted"])
@pytest.mark.parametrize("case", SMOOTH_CASES, ids=[c[0] for c in SMOOTH_CASES])
def test_smooth_fp64_matches_oracle(silu, ctx, case, variant):
    """Both sweep kernels: lanes-per-row (any R) and staged bulk-copy (R = 1;
    with R > 1 the library uses the lanes kernel, covered again), the staged
    kernel also on the length-sorted factor copies where they exist."""
    name, gen, kind, tau, fill, nrhs, sweeps = case
    A = gen()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind, tau, fill)
    F.set_kernel(variant)
    _, S = oracle_scaled(A, kind, tau, fill)
    b = synth.rhs(n, nrhs, seed=11)
    x0 = synth.rhs(n, nrhs, seed=12) * 0.5
    for mL, mU in sweeps:
        want = oracle.smooth(A, S, x0, b, mL, mU)
        x = dev(x0.copy())
        silu.ilu_smooth(F, x, dev(b), mL, mU)
        ctx.check()
        assert percol_relerr(host(x), want) < FP64_TOL, (mL, mU)
    if nrhs > 1:
        # the same columns one at a time go through the staged kernel
        for k in range(nrhs):
            want = oracle.smooth(A, S, x0[:, k:k + 1], b[:, k:k + 1], 3, 2)
            x = dev(x0[:, k:k + 1].copy())
            silu.ilu_smooth(F, x, dev(b[:, k:k + 1].copy()), 3, 2)
            ctx.check()
            assert percol_relerr(host(x), want) < FP64_TOL


@pytest.mark.parametrize("scale", ["none", "rich"])
def test_unscaled_variants_match_oracle(silu, ctx, scale):
    A = synth.cutcell7(24, 22, 20, seed=6)
    n = len(A[0]) - 1
    sc = silu.SCALE_NONE if scale == "none" else silu.SCALE_NONE_RICH
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", 1e-3, 10, scale=sc)
    OF, S = oracle_scaled(A, "ilut", 1e-3, 10)
    b = synth.rhs(n, 1, seed=3)
    # plain Richardson grows by about 1e3 per sweep here (Sec. 6.1's failure),
    # so the iterates stay finite through five sweeps, and rounding stays at
    # the 1e-15 level relative to them: the comparison is unconditional
    for mL, mU in [(3, 1), (3, 2), (2, 3), (2, 5)]:
        r = oracle.residual(A, np.zeros((n, 1)), b)
        y = oracle.richardson_lower(S.L, r, mL)
        if scale == "none":
            v = oracle.upper_jacobi(OF.U, y, mU)
        else:
            v = oracle.upper_unscaled_richardson(OF.U, y, mU)
        assert np.all(np.isfinite(v))
        x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
        silu.ilu_smooth(F, x, dev(b), mL, mU)
        got = host(x)
        assert relerr(got, v) < FP64_TOL, (mL, mU)
        assert maxabs_err(got, v) < FP64_TOL, (mL, mU)


def test_smooth_many_sweeps_equals_direct(silu, ctx):
    """Nilpotence (Sec. 5.2): #levels sweeps on each factor reproduce the
    direct triangular solves, on the device as in the oracle."""
    A = synth.cutcell7(12, 10, 9, seed=7)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    st = F.stats()
    b = dev(synth.rhs(n, 2, seed=5))
    x1 = torch.zeros(n, 2, dtype=torch.float64, device="cuda")
    x2 = torch.zeros_like(x1)
    silu.ilu_smooth(F, x1, b, st["levels_L"], st["levels_U"])
    silu.direct_trisolve(F, x2, b)
    assert relerr(host(x1), host(x2)) < FP64_TOL


DIRECT_CASES = [
    ("poisson32 R4", lambda: synth.poisson7(32), "ilu0", 0.0, 0, 4),
    ("cutcell 29x23x19 ilut R1", lambda: synth.cutcell7(29, 23, 19, seed=8), "ilut", 1e-3, 10, 1),
    ("hex27 15x13x11 ilu0 R3", lambda: synth.hex27(15, 13, 11, seed=9), "ilu0", 0.0, 0, 3),
]


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["auto", "per_level", "persistent"])
@pytest.mark.parametrize("case", DIRECT_CASES, ids=[c[0] for c in DIRECT_CASES])
def test_direct_trisolve_matches_oracle(silu, ctx, case, mode):
    name, gen, kind, tau, fill, nrhs = case
    A = gen()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind, tau, fill)
    F.set_direct(mode)
    _, S = oracle_scaled(A, kind, tau, fill)
    b = synth.rhs(n, nrhs, seed=21)
    x0 = synth.rhs(n, nrhs, seed=22)
    want = oracle.direct_apply(A, S, x0, b)
    x = dev(x0.copy())
    silu.direct_trisolve(F, x, dev(b))
    ctx.check()
    assert percol_relerr(host(x), want) < FP64_TOL


@pytest.mark.parametrize("scale,prec", [("rowcol", "fp64"), ("row", "fp32"), ("none", "fp64")])
def test_persistent_direct_scalings_and_precisions(silu, ctx, scale, prec):
    """Both exact-solve schedules on row/column-scaled factors, on FP32 sweep
    factors (the exact solves use FP64 copies) and on unscaled factors: the
    persistent launch equals the per-level launches to rounding, and, with
    row scaling, the oracle's exact application."""
    A = synth.cutcell7(27, 25, 19, seed=15)
    n = len(A[0]) - 1
    sc = {"rowcol": silu.SCALE_ROWCOL, "row": silu.SCALE_ROW, "none": silu.SCALE_NONE}[scale]
    pr = silu.FP32 if prec == "fp32" else silu.FP64
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", 1e-3, 10, scale=sc, prec=pr)
    b = synth.rhs(n, 2, seed=17)
    x0 = synth.rhs(n, 2, seed=18) * 0.5
    got = {}
    for mode in (2, 1):
        F.set_direct(mode)
        x = dev(x0.copy())
        silu.direct_trisolve(F, x, dev(b))
        ctx.check()
        got[mode] = host(x)
    assert percol_relerr(got[2], got[1]) < 1e-13
    if scale == "row":
        _, S = oracle_scaled(A, "ilut", 1e-3, 10)
        assert percol_relerr(got[2], oracle.direct_apply(A, S, x0, b)) < FP64_TOL


def test_persistent_direct_over_many_solves(silu, ctx):
    """The persistent solve alternates its readiness tag from solve to solve
    and keeps separate tagged vectors per column count: a sequence of solves
    with 1, 2, 4, 1, 3 (= 2 + 1), 4, 1 columns, from x != 0 and from x = 0
    inside FGMRES, each equals the oracle; the per-level schedule of the same
    factors agrees."""
    A = synth.cutcell7(31, 27, 21, seed=14)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", 1e-3, 10)
    F.set_direct(2)
    _, S = oracle_scaled(A, "ilut", 1e-3, 10)
    for k, R in enumerate([1, 2, 4, 1, 3, 4, 1]):
        b = synth.rhs(n, R, seed=40 + k)
        x0 = synth.rhs(n, R, seed=60 + k)
        want = oracle.direct_apply(A, S, x0, b)
        x = dev(x0.copy())
        silu.direct_trisolve(F, x, dev(b))
        ctx.check()
        assert percol_relerr(host(x), want) < FP64_TOL, (k, R)
    bv = synth.rhs(n, 1, seed=3)[:, 0]
    res = {}
    for mode in (2, 1, 2):
        F.set_direct(mode)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, its, rel = silu.fgmres_solve(F, x, dev(bv), tol=1e-10, restart=30, maxit=400, sweeps_L=0, sweeps_U=0,
                                         precond=silu.PRECOND_DIRECT)
        ctx.check()
        assert st == silu.OK and rel <= 1e-10, (mode, st, its, rel)
        res.setdefault(mode, []).append((its, host(x)))
    assert abs(res[2][0][0] - res[1][0][0]) <= 1
    assert relerr(res[2][0][1], res[1][0][1]) < 1e-8
    assert res[2][0][0] == res[2][1][0] and np.array_equal(res[2][0][1], res[2][1][1])


SORTED_CASES = [
    # rows not a multiple of the 512-row sort window; ILUT rows of uneven length
    ("cutcell 33x31x17 ilut", lambda: synth.cutcell7(33, 31, 17, seed=2), "ilut", 1e-3, 10),
    ("cutcell 41x37x23 ilut tight", lambda: synth.cutcell7(41, 37, 23, seed=6), "ilut", 1e-2, 6),
    ("hex27 13x11x9 ilut", lambda: synth.hex27(13, 11, 9, seed=5), "ilut", 1e-3, 12),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", SORTED_CASES, ids=[c[0] for c in SORTED_CASES])
def test_sorted_copy_gives_the_same_bits(silu, ctx, case, prec):
    """The length-sorted factor copy keeps each row's entries in order, so
    the staged kernel on it (variant 3) returns the same bits as on the
    natural order (variant 2), FP64 and FP32; the FP64 result also matches
    the oracle.  The copy is made on first selection, for L_s at least."""
    name, gen, kind, tau, fill = case
    A = gen()
    n = len(A[0]) - 1
    p = silu.FP32 if prec == "fp32" else silu.FP64
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind, tau, fill, prec=p)
    assert not F.layout()["in_use"].any()
    F.set_kernel(3)
    lay = F.layout()
    print(name, "pads natural", lay["pad_natural"], "sorted", lay["pad_sorted"], "in use", lay["in_use"])
    assert lay["in_use"][0], lay
    b = synth.rhs(n, 1, seed=31)
    x0 = synth.rhs(n, 1, seed=32)
    got = {}
    for variant in (2, 3, 0):
        F.set_kernel(variant)
        for mL, mU in [(4, 3), (1, 1), (0, 2)]:
            x = dev(x0.copy())
            silu.ilu_smooth(F, x, dev(b), mL, mU)
            ctx.check()
            got[variant, mL, mU] = host(x)
    for key, val in got.items():
        assert np.array_equal(val, got[(2,) + key[1:]]), key
    if p == silu.FP64:
        _, S = oracle_scaled(A, kind, tau, fill)
        for mL, mU in [(4, 3), (1, 1), (0, 2)]:
            assert relerr(got[3, mL, mU], oracle.smooth(A, S, x0, b, mL, mU)) < FP64_TOL


def test_sorted_copy_follows_refactor(silu, ctx):
    """ilu_refactor re-uploads the factors with their sorted copies (the
    27-point ILU(0) factors of a thin lattice have many short boundary rows)
    and keeps the chosen variant; results match the oracle's factors of the
    new values."""
    A = synth.hex27(9, 7, 30, seed=3)
    A2 = synth.hex27(9, 7, 30, seed=8)
    assert np.array_equal(A[1], A2[1])
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.set_kernel(3)
    assert F.layout()["in_use"].all()
    silu.ilu_refactor(F, A2[2])
    assert F.layout()["in_use"].all()
    _, S = oracle_scaled(A2, "ilu0", 0.0, 0)
    b = synth.rhs(n, 1, seed=5)
    x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    silu.ilu_smooth(F, x, dev(b), 5, 5)
    ctx.check()
    assert relerr(host(x), oracle.smooth(A2, S, np.zeros((n, 1)), b, 5, 5)) < FP64_TOL


def test_fp32_error_against_fp64_oracle(silu, ctx):
    """FP32 factors and sweeps: the error against the FP64 oracle is a number
    (printed), bounded by single-precision rounding: each sweep perturbs the
    iterate by a few units of 2^-24 relative, so 3+3 sweeps stay well below 1e-5."""
    A = synth.cutcell7(40, 36, 30, seed=10)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=silu.FP32)
    _, S = oracle_scaled(A, "ilu0", 0.0, 0)
    b = synth.rhs(n, 1, seed=1)
    for variant in (1, 2):
        F.set_kernel(variant)
        for mL, mU in [(3, 3), (5, 5), (1, 1)]:
            want = oracle.smooth(A, S, np.zeros((n, 1)), b, mL, mU)
            x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
            silu.ilu_smooth(F, x, dev(b), mL, mU)
            ctx.check()
            err = relerr(host(x), want)
            print(f"FP32 smoother kernel {variant} ({mL},{mU}) relative error vs FP64 oracle: {err:.3e}")
            assert err < 1e-5


def test_fgmres_matches_oracle(silu, ctx):
    """Same iteration count (to rounding) and both iterates below tol in true
    relative residual.  The unpreconditioned case uses a matrix without cut
    cells: on the cut-cell matrix plain GMRES(30) does not converge at all."""
    cases = (
        (silu.PRECOND_SWEEPS, (3, 3), lambda: synth.cutcell7(20, 18, 16, seed=11)),
        (silu.PRECOND_DIRECT, (0, 0), lambda: synth.cutcell7(20, 18, 16, seed=11)),
        (silu.PRECOND_NONE, (0, 0), lambda: synth.cutcell7(12, 11, 10, seed=11, sigma=0.3, frac_cut=0.0)),
    )
    for precond, (mL, mU), gen in cases:
        A = gen()
        n = len(A[0]) - 1
        F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
        _, S = oracle_scaled(A, "ilu0", 0.0, 0)
        b = synth.rhs(n, 1, seed=2)[:, 0]
        xo, sto, itso, relo = oracle.fgmres(A, S if precond != 2 else None, b, tol=1e-10, restart=30,
                                            maxit=3000, mL=mL, mU=mU, precond=precond)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, its, rel = silu.fgmres_solve(F, x, dev(b), tol=1e-10, restart=30, maxit=3000, sweeps_L=mL,
                                         sweeps_U=mU, precond=precond)
        assert st == silu.OK and sto == oracle.OK, (precond, st, sto, its, itso)
        assert rel <= 1e-10 and relo <= 1e-10
        assert abs(its - itso) <= 1 + itso // 20, (its, itso)
        r = oracle.residual(A, host(x).reshape(n, 1), b.reshape(n, 1))
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


def test_fgmres_stopping_edges(silu, ctx):
    """The device runs one inner iteration ahead of the host's stopping test:
    stopping on maxit inside a cycle, on maxit at a restart and on an exact
    (happy-breakdown) iteration must still return the iterate of exactly the
    iterations counted -- the oracle's FGMRES after the same number of
    iterations -- and a queued extra iteration must leave no trace."""
    A = synth.cutcell7(17, 15, 13, seed=21)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    _, S = oracle_scaled(A, "ilu0", 0.0, 0)
    b = synth.rhs(n, 1, seed=22)[:, 0]
    for maxit in (0, 1, 2, 7, 10, 11):
        xo, sto, itso, relo = oracle.fgmres(A, S, b, tol=1e-14, restart=10, maxit=maxit, mL=3, mU=3, precond=0)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, its, rel = silu.fgmres_solve(F, x, dev(b), tol=1e-14, restart=10, maxit=maxit, sweeps_L=3, sweeps_U=3)
        assert st == silu.ERR_NOT_CONVERGED and sto == oracle.NOT_CONVERGED
        assert its == itso == maxit
        if maxit:
            assert relerr(host(x), xo) < 1e-9, maxit
            assert abs(rel - relo) <= 1e-9 * relo
        else:
            assert not host(x).any()
    # diagonal system: ILU(0) is exact, the first iteration ends the solve with h_{1,0} = 0
    d = 1.0 + np.arange(64, dtype=np.float64)
    D = (np.arange(65, dtype=np.int64), np.arange(64, dtype=np.int32), d)
    FD = silu.ilu_setup(ctx, silu.Matrix(ctx, *D), "ilu0")
    bd = synth.rhs(64, 1, seed=23)[:, 0]
    for _ in range(2):  # the second solve reuses the captured iterations and whatever the first left behind
        x = torch.zeros(64, dtype=torch.float64, device="cuda")
        st, its, rel = silu.fgmres_solve(FD, x, dev(bd), tol=1e-12, restart=10, maxit=50, sweeps_L=1, sweeps_U=1)
        assert st == silu.OK and its == 1 and rel <= 1e-12
        assert relerr(host(x), bd / d) < 1e-14


def test_fgmres_fp32_smoother_reaches_fp64_tolerance(silu, ctx):
    A = synth.hex27(24, 22, 20, seed=12)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=silu.FP32)
    b = synth.rhs(n, 1, seed=3)[:, 0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, x, dev(b), tol=1e-10, restart=30, maxit=500, sweeps_L=3, sweeps_U=3)
    assert st == silu.OK and rel <= 1e-10
    r = oracle.residual(A, host(x).reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


def test_edge_cases(silu, ctx):
    # 1x1 system
    A1 = (np.array([0, 1], np.int64), np.array([0], np.int32), np.array([4.0]))
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A1), "ilu0")
    x = torch.zeros(1, 1, dtype=torch.float64, device="cuda")
    silu.ilu_smooth(F, x, dev(np.array([[2.0]])), 3, 3)
    assert host(x)[0, 0] == 0.5
    silu.direct_trisolve(F, x, dev(np.array([[2.0]])))
    assert host(x)[0, 0] == 0.5
    # empty system
    A0 = (np.array([0], np.int64), np.zeros(0, np.int32), np.zeros(0))
    F0 = silu.ilu_setup(ctx, silu.Matrix(ctx, *A0), "ilu0")
    assert F0.stats()["n"] == 0
    # bad arguments are rejected before any launch
    A = synth.poisson7(5)
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    xb = torch.zeros(125, 1, dtype=torch.float64, device="cuda")
    with pytest.raises(silu.SiluError):
        silu.ilu_smooth(F, xb, xb, -1, 2)
    with pytest.raises(silu.SiluError):
        silu.ilu_smooth(F, xb.float(), xb, 1, 2)
    assert silu.load().ilu_smooth(F.handle, 0, xb.data_ptr(), 1, 1, 1) == silu.ERR_INVALID_ARG


def test_fp32_27pt_error_and_staged_lanes(silu, ctx):
    """27-point rows (27 entries in A, 13 in each factor): the staged kernel runs
    A with two lanes per row.  FP64 residual parity and the FP32 smoother's
    error against the FP64 oracle (printed)."""
    A = synth.hex27(40, 36, 30, seed=4)
    n = len(A[0]) - 1
    _, S = oracle_scaled(A, "ilu0", 0.0, 0)
    b = synth.rhs(n, 1, seed=9)
    x0 = synth.rhs(n, 1, seed=10)
    F64 = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    for variant in (1, 2):
        F64.set_kernel(variant)
        want = oracle.smooth(A, S, x0, b, 3, 3)
        x = dev(x0.copy())
        silu.ilu_smooth(F64, x, dev(b), 3, 3)
        ctx.check()
        assert relerr(host(x), want) < FP64_TOL
    F32 = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=silu.FP32)
    want = oracle.smooth(A, S, np.zeros((n, 1)), b, 3, 3)
    x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    silu.ilu_smooth(F32, x, dev(b), 3, 3)
    ctx.check()
    err = relerr(host(x), want)
    print(f"27-point FP32 smoother (3,3) relative error vs FP64 oracle: {err:.3e}")
    assert err < 1e-5


def test_bounded_wait_reports_timeout_and_context_survives(silu, ctx):
    """Failure detection without a fault: a GPU wait on a flag that nothing
    sets gives up after its limit and records the timeout; the host reads
    ERR_TIMEOUT, the error word is cleared, and the context keeps working."""
    ctx.check()
    ctx.selftest_timeout(50)
    with pytest.raises(silu.SiluError) as e:
        ctx.check()
    assert e.value.status == silu.ERR_TIMEOUT
    ctx.check()  # cleared
    A = synth.cutcell7(12, seed=5)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    _, S = oracle_scaled(A, "ilu0", 0.0, 0)
    b = synth.rhs(n, 1, seed=6)
    x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    silu.ilu_smooth(F, x, dev(b), 2, 2)
    ctx.check()
    assert relerr(host(x), oracle.smooth(A, S, np.zeros((n, 1)), b, 2, 2)) < FP64_TOL


def test_sweep_overlap_gives_the_same_bits(silu):
    """Programmatic dependent launch of consecutive sweeps and levels (the
    default) only moves each kernel's first factor copies or row pointers
    ahead of the previous kernel's completion: smoother, FGMRES and direct
    results (graphs included) are the same bits with it off, and match the
    oracle."""
    A = synth.cutcell7(44, 40, 36, seed=12)
    n = len(A[0]) - 1
    b = synth.rhs(n, 1, seed=13)
    x0 = synth.rhs(n, 1, seed=14)
    out = {}
    for overlap in (True, False):
        c = silu.Context(0, torch.cuda.current_stream())
        c.set_overlap(overlap)
        F = silu.ilu_setup(c, silu.Matrix(c, *A), "ilut", 1e-3, 10)
        x = dev(x0.copy())
        silu.ilu_smooth(F, x, dev(b), 6, 5)
        c.check()
        xs = host(x)
        xf = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, its, rel = silu.fgmres_solve(F, xf, dev(b[:, 0].copy()), tol=1e-9, restart=20, maxit=400,
                                         sweeps_L=3, sweeps_U=3, precond=silu.PRECOND_SWEEPS)
        assert st == silu.OK
        xd = dev(x0.copy())
        silu.direct_trisolve(F, xd, dev(b))
        c.check()
        out[overlap] = (xs, host(xf), its, host(xd))
    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1]) and out[True][2] == out[False][2]
    assert np.array_equal(out[True][3], out[False][3])
    _, S = oracle_scaled(A, "ilut", 1e-3, 10)
    assert relerr(out[True][0], oracle.smooth(A, S, x0, b, 6, 5)) < FP64_TOL
    assert relerr(out[True][3], oracle.direct_apply(A, S, x0, b)) < FP64_TOL


def test_profile_records_sweep_runs(silu):
    """Profiling counts every launch; the L sweeps (and the U sweeps) of one
    application are timed as one run, so each class reports its launches
    and a positive total time."""
    c = silu.Context(0, torch.cuda.current_stream())
    A = synth.cutcell7(30, 28, 26, seed=2)
    n = len(A[0]) - 1
    F = silu.ilu_setup(c, silu.Matrix(c, *A), "ilut", 1e-3, 10)
    b = dev(synth.rhs(n, 1, seed=3))
    x = dev(synth.rhs(n, 1, seed=4))
    silu.ilu_smooth(F, x, b, 4, 5)
    torch.cuda.synchronize()
    l0 = c.launch_count()
    c.profile(True)
    for _ in range(3):
        silu.ilu_smooth(F, x, b, 4, 5)
    c.profile(False)
    prof = c.profile_read()
    assert c.launch_count() - l0 == 3 * (1 + 3 + 4)
    assert prof["residual"][0] == 3 and prof["sweep_L"][0] == 9 and prof["sweep_U"][0] == 12
    assert all(prof[k][1] > 0 for k in ("residual", "sweep_L", "sweep_U"))


def test_l2_reuse_settings_give_the_same_bits(silu):
    """Alternating the direction of consecutive sweeps and the L2 priorities
    of factor and vector accesses changes only which warp takes a row tile and
    how long lines stay in L2: smoother (FP64 and FP32 factors, natural and
    length-sorted layouts) and FGMRES results are the same bits for every
    setting, and the FP64 smoother matches the oracle."""
    A = synth.cutcell7(44, 40, 36, seed=12)
    n = len(A[0]) - 1
    b = synth.rhs(n, 1, seed=13)
    x0 = synth.rhs(n, 1, seed=14)
    OF = oracle.ilut(A, 1e-3, 10)
    want = oracle.smooth(A, oracle.row_scale(OF), x0, b, 7, 6)
    out = {}
    for flags in (0, 1, 3, 5, 7):
        c = silu.Context(0, torch.cuda.current_stream())
        c.set_l2_reuse(flags)
        got = []
        for prec in (silu.FP64, silu.FP32):
            F = silu.ilu_setup(c, silu.Matrix(c, *A), "ilut", 1e-3, 10, prec=prec)
            for variant in (2, 3):
                F.set_kernel(variant)
                x = dev(x0.copy())
                silu.ilu_smooth(F, x, dev(b), 7, 6)
                silu.ilu_smooth(F, x, dev(b), 4, 3)
                c.check()
                got.append(host(x))
            xf = torch.zeros(n, dtype=torch.float64, device="cuda")
            st, its, _ = silu.fgmres_solve(F, xf, dev(b[:, 0].copy()), tol=1e-9, restart=20, maxit=400,
                                           sweeps_L=3, sweeps_U=4, precond=silu.PRECOND_SWEEPS)
            assert st == silu.OK
            got.append((host(xf), its))
        out[flags] = got
        x = dev(x0.copy())
        F = silu.ilu_setup(c, silu.Matrix(c, *A), "ilut", 1e-3, 10)
        silu.ilu_smooth(F, x, dev(b), 7, 6)
        assert relerr(host(x), want) < 1e-12
    for flags in (1, 3, 5, 7):
        for a, r in zip(out[flags], out[0]):
            if isinstance(a, tuple):
                assert np.array_equal(a[0], r[0]) and a[1] == r[1], flags
            else:
                assert np.array_equal(a, r), flags
    with pytest.raises(silu.SiluError):
        silu.Context(0, torch.cuda.current_stream()).set_l2_reuse(8)
