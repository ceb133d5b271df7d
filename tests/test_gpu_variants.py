"""GPU parity of the smoother variants against the CPU oracle.

Polynomial Gauss-Seidel (Sec. 3.1), against the oracle's term-by-term Neumann
sums: on the device these are the row-scaled Richardson sweeps on the
Gauss-Seidel splitting written as factors (L_s = L_A D^{-1},
Utilde_s = D^{-1} U_A), so sweeps_L = p + 1 gives p + 1 Neumann terms.

Row/column scaling (Eq. rowcolScale): Richardson on Uhat = D_r U D_c and the
final x += D_c w, against the oracle's smoother on its own Ruiz factors.

FP64 to 1e-12 relative per right-hand side; FP32 factors report their error
against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import relerr

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


def percol(got, want):
    got = got.reshape(want.shape[0], -1)
    return max(relerr(got[:, k], want[:, k]) for k in range(want.shape[1]))


CASES = [
    ("cutcell 37x29x23 R1", lambda: synth.cutcell7(37, 29, 23, seed=1), 1),
    ("hex27 21x19x17 R3", lambda: synth.hex27(21, 19, 17, seed=3), 3),
    ("poisson 33x17x9 R2", lambda: synth.poisson7(33, 17, 9), 2),
]


@pytest.mark.parametrize("variant", [1, 2], ids=["lanes", "staged"])
@pytest.mark.parametrize("kind", ["gs", "sgs"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_poly_gs_matches_oracle(silu, ctx, case, kind, variant):
    name, gen, nrhs = case
    A = gen()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind)
    F.set_kernel(variant)
    b = synth.rhs(n, nrhs, seed=31)
    x0 = synth.rhs(n, nrhs, seed=32) * 0.25
    sym = kind == "sgs"
    for p, q in [(0, 0), (1, 0), (2, 2), (5, 3), (9, 9)]:
        want = oracle.poly_gs_smooth(A, x0, b, p, q, symmetric=sym)
        x = dev(x0.copy())
        silu.ilu_smooth(F, x, dev(b), p + 1, (q + 1) if sym else 1)
        ctx.check()
        assert percol(host(x), want) < FP64_TOL, (p, q)


@pytest.mark.parametrize("kind", ["gs", "sgs"])
def test_direct_gauss_seidel_is_exact_sweep(silu, ctx, kind):
    """direct_trisolve on the GS factors is one exact (symmetric) Gauss-Seidel
    step: the oracle's series with every term (p = #levels - 1 suffices)."""
    A = synth.cutcell7(29, 23, 19, seed=8)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind)
    st = F.stats()
    assert st["levels_L"] == 29 + 23 + 19 - 2
    b = synth.rhs(n, 1, seed=5)
    x0 = synth.rhs(n, 1, seed=6)
    want = oracle.poly_gs_smooth(A, x0, b, st["levels_L"] - 1, st["levels_U"] - 1, symmetric=(kind == "sgs"))
    x = dev(x0.copy())
    silu.direct_trisolve(F, x, dev(b))
    assert percol(host(x), want) < FP64_TOL


def test_poly_gs_fp32_error_and_fgmres(silu, ctx):
    """FP32 GS factors: error of one application against the FP64 oracle (a
    number, printed), and FGMRES(30) preconditioned by 3-term symmetric
    polynomial GS still reaches 1e-10 in FP64."""
    A = synth.cutcell7(40, 36, 30, seed=10)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "sgs", prec=silu.FP32)
    b = synth.rhs(n, 1, seed=1)
    want = oracle.poly_gs_smooth(A, np.zeros((n, 1)), b, 2, 2, symmetric=True)
    x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    silu.ilu_smooth(F, x, dev(b), 3, 3)
    err = relerr(host(x), want)
    print(f"FP32 symmetric polynomial GS (3+3 terms) relative error vs FP64 oracle: {err:.3e}")
    assert err < 1e-5
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, xs, dev(b[:, 0].copy()), tol=1e-10, restart=30, maxit=3000, sweeps_L=3,
                                     sweeps_U=3)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)
    r = oracle.residual(A, host(xs).reshape(n, 1), b)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


ROWCOL_CASES = [
    ("cutcell 37x29x23 ilu0 R1", lambda: synth.cutcell7(37, 29, 23, seed=1), "ilu0", 0.0, 0, 1),
    ("cutcell 33x31x17 ilut R2", lambda: synth.cutcell7(33, 31, 17, seed=2), "ilut", 1e-3, 10, 2),
    ("hex27 21x19x17 ilu0 R1", lambda: synth.hex27(21, 19, 17, seed=3), "ilu0", 0.0, 0, 1),
]


@pytest.mark.parametrize("variant", [1, 2], ids=["lanes", "staged"])
@pytest.mark.parametrize("case", ROWCOL_CASES, ids=[c[0] for c in ROWCOL_CASES])
def test_rowcol_smoother_matches_oracle(silu, ctx, case, variant):
    name, gen, kind, tau, fill, nrhs = case
    A = gen()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind, tau, fill, scale=silu.SCALE_ROWCOL)
    F.set_kernel(variant)
    RC = oracle.ruiz_rowcol(oracle.factor(A, kind, tau, fill), maxit=20, tol=1e-2)
    b = synth.rhs(n, nrhs, seed=41)
    x0 = synth.rhs(n, nrhs, seed=42) * 0.5
    for mL, mU in [(5, 5), (1, 1), (3, 1), (0, 4), (2, 0), (10, 10)]:
        want = oracle.smooth_rowcol(A, RC, x0, b, mL, mU)
        x = dev(x0.copy())
        silu.ilu_smooth(F, x, dev(b), mL, mU)
        ctx.check()
        assert percol(host(x), want) < FP64_TOL, (mL, mU)
        xz = torch.zeros(n, nrhs, dtype=torch.float64, device="cuda")
        silu.ilu_smooth(F, xz, dev(b), mL, mU)
        assert percol(host(xz), oracle.smooth_rowcol(A, RC, np.zeros_like(x0), b, mL, mU)) < FP64_TOL
    # the exact solve with row/column scaled factors is the exact ILU application
    S = oracle.row_scale(oracle.factor(A, kind, tau, fill))
    xd = dev(x0.copy())
    silu.direct_trisolve(F, xd, dev(b))
    assert percol(host(xd), oracle.direct_apply(A, S, x0, b)) < FP64_TOL


def test_rowcol_fp32_and_fgmres(silu, ctx):
    """FP32 row/column-scaled factors: error against the FP64 oracle (a number,
    printed) and FGMRES(30) to 1e-10 with 3+3 FP32 sweeps."""
    A = synth.cutcell7(40, 36, 30, seed=10)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", scale=silu.SCALE_ROWCOL, prec=silu.FP32)
    RC = oracle.ruiz_rowcol(oracle.ilu0(A), maxit=20, tol=1e-2)
    b = synth.rhs(n, 1, seed=1)
    want = oracle.smooth_rowcol(A, RC, np.zeros((n, 1)), b, 3, 3)
    x = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    silu.ilu_smooth(F, x, dev(b), 3, 3)
    err = relerr(host(x), want)
    print(f"FP32 row/column-scaled smoother (3+3) relative error vs FP64 oracle: {err:.3e}")
    assert err < 1e-5
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, xs, dev(b[:, 0].copy()), tol=1e-10, restart=30, maxit=3000, sweeps_L=3,
                                     sweeps_U=3)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)


@pytest.mark.parametrize("which,kind,scale", [("U", "ilut", "row"), ("U", "ilut", "rowcol"), ("L", "ilu0", "row"),
                                              ("U", "iluk", "row")])
def test_power_norms_match_oracle(silu, ctx, which, kind, scale):
    """||T^p||_2 estimates (Sec. 5.2, Fig. Up): the device's power iteration
    against the oracle's from the same start vector and iteration count; and
    exactly zero from p = #levels on (nilpotence)."""
    A = synth.cutcell7(14, 12, 11, seed=5)
    n = len(A[0]) - 1
    tau, fill = {"ilut": (1e-4, 10), "ilu0": (0.0, 0), "iluk": (0.0, 1)}[kind]
    sc = silu.SCALE_ROWCOL if scale == "rowcol" else silu.SCALE_ROW
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind, tau, fill, scale=sc)
    OF = oracle.factor(A, kind, tau, fill)
    if scale == "rowcol":
        T = oracle.ruiz_rowcol(OF, maxit=20, tol=1e-2).Us
    else:
        S = oracle.row_scale(OF)
        T = S.L if which == "L" else S.Us
    v0 = synth.rhs(n, 1, seed=9)[:, 0]
    pmax, iters = 12, 25
    got = F.power_norms(which, pmax, iters, v0)
    want = oracle.power_norms(T, pmax, iters, v0)
    for p in range(pmax):
        if want[p] == 0.0:
            assert got[p] == 0.0
        else:
            assert abs(got[p] - want[p]) <= 1e-10 * want[p], (p, got[p], want[p])
    # a 4 x 3 grid's ILU(0) upper factor has 4 + 3 + 1 - 2 = 6 levels: T^5 v != 0, T^6 = 0
    B = synth.poisson7(4, 3, 1)
    G = silu.ilu_setup(ctx, silu.Matrix(ctx, *B), "ilu0")
    assert G.stats()["levels_U"] == 6
    z = G.power_norms("U", 7, 3, synth.rhs(12, 1, seed=1)[:, 0])
    assert np.all(z[:5] > 0.0) and np.all(z[5:] == 0.0)


@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_mat_residual_matches_oracle(silu, ctx, nrhs):
    """silu_mat_residual: r = b - A x on the device, the residual step of the
    smoother (Eq. ILUsplit), against the oracle's (column blocks of up to four
    right-hand sides, and the staged kernel for one)."""
    A = synth.hex27(23, 19, 17, seed=4)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    x = synth.rhs(n, nrhs, seed=2)
    b = synth.rhs(n, nrhs, seed=3)
    r = torch.empty(n, nrhs, dtype=torch.float64, device="cuda")
    M.residual(r, dev(x), dev(b))
    assert percol(host(r), oracle.residual(A, x, b)) < FP64_TOL


def test_matrix_launch_shapes(silu, ctx):
    """silu_mat_set_shape: every launch shape of the staged kernel on A gives
    the residual to FP64 parity, and captured FGMRES iterations on A are
    rebuilt after a change (same iteration count, converged)."""
    A = synth.hex27(19, 17, 15, seed=7)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    F = silu.ilu_setup(ctx, M, "ilu0")
    x = synth.rhs(n, 1, seed=2)
    b = synth.rhs(n, 1, seed=3)
    want = oracle.residual(A, x, b)
    bd = dev(b[:, 0].copy())
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    st0, its0, _ = silu.fgmres_solve(F, xs, bd, tol=1e-10, restart=30, maxit=500, sweeps_L=3, sweeps_U=3)
    for lanes, passes, chunk in [(1, 1, 16), (1, 2, 8), (2, 1, 16), (4, 1, 8), (0, 0, 16)]:
        M.set_shape(lanes, passes, chunk)
        r = torch.empty(n, 1, dtype=torch.float64, device="cuda")
        M.residual(r, dev(x), dev(b))
        assert percol(host(r), want) < FP64_TOL, (lanes, passes, chunk)
        xs.zero_()
        st, its, rel = silu.fgmres_solve(F, xs, bd, tol=1e-10, restart=30, maxit=500, sweeps_L=3, sweeps_U=3)
        assert st == silu.OK and rel <= 1e-10 and abs(its - its0) <= 1


def test_matrix_narrow_configuration(silu, ctx):
    """The narrow configuration (gather width 10: shorter tiles, 24 warps per
    block) on a 7-point matrix gives the residual of the default one-lane
    shape bit for bit (each row sums in column order in both), and matches
    the oracle; a 27-point matrix, whose rows do not fit it, is refused with
    SILU_ERR_INVALID_ARG and keeps its shape."""
    A = synth.cutcell7(37, 29, 23, seed=6)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    x = synth.rhs(n, 1, seed=4)
    b = synth.rhs(n, 1, seed=5)
    res = {}
    for chunk in (10, 16, 0):
        M.set_shape(1, 1, chunk)
        r = torch.empty(n, 1, dtype=torch.float64, device="cuda")
        M.residual(r, dev(x), dev(b))
        res[chunk] = host(r)
    assert np.array_equal(res[10], res[16]) and np.array_equal(res[0], res[10])
    assert percol(res[10], oracle.residual(A, x, b)) < FP64_TOL
    H = synth.hex27(13, 11, 9, seed=6)
    MH = silu.Matrix(ctx, *H)
    with pytest.raises(silu.SiluError) as ei:
        MH.set_shape(1, 1, 10)
    assert ei.value.status == silu.ERR_INVALID_ARG
    nh = len(H[0]) - 1
    xh, bh = synth.rhs(nh, 1, seed=4), synth.rhs(nh, 1, seed=5)
    r = torch.empty(nh, 1, dtype=torch.float64, device="cuda")
    MH.residual(r, dev(xh), dev(bh))
    assert percol(host(r), oracle.residual(H, xh, bh)) < FP64_TOL


def test_matrix_autotune_keeps_a_valid_fastest_shape(silu, ctx):
    """silu_mat_autotune: the shape it keeps is one it timed, the residual
    with it matches the oracle to FP64 parity, FGMRES on A still converges,
    and an empty matrix keeps the automatic shape."""
    for A in (synth.hex27(21, 18, 16, seed=8), synth.cutcell7(33, 29, 25, seed=8)):
        n = len(A[0]) - 1
        M = silu.Matrix(ctx, *A)
        F = silu.ilu_setup(ctx, M, "ilu0")
        (lanes, passes, chunk), ms = M.autotune()
        assert lanes in (1, 2, 4) and passes in (1, 2, 4) and chunk in (8, 10, 16) and ms > 0
        assert chunk != 10 or (lanes == 1 and passes == 1)
        assert lanes == 1 or passes == 1
        x = synth.rhs(n, 1, seed=2)
        b = synth.rhs(n, 1, seed=3)
        r = torch.empty(n, 1, dtype=torch.float64, device="cuda")
        M.residual(r, dev(x), dev(b))
        assert percol(host(r), oracle.residual(A, x, b)) < FP64_TOL
        xs = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, its, rel = silu.fgmres_solve(F, xs, dev(b[:, 0].copy()), tol=1e-10, restart=30, maxit=800,
                                         sweeps_L=3, sweeps_U=3)
        assert st == silu.OK and rel <= 1e-10
    E = silu.Matrix(ctx, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert E.autotune()[1] == 0.0


def test_loaded_factors_smooth_like_the_originals(silu, ctx, tmp_path):
    """Factors written by silu_ilu_save and read back by silu_ilu_load on a
    device context give the same bits in the smoother and the direct solve."""
    A = synth.cutcell7(31, 27, 23, seed=9)
    n = len(A[0]) - 1
    M = silu.Matrix(ctx, *A)
    F = silu.ilu_setup(ctx, M, "ilut", 1e-3, 10, prec=silu.FP32)
    path = str(tmp_path / "f.silu")
    F.save(path)
    G = silu.ILU.load_file(M, path)
    b = dev(synth.rhs(n, 1, seed=4))
    for fn in (lambda H, x: silu.ilu_smooth(H, x, b, 4, 4), lambda H, x: silu.direct_trisolve(H, x, b)):
        x1 = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
        x2 = torch.zeros_like(x1)
        fn(F, x1)
        fn(G, x2)
        assert torch.equal(x1, x2)
