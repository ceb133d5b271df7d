"""GPU parity of the AMG V-cycle (Sec. 3, Alg. mgcycle) against the oracle's,
and FGMRES preconditioned by it.

The hierarchy is the same on both sides bit for bit (host setup, checked in
tests/test_host_setup.py); the cycle's kernels (ILU sweeps on the finest
level, l1-Jacobi, restriction, prolongation, dense coarsest solve) are
compared at 1e-12 relative (the coarsest operators here have condition
numbers below 20, so the library's explicit inverse and the oracle's
elimination agree far below that)."""
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
    # name, generator, kind, tau, fill, theta, coarse_size, nu, (mL, mU), tolerance
    ("poisson 21x19x17 ilu0", lambda: synth.poisson7(21, 19, 17), "ilu0", 0.0, 0, 0.25, 50, 1, (2, 2), 1e-12),
    ("cutcell 23x21x19 ilu0", lambda: synth.cutcell7(23, 21, 19, seed=3), "ilu0", 0.0, 0, 0.25, 100, 2, (3, 3),
     1e-12),
    ("hex27 13x12x11 ilut", lambda: synth.hex27(13, 12, 11, seed=4), "ilut", 1e-3, 10, 0.25, 60, 1, (2, 1), 1e-12),
    ("poisson 16^3 nu0", lambda: synth.poisson7(16), "ilu0", 0.0, 0, 0.5, 40, 0, (1, 1), 1e-12),
]


@pytest.mark.parametrize("coarse", ["jacobi", "gs"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_vcycle_matches_oracle(silu, ctx, case, coarse):
    name, gen, kind, tau, fill, theta, cs, nu, (mL, mU), tol = case
    A = gen()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind, tau, fill)
    terms = 3
    F.amg_setup(theta=theta, max_levels=12, coarse_size=cs, jacobi_sweeps=nu,
                coarse_smoother=silu.AMG_POLY_GS if coarse == "gs" else silu.AMG_L1_JACOBI, gs_terms=terms)
    H = oracle.AMG(A, theta=theta, max_levels=12, coarse_size=cs)
    assert F.amg_stats()["levels"] == len(H.levels) >= 3
    S = oracle.row_scale(oracle.factor(A, kind, tau, fill))
    b = synth.rhs(n, 1, seed=7)[:, 0]
    x = np.zeros(n)
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    bd = dev(b)
    for cycle in range(3):  # successive cycles from the previous iterate
        x = H.vcycle(S, x, b, mL, mU, nu=nu, coarse=coarse, terms=terms)
        F.amg_vcycle(xd, bd, mL, mU)
        ctx.check()
        err = relerr(host(xd), x)
        assert err < tol, (cycle, err)


def test_single_level_hierarchy_is_the_direct_solve(silu, ctx):
    A = synth.cutcell7(7, 6, 5, seed=2)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.amg_setup(coarse_size=1000)
    assert F.amg_stats()["levels"] == 1
    b = synth.rhs(n, 1, seed=3)[:, 0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    F.amg_vcycle(x, dev(b), 2, 2)
    from _helpers import dense
    assert relerr(host(x), np.linalg.solve(dense(A, n), b)) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fgmres_with_amg_preconditioner(silu, ctx, prec):
    """FGMRES(30) to 1e-10 with one V-cycle as the preconditioner (the
    paper's GMRES + AMG configuration, ILU smoothing on the finest level):
    converges, in far fewer iterations than with the single-level smoother,
    and the true relative residual (recomputed by the oracle) meets tol."""
    A = synth.cutcell7(40, 36, 30, seed=10)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=silu.FP32 if prec == "fp32" else silu.FP64)
    F.amg_setup(theta=0.25, coarse_size=200, jacobi_sweeps=1)
    b = synth.rhs(n, 1, seed=1)[:, 0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, x, dev(b), tol=1e-10, restart=30, maxit=2000, sweeps_L=3, sweeps_U=3,
                                     precond=silu.PRECOND_AMG)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)
    r = oracle.residual(A, host(x).reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10
    x1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    st1, its1, rel1 = silu.fgmres_solve(F, x1, dev(b), tol=1e-10, restart=30, maxit=4000, sweeps_L=3, sweeps_U=3)
    assert st1 == silu.OK
    print(f"{prec}: FGMRES(30) iterations, AMG V-cycle {its} vs single-level smoother {its1}")
    assert its * 3 < its1


def test_vcycle_with_exact_triangular_solves(silu, ctx):
    """With negative sweep counts the finest level is smoothed by the exact
    level-scheduled solves; Richardson sweeps reach the same operator once
    their count equals the factor's level count (nilpotence, Sec. 5.2), so the
    oracle's cycle with that many sweeps is the reference."""
    A = synth.cutcell7(17, 15, 13, seed=6)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.amg_setup(theta=0.25, coarse_size=60, jacobi_sweeps=1)
    st = F.stats()
    H = oracle.AMG(A, theta=0.25, coarse_size=60)
    S = oracle.row_scale(oracle.ilu0(A))
    b = synth.rhs(n, 1, seed=8)[:, 0]
    want = H.vcycle(S, np.zeros(n), b, st["levels_L"], st["levels_U"])
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    F.amg_vcycle(x, dev(b), -1, -1)
    assert relerr(host(x), want) < 1e-12
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    status, its, rel = silu.fgmres_solve(F, xs, dev(b), tol=1e-10, restart=30, maxit=500, sweeps_L=0, sweeps_U=0,
                                         precond=silu.PRECOND_AMG_DIRECT)
    assert status == silu.OK and rel <= 1e-10
    r = oracle.residual(A, host(xs).reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


@pytest.mark.parametrize("terms", [1, 2, 4])
def test_fgmres_amg_with_polynomial_gs_below(silu, ctx, terms):
    """The mixed V-cycle of Sec. 6.3 (ILU on the finest level, polynomial
    Gauss-Seidel below) as the FGMRES preconditioner reaches 1e-10."""
    A = synth.cutcell7(36, 32, 30, seed=12)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.amg_setup(coarse_size=200, jacobi_sweeps=1, coarse_smoother=silu.AMG_POLY_GS, gs_terms=terms)
    b = synth.rhs(n, 1, seed=13)[:, 0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, x, dev(b), tol=1e-10, restart=30, maxit=1000, sweeps_L=6, sweeps_U=6,
                                     precond=silu.PRECOND_AMG)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)
    r = oracle.residual(A, host(x).reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


def test_degenerate_systems(silu, ctx):
    """1 x 1 system: one V-cycle and one Schur smoother step are exact; an
    empty system is a no-op."""
    one = (np.array([0, 1], np.int64), np.array([0], np.int32), np.array([4.0]))
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *one), "ilu0")
    F.amg_setup()
    F.schur_setup(2, 1e-3, 5)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.amg_vcycle(x, dev(np.array([2.0])), 3, 3)
    assert host(x)[0] == 0.5
    x.zero_()
    F.schur_smooth(x, dev(np.array([2.0])), 3, 3)
    assert host(x)[0] == 0.5
    empty = (np.array([0], np.int64), np.zeros(0, np.int32), np.zeros(0))
    E = silu.ilu_setup(ctx, silu.Matrix(ctx, *empty), "ilu0")
    E.amg_setup()
    E.schur_setup(2, 1e-3, 5)
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    E.amg_vcycle(z, z, 1, 1)
    E.schur_smooth(z, z, 1, 1)
    ctx.check()


SCHUR_CASES = [
    # name, generator, parts, tau, fill, (mL, mU), coarse smoother
    ("poisson 21x19x17 p4", lambda: synth.poisson7(21, 19, 17), 4, 1e-3, 10, (3, 3), "jacobi"),
    ("cutcell 23x21x19 p3", lambda: synth.cutcell7(23, 21, 19, seed=3), 3, 1e-3, 8, (2, 4), "gs"),
    ("cutcell 17x15x13 p1", lambda: synth.cutcell7(17, 15, 13, seed=5), 1, 1e-3, 10, (3, 2), "jacobi"),
]


@pytest.mark.parametrize("case", SCHUR_CASES, ids=[c[0] for c in SCHUR_CASES])
def test_vcycle_with_schur_smoother_matches_oracle(silu, ctx, case):
    """The V-cycle whose finest level is smoothed by the ILUT Schur complement
    smoother (Sec. 3.1), against the oracle's, over successive cycles from the
    previous iterate, FP64 to 1e-12; then FGMRES(30) preconditioned by it
    reaches 1e-10 on the Poisson case."""
    name, gen, parts, tau, fill, (mL, mU), coarse = case
    A = gen()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    terms = 2
    F.amg_setup(theta=0.25, max_levels=12, coarse_size=60, jacobi_sweeps=1,
                coarse_smoother=silu.AMG_POLY_GS if coarse == "gs" else silu.AMG_L1_JACOBI, gs_terms=terms)
    F.schur_setup(parts, tau, fill)
    H = oracle.AMG(A, theta=0.25, max_levels=12, coarse_size=60)
    assert F.amg_stats()["levels"] == len(H.levels) >= 3
    b = synth.rhs(n, 1, seed=8)[:, 0]
    x = synth.rhs(n, 1, seed=9)[:, 0] * 0.5
    xd = dev(x.copy())
    bd = dev(b)
    for cycle in range(3):
        x = H.vcycle_schur(x, b, parts, tau, fill, mL, mU, coarse=coarse, terms=terms)
        F.amg_vcycle_schur(xd, bd, mL, mU)
        ctx.check()
        err = relerr(host(xd), x)
        assert err < 1e-12, (cycle, err)
    if name.startswith("poisson"):
        xs = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, its, rel = silu.fgmres_solve(F, xs, bd, tol=1e-10, restart=30, maxit=500, sweeps_L=mL, sweeps_U=mU,
                                         precond=silu.PRECOND_AMG_SCHUR)
        assert st == silu.OK and rel <= 1e-10, (st, its, rel)
        r = oracle.residual(A, host(xs).reshape(n, 1), b.reshape(n, 1))
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


def test_schur_cycle_refused_without_setup(silu, ctx):
    A = synth.poisson7(9)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    b = dev(synth.rhs(n, 1, seed=1)[:, 0])
    with pytest.raises(silu.SiluError):
        F.amg_vcycle_schur(x, b, 2, 2)  # no hierarchy
    F.amg_setup(coarse_size=50)
    with pytest.raises(silu.SiluError):
        F.amg_vcycle_schur(x, b, 2, 2)  # no Schur complement smoother
    with pytest.raises(silu.SiluError):
        silu.fgmres_solve(F, x, b, tol=1e-8, precond=silu.PRECOND_AMG_SCHUR)


ILU_LEVEL_CASES = [
    # name, generator, kind, tau, fill, ilu_levels, coarse smoother, (mL, mU)
    ("cutcell 23x21x19 ilu0 two levels", lambda: synth.cutcell7(23, 21, 19, seed=3), "ilu0", 0.0, 0, 2, "jacobi",
     (3, 2)),
    ("cutcell 23x21x19 ilu0 all levels", lambda: synth.cutcell7(23, 21, 19, seed=3), "ilu0", 0.0, 0, 25, "gs",
     (2, 3)),
    ("hex27 13x12x11 ilut all levels", lambda: synth.hex27(13, 12, 11, seed=4), "ilut", 1e-3, 10, 3, "jacobi",
     (2, 2)),
    ("poisson 16^3 iluk1 all levels", lambda: synth.poisson7(16), "iluk", 0.0, 1, 25, "jacobi", (1, 1)),
]


@pytest.mark.parametrize("case", ILU_LEVEL_CASES, ids=[c[0] for c in ILU_LEVEL_CASES])
def test_vcycle_with_ilu_on_several_levels_matches_oracle(silu, ctx, case):
    """ILU smoothing from the finest level down (Sec. 6): levels below the
    finest get incomplete factorisations of A_l of their own (the same kind,
    tau and fill; bit-identical host factors on both sides) and are swept
    like the finest; three successive cycles against the oracle's
    vcycle_ilu at 1e-12, then FGMRES(30) preconditioned by the cycle."""
    name, gen, kind, tau, fill, nilu, coarse, (mL, mU) = case
    A = gen()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), kind, tau, fill)
    F.amg_setup(theta=0.25, max_levels=12, coarse_size=40, jacobi_sweeps=1,
                coarse_smoother=silu.AMG_POLY_GS if coarse == "gs" else silu.AMG_L1_JACOBI, gs_terms=2,
                ilu_levels=nilu)
    H = oracle.AMG(A, theta=0.25, max_levels=12, coarse_size=40)
    assert F.amg_stats()["levels"] == len(H.levels) >= 3
    fac = H.level_factors(kind, tau, fill, count=nilu)
    assert len(fac) == min(nilu, len(H.levels) - 1) >= 2
    b = synth.rhs(n, 1, seed=11)[:, 0]
    x = synth.rhs(n, 1, seed=12)[:, 0]
    xd, bd = dev(x.copy()), dev(b)
    for cycle in range(3):
        x = H.vcycle_ilu(fac, x, b, mL, mU, nu=1, coarse=coarse, terms=2)
        F.amg_vcycle(xd, bd, mL, mU)
        ctx.check()
        got = host(xd)
        assert relerr(got, x) < 1e-12, (cycle, relerr(got, x))
        assert maxabs_err(got, x) < 1e-12, cycle
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, xs, bd, tol=1e-10, restart=30, maxit=500, sweeps_L=max(mL, 2),
                                     sweeps_U=max(mU, 2), precond=silu.PRECOND_AMG)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)
    r = oracle.residual(A, host(xs).reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


def test_vcycle_with_exact_solves_on_several_levels(silu, ctx):
    """With negative sweep counts every ILU level is smoothed by its exact
    triangular solves; the oracle reaches the same operator with as many
    sweeps as each factor has levels (nilpotence, Sec. 5.2), per level."""
    A = synth.cutcell7(17, 15, 13, seed=6)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.amg_setup(theta=0.25, coarse_size=40, jacobi_sweeps=1, ilu_levels=3)
    H = oracle.AMG(A, theta=0.25, coarse_size=40)
    fac = H.level_factors("ilu0", count=3)
    assert len(fac) == 3
    mL = [oracle.levels_lower(S.L)[0] for S in fac]
    mU = [oracle.levels_upper(S.Us)[0] for S in fac]
    b = synth.rhs(n, 1, seed=8)[:, 0]
    want = H.vcycle_ilu(fac, np.zeros(n), b, mL, mU)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    F.amg_vcycle(x, dev(b), -1, -1)
    assert relerr(host(x), want) < 1e-12
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, xs, dev(b), tol=1e-10, restart=30, maxit=500, sweeps_L=0, sweeps_U=0,
                                     precond=silu.PRECOND_AMG_DIRECT)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)
    r = oracle.residual(A, host(xs).reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


def test_ilu_levels_refused_for_gauss_seidel_factors(silu, ctx):
    A = synth.poisson7(10)
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "gs")
    with pytest.raises(silu.SiluError):
        F.amg_setup(coarse_size=40, ilu_levels=2)
    with pytest.raises(silu.SiluError):
        F.amg_setup(coarse_size=40, ilu_levels=-1)
    F.amg_setup(coarse_size=40, ilu_levels=1)  # the finest level alone takes any kind


def test_schur_smoothed_cycle_with_ilu_below_matches_oracle(silu, ctx):
    """The Schur complement smoother on the finest level and ILU smoothers of
    their own on the next two levels, three successive cycles against the
    oracle at 1e-12, and FGMRES(30) preconditioned by it."""
    A = synth.poisson7(21, 19, 17)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.amg_setup(theta=0.25, max_levels=12, coarse_size=40, jacobi_sweeps=1, ilu_levels=3)
    F.schur_setup(4, 1e-3, 10)
    H = oracle.AMG(A, theta=0.25, max_levels=12, coarse_size=40)
    assert len(H.levels) >= 4
    fac = H.level_factors("ilu0", count=3)
    b = synth.rhs(n, 1, seed=8)[:, 0]
    x = synth.rhs(n, 1, seed=9)[:, 0]
    xd, bd = dev(x.copy()), dev(b)
    for cycle in range(3):
        x = H.vcycle_ilu(fac, x, b, 3, 2, schur=(4, 1e-3, 10))
        F.amg_vcycle_schur(xd, bd, 3, 2)
        ctx.check()
        assert relerr(host(xd), x) < 1e-12, cycle
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, xs, bd, tol=1e-10, restart=30, maxit=500, sweeps_L=3, sweeps_U=2,
                                     precond=silu.PRECOND_AMG_SCHUR)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)


def test_fp32_factors_on_every_ilu_level(silu, ctx):
    """FP32 factors and sweeps on the finest and every coarser ILU level (the
    rest of the cycle and FGMRES in FP64): one cycle within FP32 rounding of
    the oracle's FP64 cycle, and FGMRES(30) still reaches 1e-10."""
    A = synth.cutcell7(40, 36, 30, seed=10)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=silu.FP32)
    F.amg_setup(theta=0.25, coarse_size=200, jacobi_sweeps=1, ilu_levels=25)
    H = oracle.AMG(A, theta=0.25, coarse_size=200)
    fac = H.level_factors("ilu0")
    b = synth.rhs(n, 1, seed=1)[:, 0]
    want = H.vcycle_ilu(fac, np.zeros(n), b, 3, 3)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    F.amg_vcycle(x, dev(b), 3, 3)
    assert relerr(host(x), want) < 1e-5
    xs = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, xs, dev(b), tol=1e-10, restart=30, maxit=2000, sweeps_L=3, sweeps_U=3,
                                     precond=silu.PRECOND_AMG)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)
    r = oracle.residual(A, host(xs).reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


def test_schur_smoothed_cycle_with_the_preconditioned_interface_step(silu, ctx):
    """The V-cycle whose finest level is smoothed by the Schur complement
    smoother with the diag(C)-preconditioned interface iteration, against the
    oracle's, three successive cycles at 1e-12 on a cut-cell matrix."""
    A = synth.cutcell7(23, 21, 19, seed=3)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.amg_setup(theta=0.25, max_levels=12, coarse_size=60, jacobi_sweeps=1)
    F.schur_setup(3, 1e-3, 8)
    F.schur_set_interface_prec(silu.SCHUR_IFACE_DIAG)
    H = oracle.AMG(A, theta=0.25, max_levels=12, coarse_size=60)
    b = synth.rhs(n, 1, seed=8)[:, 0]
    x = synth.rhs(n, 1, seed=9)[:, 0] * 0.5
    xd, bd = dev(x.copy()), dev(b)
    for cycle in range(3):
        x = H.vcycle_schur(x, b, 3, 1e-3, 8, 2, 4, iface_prec=1)
        F.amg_vcycle_schur(xd, bd, 2, 4)
        ctx.check()
        assert relerr(host(xd), x) < 1e-12, cycle
