"""GPU parity of the ILUT Schur complement smoother (Sec. 3.1, Eq. schur)
against the oracle's, and FGMRES preconditioned by it.  FP64 to 1e-12
relative; FP32 factors of B report their error against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from _helpers import relerr

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
    ("cutcell 31x27x23 p4", lambda: synth.cutcell7(31, 27, 23, seed=1), 4, 1e-3, 10, (3, 3)),
    ("hex27 17x15x14 p3", lambda: synth.hex27(17, 15, 14, seed=2), 3, 1e-3, 12, (2, 2)),
    ("poisson 24^3 p8", lambda: synth.poisson7(24), 8, 1e-2, 6, (4, 1)),
    ("poisson 12^3 p1", lambda: synth.poisson7(12), 1, 1e-3, 10, (3, 3)),
    # no interior rows: every row its own part, and more parts than rows (B is empty, S = A)
    ("poisson 6^3 every row a part", lambda: synth.poisson7(6), 216, 1e-3, 10, (3, 3)),
    ("poisson 6^3 more parts than rows", lambda: synth.poisson7(6), 300, 1e-3, 10, (2, 1)),
]


@pytest.mark.parametrize("iface_prec", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_schur_smoother_matches_oracle(silu, ctx, case, iface_prec):
    """The smoother with the paper's unpreconditioned interface iteration and
    with the diag(C) right preconditioner, against the oracle's, from zero and
    from a nonzero iterate."""
    name, gen, parts, tau, fill, (mL, mU) = case
    A = gen()
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.schur_setup(parts, tau, fill)
    F.schur_set_interface_prec(iface_prec)
    b = synth.rhs(n, 1, seed=3)[:, 0]
    x0 = synth.rhs(n, 1, seed=4)[:, 0] * 0.5
    for start in (np.zeros(n), x0):
        r = oracle.residual(A, start.reshape(n, 1), b.reshape(n, 1))[:, 0]
        want = start + oracle.schur_apply(A, r, parts, tau, fill, mL, mU, iface_prec)
        x = dev(start.copy())
        F.schur_smooth(x, dev(b), mL, mU)
        ctx.check()
        assert relerr(host(x), want) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fgmres_with_schur_preconditioner(silu, ctx, prec):
    """FGMRES(30) to 1e-10 preconditioned by one Schur complement smoother
    application, on the 27-point matrix (the paper applies this smoother to
    the Nalu-Wind systems the 27-point generator stands in for).  On the
    cut-cell matrices the single GMRES step on the interface system is too
    weak and FGMRES stalls, in the oracle as on the device."""
    A = synth.hex27(28, 26, 24, seed=5)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=silu.FP32 if prec == "fp32" else silu.FP64)
    F.schur_setup(4, 1e-3, 10)
    b = synth.rhs(n, 1, seed=6)[:, 0]
    if prec == "fp32":
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        F.schur_smooth(z, dev(b), 3, 3)
        err = relerr(host(z), oracle.schur_apply(A, b, 4, 1e-3, 10, 3, 3))
        print(f"FP32 Schur complement smoother (3+3) relative error vs FP64 oracle: {err:.3e}")
        assert err < 1e-4
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.fgmres_solve(F, x, dev(b), tol=1e-10, restart=30, maxit=3000, sweeps_L=3, sweeps_U=3,
                                     precond=silu.PRECOND_SCHUR)
    assert st == silu.OK and rel <= 1e-10, (st, its, rel)
    r = oracle.residual(A, host(x).reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10


def test_fgmres_on_cut_cell_with_the_preconditioned_interface_step(silu, ctx):
    """With the interface iteration right-preconditioned by diag(C) the
    smoother makes FGMRES converge on a cut-cell matrix, where the paper's
    unpreconditioned iteration stalls (checked here over the same number of
    iterations)."""
    A = synth.cutcell7(31, 27, 23, seed=1)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0")
    F.schur_setup(4, 1e-3, 10)
    b = synth.rhs(n, 1, seed=6)[:, 0]
    its, xs = {}, {}
    for mode in (silu.SCHUR_IFACE_DIAG, silu.SCHUR_IFACE_NONE):
        F.schur_set_interface_prec(mode)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, k, rel = silu.fgmres_solve(F, x, dev(b), tol=1e-10, restart=30, maxit=1500, sweeps_L=3, sweeps_U=3,
                                       precond=silu.PRECOND_SCHUR)
        its[mode], xs[mode] = (st, k, rel), host(x)
    st, k, rel = its[silu.SCHUR_IFACE_DIAG]
    assert st == silu.OK and rel <= 1e-10, its
    r = oracle.residual(A, xs[silu.SCHUR_IFACE_DIAG].reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-10
    assert its[silu.SCHUR_IFACE_NONE][0] != silu.OK or its[silu.SCHUR_IFACE_NONE][1] > k, its
    with pytest.raises(silu.SiluError):
        F.schur_set_interface_prec(2)
