"""The solve server on the GPU: a served request gives the same solution as a
direct fgmres_solve of the same system (both reach tol in true relative
residual, checked by the oracle's residual), and the result of a request is
bitwise the same alone and in a mix of concurrent requests; admitted
requests overlap on the device."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def silu():
    import paper_2111_09512_gb300 as s
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s.build()
    return s


def test_served_solution_matches_direct_solve(silu):
    A = synth.cutcell7(30, 28, 26, seed=31)
    n = len(A[0]) - 1
    b = synth.rhs(n, 1, seed=32)[:, 0]
    S = silu.Server(device=0, hbm_budget=8 << 30, workers=2, max_queue=8)
    st, t = S.submit(A, b, prec=silu.FP32, tol=1e-8, restart=30)
    assert st == silu.OK
    done, res, x = S.poll(t, wait=True)
    S.close()
    assert res.status == silu.OK and res.relres <= 1e-8
    r = oracle.residual(A, x.reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-8
    ctx = silu.Context(0, torch.cuda.current_stream())
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=silu.FP32)
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    st1, its1, rel1 = silu.fgmres_solve(F, xd, torch.from_numpy(b).cuda(), tol=1e-8, restart=30, maxit=5000)
    assert st1 == silu.OK and its1 == res.iterations
    assert np.array_equal(xd.cpu().numpy(), x)


def test_result_same_alone_and_in_the_mix(silu):
    probe = synth.cutcell7(40, 36, 33, seed=41)
    pb = synth.rhs(len(probe[0]) - 1, 1, seed=42)[:, 0]
    S = silu.Server(device=0, hbm_budget=16 << 30, workers=4, max_queue=64)
    _, t = S.submit(probe, pb, prec=silu.FP32, tol=1e-8)
    _, res_alone, x_alone = S.poll(t, wait=True)
    # the same request among concurrent others of uneven sizes
    others = [synth.cutcell7(e, seed=100 + e) for e in (48, 20, 56, 33, 64, 27, 44)]
    tickets = []
    for k, A in enumerate(others):
        st, tk = S.submit(A, synth.rhs(len(A[0]) - 1, 1, seed=200 + k)[:, 0], prec=silu.FP32, tol=1e-8)
        assert st == silu.OK
        tickets.append(tk)
        if k == 3:
            _, t_mix = S.submit(probe, pb, prec=silu.FP32, tol=1e-8)
    _, res_mix, x_mix = S.poll(t_mix, wait=True)
    spans = []
    for tk in tickets:
        _, r, _ = S.poll(tk, wait=True, want_x=False)
        assert r.status == silu.OK
        spans.append((r.t_admit, r.t_done))
    S.close()
    assert res_alone.status == res_mix.status == silu.OK
    assert res_alone.iterations == res_mix.iterations
    assert np.array_equal(x_alone, x_mix)
    # admitted requests overlapped on the device
    spans.sort()
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_served_amg_request_matches_direct_solve(silu):
    """A request with the AMG V-cycle preconditioner (the paper's GMRES + AMG,
    FP32 ILU smoothing the finest level) gives the same bits through the
    server, alone and next to a sweeps-only request, as a direct call."""
    A = synth.cutcell7(34, 30, 27, seed=51)
    n = len(A[0]) - 1
    b = synth.rhs(n, 1, seed=52)[:, 0]
    S = silu.Server(device=0, hbm_budget=8 << 30, workers=2, max_queue=8)
    kw = dict(prec=silu.FP32, tol=1e-8, restart=30, maxit=2000, sweeps_L=8, sweeps_U=8, precond=silu.PRECOND_AMG)
    st, t = S.submit(A, b, **kw)
    assert st == silu.OK
    other = synth.cutcell7(40, 40, 40, seed=53)
    st2, t2 = S.submit(other, synth.rhs(len(other[0]) - 1, 1, seed=54)[:, 0], prec=silu.FP32, tol=1e-8)
    assert st2 == silu.OK
    _, res, x = S.poll(t, wait=True)
    _, res2, _ = S.poll(t2, wait=True, want_x=False)
    S.close()
    assert res.status == silu.OK and res.relres <= 1e-8 and res2.status == silu.OK
    r = oracle.residual(A, x.reshape(n, 1), b.reshape(n, 1))
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.5e-8
    ctx = silu.Context(0, torch.cuda.current_stream())
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=silu.FP32)
    F.amg_setup()
    xd = torch.zeros(n, dtype=torch.float64, device="cuda")
    st1, its1, _ = silu.fgmres_solve(F, xd, torch.from_numpy(b).cuda(), tol=1e-8, restart=30, maxit=2000,
                                     sweeps_L=8, sweeps_U=8, precond=silu.PRECOND_AMG)
    assert st1 == silu.OK and its1 == res.iterations
    assert np.array_equal(xd.cpu().numpy(), x)
