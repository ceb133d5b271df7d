"""Batches of uneven systems on the GPU: the packed smoother equals each
system's oracle smoother; the batched FGMRES gives each system what a
single-system solve gives (iterations within rounding, true residual below
tol); the autotuner keeps results unchanged."""
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


def systems_for(edges, seed0):
    return [synth.cutcell7(e, seed=seed0 + k) for k, e in enumerate(edges)]


def test_batch_smooth_matches_each_system(silu, ctx):
    edges = [5, 11, 8, 16, 3, 13, 9, 20, 7]
    systems = systems_for(edges, 300)
    B = silu.Batch(ctx, systems, "ilu0")
    n = B.n
    b = synth.rhs(n, 1, seed=4)[:, 0]
    x0 = synth.rhs(n, 1, seed=5)[:, 0]
    for variant in (1, 2):
        B.factors.set_kernel(variant)
        x = torch.from_numpy(x0.copy()).cuda()
        silu.silu_batch_smooth(B, x, torch.from_numpy(b).cuda(), 3, 4)
        ctx.check()
        got = x.cpu().numpy()
        for k, A in enumerate(systems):
            r0, r1 = B.offsets[k], B.offsets[k + 1]
            S = oracle.row_scale(oracle.ilu0(A))
            want = oracle.smooth(A, S, x0[r0:r1], b[r0:r1], 3, 4)[:, 0]
            assert relerr(got[r0:r1], want) < 1e-12, (variant, k)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_fgmres_matches_single_system_solves(silu, ctx, prec):
    edges = [6, 14, 9, 18, 4, 12, 22, 10]
    systems = systems_for(edges, 400)
    p = silu.FP32 if prec == "fp32" else silu.FP64
    B = silu.Batch(ctx, systems, "ilu0", prec=p)
    n = B.n
    b = synth.rhs(n, 1, seed=7)[:, 0]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, rel = silu.silu_batch_fgmres(B, x, torch.from_numpy(b).cuda(), tol=1e-8, restart=20, maxit=2000,
                                          sweeps_L=3, sweeps_U=3)
    assert st == silu.OK
    xb = x.cpu().numpy()
    for k, A in enumerate(systems):
        r0, r1 = B.offsets[k], B.offsets[k + 1]
        # the same system alone through the single-system solver
        F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilu0", prec=p)
        xs = torch.zeros(r1 - r0, dtype=torch.float64, device="cuda")
        st1, its1, rel1 = silu.fgmres_solve(F, xs, torch.from_numpy(b[r0:r1].copy()).cuda(), tol=1e-8, restart=20,
                                            maxit=2000, sweeps_L=3, sweeps_U=3)
        assert st1 == silu.OK
        assert abs(int(its[k]) - its1) <= 1 + its1 // 20, (k, its[k], its1)
        assert rel[k] <= 1e-8
        r = oracle.residual(A, xb[r0:r1].reshape(-1, 1), b[r0:r1].reshape(-1, 1))
        assert np.linalg.norm(r) / np.linalg.norm(b[r0:r1]) <= 1.5e-8


def test_batch_fgmres_is_deterministic_and_graph_replays(silu, ctx):
    """Two solves of the same batch give bitwise the same iterates (fixed
    reduction order; the second solve replays the captured iterations)."""
    systems = systems_for([7, 15, 10, 12], 500)
    B = silu.Batch(ctx, systems, "ilu0", prec=silu.FP32)
    b = torch.from_numpy(synth.rhs(B.n, 1, seed=8)[:, 0]).cuda()
    x1 = torch.zeros(B.n, dtype=torch.float64, device="cuda")
    x2 = torch.zeros_like(x1)
    r1 = silu.silu_batch_fgmres(B, x1, b, tol=1e-9, restart=20, maxit=1000)
    r2 = silu.silu_batch_fgmres(B, x2, b, tol=1e-9, restart=20, maxit=1000)
    assert r1[0] == r2[0] == silu.OK
    assert np.array_equal(r1[1], r2[1])
    assert torch.equal(x1, x2)


def test_autotune_keeps_results(silu, ctx):
    systems = systems_for([12, 20, 16, 9], 600)
    B = silu.Batch(ctx, systems, "ilu0")
    b = torch.from_numpy(synth.rhs(B.n, 1, seed=9)[:, 0]).cuda()
    x1 = torch.zeros(B.n, dtype=torch.float64, device="cuda")
    silu.silu_batch_smooth(B, x1, b, 3, 3)
    choice, ms = B.factors.autotune(3, 3)
    table = B.factors.tune_table()
    run = [row[4] for row in table if row[4] >= 0]
    assert 0 <= choice < len(table) and ms > 0 and table[choice][4] == ms == min(run)
    x2 = torch.zeros_like(x1)
    silu.silu_batch_smooth(B, x2, b, 3, 3)
    ctx.check()
    assert relerr(x2.cpu().numpy(), x1.cpu().numpy()) < 1e-12


def test_autotune_tries_sorted_copies_where_they_pay(silu, ctx):
    """ILUT factors of a cut-cell matrix have rows of uneven length, so the
    autotuner also times the length-sorted copies (variant 3); whatever it
    picks, results stay within FP64 rounding of the untuned ones."""
    A = synth.cutcell7(40, 36, 30, seed=4)
    n = len(A[0]) - 1
    F = silu.ilu_setup(ctx, silu.Matrix(ctx, *A), "ilut", 1e-3, 10)
    b = torch.from_numpy(synth.rhs(n, 1, seed=3)).cuda()
    x1 = torch.zeros(n, 1, dtype=torch.float64, device="cuda")
    silu.ilu_smooth(F, x1, b, 4, 4)
    choice, ms = F.autotune(4, 4)
    table = F.tune_table()
    sorted_rows = [row for row in table if row[0] == 3]
    assert sorted_rows and all(row[4] > 0 for row in sorted_rows)
    assert table[choice][4] == ms == min(row[4] for row in table if row[4] >= 0)
    x2 = torch.zeros_like(x1)
    silu.ilu_smooth(F, x2, b, 4, 4)
    ctx.check()
    assert relerr(x2.cpu().numpy(), x1.cpu().numpy()) < 1e-12
