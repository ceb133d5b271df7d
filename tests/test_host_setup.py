"""Host-side logic of libsilu on the CPU: the C ABI loads and exports every
declared symbol, input validation, and the host factorisation / scaling /
level sets against the oracle (patterns and levels bit-exact, values to
1e-14 relative; both sides round every operation as written)."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2111_09512_gb300 as silu
import synth
from _helpers import csr_from_dense

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    silu.build()
    return silu.Context(device=-1)


def header_functions():
    text = open(os.path.join(ROOT, "include", "silu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)
    return sorted({n for n in names if n.startswith(("silu_", "ilu_", "direct_", "fgmres_"))})


def test_library_exports_every_declared_symbol():
    silu.build()
    import ctypes
    lib = ctypes.CDLL(silu.LIB_PATH)
    declared = header_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(silu.exported_symbols()) <= set(declared)
    assert "sm_103a" in silu.silu_version()


def test_host_only_context_refuses_device_calls(ctx):
    A = synth.poisson7(4)
    M = silu.Matrix(ctx, *A)
    F = silu.ILU(M, "ilu0")
    st = silu.load().ilu_smooth(F.handle, 8, 8, 1, 1, 1)
    assert st == silu.ERR_NO_DEVICE
    assert b"host-only" in silu.load().silu_last_error(ctx.handle)


def test_csr_validation(ctx):
    rp = np.array([0, 2, 3], np.int64)
    with pytest.raises(silu.SiluError) as e:
        silu.Matrix(ctx, rp, np.array([0, 5, 1], np.int32), np.ones(3))
    assert e.value.status == silu.ERR_INVALID_ARG
    with pytest.raises(silu.SiluError):
        silu.Matrix(ctx, rp, np.array([0, 1, 1], np.int32), np.array([1.0, np.nan, 1.0]))
    with pytest.raises(silu.SiluError):
        silu.Matrix(ctx, np.array([0, 2, 1], np.int64), np.array([0, 1, 1], np.int32), np.ones(3))
    # unsorted columns and duplicates are canonicalised: same factors as the sorted matrix
    Mu = silu.Matrix(ctx, np.array([0, 3, 5], np.int64), np.array([1, 0, 0, 1, 0], np.int32),
                     np.array([-1.0, 2.0, 2.0, 4.0, -1.0]))
    F = silu.ILU(Mu, "ilu0").export()
    assert np.array_equal(F["U"][1], [0, 1, 1]) and np.array_equal(F["U"][2], [4.0, -1.0, 3.75])
    assert np.array_equal(F["L"][2], [-0.25])


def test_zero_pivot_reported(ctx):
    M = silu.Matrix(ctx, np.array([0, 2, 4], np.int64), np.array([0, 1, 0, 1], np.int32),
                    np.array([0.0, 1.0, 1.0, 2.0]))
    for kind in ("ilu0", "ilut", "iluk"):
        with pytest.raises(silu.SiluError) as e:
            silu.ILU(M, kind, tau=0.0, fill=2)
        assert e.value.status == silu.ERR_ZERO_PIVOT


def compare_with_oracle(F, OF, OS):
    ex = F.export()
    for mine, theirs in ((ex["L"], OF.L), (ex["U"], OF.U), (ex["Us"], OS.Us)):
        assert np.array_equal(mine[0], theirs[0])
        assert np.array_equal(mine[1], theirs[1])
        d = np.abs(mine[2] - theirs[2])
        assert np.all(d <= 1e-14 * np.abs(theirs[2]))
    assert np.all(np.abs(ex["dinv"] - OS.dinv) <= 1e-14 * np.abs(OS.dinv))
    return ex


CASES = [
    ("poisson 9x7x5 ilu0", lambda: synth.poisson7(9, 7, 5), "ilu0", 0.0, 0),
    ("cutcell 10x9x8 ilu0", lambda: synth.cutcell7(10, 9, 8, seed=3), "ilu0", 0.0, 0),
    ("hex27 6x5x4 ilu0", lambda: synth.hex27(6, 5, 4, seed=2), "ilu0", 0.0, 0),
    ("cutcell 8x8x6 iluk1", lambda: synth.cutcell7(8, 8, 6, seed=4), "iluk", 0.0, 1),
    ("cutcell 7x6x5 iluk3", lambda: synth.cutcell7(7, 6, 5, seed=5), "iluk", 0.0, 3),
    ("hex27 5x4x4 iluk2", lambda: synth.hex27(5, 4, 4, seed=6), "iluk", 0.0, 2),
    ("cutcell 12x11x10 ilut", lambda: synth.cutcell7(12, 11, 10, seed=1), "ilut", 1e-3, 10),
    ("cutcell 10x10x10 ilut tight", lambda: synth.cutcell7(10, 10, 10, seed=7), "ilut", 1e-2, 3),
    ("hex27 6x6x5 ilut", lambda: synth.hex27(6, 6, 5, seed=8), "ilut", 1e-3, 8),
]


@pytest.mark.parametrize("name,gen,kind,tau,fill", CASES, ids=[c[0] for c in CASES])
def test_host_factors_match_oracle(ctx, name, gen, kind, tau, fill):
    A = gen()
    F = silu.ILU(silu.Matrix(ctx, *A), kind, tau=tau, fill=fill)
    OF = oracle.factor(A, kind, tau, fill)
    OS = oracle.row_scale(OF)
    ex = compare_with_oracle(F, OF, OS)
    nl, levL = oracle.levels_lower(OS.L)
    nu, levU = oracle.levels_upper(OS.Us)
    st = F.stats()
    assert st["levels_L"] == nl and st["levels_U"] == nu
    assert np.array_equal(ex["levL"], levL) and np.array_equal(ex["levU"], levU)


def test_host_ilut_cut_cell_64(ctx):
    """A larger ILUT(1e-3, 10) cut-cell case: 262,144 rows, several thousand
    drop decisions near the threshold, all identical to the oracle's."""
    A = synth.cutcell7(64, 64, 64, seed=1)
    F = silu.ILU(silu.Matrix(ctx, *A), "ilut", tau=1e-3, fill=10)
    OF = oracle.ilut(A, 1e-3, 10)
    compare_with_oracle(F, OF, oracle.row_scale(OF))


def test_refactor_reuses_the_pattern(ctx):
    A = synth.cutcell7(8, 7, 6, seed=2)
    A2 = synth.cutcell7(8, 7, 6, seed=9)
    assert np.array_equal(A[1], A2[1])
    for kind, fill in (("ilu0", 0), ("iluk", 2)):
        M = silu.Matrix(ctx, *A)
        F = silu.ILU(M, kind, fill=fill)
        silu.ilu_refactor(F, A2[2])
        OF = oracle.factor(A2, kind, 0.0, fill)
        compare_with_oracle(F, OF, oracle.row_scale(OF))
    F = silu.ILU(silu.Matrix(ctx, *A), "ilut", tau=1e-3, fill=5)
    with pytest.raises(silu.SiluError):
        silu.ilu_refactor(F, A2[2])


def test_batch_factors_are_the_systems_factors(ctx):
    """silu_batch_setup factors each system on its own (in parallel) and packs
    them block-diagonally: the packed factors equal the oracle's factors of
    each system with columns shifted by the system's offset."""
    edges = [3, 7, 4, 9, 5, 6, 8, 2]
    systems = [synth.cutcell7(e, e + 1, e, seed=50 + k) for k, e in enumerate(edges)]
    for kind, tau, fill in (("ilu0", 0.0, 0), ("ilut", 1e-3, 6), ("iluk", 0.0, 1)):
        B = silu.Batch(ctx, systems, kind, tau=tau, fill=fill)
        ex = B.factors.export()
        off = B.offsets
        for k, A in enumerate(systems):
            OF = oracle.factor(A, kind, tau, fill)
            OS = oracle.row_scale(OF)
            r0, r1 = off[k], off[k + 1]
            for mine, theirs in ((ex["L"], OS.L), (ex["Us"], OS.Us)):
                rp = mine[0][r0:r1 + 1]
                seg = slice(rp[0], rp[-1])
                assert np.array_equal(rp - rp[0], theirs[0])
                assert np.array_equal(mine[1][seg] - r0, theirs[1])
                assert np.all(np.abs(mine[2][seg] - theirs[2]) <= 1e-14 * np.abs(theirs[2]))
            assert np.allclose(ex["dinv"][r0:r1], OS.dinv, rtol=1e-14, atol=0)
        B.close()


def _tile_slots_per_entry(rp, rows=32, cap=416):
    """FMA slots per entry of one-lane-per-row warp tiles (32 rows, at most
    `cap` entries per tile), each costing 32 times its longest row."""
    n = len(rp) - 1
    lens = np.diff(rp)
    slots, r0 = 0, 0
    while r0 < n:
        r1 = r0
        while r1 < n and r1 - r0 < rows and rp[r1 + 1] - rp[r0] <= cap:
            r1 += 1
        slots += 32 * int(lens[r0:r1].max())
        r0 = r1
    return slots / rp[-1]


def _window_sorted_rp(rp, window=512):
    lens = np.diff(rp)
    order = np.concatenate([w0 + np.argsort(-lens[w0:w0 + window], kind="stable")
                            for w0 in range(0, len(lens), window)])
    return np.concatenate([[0], np.cumsum(lens[order])])


def test_layout_pads(ctx):
    """silu_ilu_layout's padding figures equal a direct count over the
    exported factors; ILUT's uneven L rows get a sorted copy, Poisson's
    uniform rows do not, and a host-only context sweeps nothing."""
    for A, kind, tau, fill, sorted_L in ((synth.cutcell7(20, 18, 16, seed=1), "ilut", 1e-3, 10, True),
                                         (synth.poisson7(17, 15, 13), "ilu0", 0.0, 0, False)):
        F = silu.ILU(silu.Matrix(ctx, *A), kind, tau=tau, fill=fill)
        lay = F.layout()
        ex = F.export()
        for k, fac in enumerate(("L", "Us")):
            rp = ex[fac][0]
            nat, srt = _tile_slots_per_entry(rp), _tile_slots_per_entry(_window_sorted_rp(rp))
            assert lay["pad_natural"][k] == pytest.approx(nat, rel=1e-12)
            assert lay["pad_sorted"][k] == pytest.approx(srt, rel=1e-12)
            assert srt <= nat + 1e-12
        pays = lay["pad_natural"][0] >= 1.08 and lay["pad_natural"][0] - lay["pad_sorted"][0] >= 0.05
        assert pays == sorted_L
        assert not lay["in_use"].any()


@pytest.mark.parametrize("kind", ["gs", "sgs"])
def test_gauss_seidel_factors(ctx, kind):
    """GS / SGS as factors (Sec. 3.1): L_s = L_A D^{-1}, Utilde_s = D^{-1} U_A
    (SGS only), dinv = 1 / diag(A), each one division of A's entries; and the
    row-scaled Richardson sweeps on them reproduce the oracle's polynomial
    Gauss-Seidel, sum_{j<=p} (-D^{-1} L_A)^j D^{-1} r, formed term by term."""
    from _helpers import dense
    A = synth.cutcell7(6, 5, 4, seed=9)
    n = len(A[0]) - 1
    M = dense(A)
    d = np.diag(M)
    ex = silu.ILU(silu.Matrix(ctx, *A), kind).export()
    assert np.array_equal(ex["dinv"], 1.0 / d)
    assert np.array_equal(dense(ex["L"], n), np.tril(M, -1) / d[None, :])
    want_us = np.triu(M, 1) / d[:, None] if kind == "sgs" else np.zeros((n, n))
    assert np.array_equal(dense(ex["Us"], n), want_us)
    S = oracle.Scaled(n, ex["L"], ex["Us"], ex["dinv"])
    b = synth.rhs(n, 2, seed=3)
    x0 = synth.rhs(n, 2, seed=4)
    for p, q in ((0, 0), (1, 0), (3, 2), (6, 5)):
        mine = oracle.smooth(A, S, x0, b, p + 1, q + 1)
        want = oracle.poly_gs_smooth(A, x0, b, p, q, symmetric=(kind == "sgs"))
        assert np.linalg.norm(mine - want) / np.linalg.norm(want) < 1e-13
    # zero diagonal refused
    Z = silu.Matrix(ctx, np.array([0, 2, 4], np.int64), np.array([0, 1, 0, 1], np.int32),
                    np.array([0.0, 1.0, 1.0, 2.0]))
    with pytest.raises(silu.SiluError) as e:
        silu.ILU(Z, kind)
    assert e.value.status == silu.ERR_ZERO_PIVOT


@pytest.mark.parametrize("kind,tau,fill", [("ilu0", 0.0, 0), ("ilut", 1e-3, 6)])
def test_rowcol_scaling_matches_oracle(ctx, kind, tau, fill):
    """Row/column scaling (Eq. rowcolScale): the library's Ruiz equilibration
    and unit-diagonal row fix reproduce the oracle's bit for bit (both round
    every operation as written); the Richardson smoother on the host copies
    equals the row-scaled one (Uhat = D_c^{-1} (D^{-1} U) D_c)."""
    A = synth.cutcell7(9, 8, 7, seed=12)
    n = len(A[0]) - 1
    F = silu.ILU(silu.Matrix(ctx, *A), kind, tau, fill, scale=silu.SCALE_ROWCOL)
    ex = F.export()
    dc, steps = F.colscale()
    OF = oracle.factor(A, kind, tau, fill)
    RC = oracle.ruiz_rowcol(OF, maxit=20, tol=1e-2)
    assert steps == RC.steps and 1 <= steps <= 20
    assert np.array_equal(dc, RC.dc)
    assert np.array_equal(ex["dinv"], RC.dr)
    for mine, theirs in zip(ex["Us"], RC.Us):
        assert np.array_equal(mine, theirs)
    b = synth.rhs(n, 1, seed=2)
    S = oracle.row_scale(OF)
    want = oracle.smooth(A, S, np.zeros((n, 1)), b, 4, 4)
    got = oracle.smooth_rowcol(A, RC, np.zeros((n, 1)), b, 4, 4)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-13
    # another scaling has no column factor
    G = silu.ILU(silu.Matrix(ctx, *A), kind, tau, fill)
    with pytest.raises(silu.SiluError):
        G.colscale()


@pytest.mark.parametrize("gen,theta", [("cutcell", 0.25), ("hex27", 0.25), ("poisson", 0.5), ("cutcell", 0.05)])
def test_amg_hierarchy_matches_oracle(ctx, gen, theta):
    """AMG setup (Sec. 3): the library's C/F splits, interpolation and Galerkin
    operators equal the oracle's bit for bit on every level (both sum in the
    same stated orders without FMA contraction)."""
    A = {"cutcell": lambda: synth.cutcell7(11, 10, 9, seed=4), "hex27": lambda: synth.hex27(9, 8, 8, seed=5),
         "poisson": lambda: synth.poisson7(12, 11, 10)}[gen]()
    F = silu.ILU(silu.Matrix(ctx, *A), "ilu0")
    F.amg_setup(theta=theta, max_levels=10, coarse_size=30, jacobi_sweeps=1)
    H = oracle.AMG(A, theta=theta, max_levels=10, coarse_size=30)
    st = F.amg_stats()
    assert st["levels"] == len(H.levels) and st["levels"] >= 3
    for l, OL in enumerate(H.levels):
        mine = F.amg_level(l)
        for a, b in zip(mine["A"], OL.A):
            assert np.array_equal(a, b), (l, "A")
        if OL.P is None:
            assert mine["P"] is None
            continue
        assert np.array_equal(mine["cf"], OL.cf), l
        for a, b in zip(mine["P"], OL.P):
            assert np.array_equal(a, b), (l, "P")


def test_amg_bad_parameters(ctx):
    A = synth.poisson7(5)
    F = silu.ILU(silu.Matrix(ctx, *A), "ilu0")
    for kw in ({"theta": 0.0}, {"theta": 1.5}, {"max_levels": 0}, {"coarse_size": 0}, {"jacobi_sweeps": -1}):
        with pytest.raises(silu.SiluError) as e:
            F.amg_setup(**kw)
        assert e.value.status == silu.ERR_INVALID_ARG
    with pytest.raises(silu.SiluError):
        F.amg_stats()


@pytest.mark.parametrize("parts", [1, 3, 8])
def test_schur_interface_matches_oracle(ctx, parts):
    """Schur complement smoother setup (Sec. 3.1): the interface rows of the
    contiguous block partition are the oracle's (integer, exact)."""
    A = synth.cutcell7(9, 8, 7, seed=2)
    F = silu.ILU(silu.Matrix(ctx, *A), "ilu0")
    F.schur_setup(parts, 1e-3, 10)
    st = F.schur_stats()
    k, marks = oracle.schur_interface(A, parts)
    assert st["interface"] == k and st["interior"] == len(marks) - k
    assert np.array_equal(st["marks"], marks)
    with pytest.raises(silu.SiluError):
        F.schur_setup(0, 1e-3, 10)


def test_amg_rejects_bad_coarse_smoother(ctx):
    A = synth.poisson7(6)
    F = silu.ILU(silu.Matrix(ctx, *A), "ilu0")
    for kw in ({"coarse_smoother": 7}, {"coarse_smoother": silu.AMG_POLY_GS, "gs_terms": 0}):
        with pytest.raises(silu.SiluError) as e:
            F.amg_setup(coarse_size=20, **kw)
        assert e.value.status == silu.ERR_INVALID_ARG
    F.amg_setup(coarse_size=20, coarse_smoother=silu.AMG_POLY_GS, gs_terms=3)
    assert F.amg_stats()["levels"] >= 2


@pytest.mark.parametrize("scale", ["row", "rowcol"])
def test_dep_matches_oracle(ctx, scale):
    """Departure from normality (Eq. depB) of L, U and the scaled upper
    factor against the oracle's; for symmetric A under ILU(0) with row
    scaling dep(L) = dep(D^{-1} U) (Table dep)."""
    A = synth.cutcell7(10, 9, 8, seed=3)
    sc = silu.SCALE_ROWCOL if scale == "rowcol" else silu.SCALE_ROW
    F = silu.ILU(silu.Matrix(ctx, *A), "ilu0", scale=sc)
    d = F.dep()
    OF = oracle.ilu0(A)
    assert abs(d["L"] - oracle.dep_triangular(OF.L, unit_diag=True)) <= 1e-14 * d["L"]
    assert abs(d["U"] - oracle.dep_triangular(OF.U)) <= 1e-14 * d["U"]
    Us = oracle.ruiz_rowcol(OF).Us if scale == "rowcol" else oracle.row_scale(OF).Us
    assert abs(d["scaled"] - oracle.dep_triangular(Us, unit_diag=True)) <= 1e-14 * d["scaled"]
    if scale == "row":
        assert abs(d["L"] - d["scaled"]) <= 1e-13 * d["L"]
        assert d["U"] > 10 * d["scaled"]


def test_amg_and_schur_on_degenerate_systems(ctx):
    """Empty and 1x1 systems: the AMG hierarchy is a single (directly solved)
    level, the Schur partition has no interface."""
    one = (np.array([0, 1], np.int64), np.array([0], np.int32), np.array([4.0]))
    empty = (np.array([0], np.int64), np.zeros(0, np.int32), np.zeros(0))
    for A in (one, empty):
        F = silu.ILU(silu.Matrix(ctx, *A), "ilu0")
        F.amg_setup()
        st = F.amg_stats()
        assert st["levels"] == 1 and st["rows"] == [len(A[0]) - 1]
        F.amg_setup(ilu_levels=5)  # no level below the finest to give an ILU smoother
        assert F.amg_stats()["levels"] == 1 and F.amg_level_ilu(0) is F
        F.schur_setup(4, 1e-3, 5)
        sst = F.schur_stats()
        assert sst["interface"] == 0 and sst["interior"] == len(A[0]) - 1


@pytest.mark.parametrize("kind,tau,fill,scale", [("ilut", 1e-3, 6, "row"), ("iluk", 0.0, 1, "rowcol"),
                                                 ("sgs", 0.0, 0, "row")])
def test_factor_save_and_load(ctx, tmp_path, kind, tau, fill, scale):
    """silu_ilu_save / silu_ilu_load: the loaded object has the saved factors,
    scaling and level sets bit for bit, without factoring again; a file that
    does not fit the matrix, or is corrupt, is refused."""
    A = synth.cutcell7(9, 8, 7, seed=6)
    M = silu.Matrix(ctx, *A)
    sc = silu.SCALE_ROWCOL if scale == "rowcol" else silu.SCALE_ROW
    F = silu.ILU(M, kind, tau, fill, scale=sc)
    path = str(tmp_path / "f.silu")
    F.save(path)
    G = silu.ILU.load_file(M, path)
    a, b = F.export(), G.export()
    for key in a:
        if isinstance(a[key], tuple):
            for u, v in zip(a[key], b[key]):
                assert np.array_equal(u, v), key
        else:
            assert np.array_equal(a[key], b[key]), key
    assert F.stats() == G.stats()
    other = silu.Matrix(ctx, *synth.cutcell7(5, 5, 5, seed=1))
    with pytest.raises(silu.SiluError):
        silu.ILU.load_file(other, path)
    raw = bytearray(open(path, "rb").read())
    raw[-200:] = b"\xff" * 200
    bad = str(tmp_path / "bad.silu")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(silu.SiluError):
        silu.ILU.load_file(M, bad)
    with pytest.raises(silu.SiluError):
        silu.ILU.load_file(M, str(tmp_path / "missing.silu"))


def test_threaded_setup_matches_oracle_bit_for_bit(ctx):
    """Above a million entries the host setup runs on threads: row ranges for
    the canonical CSR, the L/U split and the row scaling, level sets of the
    lower pattern for the numeric ILU(0).  Every row keeps its arithmetic and
    order, so the factors equal the oracle's bit for bit.  The same matrix
    given with every row's columns shuffled and every value split into two
    halves (exact in binary) canonicalises to the same factors."""
    A = synth.hex27(52, 50, 48, seed=9)
    assert len(A[1]) > (1 << 20)
    F = silu.ILU(silu.Matrix(ctx, *A), "ilu0")
    OF = oracle.ilu0(A)
    OS = oracle.row_scale(OF)
    ex = F.export()
    for mine, theirs in ((ex["L"], OF.L), (ex["U"], OF.U), (ex["Us"], OS.Us)):
        for k in range(3):
            assert np.array_equal(mine[k], theirs[k])
    assert np.array_equal(ex["dinv"], OS.dinv)
    rp, ci, va = A
    rng = np.random.default_rng(3)
    n = len(rp) - 1
    lens = np.diff(rp)
    rows = np.repeat(np.arange(n), lens)
    key = rows * 4.0 + rng.random(len(ci))  # shuffle within each row
    order = np.argsort(key, kind="stable")
    ci2 = np.repeat(ci[order], 2)
    va2 = np.repeat(va[order] * 0.5, 2)
    rp2 = (2 * rp).astype(np.int64)
    G = silu.ILU(silu.Matrix(ctx, rp2, ci2.astype(np.int32), va2), "ilu0").export()
    for part in ("L", "U", "Us"):
        for k in range(3):
            assert np.array_equal(G[part][k], ex[part][k])


@pytest.mark.parametrize("gen,kind,tau,fill", [("cutcell", "ilu0", 0.0, 0), ("hex27", "ilut", 1e-3, 8),
                                               ("cutcell", "iluk", 0.0, 1), ("poisson", "ilut", 1e-2, 3)])
def test_amg_ilu_levels_factors_match_oracle(ctx, gen, kind, tau, fill):
    """ILU smoothing below the finest level (Sec. 6): the factor object of
    every ILU level holds the row-scaled factorisation of that level's A_l of
    the finest level's kind: the oracle's patterns exactly and its values to
    1e-14 (the hierarchy is bit for bit the oracle's), with the oracle's level
    counts; a level without one is refused."""
    A = {"cutcell": lambda: synth.cutcell7(11, 10, 9, seed=4), "hex27": lambda: synth.hex27(9, 8, 8, seed=5),
         "poisson": lambda: synth.poisson7(12, 11, 10)}[gen]()
    F = silu.ILU(silu.Matrix(ctx, *A), kind, tau=tau, fill=fill)
    F.amg_setup(theta=0.25, max_levels=10, coarse_size=30, jacobi_sweeps=1, ilu_levels=25)
    H = oracle.AMG(A, theta=0.25, max_levels=10, coarse_size=30)
    nlev = F.amg_stats()["levels"]
    assert nlev == len(H.levels) >= 3
    fac = H.level_factors(kind, tau, fill)
    assert len(fac) == nlev - 1
    assert F.amg_level_ilu(0) is F
    for l in range(1, nlev - 1):
        G = F.amg_level_ilu(l)
        OF = oracle.factor(H.levels[l].A, kind, tau, fill)
        ex = compare_with_oracle(G, OF, fac[l])
        st = G.stats()
        assert st["levels_L"] == oracle.levels_lower(fac[l].L)[0], l
        assert st["levels_U"] == oracle.levels_upper(fac[l].Us)[0], l
        assert len(ex["dinv"]) == H.levels[l].n
    with pytest.raises(silu.SiluError):
        F.amg_level_ilu(nlev - 1)  # the coarsest level is solved directly
    F.amg_setup(theta=0.25, max_levels=10, coarse_size=30, ilu_levels=2)
    F.amg_level_ilu(1)
    with pytest.raises(silu.SiluError):
        F.amg_level_ilu(2)


def test_schur_interface_prec_modes(ctx):
    """silu_schur_set_interface_prec: refused before silu_schur_setup and for
    an unknown mode; the diag(C) mode is refused when an interface row has no
    diagonal entry (its c_kk is zero), the plain mode is always accepted."""
    A = synth.cutcell7(8, 7, 6, seed=2)
    F = silu.ILU(silu.Matrix(ctx, *A), "ilu0")
    with pytest.raises(silu.SiluError):
        F.schur_set_interface_prec(silu.SCHUR_IFACE_DIAG)
    F.schur_setup(3, 1e-3, 8)
    F.schur_set_interface_prec(silu.SCHUR_IFACE_DIAG)
    F.schur_set_interface_prec(silu.SCHUR_IFACE_NONE)
    with pytest.raises(silu.SiluError) as e:
        F.schur_set_interface_prec(3)
    assert e.value.status == silu.ERR_INVALID_ARG
    M = np.array([[2.0, 1.0], [1.0, 0.0]])  # two parts: both rows interface, C = M, c_11 = 0
    G = silu.ILU(silu.Matrix(ctx, *csr_from_dense(M)), "ilu0")
    G.schur_setup(2, 0.0, 2)
    with pytest.raises(silu.SiluError) as e:
        G.schur_set_interface_prec(silu.SCHUR_IFACE_DIAG)
    assert e.value.status == silu.ERR_ZERO_PIVOT
    G.schur_set_interface_prec(silu.SCHUR_IFACE_NONE)
