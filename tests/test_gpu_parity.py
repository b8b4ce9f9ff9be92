"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle,
one half-step at a time from the same input iterate (the top-t selection is
discontinuous, so whole trajectories are not compared).

Tolerances: FP64 1e-12 and FP32 2e-5, relative to the largest oracle value
of each column (entries close to the clamp at 0 have no meaningful
entrywise relative error).  Supports must agree except where the oracle's
projected value lies within the tolerance of the t-th largest value or of
zero.  For FP32 the oracle receives the same FP32-rounded A and iterate the
GPU uses, so only the arithmetic differs.
"""
import numpy as np
import pytest

import oracle
import paper_1510_05237_gb300 as E
from gen import Corpus, planted_50k_100k, planted_corpus, small_zipf, uniform_init, zipf_corpus
from helpers import compare_factor, make_ctx

pytestmark = pytest.mark.gpu

TOL = {E.F64: 1e-12, E.F32: 2e-5}
# E through <U, AV>: the cross term carries the sparse product's rounding
# (FP32: ~1e-7 relative), so E agrees to ~1e-10 in FP64 and ~1e-6 in FP32.
ETOL = {E.F64: 1e-10, E.F32: 1e-6}
OMODE = {E.TOPT_COLUMN: oracle.COLUMN, E.TOPT_MATRIX: oracle.MATRIX, E.TOPT_NONE: oracle.NONE}


def as_used(A: Corpus, U0: np.ndarray, compute: int):
    """The A and U0 the GPU actually computes with."""
    if compute == E.F32:
        return A.astype(np.float32), U0.astype(np.float32).astype(np.float64)
    return A, U0


def step_parity(A, k, t_u, t_v, U0, mode, compute, what=""):
    """update_V then update_U on the GPU, each compared with the oracle from
    the GPU's own input iterate; R and E compared on the GPU's iterates."""
    tol = TOL[compute]
    Ao, U0o = as_used(A, U0, compute)
    ctx = make_ctx(A, k, t_u, t_v, U0, mode, compute)
    E.espnmf_als_update_V(ctx)
    Vg = E.espnmf_get_factor(ctx, E.V)
    Vo, Vpre = oracle.update_V(Ao, U0o, t_v, OMODE[mode], return_pre=True)
    compare_factor(Vg, Vo, Vpre, t_v, mode, tol, what + " V")
    E.espnmf_als_update_U(ctx)
    Ug = E.espnmf_get_factor(ctx, E.U)
    Uo, Upre = oracle.update_U(Ao, Vg, t_u, OMODE[mode], return_pre=True)
    compare_factor(Ug, Uo, Upre, t_u, mode, tol, what + " U")
    R, Eg = E.espnmf_residual(ctx), E.espnmf_error(ctx)
    Ro = oracle.residual(Ug, U0o)
    Eo = oracle.error_identity(Ao, Ug, Vg)
    assert abs(R - Ro) <= 1e-10 * max(1.0, Ro), (R, Ro)
    assert abs(Eg - Eo) <= ETOL[compute], (Eg, Eo)
    # invariants of the enforced factors
    for F, t in ((Vg, t_v), (Ug, t_u)):
        assert np.all(F >= 0) and not np.any(np.signbit(F))
        if mode == E.TOPT_COLUMN:
            assert np.count_nonzero(F, axis=0).max() <= t
        elif mode == E.TOPT_MATRIX:
            assert np.count_nonzero(F) <= t
    return ctx, Ug, Vg


@pytest.mark.parametrize("compute", [E.F64, E.F32])
@pytest.mark.parametrize("mode,t", [(E.TOPT_COLUMN, 100), (E.TOPT_MATRIX, 700), (E.TOPT_NONE, 0)])
def test_step_parity_zipf_2000x500(compute, mode, t):
    A = small_zipf(1)
    U0 = uniform_init(A.n, 10, 1)
    step_parity(A, 10, t, t, U0, mode, compute, "zipf")


@pytest.mark.parametrize("compute", [E.F64, E.F32])
def test_step_parity_planted_scaled(compute):
    A = planted_50k_100k(seed=2, scale=0.05)
    assert np.diff(A.rowptr).max() > 256   # long rows are cut into segments
    U0 = uniform_init(A.n, 50, 2)
    ctx, Ug, Vg = step_parity(A, 50, 120, 150, U0, E.TOPT_COLUMN, compute, "planted")
    # a second sweep from the enforced iterate (sparse factors this time)
    Ao, _ = as_used(A, U0, compute)
    E.espnmf_als_update_V(ctx)
    V2 = E.espnmf_get_factor(ctx, E.V)
    Vo, Vpre = oracle.update_V(Ao, Ug, 150, oracle.COLUMN, return_pre=True)
    compare_factor(V2, Vo, Vpre, 150, E.TOPT_COLUMN, TOL[compute], "planted V2")
    E.espnmf_als_update_U(ctx)
    U2 = E.espnmf_get_factor(ctx, E.U)
    Uo, Upre = oracle.update_U(Ao, V2, 120, oracle.COLUMN, return_pre=True)
    compare_factor(U2, Uo, Upre, 120, E.TOPT_COLUMN, TOL[compute], "planted U2")
    assert abs(E.espnmf_residual(ctx) - oracle.residual(U2, Ug)) < 1e-9


def test_selector_threshold_hint_miss_falls_back():
    """The FP32 selector starts each column's search from the threshold that
    column had in the previous sweep.  Scaling U by 2^10 moves every
    threshold ten binades away from its hint: the search must fall back to
    the full radix selection, and the steps (the fallback one, then a warm
    one) still match the oracle."""
    A = planted_50k_100k(seed=2, scale=0.05)
    U0 = uniform_init(A.n, 50, 2)
    ctx = make_ctx(A, 50, 120, 150, U0, E.TOPT_COLUMN, E.F32)
    E.espnmf_iterate(ctx, 3)
    w0, f0 = E.espnmf_select_stats(ctx)
    assert w0 + f0 >= 3 * 2 * 50 and f0 >= 2 * 50   # the first sweep has no hints
    Ucur = E.espnmf_get_factor(ctx, E.U).astype(np.float32) * np.float32(1024.0)
    E.espnmf_set_factor(ctx, E.U, Ucur)
    Ucur = Ucur.astype(np.float64)
    Ao, _ = as_used(A, U0, E.F32)
    for step in range(2):
        E.espnmf_als_update_V(ctx)
        if step == 0:
            w1, f1 = E.espnmf_select_stats(ctx)
            assert (w1, f1) == (w0, f0 + 50)   # every V column missed its hint
        Vg = E.espnmf_get_factor(ctx, E.V)
        Vo, Vpre = oracle.update_V(Ao, Ucur, 150, oracle.COLUMN, return_pre=True)
        compare_factor(Vg, Vo, Vpre, 150, E.TOPT_COLUMN, 2e-5, f"hint miss V{step}")
        E.espnmf_als_update_U(ctx)
        Ug = E.espnmf_get_factor(ctx, E.U)
        Uo, Upre = oracle.update_U(Ao, Vg, 120, oracle.COLUMN, return_pre=True)
        compare_factor(Ug, Uo, Upre, 120, E.TOPT_COLUMN, 2e-5, f"hint miss U{step}")
        Ucur = Ug
    w2, f2 = E.espnmf_select_stats(ctx)
    assert w2 + f2 == w0 + f0 + 2 * 2 * 50


@pytest.mark.parametrize("compute", [E.F64, E.F32])
@pytest.mark.parametrize("k", [1, 3, 33, 64, 72])
def test_step_parity_factor_widths(compute, k):
    """Every factor row width: one 16-byte chunk (k <= 4), a partial second
    chunk (k = 33), two full chunks (k = 64) and the per-lane gathers of
    k > 64, each from a dense start (all rows heavy) and then from the
    enforced iterate (light and heavy rows mixed)."""
    A = planted_50k_100k(seed=7, scale=0.02)
    U0 = uniform_init(A.n, k, 7)
    t_u, t_v = max(1, A.n // 12), max(1, A.m // 15)
    ctx, Ug, Vg = step_parity(A, k, t_u, t_v, U0, E.TOPT_COLUMN, compute, f"k={k}")
    Ao, _ = as_used(A, U0, compute)
    E.espnmf_als_update_V(ctx)
    V2 = E.espnmf_get_factor(ctx, E.V)
    Vo, Vpre = oracle.update_V(Ao, Ug, t_v, oracle.COLUMN, return_pre=True)
    compare_factor(V2, Vo, Vpre, t_v, E.TOPT_COLUMN, TOL[compute], f"k={k} V2")
    E.espnmf_als_update_U(ctx)
    U2 = E.espnmf_get_factor(ctx, E.U)
    Uo, Upre = oracle.update_U(Ao, V2, t_u, oracle.COLUMN, return_pre=True)
    compare_factor(U2, Uo, Upre, t_u, E.TOPT_COLUMN, TOL[compute], f"k={k} U2")


def test_full_size_planted_50k_100k_fp32():
    """The benchmarked workload (~10M nnz, k=50, t=1000) in FP32, launched as
    the benchmark launches it, both half-steps compared in full."""
    A = planted_50k_100k(seed=2)
    U0 = uniform_init(A.n, 50, 2)
    ctx, Ug, Vg = step_parity(A, 50, 1000, 1000, U0, E.TOPT_COLUMN, E.F32, "C2")
    # one more sweep through the captured graph, from the enforced iterate
    Ao = A.astype(np.float32)
    R, Es = E.espnmf_iterate(ctx, 1)
    U2 = E.espnmf_get_factor(ctx, E.U)
    V2 = E.espnmf_get_factor(ctx, E.V)
    Vo, Vpre = oracle.update_V(Ao, Ug, 1000, oracle.COLUMN, return_pre=True)
    compare_factor(V2, Vo, Vpre, 1000, E.TOPT_COLUMN, 2e-5, "C2 V2")
    Uo, Upre = oracle.update_U(Ao, V2, 1000, oracle.COLUMN, return_pre=True)
    compare_factor(U2, Uo, Upre, 1000, E.TOPT_COLUMN, 2e-5, "C2 U2")
    assert abs(R[0] - oracle.residual(U2, Ug)) < 1e-9
    assert abs(Es[0] - oracle.error_identity(Ao, U2, V2)) < ETOL[E.F32]


@pytest.mark.parametrize("compute", [E.F64, E.F32])
def test_exact_ties_keep_lower_index(compute):
    """Duplicated documents give bitwise-equal rows of V on both sides; the
    enforcement must keep the lower row index."""
    rng = np.random.default_rng(3)
    D = rng.random((40, 30)) * (rng.random((40, 30)) < 0.3) + 0.01 * (rng.random((40, 30)) < 0.05)
    D[:, 20:30] = D[:, 0:10]          # docs 20..29 duplicate docs 0..9
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(41, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=40), out=rowptr[1:])
    A = Corpus(40, 30, rowptr, cols.astype(np.int32), D[rows, cols])
    U0 = uniform_init(40, 3, 3)
    Ao, U0o = as_used(A, U0, compute)
    for t in [1, 3, 5, 11]:
        ctx = make_ctx(A, 3, 10, t, U0, E.TOPT_COLUMN, compute)
        E.espnmf_als_update_V(ctx)
        Vg = E.espnmf_get_factor(ctx, E.V)
        Vo = oracle.update_V(Ao, U0o, t, oracle.COLUMN)
        if compute == E.F64:
            np.testing.assert_array_equal(Vg != 0, Vo != 0)
        # the GPU's own ties are resolved toward the lower index
        for c in range(3):
            for j in range(10):
                if Vg[20 + j, c] != 0:
                    assert Vg[j, c] != 0


@pytest.mark.parametrize("compute", [E.F64, E.F32])
def test_edge_cases(compute):
    rng = np.random.default_rng(5)
    n, m = 300, 200
    D = rng.random((n, m)) * (rng.random((n, m)) < 0.05)
    D[7, :] = rng.random(m) + 0.1          # a dense row (cut into segments)
    D[:, 11] = 0.0                          # an empty document
    D[13, :] = 0.0                          # an empty term
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    A = Corpus(n, m, rowptr, cols.astype(np.int32), D[rows, cols])
    # k = 1: the solve is a division
    step_parity(A, 1, 10, 10, uniform_init(n, 1, 5), E.TOPT_COLUMN, compute, "k1")
    # t >= column length: Alg. 1
    step_parity(A, 4, n, m, uniform_init(n, 4, 6), E.TOPT_COLUMN, compute, "t=len")
    # ragged sizes, k not a multiple of 8
    step_parity(A, 13, 17, 9, uniform_init(n, 13, 7), E.TOPT_COLUMN, compute, "k13")
    # t = 0 empties V; the U step then drops every column of the Gram
    ctx = make_ctx(A, 3, 5, 0, uniform_init(n, 3, 8), E.TOPT_COLUMN, compute)
    E.espnmf_als_update_V(ctx)
    assert E.espnmf_factor_nnz(ctx, E.V) == 0
    E.espnmf_als_update_U(ctx)
    assert E.espnmf_factor_nnz(ctx, E.U) == 0
    assert E.espnmf_residual(ctx) == np.inf


def test_singular_and_nonfinite_are_reported():
    A = small_zipf(2)
    U0 = uniform_init(A.n, 4, 2)
    U0[:, 3] = U0[:, 1]
    ctx = make_ctx(A, 4, 50, 50, U0, E.TOPT_COLUMN, E.F64)
    E.espnmf_als_update_V(ctx)
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_sync(ctx)
    assert ei.value.status == E.ERR_SINGULAR
    U0 = uniform_init(A.n, 4, 2)
    U0[5, 2] = np.nan
    with pytest.raises(E.EspnmfError) as ei:
        make_ctx(A, 4, 50, 50, U0, E.TOPT_COLUMN, E.F64)
    assert ei.value.status == E.ERR_NONFINITE
    U0 = uniform_init(A.n, 4, 2)
    U0[5, 2] = -1.0
    with pytest.raises(E.EspnmfError) as ei:
        make_ctx(A, 4, 50, 50, U0, E.TOPT_COLUMN, E.F64)
    assert ei.value.status == E.ERR_INVALID_ARG


def test_bad_matrix_is_rejected():
    A = small_zipf(2)
    U0 = uniform_init(A.n, 4, 2)
    bad = A.val.copy()
    bad[3] = -1.0
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_init(A.rowptr, A.colidx, bad, A.n, A.m, 4, 5, 5, E.TOPT_COLUMN, E.F64, U0)
    assert ei.value.status == E.ERR_BAD_MATRIX
    ci = A.colidx.copy()
    ci[A.rowptr[1]] = A.m
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_init(A.rowptr, ci, A.val, A.n, A.m, 4, 5, 5, E.TOPT_COLUMN, E.F64, U0)
    assert ei.value.status == E.ERR_BAD_MATRIX


@pytest.mark.parametrize("compute", [E.F64, E.F32])
@pytest.mark.parametrize("mode", [E.TOPT_COLUMN, E.TOPT_MATRIX])
def test_enforce_topt_on_context_and_buffer(compute, mode):
    import torch
    A = small_zipf(3)
    U0 = uniform_init(A.n, 6, 3)
    ctx = make_ctx(A, 6, 2000, 500, U0, mode, compute)
    E.espnmf_iterate(ctx, 2)
    Ug = E.espnmf_get_factor(ctx, E.U)
    for t in [0, 1, 7, 40]:
        tt = t if mode == E.TOPT_COLUMN else 6 * t
        ctx2 = make_ctx(A, 6, 2000, 500, U0, mode, compute)
        E.espnmf_iterate(ctx2, 2)
        E.espnmf_enforce_topt(ctx2, E.U, tt)
        got = E.espnmf_get_factor(ctx2, E.U)
        np.testing.assert_array_equal(got, oracle.topt(Ug, tt, OMODE[mode]))
    # stand-alone selector on a device buffer with ties and negatives
    rng = np.random.default_rng(9)
    X = (rng.integers(-3, 6, (1000, 7)) * 0.25).astype(np.float64)
    dt = torch.float64 if compute == E.F64 else torch.float32
    for t in [0, 1, 5, 333, 5000]:
        Xd = torch.tensor(X, dtype=dt, device="cuda")
        E.espnmf_enforce_topt_buffer(Xd, t, mode)
        ref = oracle.topt(np.maximum(X, 0), t, OMODE[mode])
        np.testing.assert_array_equal(Xd.double().cpu().numpy(), ref)


def test_factor_export_layouts_agree():
    A = small_zipf(4)
    ctx = make_ctx(A, 8, 90, 60, uniform_init(A.n, 8, 4), E.TOPT_COLUMN, E.F32)
    E.espnmf_iterate(ctx, 3)
    for which, rows in ((E.U, A.n), (E.V, A.m)):
        D = E.espnmf_get_factor(ctx, which)
        cp, ci, cv = E.espnmf_get_factor(ctx, which, E.CSC)
        rp, ri, rv = E.espnmf_get_factor(ctx, which, E.CSR)
        assert cp[-1] == rp[-1] == np.count_nonzero(D) == E.espnmf_factor_nnz(ctx, which)
        Dc = np.zeros_like(D)
        for c in range(8):
            seg = slice(cp[c], cp[c + 1])
            assert np.all(np.diff(ci[seg]) > 0)
            Dc[ci[seg], c] = cv[seg]
        Dr = np.zeros_like(D)
        for r in range(rows):
            seg = slice(rp[r], rp[r + 1])
            assert np.all(np.diff(ri[seg]) > 0)
            Dr[r, ri[seg]] = rv[seg]
        np.testing.assert_array_equal(Dc, D)
        np.testing.assert_array_equal(Dr, D)


def test_error_after_set_factor_matches_oracle():
    A = small_zipf(5)
    rng = np.random.default_rng(6)
    U0 = uniform_init(A.n, 5, 5)
    ctx = make_ctx(A, 5, 100, 100, U0, E.TOPT_COLUMN, E.F64)
    E.espnmf_iterate(ctx, 1)
    V = rng.random((A.m, 5)) * (rng.random((A.m, 5)) < 0.3)
    U = rng.random((A.n, 5)) * (rng.random((A.n, 5)) < 0.2)
    E.espnmf_set_factor(ctx, E.V, V)
    E.espnmf_set_factor(ctx, E.U, U)
    assert abs(E.espnmf_error(ctx) - oracle.error_identity(A, U, V)) < 1e-12
    assert abs(oracle.error_identity(A, U, V) - oracle.error_direct(A, U, V)) < 1e-12


def test_graph_replay_equals_eager_and_is_deterministic():
    A = planted_50k_100k(seed=4, scale=0.03)
    U0 = uniform_init(A.n, 20, 4)
    out = []
    for graph in (1, 0, 1):
        ctx = make_ctx(A, 20, 80, 100, U0, E.TOPT_COLUMN, E.F32)
        E.espnmf_set_option(ctx, E.OPT_USE_GRAPH, graph)
        R, Es = E.espnmf_iterate(ctx, 6)
        out.append((R, Es, E.espnmf_get_factor(ctx, E.U), E.espnmf_get_factor(ctx, E.V)))
    for a, b in ((out[0], out[1]), (out[0], out[2])):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    R, Es = out[0][0], out[0][1]
    assert np.all(np.isfinite(R)) and np.all((Es > 0) & (Es < 1))


def test_sweep_measures_on_gpu_iterates():
    A = zipf_corpus(3000, 2000, 40, 1.1, 8, sigma=0.5)
    U0 = uniform_init(A.n, 12, 8)
    ctx = make_ctx(A, 12, 150, 120, U0, E.TOPT_COLUMN, E.F64)
    E.espnmf_iterate(ctx, 4)
    U4 = E.espnmf_get_factor(ctx, E.U)
    R, Es = E.espnmf_iterate(ctx, 1)
    U5, V5 = E.espnmf_get_factor(ctx, E.U), E.espnmf_get_factor(ctx, E.V)
    assert abs(R[0] - oracle.residual(U5, U4)) < 1e-12
    assert abs(Es[0] - oracle.error_direct(A, U5, V5)) < 1e-11


def test_spmm_launch_shapes_give_identical_results():
    """Every FP32 sparse-product shape (1, 2 or 4 warps per slice, any
    shared-memory carveout, any way of skipping zero factor rows, or the
    tuner's choice) adds the same products in the same order: the sweeps
    agree bitwise."""
    A = planted_50k_100k(seed=2, scale=0.05)
    U0 = uniform_init(A.n, 50, 2)
    runs = []
    for opts in [{}, {E.OPT_SPMM_SPLIT: 1}, {E.OPT_SPMM_SPLIT: 2}, {E.OPT_SPMM_SPLIT: 4},
                 {E.OPT_SPMM_SPLIT: 2, E.OPT_SPMM_CARVEOUT: 25},
                 {E.OPT_SPMM_SPLIT: 4, E.OPT_SPMM_CARVEOUT: 100},
                 {E.OPT_SPMM_SPLIT: 1, E.OPT_SPMM_MASK: 0},
                 {E.OPT_SPMM_SPLIT: 1, E.OPT_SPMM_MASK: 2},
                 {E.OPT_SPMM_SPLIT: 2, E.OPT_SPMM_MASK: 2}]:
        ctx = make_ctx(A, 50, 120, 150, U0, E.TOPT_COLUMN, E.F32)
        for o, v in opts.items():
            E.espnmf_set_option(ctx, o, v)
        R1, E1 = E.espnmf_iterate(ctx, 1)
        R2, E2 = E.espnmf_iterate(ctx, 3)
        runs.append((np.concatenate([R1, R2]), np.concatenate([E1, E2]),
                     E.espnmf_get_factor(ctx, E.U), E.espnmf_get_factor(ctx, E.V)))
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            np.testing.assert_array_equal(a, b)


def _transpose(A: Corpus) -> Corpus:
    """The corpus with terms and documents exchanged (CSR of A^T)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    order = np.lexsort((rows, A.colidx))
    rowptr = np.zeros(A.m + 1, dtype=np.int64)
    np.cumsum(np.bincount(A.colidx, minlength=A.m), out=rowptr[1:])
    return Corpus(A.m, A.n, rowptr, rows[order].astype(np.int32), A.val[order].copy())


@pytest.mark.parametrize("transposed", [False, True])
@pytest.mark.parametrize("sparse_start", [False, True])
def test_frequent_part_matches_oracle(transposed, sparse_start):
    """The frequent terms' entries go through the dense-table kernel: A^T U on
    the Zipf corpus, A V on its transpose (whose documents are Zipf); from a
    dense start, and from a sparse one whose frequent rows are partly zero;
    two sweeps, each half-step from the GPU's own iterate."""
    from gen import sparse_init
    A = small_zipf(3)
    if transposed:
        A = _transpose(A)
    k, t = 12, 40
    U0 = sparse_init(A.n, k, 6, 3) if sparse_start else uniform_init(A.n, k, 3)
    ctx = make_ctx(A, k, t, t, U0, E.TOPT_COLUMN, E.F32)
    h, hnnz = E.espnmf_spmm_frequent(ctx, 0 if transposed else 1)
    assert h > 0 and hnnz * 10 >= A.nnz, (h, hnnz)
    Ao = A.astype(np.float32)
    Ucur = U0.astype(np.float32).astype(np.float64)
    for sweep in range(2):
        E.espnmf_als_update_V(ctx)
        Vg = E.espnmf_get_factor(ctx, E.V)
        Vo, Vpre = oracle.update_V(Ao, Ucur, t, oracle.COLUMN, return_pre=True)
        compare_factor(Vg, Vo, Vpre, t, E.TOPT_COLUMN, 2e-5, f"freq V{sweep}")
        E.espnmf_als_update_U(ctx)
        Ug = E.espnmf_get_factor(ctx, E.U)
        Uo, Upre = oracle.update_U(Ao, Vg, t, oracle.COLUMN, return_pre=True)
        compare_factor(Ug, Uo, Upre, t, E.TOPT_COLUMN, 2e-5, f"freq U{sweep}")
        assert abs(E.espnmf_error(ctx) - oracle.error_identity(Ao, Ug, Vg)) < ETOL[E.F32]
        assert abs(E.espnmf_residual(ctx) - oracle.residual(Ug, Ucur)) < 1e-9
        Ucur = Ug


def test_benchmark_corpus_uses_the_frequent_part():
    """The planted corpus routes its frequent terms through the dense table
    (A^T U) and leaves A V, whose documents are not skewed, to the SELL part."""
    A = planted_50k_100k(seed=2, scale=0.05)
    ctx = make_ctx(A, 50, 120, 150, uniform_init(A.n, 50, 2), E.TOPT_COLUMN, E.F32)
    h_atu, e_atu = E.espnmf_spmm_frequent(ctx, 1)
    h_av, e_av = E.espnmf_spmm_frequent(ctx, 0)
    assert h_atu > 0 and e_atu * 10 >= A.nnz
    assert h_av == 0 and e_av == 0
    ctx64 = make_ctx(A, 50, 120, 150, uniform_init(A.n, 50, 2), E.TOPT_COLUMN, E.F64)
    assert E.espnmf_spmm_frequent(ctx64, 1) == (0, 0)


@pytest.mark.parametrize("scale", [1e14, 1e-17])
def test_step_parity_with_factor_scaled_far_from_one(scale):
    """A factor scaled by 1e14 (or 1e-17) puts the Gram pivots beyond 1e30
    (below 1e-30), outside the range where the FP32 seed of the Cholesky
    pivot's inverse square root is used; the FP32 form must still solve the
    system (V scales by 1/scale, and the U half meets pivots on the other
    side) and match the oracle.  (The FP32 form's Gram sums square FP32
    factor entries, so entries beyond about 1e18 or below 1e-18 are outside
    its range; the FP64 form has no such limit.)"""
    A = small_zipf(6)
    U0 = uniform_init(A.n, 8, 6) * scale
    step_parity(A, 8, 90, 70, U0, E.TOPT_COLUMN, E.F32, f"scale={scale:g}")


@pytest.mark.parametrize("compute", [E.F64, E.F32])
def test_enforce_topt_buffer_leaves_nonfinite_input_unchanged(compute):
    import torch
    rng = np.random.default_rng(10)
    X = (rng.integers(-3, 6, (500, 7)) * 0.25).astype(np.float64)
    X[17, 3] = np.nan
    X[40, 0] = np.inf
    dt = torch.float64 if compute == E.F64 else torch.float32
    Xd = torch.tensor(X, dtype=dt, device="cuda")
    before = Xd.clone()
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_enforce_topt_buffer(Xd, 10, E.TOPT_COLUMN)
    assert ei.value.status == E.ERR_NONFINITE
    assert torch.equal(torch.isnan(Xd), torch.isnan(before))
    assert torch.equal(torch.nan_to_num(Xd), torch.nan_to_num(before))
