"""The FP32 column selector on columns long enough to be split over a
cluster of two CTAs (at least 32768 rows): the warm start sums its counts
over the cluster, a hint miss falls back to the full search on both CTAs,
and exact ties between rows held by different CTAs go to the lower row."""
import numpy as np
import pytest

import oracle
import paper_1510_05237_gb300 as E
from gen import Corpus, planted_50k_100k, uniform_init
from helpers import compare_factor, make_ctx

pytestmark = pytest.mark.gpu

M_SPLIT = 40000   # documents: rows of V, split 20000 / 20000 over the cluster


def test_ties_across_the_two_ctas_keep_the_lower_row():
    rng = np.random.default_rng(12)
    n = 40
    D = (rng.random((n, M_SPLIT)) * (rng.random((n, M_SPLIT)) < 0.2)).astype(np.float32)
    D[:, 30000:30010] = D[:, 5:15]      # documents 30000.. duplicate 5.. (other CTA)
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    A = Corpus(n, M_SPLIT, rowptr, cols.astype(np.int32), D[rows, cols].astype(np.float64))
    U0 = uniform_init(n, 3, 4).astype(np.float32).astype(np.float64)
    for t in (5, 11, 997):
        ctx = make_ctx(A, 3, 10, t, U0, E.TOPT_COLUMN, E.F32)
        E.espnmf_als_update_V(ctx)
        Vg = E.espnmf_get_factor(ctx, E.V)
        assert np.count_nonzero(Vg, axis=0).max() <= t
        for c in range(3):
            for j in range(10):
                assert Vg[30000 + j, c] == Vg[5 + j, c] or Vg[30000 + j, c] == 0
                if Vg[30000 + j, c] != 0:
                    assert Vg[5 + j, c] != 0, (t, c, j)
        Vo, Vpre = oracle.update_V(A, U0, t, oracle.COLUMN, return_pre=True)
        compare_factor(Vg, Vo, Vpre, t, E.TOPT_COLUMN, 2e-5, f"ties t={t}")
        E.espnmf_destroy(ctx)


def test_two_cta_warm_start_and_hint_miss_match_the_oracle():
    A = planted_50k_100k(seed=2, scale=0.36)          # 18000 terms x 36000 documents
    assert A.m >= 32768
    U0 = uniform_init(A.n, 50, 2)
    ctx = make_ctx(A, 50, 150, 200, U0, E.TOPT_COLUMN, E.F32)
    E.espnmf_iterate(ctx, 3)
    w0, f0 = E.espnmf_select_stats(ctx)
    assert w0 > 0                                   # warm starts held on the split columns
    Ao = A.astype(np.float32)
    # every V column misses its hint after U is scaled by 2^10
    Ucur = E.espnmf_get_factor(ctx, E.U).astype(np.float32) * np.float32(1024.0)
    E.espnmf_set_factor(ctx, E.U, Ucur)
    Ucur = Ucur.astype(np.float64)
    for step in range(2):
        E.espnmf_als_update_V(ctx)
        if step == 0:
            w1, f1 = E.espnmf_select_stats(ctx)
            assert (w1, f1) == (w0, f0 + 50)
        Vg = E.espnmf_get_factor(ctx, E.V)
        Vo, Vpre = oracle.update_V(Ao, Ucur, 200, oracle.COLUMN, return_pre=True)
        compare_factor(Vg, Vo, Vpre, 200, E.TOPT_COLUMN, 2e-5, f"split V{step}")
        E.espnmf_als_update_U(ctx)
        Ug = E.espnmf_get_factor(ctx, E.U)
        Uo, Upre = oracle.update_U(Ao, Vg, 150, oracle.COLUMN, return_pre=True)
        compare_factor(Ug, Uo, Upre, 150, E.TOPT_COLUMN, 2e-5, f"split U{step}")
        R, Eg = E.espnmf_residual(ctx), E.espnmf_error(ctx)
        assert abs(Eg - oracle.error_identity(Ao, Ug, Vg)) < 1e-6
        Ucur = Ug
    w2, f2 = E.espnmf_select_stats(ctx)
    assert w2 > w1      # the second step's V columns started warm again
