"""The second tier of the frequent part: with k = 100 a 200 KB shared-memory
table holds 457 factor rows, and in column mode the frequent part takes up
to t of the candidate rows; the rows beyond the shared-memory table are read
from the factor's table in global memory by a second launch.  A Zipf corpus
with 1568 candidate terms and t_u = 1200 gets both tiers; half-steps from
a dense start and from converged iterates match the oracle."""
import numpy as np
import pytest

import oracle
import paper_1510_05237_gb300 as E
from gen import uniform_init, zipf_corpus
from helpers import compare_factor, make_ctx

pytestmark = pytest.mark.gpu

K, T_U, T_V = 100, 1200, 400


@pytest.fixture(scope="module")
def corpus():
    return zipf_corpus(60000, 40000, 60.0, 1.05, 7, sigma=0.7)


def test_both_tiers_match_the_oracle(corpus):
    A = corpus
    Ao = A.astype(np.float32)
    U0 = uniform_init(A.n, K, 7).astype(np.float32).astype(np.float64)
    ctx = make_ctx(A, K, T_U, T_V, U0, E.TOPT_COLUMN, E.F32)
    h, hnnz = E.espnmf_spmm_frequent(ctx, 1)
    assert h == T_U, h                       # 457 staged, the rest in the second tier
    assert hnnz > 0
    Ucur = U0
    for step in range(2):
        E.espnmf_als_update_V(ctx)
        Vg = E.espnmf_get_factor(ctx, E.V)
        Vo, Vpre = oracle.update_V(Ao, Ucur, T_V, oracle.COLUMN, return_pre=True)
        compare_factor(Vg, Vo, Vpre, T_V, E.TOPT_COLUMN, 2e-5, f"tier2 V{step}")
        E.espnmf_als_update_U(ctx)
        Ug = E.espnmf_get_factor(ctx, E.U)
        Uo, Upre = oracle.update_U(Ao, Vg, T_U, oracle.COLUMN, return_pre=True)
        compare_factor(Ug, Uo, Upre, T_U, E.TOPT_COLUMN, 2e-5, f"tier2 U{step}")
        Ucur = Ug
        if step == 0:
            # a few graph-replayed sweeps between the two compared steps
            E.espnmf_iterate(ctx, 3)
            Ucur = E.espnmf_get_factor(ctx, E.U)
    E.espnmf_destroy(ctx)


def test_both_tiers_in_the_document_product(corpus):
    """The transposed corpus: its documents are Zipf-skewed, so the product
    A V (the U half) gets both tiers.  The half-steps match the oracle, and
    so do R and E of the sweep: E needs ||A||^2 over every entry of A, the
    two tiers' included.  A sparse start (400 nonzeros per column) keeps the
    first Gram well conditioned for the FP32 tolerance at k = 100."""
    from gen import sparse_init
    from test_gpu_parity import _transpose
    A = _transpose(corpus)
    Ao = A.astype(np.float32)
    t_u, t_v = T_V, T_U                      # t of the gathered factor V: 1200
    U0 = sparse_init(A.n, K, 400, 9).astype(np.float32).astype(np.float64)
    ctx = make_ctx(A, K, t_u, t_v, U0, E.TOPT_COLUMN, E.F32)
    h, hnnz = E.espnmf_spmm_frequent(ctx, 0)
    assert h == t_v, h
    assert hnnz > 0
    Rg, Eg = E.espnmf_iterate(ctx, 1)
    Vg = E.espnmf_get_factor(ctx, E.V)
    Ug = E.espnmf_get_factor(ctx, E.U)
    Vo, Vpre = oracle.update_V(Ao, U0, t_v, oracle.COLUMN, return_pre=True)
    compare_factor(Vg, Vo, Vpre, t_v, E.TOPT_COLUMN, 2e-5, "tier2 A V: V")
    Uo, Upre = oracle.update_U(Ao, Vg, t_u, oracle.COLUMN, return_pre=True)
    compare_factor(Ug, Uo, Upre, t_u, E.TOPT_COLUMN, 2e-5, "tier2 A V: U")
    assert abs(Eg[0] - oracle.error_identity(Ao, Ug, Vg)) < 1e-6
    assert abs(Rg[0] - oracle.residual(Ug, U0)) < 1e-9
    E.espnmf_destroy(ctx)
