"""Sequential ALS (Sec. 4, Alg. 3; rank-1 topics and blocks of k2 > 1) on
the GPU against the oracle.  In FP64 the whole run is compared (supports exactly, values to
1e-10 of each column's largest: the data are continuous, so a threshold tie
within rounding is improbable); in FP32 the final reconstruction error.
Invalid arguments are rejected before any work."""
import numpy as np
import pytest
import torch

import oracle
import paper_1510_05237_gb300 as E
from gen import planted_corpus, small_zipf, uniform_init

pytestmark = pytest.mark.gpu


def run_gpu(A, k, t_u, t_v, iters, u0, compute, k2=1):
    vals = A.val if compute == E.F64 else A.val.astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    u = u0 if compute == E.F64 else u0.astype(np.float32)
    U, V = E.espnmf_sequential(dev(A.rowptr), dev(A.colidx), dev(vals), A.n, A.m, k, t_u, t_v,
                               iters, dev(u), compute, k2=k2)
    return U.double().cpu().numpy(), V.double().cpu().numpy()


def assert_same(G, O, what):
    assert G.shape == O.shape
    np.testing.assert_array_equal(G > 0, O > 0, err_msg=f"{what}: supports differ")
    scale = np.maximum(np.abs(O).max(axis=0), 1e-300)
    assert (np.abs(G - O) / scale).max() < 1e-10, what


@pytest.mark.parametrize("k,iters", [(1, 2), (3, 3), (5, 2)])
def test_sequential_matches_oracle_fp64(k, iters):
    A = small_zipf(seed=3)
    u0 = uniform_init(A.n, 1, 4)[:, 0]
    U, V = run_gpu(A, k, 150, 120, iters, u0, E.F64)
    Uo, Vo = oracle.sequential(A, u0, k, 150, 120, iters)
    assert_same(U, Uo, "U")
    assert_same(V, Vo, "V")


@pytest.mark.parametrize("k,k2,iters", [(4, 2, 2), (6, 3, 3), (6, 6, 2), (9, 3, 1)])
def test_sequential_blocks_match_oracle_fp64(k, k2, iters):
    A = small_zipf(seed=3)
    U0 = uniform_init(A.n, k2, 4)
    U, V = run_gpu(A, k, 150, 120, iters, U0, E.F64, k2=k2)
    Uo, Vo = oracle.sequential(A, U0, k, 150, 120, iters, k2=k2)
    assert_same(U, Uo, "U")
    assert_same(V, Vo, "V")


def test_sequential_blocks_planted_fp64_and_fp32():
    """k2 = 3 on a planted corpus: FP64 whole run against the oracle, FP32
    final error within 1e-4 of the oracle's."""
    A = planted_corpus(3000, 2000, 6, 60, 40.0, 0.6, 0.1, 0.05, 7)
    U0 = uniform_init(A.n, 3, 8)
    Uo, Vo = oracle.sequential(A, U0, 6, 200, 150, 4, k2=3)
    U, V = run_gpu(A, 6, 200, 150, 4, U0, E.F64, k2=3)
    assert_same(U, Uo, "U")
    assert_same(V, Vo, "V")
    U32, V32 = run_gpu(A, 6, 200, 150, 4, U0, E.F32, k2=3)
    assert (U32 >= 0).all() and (V32 >= 0).all()
    assert ((U32 > 0).sum(axis=0) <= 200).all() and ((V32 > 0).sum(axis=0) <= 150).all()
    e32 = oracle.error_direct(A.astype(np.float32), U32, V32)
    eo = oracle.error_direct(A, Uo, Vo)
    assert abs(e32 - eo) < 1e-4


def test_sequential_planted_fp64_and_fp32():
    A = planted_corpus(3000, 2000, 6, 60, 40.0, 0.6, 0.1, 0.05, 7)
    u0 = uniform_init(A.n, 1, 7)[:, 0]
    Uo, Vo = oracle.sequential(A, u0, 6, 200, 150, 4)
    U, V = run_gpu(A, 6, 200, 150, 4, u0, E.F64)
    assert_same(U, Uo, "U")
    assert_same(V, Vo, "V")
    U32, V32 = run_gpu(A, 6, 200, 150, 4, u0, E.F32)
    assert (U32 >= 0).all() and (V32 >= 0).all()
    assert ((U32 > 0).sum(axis=0) <= 200).all() and ((V32 > 0).sum(axis=0) <= 150).all()
    A32 = A.astype(np.float32)
    e32 = oracle.error_direct(A32, U32, V32)
    eo = oracle.error_direct(A, Uo, Vo)
    assert abs(e32 - eo) < 1e-4


def test_sequential_rejects_bad_arguments():
    A = small_zipf(seed=3)
    u0 = uniform_init(A.n, 1, 4)[:, 0]
    with pytest.raises(E.EspnmfError):
        run_gpu(A, 0, 10, 10, 1, u0, E.F64)
    with pytest.raises(E.EspnmfError):
        run_gpu(A, 2, 10, 10, 0, u0, E.F64)
    with pytest.raises(E.EspnmfError):                       # k not a multiple of k2
        run_gpu(A, 5, 10, 10, 1, uniform_init(A.n, 2, 4), E.F64, k2=2)
