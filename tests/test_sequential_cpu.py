"""Sequential ALS (Sec. 4, Alg. 3): the oracle pinned against independent
formulations -- the first block is Alg. 2 with k2 topics, and every update
of a later block is the dense least-squares fit of the deflated matrix
A - U1 V1^T (numpy lstsq, QR/SVD based, not the normal equations), then the
projection and the top-t rule (brute force, per column); plus the
invariants of the result.  Rank-1 topics (k2 = 1, the case the paper times)
and blocks of k2 = 2, 3."""
import numpy as np
import pytest

import oracle
from gen import small_zipf, uniform_init


def keep_top(x, t):
    """Projection and top-t of one column by brute force (ties: lower index)."""
    x = np.where(x > 0, x, 0.0)
    pos = np.nonzero(x > 0)[0]
    if len(pos) > t:
        order = sorted(pos, key=lambda i: (-x[i], i))
        y = np.zeros_like(x)
        y[order[:t]] = x[order[:t]]
        return y
    return x


@pytest.fixture(scope="module")
def corpus():
    return small_zipf(seed=3)


def test_first_topic_is_alg2_with_one_topic(corpus):
    A = corpus
    u0 = uniform_init(A.n, 1, 4)[:, 0]
    U, V = oracle.sequential(A, u0, 1, 150, 120, 1)
    V2 = oracle.update_V(A, u0[:, None], 120, oracle.COLUMN)
    U2 = oracle.update_U(A, V2, 150, oracle.COLUMN)
    np.testing.assert_allclose(V[:, 0], V2[:, 0], rtol=1e-13, atol=0)
    np.testing.assert_allclose(U[:, 0], U2[:, 0], rtol=1e-13, atol=0)


def test_updates_fit_the_deflated_matrix(corpus):
    """Topic j's first V and U updates equal the least-squares fit of
    R = A - U1 V1^T (dense), then projection and top-t."""
    A = corpus
    Ad = A.dense()
    u0 = uniform_init(A.n, 1, 9)[:, 0]
    t_u, t_v = 200, 90
    for k in (2, 3):
        U, V, vpre, upre = oracle.sequential(A, u0, k, t_u, t_v, 1, return_pre=True)
        R = Ad - U[:, :k - 1] @ V[:, :k - 1].T
        v_ls = np.linalg.lstsq(u0[:, None], R, rcond=None)[0][0]       # min ||R - u0 v^T||
        np.testing.assert_allclose(vpre, v_ls, rtol=0, atol=1e-12 * np.abs(v_ls).max())
        v = keep_top(v_ls, t_v)
        np.testing.assert_allclose(V[:, k - 1], v, rtol=0, atol=1e-12 * np.abs(v).max())
        u_ls = np.linalg.lstsq(V[:, k - 1][:, None], R.T, rcond=None)[0][0]   # min ||R - u v^T||
        np.testing.assert_allclose(upre, u_ls, rtol=0, atol=1e-12 * np.abs(u_ls).max())
        np.testing.assert_allclose(U[:, k - 1], keep_top(u_ls, t_u), rtol=0,
                                   atol=1e-12 * np.abs(u_ls).max())


def test_result_is_nonnegative_and_sparse_per_topic(corpus):
    A = corpus
    u0 = uniform_init(A.n, 1, 2)[:, 0]
    U, V = oracle.sequential(A, u0, 4, 100, 60, 5)
    assert (U >= 0).all() and (V >= 0).all()
    assert ((U > 0).sum(axis=0) <= 100).all() and ((V > 0).sum(axis=0) <= 60).all()
    # later topics explain what the earlier ones left: the error decreases
    Ad = A.dense()
    errs = [np.linalg.norm(Ad - U[:, :j] @ V[:, :j].T) for j in range(1, 5)]
    assert all(b <= a + 1e-9 for a, b in zip(errs, errs[1:]))


def test_zero_initial_guess_gives_zero_topics(corpus):
    A = corpus
    U, V = oracle.sequential(A, np.zeros(A.n), 2, 50, 50, 2)
    assert not U.any() and not V.any()


def keep_top_cols(X, t):
    return np.stack([keep_top(X[:, j], t) for j in range(X.shape[1])], axis=1)


@pytest.mark.parametrize("k2,iters", [(2, 1), (3, 2)])
def test_one_block_is_alg2(corpus, k2, iters):
    """eta = 1: Alg. 3 is its START, Alg. 2 with k2 topics from U0."""
    A = corpus
    U0 = uniform_init(A.n, k2, 5)
    U, V = oracle.sequential(A, U0, k2, 150, 120, iters, k2=k2)
    Ua, Va, _, _ = oracle.iterate(A, U0, 150, 120, oracle.COLUMN, iters)
    np.testing.assert_array_equal(U, Ua)
    np.testing.assert_array_equal(V, Va)


@pytest.mark.parametrize("k2,k", [(2, 4), (2, 6), (3, 6)])
def test_block_updates_fit_the_deflated_matrix(corpus, k2, k):
    """The last block's first V2 and U2 (Eq. 7, Eq. 8) equal the
    least-squares fits of R = A - U1 V1^T: V2^T = argmin ||R - U0 X||,
    U2^T = argmin ||R^T - V2 X|| (numpy lstsq), then projection and top-t
    per column."""
    A = corpus
    Ad = A.dense()
    U0 = uniform_init(A.n, k2, 11)
    t_u, t_v = 200, 90
    U, V, vpre, upre = oracle.sequential(A, U0, k, t_u, t_v, 1, return_pre=True, k2=k2)
    k1 = k - k2
    R = Ad - U[:, :k1] @ V[:, :k1].T
    v_ls = np.linalg.lstsq(U0, R, rcond=None)[0].T                      # m x k2
    np.testing.assert_allclose(vpre, v_ls, rtol=0, atol=1e-11 * np.abs(v_ls).max())
    V2 = keep_top_cols(v_ls, t_v)
    np.testing.assert_array_equal(V[:, k1:] > 0, V2 > 0)
    np.testing.assert_allclose(V[:, k1:], V2, rtol=0, atol=1e-11 * np.abs(V2).max())
    u_ls = np.linalg.lstsq(V[:, k1:], R.T, rcond=None)[0].T             # n x k2
    np.testing.assert_allclose(upre, u_ls, rtol=0, atol=1e-11 * np.abs(u_ls).max())
    U2 = keep_top_cols(u_ls, t_u)
    np.testing.assert_array_equal(U[:, k1:] > 0, U2 > 0)
    np.testing.assert_allclose(U[:, k1:], U2, rtol=0, atol=1e-11 * np.abs(u_ls).max())


def test_blocks_are_nonnegative_and_sparse_per_column(corpus):
    A = corpus
    U0 = uniform_init(A.n, 2, 6)
    U, V = oracle.sequential(A, U0, 6, 100, 60, 4, k2=2)
    assert (U >= 0).all() and (V >= 0).all()
    assert ((U > 0).sum(axis=0) <= 100).all() and ((V > 0).sum(axis=0) <= 60).all()
    assert ((U > 0).sum(axis=0) > 0).all() and ((V > 0).sum(axis=0) > 0).all()


def test_block_size_must_divide_k(corpus):
    A = corpus
    with pytest.raises(oracle.OracleError):
        oracle.sequential(A, uniform_init(A.n, 2, 1), 5, 10, 10, 1, k2=2)
