"""Sequential ALS (Sec. 4, Alg. 3, rank-1 topics): the oracle pinned against
independent formulations -- the first topic is Alg. 2 with k = 1, and every
update is the dense least-squares fit of the deflated matrix
A - U1 V1^T (numpy lstsq), then the projection and the top-t rule (brute
force); plus the invariants of the result."""
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
