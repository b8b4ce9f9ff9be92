"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these re-type the oracle's own formulas: each compares it with an
independent route -- a QR least-squares solve, a brute-force sort, a dense
reconstruction, a closed form, an exact planted factorisation, an invariance
of the method, a hand-derived worked example or finite differences -- so that
a dropped term, a wrong sign, a swapped index or a transposed operand fails
at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle
from gen import Corpus, small_zipf, uniform_init

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def corpus_from_dense(D: np.ndarray) -> Corpus:
    n, m = D.shape
    rows, cols = np.nonzero(D)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return Corpus(n, m, rowptr, cols.astype(np.int32), D[rows, cols].astype(np.float64))


def rand_sparse(rng, n, m, density):
    D = rng.random((n, m)) * (rng.random((n, m)) < density)
    D[rng.integers(0, n), :] += 0.1   # no empty document
    return D


def qr_lstsq(M: np.ndarray, B: np.ndarray) -> np.ndarray:
    """min ||M x - b|| for every column b of B by Householder QR."""
    Q, R = np.linalg.qr(M)
    return np.linalg.solve(R, Q.T @ B)


# ---------------------------------------------------------------------------
# Alg. 2 steps 1 and 3: the least-squares step

@pytest.mark.parametrize("n,m,k", [(12, 9, 3), (10, 7, 4), (8, 11, 2)])
def test_ls_step_equals_qr_least_squares(n, m, k):
    rng = np.random.default_rng(n * 100 + k)
    D = rand_sparse(rng, n, m, 0.5)
    A = corpus_from_dense(D)
    U = rng.random((n, k))
    _, Vpre = oracle.update_V(A, U, t_v=m, mode=oracle.NONE, return_pre=True)
    # V = argmin ||A - U V^T||: column j of A^T is fitted by U v_j
    Vref = qr_lstsq(U, D).T
    np.testing.assert_allclose(Vpre, Vref, rtol=0, atol=1e-12 * np.abs(Vref).max())
    V = rng.random((m, k))
    _, Upre = oracle.update_U(A, V, t_u=n, mode=oracle.NONE, return_pre=True)
    Uref = qr_lstsq(V, D.T).T
    np.testing.assert_allclose(Upre, Uref, rtol=0, atol=1e-12 * np.abs(Uref).max())


def test_k1_is_a_division():
    """Rank 1: the k x k inverse is one floating-point division."""
    rng = np.random.default_rng(3)
    D = rand_sparse(rng, 15, 10, 0.4)
    A = corpus_from_dense(D)
    u = rng.random((15, 1))
    V = oracle.update_V(A, u, t_v=10, mode=oracle.COLUMN)
    ref = np.maximum(0.0, (D.T @ u) / float(u[:, 0] @ u[:, 0]))
    np.testing.assert_allclose(V, ref, rtol=1e-14, atol=0)


def test_projection_clamps_negatives_and_signed_zero():
    X = np.array([[-1.0, -0.0], [0.0, 2.5], [3.0, -1e-300]])
    P = oracle.project(X)
    assert np.all(P >= 0)
    assert not np.any(np.signbit(P))
    np.testing.assert_array_equal(P, [[0, 0], [0, 2.5], [3.0, 0]])
    with pytest.raises(oracle.OracleError) as e:
        oracle.project(np.array([[1.0, np.nan]]))
    assert e.value.status == oracle.NONFINITE


def test_t_at_least_column_length_equals_alg1():
    """With t >= the column length, Alg. 2 reduces to Alg. 1 (clamped LS)."""
    rng = np.random.default_rng(5)
    D = rand_sparse(rng, 14, 9, 0.4)
    A = corpus_from_dense(D)
    U = rng.random((14, 3))
    V2 = oracle.update_V(A, U, t_v=9, mode=oracle.COLUMN)
    V1 = oracle.update_V(A, U, t_v=0, mode=oracle.NONE)
    np.testing.assert_array_equal(V2, V1)
    np.testing.assert_allclose(V1, np.maximum(qr_lstsq(U, D).T, 0), atol=1e-12)


# ---------------------------------------------------------------------------
# Alg. 2 steps 2 and 4: the top-t rule

def brute_topt(X, t, mode):
    X = np.array(X, dtype=float)
    out = np.zeros_like(X)
    rows, k = X.shape
    if mode == oracle.NONE:
        return X
    if mode == oracle.COLUMN:
        for c in range(k):
            cand = sorted([(-X[i, c], i) for i in range(rows) if X[i, c] > 0])
            for _, i in cand[:t]:
                out[i, c] = X[i, c]
        return out
    cand = sorted([(-X[i, c], i * k + c) for i in range(rows) for c in range(k)
                   if X[i, c] > 0])
    for _, q in cand[:t]:
        out[q // k, q % k] = X[q // k, q % k]
    return out


@pytest.mark.parametrize("mode", [oracle.COLUMN, oracle.MATRIX])
@pytest.mark.parametrize("seed", range(6))
def test_topt_equals_brute_force_sort(mode, seed):
    rng = np.random.default_rng(seed)
    rows, k = int(rng.integers(1, 30)), int(rng.integers(1, 6))
    # few distinct values so that ties at the threshold are common
    X = rng.integers(0, 5, (rows, k)).astype(float) * rng.choice([1.0, 0.5], (rows, k))
    for t in [0, 1, 2, 3, 7, rows, rows * k + 1]:
        np.testing.assert_array_equal(oracle.topt(X, t, mode), brute_topt(X, t, mode))


def test_topt_counts_and_tie_order():
    X = np.array([[1.0, 2.0], [1.0, 0.0], [1.0, 2.0], [0.5, 2.0]])
    Y = oracle.topt(X, 2, oracle.COLUMN)
    np.testing.assert_array_equal(Y, [[1, 2], [1, 0], [0, 2], [0, 0]])
    Z = oracle.topt(X, 3, oracle.MATRIX)
    np.testing.assert_array_equal(Z, [[0, 2], [0, 0], [0, 2], [0, 2]])


# ---------------------------------------------------------------------------
# Sec. 3.1 measures

def test_error_identity_equals_dense_reconstruction():
    rng = np.random.default_rng(11)
    for n, m, k in [(9, 7, 2), (13, 6, 3), (5, 12, 4)]:
        D = rand_sparse(rng, n, m, 0.5)
        A = corpus_from_dense(D)
        U, V = rng.random((n, k)), rng.random((m, k))
        ref = np.linalg.norm(D - U @ V.T) / np.linalg.norm(D)
        assert abs(oracle.error_identity(A, U, V) - ref) <= 1e-12 * ref
        assert abs(oracle.error_direct(A, U, V) - ref) <= 1e-12 * ref
        f = np.linalg.norm(D - U @ V.T) ** 2
        assert abs(oracle.loss(A, U, V) - f) <= 1e-12 * np.linalg.norm(D) ** 2


def test_residual_matches_frobenius_definition():
    rng = np.random.default_rng(2)
    a, b = rng.random((7, 3)), rng.random((7, 3))
    assert abs(oracle.residual(a, b) - np.linalg.norm(a - b) / np.linalg.norm(a)) < 1e-15
    z = np.zeros((7, 3))
    assert oracle.residual(z, z) == 0.0
    assert oracle.residual(z, b) == np.inf


# ---------------------------------------------------------------------------
# Hand-derived worked examples

def test_golden_k1_worked_example():
    g = json.load(open(os.path.join(GOLD, "k1_worked_example.json")))
    A = corpus_from_dense(np.array(g["dense_A"]))
    U0 = np.array(g["U0"])
    V1 = oracle.update_V(A, U0, g["t_v"], oracle.COLUMN)
    np.testing.assert_allclose(V1, g["V1"], rtol=1e-15, atol=0)
    U1 = oracle.update_U(A, V1, g["t_u"], oracle.COLUMN)
    np.testing.assert_allclose(U1, g["U1"], rtol=1e-15, atol=0)
    U, V, R, E = oracle.iterate(A, U0, g["t_u"], g["t_v"], oracle.COLUMN, 1)
    assert abs(R[0] ** 2 - g["R1_squared"]) < 1e-14
    assert abs(E[0] ** 2 - g["E1_squared"]) < 1e-14


def test_golden_k2_worked_example():
    g = json.load(open(os.path.join(GOLD, "k2_worked_example.json")))
    A = corpus_from_dense(np.array(g["dense_A"]))
    U = np.array(g["U"])
    _, pre = oracle.update_V(A, U, 3, oracle.NONE, return_pre=True)
    np.testing.assert_allclose(pre, g["V_pre"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.update_V(A, U, 1, oracle.COLUMN),
                               g["V_column_t1"], rtol=0, atol=1e-15)
    np.testing.assert_array_equal(oracle.update_V(A, np.array(g["U2"]), 3, oracle.MATRIX),
                                  g["V2_matrix_t3"])


# ---------------------------------------------------------------------------
# Exact factorisation: a fixed point that reaches machine precision

def test_planted_exact_factorisation_is_a_fixed_point():
    rng = np.random.default_rng(7)
    n, m, k, t = 40, 30, 4, 6
    Us, Vs = np.zeros((n, k)), np.zeros((m, k))
    for c in range(k):   # disjoint supports, t nonzeros per column
        Us[c * t:(c + 1) * t, c] = rng.random(t) + 0.5
        Vs[c * t + 1:(c + 1) * t + 1, c] = rng.random(t) + 0.5
    A = corpus_from_dense(Us @ Vs.T)
    U, V, R, E = oracle.iterate(A, Us, t, t, oracle.COLUMN, 1)
    np.testing.assert_allclose(V, Vs, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(U, Us, rtol=1e-12, atol=1e-14)
    assert E[0] < 1e-7 and R[0] < 1e-12


# ---------------------------------------------------------------------------
# Invariances

def test_scale_by_two_scales_factor_exactly():
    """Scaling A by a power of two scales V by the same, bitwise; supports
    and E are unchanged (the top-t rule does not depend on scaling)."""
    A = small_zipf(3)
    U0 = uniform_init(A.n, 6, 3)
    A2 = Corpus(A.n, A.m, A.rowptr, A.colidx, A.val * 2.0)
    V = oracle.update_V(A, U0, 50)
    V2 = oracle.update_V(A2, U0, 50)
    np.testing.assert_array_equal(V2, 2.0 * V)
    _, _, _, E = oracle.iterate(A, U0, 80, 50, oracle.COLUMN, 2)
    _, _, _, E2 = oracle.iterate(A2, U0, 80, 50, oracle.COLUMN, 2)
    np.testing.assert_allclose(E2, E, rtol=1e-13)


def test_permutation_equivariance():
    rng = np.random.default_rng(13)
    D = rand_sparse(rng, 25, 18, 0.3)
    U = rng.random((25, 3))
    pr, pc, pk = rng.permutation(25), rng.permutation(18), rng.permutation(3)
    A = corpus_from_dense(D)
    Ap = corpus_from_dense(D[pr][:, pc])
    V = oracle.update_V(A, U, 5)
    Vp = oracle.update_V(Ap, U[pr][:, pk], 5)
    np.testing.assert_allclose(Vp, V[pc][:, pk], rtol=1e-12, atol=1e-15)


def test_sweep_invariants_both_modes():
    A = small_zipf(1)
    U0 = uniform_init(A.n, 10, 1)
    for mode, t in [(oracle.COLUMN, 100), (oracle.MATRIX, 400)]:
        U, V, R, E = oracle.iterate(A, U0, t, t, mode, 3)
        assert np.all(U >= 0) and np.all(V >= 0)
        if mode == oracle.COLUMN:
            assert np.count_nonzero(U, axis=0).max() <= t
            assert np.count_nonzero(V, axis=0).max() <= t
        else:
            assert np.count_nonzero(U) <= t and np.count_nonzero(V) <= t
        assert np.all(np.isfinite(R)) and np.all((E >= 0) & (E <= 1.0 + 1e-12))


# ---------------------------------------------------------------------------
# Singular Gram readings

def test_zero_factor_column_gives_minimum_norm_solution():
    rng = np.random.default_rng(17)
    D = rand_sparse(rng, 12, 8, 0.5)
    A = corpus_from_dense(D)
    U = rng.random((12, 3))
    U[:, 1] = 0.0
    _, pre = oracle.update_V(A, U, 8, oracle.NONE, return_pre=True)
    ref = np.linalg.pinv(U) @ D   # minimum-norm least squares
    np.testing.assert_allclose(pre, ref.T, atol=1e-12)
    assert np.all(pre[:, 1] == 0)


def test_dependent_columns_are_singular():
    rng = np.random.default_rng(19)
    A = corpus_from_dense(rand_sparse(rng, 10, 6, 0.5))
    U = rng.random((10, 3))
    U[:, 2] = U[:, 0]
    with pytest.raises(oracle.OracleError) as e:
        oracle.update_V(A, U, 6)
    assert e.value.status == oracle.SINGULAR


def test_nonfinite_factor_is_an_error():
    rng = np.random.default_rng(23)
    A = corpus_from_dense(rand_sparse(rng, 10, 6, 0.5))
    U = rng.random((10, 2))
    U[3, 1] = np.inf
    with pytest.raises(oracle.OracleError) as e:
        oracle.update_V(A, U, 6)
    assert e.value.status == oracle.NONFINITE


# ---------------------------------------------------------------------------
# Loss gradients (Eq. 6 objective) and the polish step

def test_gradients_match_central_differences():
    rng = np.random.default_rng(29)
    D = rand_sparse(rng, 9, 7, 0.5)
    A = corpus_from_dense(D)
    U, V = rng.random((9, 3)), rng.random((7, 3))
    f = lambda U_, V_: np.linalg.norm(D - U_ @ V_.T) ** 2
    gU, gV = oracle.grad_U(A, U, V), oracle.grad_V(A, U, V)
    h = 1e-3
    for (i, c) in [(0, 0), (4, 2), (8, 1)]:
        Up, Um = U.copy(), U.copy()
        Up[i, c] += h
        Um[i, c] -= h
        fd = (f(Up, V) - f(Um, V)) / (2 * h)   # exact for a quadratic
        assert abs(fd - gU[i, c]) < 1e-8 * max(1.0, abs(fd))
        Vp, Vm = V.copy(), V.copy()
        Vp[i % 7, c] += h
        Vm[i % 7, c] -= h
        fd = (f(U, Vp) - f(U, Vm)) / (2 * h)
        assert abs(fd - gV[i % 7, c]) < 1e-8 * max(1.0, abs(fd))


def test_lambda_max_and_pg_step_descends():
    rng = np.random.default_rng(31)
    M = rng.random((6, 6))
    G = M @ M.T
    lam = oracle.lambda_max(G)
    assert abs(lam - np.linalg.eigvalsh(G)[-1]) < 1e-9 * lam
    A = small_zipf(2)
    U0 = uniform_init(A.n, 5, 2)
    U, V, _, _ = oracle.iterate(A, U0, 60, 40, oracle.COLUMN, 2)
    f0 = oracle.loss(A, U, V)
    U1, V1 = oracle.pg_step(A, U, V, 0)
    f1 = oracle.loss(A, U1, V1)
    assert f1 <= f0 * (1 + 1e-14)
    assert np.all((U1 != 0) <= (U != 0))   # support only shrinks
    U2, V2 = oracle.pg_step(A, U1, V1, 1)
    assert oracle.loss(A, U2, V2) <= f1 * (1 + 1e-14)
    assert np.all(U2 >= 0) and np.all(V2 >= 0)


def test_pg_step_size_is_pinned_by_the_rank_one_minimiser():
    """With k = 1 the objective is a 1-D quadratic in each entry of u:
    f(u) = ||A - u v^T||^2 has gradient 2 (u v^T v - A v) and curvature
    2 v^T v, so a step of length 1 / (2 v^T v) from any u lands exactly on
    the unconstrained minimiser A v / v^T v; the projection then clamps it
    at 0 and keeps u's support.  The expected value below is that closed
    form, written out independently of the oracle: a step of twice the
    length (1 / v^T v) would land on 2 A v / v^T v - u instead."""
    rng = np.random.default_rng(37)
    D = rand_sparse(rng, 11, 8, 0.6)
    A = corpus_from_dense(D)
    u = rng.random((11, 1)) + 0.1
    u[[2, 7]] = 0.0                     # outside the support: stays 0
    v = rng.random((8, 1)) + 0.1
    U1, V1 = oracle.pg_step(A, u, v, 0)
    ls = (D @ v[:, 0]) / float(v[:, 0] @ v[:, 0])
    expect = np.where(u[:, 0] > 0, np.maximum(ls, 0.0), 0.0)
    assert np.allclose(U1[:, 0], expect, rtol=1e-12, atol=1e-14)
    assert np.array_equal(V1, v)
    # and the V step from the same closed form with the roles swapped
    U2, V2 = oracle.pg_step(A, u, v, 1)
    ls_v = (D.T @ u[:, 0]) / float(u[:, 0] @ u[:, 0])
    expect_v = np.where(v[:, 0] > 0, np.maximum(ls_v, 0.0), 0.0)
    assert np.allclose(V2[:, 0], expect_v, rtol=1e-12, atol=1e-14)


def test_openmp_build_gives_bitwise_the_same_sweeps():
    """The all-cores CPU baseline runs the oracle's OpenMP build; its loops
    split work between threads without reordering any sum, so its sweeps
    equal the single-threaded build's bit for bit."""
    A = small_zipf(3)
    U0 = uniform_init(A.n, 7, 3)
    for mode, t in ((oracle.COLUMN, 40), (oracle.MATRIX, 300), (oracle.NONE, 0)):
        a = oracle.iterate(A, U0, t, t, mode, 3)
        b = oracle.iterate(A, U0, t, t, mode, 3, threads=4)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
