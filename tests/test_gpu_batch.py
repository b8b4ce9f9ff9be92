"""Batched sweeps of independent problems (uneven n, m, k, t) against each
problem's own context run alone (bitwise: batching adds no arithmetic) and,
for a few problems, one step against the FP64 oracle.  A problem with a
singular start fails alone; the others go on."""
import numpy as np
import pytest

import oracle
import paper_1510_05237_gb300 as E
from gen import batch_problems, uniform_init
from helpers import compare_factor, make_ctx

pytestmark = pytest.mark.gpu


def problem_args(A, k, t_u, t_v, U0, compute):
    vals = A.val if compute == E.F64 else A.val.astype(np.float32)
    return (A.rowptr, A.colidx, vals, A.n, A.m, k, t_u, t_v, U0)


@pytest.mark.parametrize("compute", [E.F64, E.F32])
def test_batch_equals_each_problem_alone(compute):
    probs = batch_problems(12, seed=4, max_scale=0.25)
    U0s = [uniform_init(A.n, k, 100 + i) for i, (A, k, tu, tv) in enumerate(probs)]
    b = E.espnmf_batch_init([problem_args(A, k, tu, tv, U0s[i], compute)
                             for i, (A, k, tu, tv) in enumerate(probs)],
                            compute=compute, streams=4)
    status, R, Es = E.espnmf_batch_iterate(b, 4)
    assert (status == 0).all(), status
    for i, (A, k, tu, tv) in enumerate(probs):
        ctx = make_ctx(A, k, tu, tv, U0s[i], compute=compute)
        R1, E1 = E.espnmf_iterate(ctx, 4)
        np.testing.assert_array_equal(R[i], R1)
        np.testing.assert_array_equal(Es[i], E1)
        bc = b.ctx(i)
        for which in (E.U, E.V):
            np.testing.assert_array_equal(E.espnmf_get_factor(bc, which),
                                          E.espnmf_get_factor(ctx, which))


def test_batch_step_parity_with_oracle():
    probs = batch_problems(6, seed=9, max_scale=0.2)
    U0s = [uniform_init(A.n, k, 7 + i) for i, (A, k, tu, tv) in enumerate(probs)]
    b = E.espnmf_batch_init([problem_args(A, k, tu, tv, U0s[i], E.F64)
                             for i, (A, k, tu, tv) in enumerate(probs)], compute=E.F64)
    status, _, _ = E.espnmf_batch_iterate(b, 2)
    assert (status == 0).all()
    Us = [E.espnmf_get_factor(b.ctx(i), E.U) for i in range(len(probs))]
    status, _, _ = E.espnmf_batch_iterate(b, 1)
    assert (status == 0).all()
    for i, (A, k, tu, tv) in enumerate(probs):
        V = E.espnmf_get_factor(b.ctx(i), E.V)
        Vo, Vpre = oracle.update_V(A, Us[i], tv, oracle.COLUMN, return_pre=True)
        compare_factor(V, Vo, Vpre, tv, E.TOPT_COLUMN, 1e-12, f"batch {i} V")
        U = E.espnmf_get_factor(b.ctx(i), E.U)
        Uo, Upre = oracle.update_U(A, V, tu, oracle.COLUMN, return_pre=True)
        compare_factor(U, Uo, Upre, tu, E.TOPT_COLUMN, 1e-12, f"batch {i} U")


def test_one_singular_problem_fails_alone():
    probs = batch_problems(5, seed=11, max_scale=0.2)
    U0s = [uniform_init(A.n, k, 3 + i) for i, (A, k, tu, tv) in enumerate(probs)]
    U0s[2][:, 1] = U0s[2][:, 0]        # two equal columns: U0^T U0 is singular
    b = E.espnmf_batch_init([problem_args(A, k, tu, tv, U0s[i], E.F64)
                             for i, (A, k, tu, tv) in enumerate(probs)], compute=E.F64)
    status, R, Es = E.espnmf_batch_iterate(b, 3)
    assert status[2] == E.ERR_SINGULAR
    assert all(status[i] == 0 for i in range(5) if i != 2), status
    assert np.all(np.isfinite(Es[[0, 1, 3, 4]]))


def test_batch_without_graph_is_identical():
    probs = batch_problems(4, seed=13, max_scale=0.2)
    U0s = [uniform_init(A.n, k, 5 + i) for i, (A, k, tu, tv) in enumerate(probs)]
    args = [problem_args(A, k, tu, tv, U0s[i], E.F32) for i, (A, k, tu, tv) in enumerate(probs)]
    b1 = E.espnmf_batch_init(args)
    b2 = E.espnmf_batch_init(args)
    E.espnmf_batch_set_option(b2, E.OPT_USE_GRAPH, 0)
    _, R1, E1 = E.espnmf_batch_iterate(b1, 3)
    _, R2, E2 = E.espnmf_batch_iterate(b2, 3)
    np.testing.assert_array_equal(R1, R2)
    np.testing.assert_array_equal(E1, E2)
