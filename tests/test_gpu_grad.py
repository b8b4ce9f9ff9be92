"""GPU parity of the squared objective f = ||A - U V^T||_F^2, its gradients,
the projected-gradient polish and the autograd Function, against the FP64
oracle and against central differences of the GPU's own FP64 loss.

f is quadratic in U for fixed V (and in V for fixed U), so a central
difference is exact up to rounding for any step h: with h = 1e-3 the
difference carries an error of about eps |f| / h.  Entries are perturbed on
the support (value > 2h), since a factor must stay non-negative.
"""
import numpy as np
import pytest

import oracle
import paper_1510_05237_gb300 as E
from gen import small_zipf, uniform_init, zipf_100k_200k
from helpers import compare_factor, make_ctx

pytestmark = pytest.mark.gpu

TOL = {E.F64: 1e-12, E.F32: 2e-5}
FTOL = {E.F64: 1e-11, E.F32: 1e-6}


def as_used(A, compute):
    return A.astype(np.float32) if compute == E.F32 else A


def grad_scale(Ao, U, V):
    """Size of the two terms of 2 (U G_V - A V): the error bound's scale."""
    AV = oracle.spmm_A(Ao, V)
    UG = U @ oracle.gram(V)
    AtU = oracle.spmm_At(Ao, U)
    VG = V @ oracle.gram(U)
    return (2 * max(np.abs(AV).max(), np.abs(UG).max()),
            2 * max(np.abs(AtU).max(), np.abs(VG).max()))


@pytest.mark.parametrize("compute", [E.F64, E.F32])
def test_loss_and_gradients_match_oracle(compute):
    A = small_zipf()
    k, t = 10, 100
    ctx = make_ctx(A, k, t, t, uniform_init(A.n, k, 1), compute=compute)
    E.espnmf_iterate(ctx, 2, want_measures=False)
    U = E.espnmf_get_factor(ctx, E.U)
    V = E.espnmf_get_factor(ctx, E.V)
    Ao = as_used(A, compute)
    f = E.espnmf_loss(ctx)
    fo = oracle.loss(Ao, U, V)
    a2 = float(np.sum(Ao.val ** 2))
    assert abs(f - fo) <= FTOL[compute] * a2, (f, fo)
    su, sv = grad_scale(Ao, U, V)
    for which, ref, sc in ((E.U, oracle.grad_U(Ao, U, V), su),
                           (E.V, oracle.grad_V(Ao, U, V), sv)):
        for dt in (np.float64, np.float32):
            g = E.espnmf_grad(ctx, which, dtype=dt)
            err = np.abs(g.astype(np.float64) - ref).max() / sc
            lim = TOL[compute] if dt == np.float64 else max(TOL[compute], 1e-7)
            assert err <= lim, (which, dt, err)


def test_gradient_into_device_tensor_and_host_agree():
    import torch
    A = small_zipf()
    ctx = make_ctx(A, 8, 80, 80, uniform_init(A.n, 8, 3))
    E.espnmf_iterate(ctx, 1, want_measures=False)
    h = E.espnmf_grad(ctx, E.V)
    d = torch.empty((A.m, 8), dtype=torch.float64, device="cuda")
    E.espnmf_grad(ctx, E.V, d)
    assert np.array_equal(d.cpu().numpy(), h)


def central_difference_check(ctx, U, V, which, entries, h=1e-3):
    g = E.espnmf_grad(ctx, which)
    F = U if which == E.U else V
    worst = 0.0
    for (i, j) in entries:
        vals = []
        for s in (+h, -h):
            Fp = F.copy()
            Fp[i, j] += s
            E.espnmf_set_factor(ctx, which, Fp)
            vals.append(E.espnmf_loss(ctx))
        E.espnmf_set_factor(ctx, which, F)
        fd = (vals[0] - vals[1]) / (2 * h)
        bound = 64 * np.finfo(float).eps * max(abs(vals[0]), 1.0) / h
        assert abs(fd - g[i, j]) <= bound + 1e-9 * abs(g[i, j]), (i, j, fd, g[i, j], bound)
        worst = max(worst, abs(fd - g[i, j]))
    return worst


def support_entries(F, count, seed, h=1e-3):
    rng = np.random.default_rng(seed)
    rows, cols = np.nonzero(F > 2 * h)
    pick = rng.choice(len(rows), size=min(count, len(rows)), replace=False)
    return list(zip(rows[pick].tolist(), cols[pick].tolist()))


def test_gradients_match_central_differences_small():
    A = small_zipf()
    k, t = 10, 100
    ctx = make_ctx(A, k, t, t, uniform_init(A.n, k, 1))
    E.espnmf_iterate(ctx, 2, want_measures=False)
    U = E.espnmf_get_factor(ctx, E.U)
    V = E.espnmf_get_factor(ctx, E.V)
    central_difference_check(ctx, U, V, E.U, support_entries(U, 16, 1))
    central_difference_check(ctx, U, V, E.V, support_entries(V, 16, 2))


@pytest.mark.parametrize("which", [E.U, E.V])
def test_pg_step_matches_oracle_and_descends(which):
    A = small_zipf()
    k, t = 10, 100
    ctx = make_ctx(A, k, t, t, uniform_init(A.n, k, 1))
    E.espnmf_iterate(ctx, 2, want_measures=False)
    U = E.espnmf_get_factor(ctx, E.U)
    V = E.espnmf_get_factor(ctx, E.V)
    f0 = E.espnmf_loss(ctx)
    eta = E.espnmf_pg_step(ctx, which)
    G = oracle.gram(V if which == E.U else U)
    lam = oracle.lambda_max(G)
    assert abs(eta - 1.0 / (2.0 * lam)) <= 1e-13 * eta
    Uo, Vo = oracle.pg_step(A, U, V, 0 if which == E.U else 1)
    ref = Uo if which == E.U else Vo
    got = E.espnmf_get_factor(ctx, which)
    # same support or a subset: entries that reached 0 leave it
    before = U if which == E.U else V
    assert np.all((got != 0) <= (before != 0))
    compare_factor(got, ref, ref, 10 ** 9, E.TOPT_NONE, TOL[E.F64], "pg")
    f1 = E.espnmf_loss(ctx)
    assert f1 <= f0 * (1 + 1e-12), (f0, f1)
    # a caller's step is used as given
    eta2 = E.espnmf_pg_step(ctx, which, 0.25 * eta)
    assert eta2 == 0.25 * eta


def test_autograd_function_backward_is_the_gradient():
    import torch
    from paper_1510_05237_gb300.autograd import reconstruction_loss
    A = small_zipf()
    k, t = 10, 100
    ctx = make_ctx(A, k, t, t, uniform_init(A.n, k, 1))
    E.espnmf_iterate(ctx, 2, want_measures=False)
    Un = E.espnmf_get_factor(ctx, E.U)
    Vn = E.espnmf_get_factor(ctx, E.V)
    U = torch.tensor(Un, device="cuda", requires_grad=True)
    V = torch.tensor(Vn, device="cuda", requires_grad=True)
    f = reconstruction_loss(U, V, ctx)
    assert abs(f.item() - oracle.loss(A, Un, Vn)) <= 1e-11 * float(np.sum(A.val ** 2))
    (3.0 * f).backward()
    su, sv = grad_scale(A, Un, Vn)
    assert np.abs(U.grad.cpu().numpy() - 3.0 * oracle.grad_U(A, Un, Vn)).max() <= 3e-12 * su
    assert np.abs(V.grad.cpu().numpy() - 3.0 * oracle.grad_V(A, Un, Vn)).max() <= 3e-12 * sv


@pytest.fixture(scope="module")
def c5():
    """100k terms x 200k docs, ~20M nnz, Zipf(1.1); k = 64, t = 2000."""
    A = zipf_100k_200k()
    k, t = 64, 2000
    ctx = make_ctx(A, k, t, t, uniform_init(A.n, k, 5))
    E.espnmf_iterate(ctx, 1, want_measures=False)
    return A, ctx


def test_full_size_gradients_finite_differences_and_oracle(c5):
    A, ctx = c5
    U = E.espnmf_get_factor(ctx, E.U)
    V = E.espnmf_get_factor(ctx, E.V)
    # 64 random support entries of each factor against central differences
    central_difference_check(ctx, U, V, E.U, support_entries(U, 64, 11))
    central_difference_check(ctx, U, V, E.V, support_entries(V, 64, 12))
    # 64 random entries (any, zero or not) against the oracle's gradient
    rng = np.random.default_rng(13)
    su, sv = grad_scale(A, U, V)
    for which, ref_fn, sc in ((E.U, oracle.grad_U, su), (E.V, oracle.grad_V, sv)):
        g = E.espnmf_grad(ctx, which)
        ref = ref_fn(A, U, V)
        ii = rng.integers(0, g.shape[0], 64)
        jj = rng.integers(0, g.shape[1], 64)
        assert np.abs(g[ii, jj] - ref[ii, jj]).max() <= 1e-12 * sc


def test_full_size_pg_polish_interleaved_with_als(c5):
    A, ctx = c5
    for step in range(5):
        E.espnmf_iterate(ctx, 1, want_measures=False)
        f0 = E.espnmf_loss(ctx)
        E.espnmf_pg_step(ctx, E.U)
        f1 = E.espnmf_loss(ctx)
        E.espnmf_pg_step(ctx, E.V)
        f2 = E.espnmf_loss(ctx)
        assert f1 <= f0 * (1 + 1e-12) and f2 <= f1 * (1 + 1e-12), (step, f0, f1, f2)
        assert E.espnmf_factor_nnz(ctx, E.U) <= 64 * 2000
        assert E.espnmf_factor_nnz(ctx, E.V) <= 64 * 2000
