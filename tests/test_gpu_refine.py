"""One step of iterative refinement of the FP32 form's solve X = Y G^-1:
against the FP64 solution of the same FP32 system, the refined X is the
FP64 answer rounded to FP32 within a few ulps, while the plain FP32
substitution is off by about cond(G) 2^-24; and sweeps with the refinement
switched on still match the oracle step by step."""
import numpy as np
import pytest

import oracle
import paper_1510_05237_gb300 as E
from gen import planted_50k_100k, uniform_init
from helpers import compare_factor, make_ctx

pytestmark = pytest.mark.gpu


def spd(rng, k, cond):
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    lam = np.geomspace(1.0, 1.0 / cond, k)
    return (Q * lam) @ Q.T


@pytest.mark.parametrize("k,cond", [(1, 1.0), (13, 1e3), (50, 1e4), (64, 1e4)])
def test_refined_solve_is_the_fp64_solution_rounded(k, cond):
    import torch
    rng = np.random.default_rng(k)
    G = spd(rng, k, cond)
    Y = rng.standard_normal((3000, k)).astype(np.float32)
    X64 = np.linalg.solve(G.T, Y.astype(np.float64).T).T      # x G = y
    Yd = torch.from_numpy(Y).cuda()
    Gd = torch.from_numpy(G).cuda()
    plain = E.espnmf_solve_gram(Yd, Gd, refine=False).cpu().numpy().astype(np.float64)
    refined = E.espnmf_solve_gram(Yd, Gd, refine=True).cpu().numpy().astype(np.float64)
    rownorm = np.abs(X64).max(axis=1, keepdims=True)
    err_plain = (np.abs(plain - X64) / rownorm).max()
    err_ref = (np.abs(refined - X64) / rownorm).max()
    assert err_ref <= 4 * 2.0 ** -24, (err_ref, err_plain)
    if cond >= 1e3:
        assert err_ref * 8 < err_plain, (err_ref, err_plain)


def test_solve_gram_drops_zero_columns_and_reports_singular():
    import torch
    rng = np.random.default_rng(3)
    G = spd(rng, 6, 10.0)
    G[2, :] = 0.0
    G[:, 2] = 0.0
    Y = rng.standard_normal((100, 6)).astype(np.float32)
    Y[:, 2] = 0.0
    X = E.espnmf_solve_gram(torch.from_numpy(Y).cuda(), torch.from_numpy(G).cuda(), True)
    X = X.cpu().numpy()
    keep = [0, 1, 3, 4, 5]
    ref = np.linalg.solve(G[np.ix_(keep, keep)].T, Y[:, keep].astype(np.float64).T).T
    assert np.all(X[:, 2] == 0.0)
    assert np.abs(X[:, keep] - ref).max() <= 1e-6 * np.abs(ref).max()
    G2 = spd(rng, 6, 10.0)
    G2[4] = G2[1]
    G2[:, 4] = G2[:, 1]
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_solve_gram(torch.from_numpy(Y).cuda(), torch.from_numpy(G2).cuda(), True)
    assert ei.value.status == E.ERR_SINGULAR


def test_sweeps_with_refinement_match_the_oracle():
    A = planted_50k_100k(seed=2, scale=0.05)
    U0 = uniform_init(A.n, 50, 2)
    Ao = A.astype(np.float32)
    ctx = make_ctx(A, 50, 120, 150, U0, E.TOPT_COLUMN, E.F32)
    E.espnmf_set_option(ctx, E.OPT_REFINE, 1)
    E.espnmf_iterate(ctx, 2)
    U2 = E.espnmf_get_factor(ctx, E.U)
    E.espnmf_als_update_V(ctx)
    Vg = E.espnmf_get_factor(ctx, E.V)
    Vo, Vpre = oracle.update_V(Ao, U2, 150, oracle.COLUMN, return_pre=True)
    compare_factor(Vg, Vo, Vpre, 150, E.TOPT_COLUMN, 2e-5, "refined V")
    E.espnmf_als_update_U(ctx)
    Ug = E.espnmf_get_factor(ctx, E.U)
    Uo, Upre = oracle.update_U(Ao, Vg, 120, oracle.COLUMN, return_pre=True)
    compare_factor(Ug, Uo, Upre, 120, E.TOPT_COLUMN, 2e-5, "refined U")
    assert abs(E.espnmf_error(ctx) - oracle.error_identity(Ao, Ug, Vg)) < 1e-6
