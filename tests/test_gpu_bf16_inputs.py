"""BF16 inputs: A's values and U0 given as BF16 are widened exactly to the
compute type at set-up, so a context built from BF16 tensors must give
bitwise the results of one built from the same values in FP32 (or FP64),
and one step matches the oracle on those values.  The arithmetic is not
BF16: BF16 compute stays unsupported."""
import numpy as np
import pytest
import torch

import oracle
import paper_1510_05237_gb300 as E
from gen import planted_50k_100k, uniform_init
from helpers import compare_factor

pytestmark = pytest.mark.gpu


def _ctx(A, vals, U0, compute, k=50, t=150):
    dev = lambda a: (a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))).cuda()
    return E.espnmf_init(dev(A.rowptr), dev(A.colidx), dev(vals), A.n, A.m, k, t, t,
                         E.TOPT_COLUMN, compute, dev(U0))


@pytest.mark.parametrize("compute", [E.F32, E.F64])
def test_bf16_inputs_equal_the_same_values_in_a_wider_type(compute):
    A = planted_50k_100k(seed=2, scale=0.1)
    vb = torch.from_numpy(A.val.astype(np.float32)).to(torch.bfloat16)
    ub = torch.from_numpy(uniform_init(A.n, 50, 2).astype(np.float32)).to(torch.bfloat16)
    wide = torch.float64 if compute == E.F64 else torch.float32
    c1 = _ctx(A, vb, ub, compute)
    c2 = _ctx(A, vb.to(wide), ub.to(wide), compute)
    R1, E1 = E.espnmf_iterate(c1, 3)
    R2, E2 = E.espnmf_iterate(c2, 3)
    np.testing.assert_array_equal(E1, E2)
    np.testing.assert_array_equal(R1, R2)
    for which in (E.U, E.V):
        np.testing.assert_array_equal(E.espnmf_get_factor(c1, which), E.espnmf_get_factor(c2, which))
    # set_factor with a BF16 factor
    Vb = torch.from_numpy(E.espnmf_get_factor(c1, E.V).astype(np.float32)).to(torch.bfloat16)
    E.espnmf_set_factor(c1, E.V, Vb.cuda())
    E.espnmf_set_factor(c2, E.V, Vb.to(wide).cuda())
    assert E.espnmf_error(c1) == E.espnmf_error(c2)
    E.espnmf_destroy(c1)
    E.espnmf_destroy(c2)


def test_bf16_inputs_one_step_matches_the_oracle():
    A = planted_50k_100k(seed=3, scale=0.05)
    vb = torch.from_numpy(A.val.astype(np.float32)).to(torch.bfloat16)
    ub = torch.from_numpy(uniform_init(A.n, 50, 3).astype(np.float32)).to(torch.bfloat16)
    Ao = A.__class__(A.n, A.m, A.rowptr, A.colidx, vb.float().double().numpy())
    U0o = ub.float().double().numpy()
    ctx = _ctx(A, vb, ub, E.F32)
    E.espnmf_als_update_V(ctx)
    Vg = E.espnmf_get_factor(ctx, E.V)
    Vo, Vpre = oracle.update_V(Ao, U0o, 150, oracle.COLUMN, return_pre=True)
    compare_factor(Vg, Vo, Vpre, 150, E.TOPT_COLUMN, 2e-5, "bf16 V")
    E.espnmf_destroy(ctx)


def test_bf16_compute_is_unsupported():
    A = planted_50k_100k(seed=3, scale=0.02)
    with pytest.raises(E.EspnmfError):
        _ctx(A, A.val.astype(np.float32), uniform_init(A.n, 50, 3).astype(np.float32), E.BF16)
