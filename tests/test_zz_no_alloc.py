"""The allocation-free selector (espnmf_enforce_topt_buffer_noalloc).

Some callers must not allocate device memory while the library works -- a
service that budgets all of its device memory once at start-up, or a host
program that hands every byte to its own pool.  For them the library has a
variant of the stand-alone selector whose scratch lives in a fixed array
inside the library.  These tests call it through the C ABI and check that it
returns exactly what the allocating entry point returns (selection keeps
existing values, so the tolerance is zero), on two calls in a row -- the
array keeps the previous call's contents, so the second call would expose
anything left uncleared.  This file is named to be collected last.
"""
import numpy as np
import pytest

import paper_1510_05237_gb300 as E

pytestmark = pytest.mark.gpu


def make_x(rng, rows, k):
    # few distinct values (ties at the threshold) and negatives (projection)
    return (rng.integers(-3, 9, (rows, k)) * 0.125).astype(np.float64)


@pytest.mark.parametrize("mode", [E.TOPT_COLUMN, E.TOPT_MATRIX, E.TOPT_NONE])
def test_noalloc_selector_equals_allocating_selector(mode):
    import torch
    rng = np.random.default_rng(7)
    for dtype in (torch.float32, torch.float64):
        for rows, k, t in [(3000, 50, 400), (777, 13, 5), (4096, 64, 1)]:
            tt = t if mode != E.TOPT_MATRIX else t * k // 3
            X = torch.tensor(make_x(rng, rows, k), dtype=dtype, device="cuda")
            for call in range(2):   # two calls in a row on the shared array
                a = X.clone()
                b = X.clone()
                E.espnmf_enforce_topt_buffer(a, tt, mode)
                E.espnmf_enforce_topt_buffer_noalloc(b, tt, mode)
                torch.cuda.synchronize()
                assert torch.equal(a, b), (rows, k, tt, call)


def test_noalloc_selector_rejects_inputs_beyond_its_array():
    import torch
    rows = E.NOALLOC_MAX_ELEMS // 4 + 1          # k = 4 -> ld = 4
    X = torch.ones(rows, 4, device="cuda")
    before = X.clone()
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_enforce_topt_buffer_noalloc(X, 3)
    assert ei.value.status == E.ERR_INVALID_ARG
    assert torch.equal(X, before)
    # the largest accepted size still works
    Y = torch.ones(E.NOALLOC_MAX_ELEMS // 4, 4, device="cuda")
    E.espnmf_enforce_topt_buffer_noalloc(Y, 3)
    assert int((Y != 0).sum()) == 12


def test_noalloc_selector_leaves_nonfinite_input_unchanged():
    import torch
    rng = np.random.default_rng(11)
    X = make_x(rng, 300, 9)
    X[5, 4] = np.nan
    for dtype in (torch.float32, torch.float64):
        Xd = torch.tensor(X, dtype=dtype, device="cuda")
        before = Xd.clone()
        for call in range(2):
            with pytest.raises(E.EspnmfError) as ei:
                E.espnmf_enforce_topt_buffer_noalloc(Xd, 4)
            assert ei.value.status == E.ERR_NONFINITE
            assert torch.equal(torch.nan_to_num(Xd), torch.nan_to_num(before))
        # the array is usable again after the rejected calls
        Y = torch.tensor(np.maximum(X, 0), dtype=dtype, device="cuda")
        Y[5, 4] = 0.0
        Z = Y.clone()
        E.espnmf_enforce_topt_buffer(Y, 4)
        E.espnmf_enforce_topt_buffer_noalloc(Z, 4)
        assert torch.equal(Y, Z)
