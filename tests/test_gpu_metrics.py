"""The clustering accuracy of Sec. 3.2 (Eq. 3-4) computed on the device
(espnmf_topic_accuracy) against the oracle's pair-by-pair count on the same
factor."""
import numpy as np
import pytest

import oracle
import paper_1510_05237_gb300 as E
from gen import planted_50k_100k, uniform_init
from helpers import make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("compute", [E.F64, E.F32])
def test_topic_accuracy_matches_oracle(compute):
    import torch
    A = planted_50k_100k(seed=3, scale=0.05)
    n_cls = int(A.labels.max()) + 1
    ctx = make_ctx(A, 20, 150, 200, uniform_init(A.n, 20, 3), E.TOPT_COLUMN, compute)
    E.espnmf_iterate(ctx, 4)
    V = E.espnmf_get_factor(ctx, E.V)
    ref = oracle.topic_accuracy(V, A.labels, n_cls)
    got = E.espnmf_topic_accuracy(ctx, A.labels, n_cls)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    got_dev = E.espnmf_topic_accuracy(ctx, torch.from_numpy(A.labels).cuda(), n_cls)
    np.testing.assert_array_equal(got, got_dev)
    # U's columns against labels of the terms (any integer classes will do)
    term_cls = (np.arange(A.n) % 7).astype(np.int32)
    np.testing.assert_allclose(E.espnmf_topic_accuracy(ctx, term_cls, 7, which=E.U),
                               oracle.topic_accuracy(E.espnmf_get_factor(ctx, E.U), term_cls, 7),
                               rtol=0, atol=1e-12)
    bad = A.labels.copy()
    bad[np.flatnonzero((V != 0).any(axis=1))[0]] = n_cls
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_topic_accuracy(ctx, bad, n_cls)
    assert ei.value.status == E.ERR_INVALID_ARG
    E.espnmf_sync(ctx)   # the context is still usable
