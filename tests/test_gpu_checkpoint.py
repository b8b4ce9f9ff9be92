"""Checkpoint and resume (espnmf_save / espnmf_load): a run that stops,
saves its state and continues in a fresh context repeats the uninterrupted
run bit for bit -- factors, residuals and errors."""
import os

import numpy as np
import pytest

import paper_1510_05237_gb300 as E
from gen import planted_50k_100k, small_zipf, uniform_init
from helpers import make_ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("compute", [E.F64, E.F32])
@pytest.mark.parametrize("corpus", ["zipf", "planted"])
def test_resumed_run_equals_uninterrupted_run(tmp_path, compute, corpus):
    if corpus == "zipf":
        A, k, t_u, t_v = small_zipf(2), 9, 120, 60
    else:
        A, k, t_u, t_v = planted_50k_100k(seed=5, scale=0.04), 24, 90, 110
    U0 = uniform_init(A.n, k, 5)
    path = str(tmp_path / "state.ckpt")
    a = make_ctx(A, k, t_u, t_v, U0, E.TOPT_COLUMN, compute)
    E.espnmf_iterate(a, 3)
    E.espnmf_save(a, path, tag=1234)
    R1, E1 = E.espnmf_iterate(a, 4)
    Ua, Va = E.espnmf_get_factor(a, E.U), E.espnmf_get_factor(a, E.V)
    assert E.espnmf_sweeps_done(a) == 7
    # a fresh context from the same A (another initial guess), then the state
    b = make_ctx(A, k, t_u, t_v, uniform_init(A.n, k, 99), E.TOPT_COLUMN, compute)
    assert E.espnmf_load(b, path) == (1234, 3)
    R2, E2 = E.espnmf_iterate(b, 4)
    assert E.espnmf_sweeps_done(b) == 7
    np.testing.assert_array_equal(R1, R2)
    np.testing.assert_array_equal(E1, E2)
    np.testing.assert_array_equal(Ua, E.espnmf_get_factor(b, E.U))
    np.testing.assert_array_equal(Va, E.espnmf_get_factor(b, E.V))


def test_load_rejects_other_contexts_and_damaged_files(tmp_path):
    A = small_zipf(2)
    U0 = uniform_init(A.n, 6, 2)
    path = str(tmp_path / "s.ckpt")
    a = make_ctx(A, 6, 50, 40, U0, E.TOPT_COLUMN, E.F32)
    E.espnmf_iterate(a, 2)
    E.espnmf_save(a, path)
    Ua = E.espnmf_get_factor(a, E.U)
    for other in (dict(t_u=51, t_v=40, compute=E.F32), dict(t_u=50, t_v=40, compute=E.F64)):
        b = make_ctx(A, 6, other["t_u"], other["t_v"], U0, E.TOPT_COLUMN, other["compute"])
        with pytest.raises(E.EspnmfError) as ei:
            E.espnmf_load(b, path)
        assert ei.value.status == E.ERR_INVALID_ARG
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(bytes(raw))
    b = make_ctx(A, 6, 50, 40, U0, E.TOPT_COLUMN, E.F32)
    before = E.espnmf_get_factor(b, E.U)
    with pytest.raises(E.EspnmfError) as ei:
        E.espnmf_load(b, bad)
    assert ei.value.status == E.ERR_INVALID_ARG and "checksum" in str(ei.value)
    np.testing.assert_array_equal(E.espnmf_get_factor(b, E.U), before)
    open(bad, "wb").write(bytes(raw[:100]))
    with pytest.raises(E.EspnmfError):
        E.espnmf_load(b, bad)
    E.espnmf_load(b, path)
    np.testing.assert_array_equal(E.espnmf_get_factor(b, E.U), Ua)
    assert not os.path.exists(path + ".tmp")
