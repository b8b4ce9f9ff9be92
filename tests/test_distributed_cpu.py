"""The row-slab sharded sweep (world size 2, gloo on CPU): the exchanges of
``paper_1510_05237_gb300.distributed`` with the oracle's arithmetic for the
local steps must reproduce the single-rank oracle sweep.  Slabs are chosen
so that some column's top-t straddles the two ranks, and one case has exact
ties across the slab boundary (the lower global row must win)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from gen import Corpus, small_zipf, uniform_init  # noqa: E402
from paper_1510_05237_gb300 import distributed as D  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _np(fn):
    """An oracle step (numpy in, numpy out) as a step on CPU tensors."""
    return lambda *ts: torch.from_numpy(np.ascontiguousarray(fn(*(t.numpy() for t in ts))))


def _sweep_rank(rank, world, port, A, U0, t_u, t_v, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r0, r1 = D.slab(A.n, world, rank)      # my terms: rows of U
        d0, d1 = D.slab(A.m, world, rank)      # my documents: rows of V
        T = lambda a: torch.from_numpy(np.ascontiguousarray(a))  # noqa: E731
        solve_project = _np(lambda Y, G: oracle.project(oracle.ls_solve(Y, G)))
        gram, topt = _np(oracle.gram), lambda X, t: _np(lambda x: oracle.topt(x, t))(X)
        # V half: my rows of A^T U from the gathered U
        V_loc = D.sharded_half_update(_np(lambda U: oracle.spmm_At(A, U)[d0:d1]), gram,
                                      solve_project, T(U0[r0:r1]), d0, t_v, world, topt)
        # U half: my rows of A V
        AV = {}

        def prod_U(V):
            AV["Y"] = oracle.spmm_A(A, V.numpy())[r0:r1]
            return T(AV["Y"])

        U_loc = D.sharded_half_update(prod_U, gram, solve_project, V_loc, r0, t_u,
                                      world, topt)
        G_U = D.allreduce_sum(gram(U_loc))
        G_V = D.allreduce_sum(gram(V_loc))
        rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
        a2 = float(np.sum(A.val[(rows >= r0) & (rows < r1)] ** 2))
        Un = U_loc.numpy()
        sums = T(np.array([np.sum((Un - U0[r0:r1]) ** 2), np.sum(Un ** 2),
                           np.sum(Un * AV["Y"]), a2], dtype=np.float64))
        R, E = D.sharded_measures(sums, G_U, G_V)
        assert R.dim() == 0 and E.dim() == 0 and R.dtype == torch.float64
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), U=Un, V=V_loc.numpy(), R=float(R),
                 E=float(E), r=np.array([r0, r1, d0, d1]))
    finally:
        dist.destroy_process_group()


def _run(A, U0, t_u, t_v, tmp_path, world=2):
    mp.start_processes(_sweep_rank, args=(world, _free_port(), A, U0, t_u, t_v, str(tmp_path)),
                       nprocs=world, start_method="spawn", join=True)
    U = np.zeros((A.n, U0.shape[1]))
    V = np.zeros((A.m, U0.shape[1]))
    meas = []
    for r in range(world):
        z = np.load(tmp_path / f"rank{r}.npz")
        r0, r1, d0, d1 = z["r"]
        U[r0:r1], V[d0:d1] = z["U"], z["V"]
        meas.append((float(z["R"]), float(z["E"])))
    return U, V, meas


def test_two_rank_sweep_equals_single_rank_oracle(tmp_path):
    A = small_zipf()
    k, t = 10, 100
    U0 = uniform_init(A.n, k, 1)
    U, V, meas = _run(A, U0, t, t, tmp_path)
    Vo = oracle.update_V(A, U0, t)
    Uo = oracle.update_U(A, Vo, t)
    # the selection sees the same FP64 candidates on both sides: the same support
    np.testing.assert_array_equal(V != 0, Vo != 0)
    np.testing.assert_array_equal(U != 0, Uo != 0)
    assert np.abs(V - Vo).max() <= 1e-12 * np.abs(Vo).max()
    assert np.abs(U - Uo).max() <= 1e-12 * np.abs(Uo).max()
    Ro, Eo = oracle.residual(Uo, U0), oracle.error_identity(A, Uo, Vo)
    for R, E in meas:                     # every rank holds the same measures
        assert abs(R - Ro) <= 1e-12 * Ro and abs(E - Eo) <= 1e-12
    # some column's kept set spans both ranks' slabs
    half = A.m // 2
    assert any((Vo[:half, c] != 0).any() and (Vo[half:, c] != 0).any() for c in range(k))


def test_ties_across_the_slab_boundary_go_to_the_lower_row(tmp_path):
    # documents 0..9 (rank 0) and 30..39 (rank 1) are identical: their V rows
    # tie exactly and the lower global rows must be kept
    rng = np.random.default_rng(8)
    D_ = rng.random((24, 40)) * (rng.random((24, 40)) < 0.4)
    D_[:, 30:40] = D_[:, 0:10]
    rows, cols = np.nonzero(D_)
    rowptr = np.zeros(25, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=24), out=rowptr[1:])
    A = Corpus(24, 40, rowptr, cols.astype(np.int32), D_[rows, cols])
    U0 = uniform_init(24, 3, 2)
    U, V, _ = _run(A, U0, 10, 6, tmp_path)
    Vo = oracle.update_V(A, U0, 6)
    np.testing.assert_array_equal(V != 0, Vo != 0)
    for c in range(3):
        for j in range(10):
            if V[30 + j, c] != 0:
                assert V[j, c] != 0
