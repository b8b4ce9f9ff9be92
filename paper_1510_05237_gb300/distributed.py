"""Row-slab sharding of one factorisation over N ranks (the exchanges of a
multi-GPU sweep of Alg. 2).

Rank g owns a contiguous slab of the documents (rows of A^T: its rows of V)
and a contiguous slab of the terms (rows of A: its rows of U).  A half-step
needs every rank's sparse product rows of its own slab, which read the whole
other factor, and three exchanges:

  * the other factor in full: an all-gather of the slabs (the enforced factor
    holds at most t*k nonzeros);
  * its Gram matrix: a sum of the slabs' Grams (all-reduce, FP64);
  * the enforcement: the global top-t of a column lies inside the union of
    the ranks' local top-t, so each rank selects its local top-t, the
    candidates are all-gathered in global row order, the same selection is
    run again on the union (identical on every rank), and each rank keeps
    those of its candidates that survive.  Ties go to the lower global row,
    as in the single-GPU selector, because the union is laid out in global
    row order.

The residual and the error need only sums of per-slab scalars (all-reduce).

The local steps (sparse product, solve and projection, selection) are passed
in as functions: on GPU ranks they are the library's kernels (the selection
defaults to ``espnmf_enforce_topt_buffer``); the collectives come from
``torch.distributed`` (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np


def slab(total: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous share of `total` rows."""
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    return dist


def allreduce_sum(x: np.ndarray) -> np.ndarray:
    """Sum over ranks (FP64 arrays stay FP64)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x)).clone()
    _dist().all_reduce(t)
    return t.numpy()


def allgather_rows(local: np.ndarray, world: int) -> np.ndarray:
    """Concatenation of every rank's rows, in rank order."""
    import torch
    dist = _dist()
    t = torch.from_numpy(np.ascontiguousarray(local))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([t.shape[0]], dtype=torch.int64))
    cap = int(max(int(s) for s in sizes))
    pad = torch.zeros((cap,) + tuple(t.shape[1:]), dtype=t.dtype)
    pad[: t.shape[0]] = t
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return np.concatenate([p[: int(s)].numpy() for p, s in zip(parts, sizes)], axis=0)


def default_select(X: np.ndarray, t: int) -> np.ndarray:
    """Per-column top-t of a projected candidate with the library's selector
    (lower row index wins ties); X is rows x k, returned enforced."""
    import torch
    from . import binding as B
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    B.espnmf_enforce_topt_buffer(Xd, t, B.TOPT_COLUMN)
    torch.cuda.synchronize()
    return Xd.cpu().numpy()


def global_topt(X_local: np.ndarray, row0: int, t: int, world: int,
                select: Callable[[np.ndarray, int], np.ndarray] = default_select) -> np.ndarray:
    """Exact per-column top-t of the row-sharded projected candidate whose
    rows [row0, row0 + len) this rank holds; returns this rank's enforced
    rows."""
    k = X_local.shape[1]
    mine = select(X_local.copy(), t)                     # local top-t (superset of the final)
    rows = np.flatnonzero((mine != 0).any(axis=1))
    cand = np.concatenate([(rows + row0)[:, None].astype(np.float64), mine[rows]], axis=1)
    union = allgather_rows(cand, world)                  # global row order (slabs ascend)
    kept = select(union[:, 1:].copy(), t)                # the same on every rank
    out = np.zeros_like(X_local)
    grows = union[:, 0].astype(np.int64)
    here = (grows >= row0) & (grows < row0 + X_local.shape[0])
    out[grows[here] - row0] = kept[here]
    assert out.shape[1] == k
    return out


def sharded_half_update(product_rows: Callable[[np.ndarray], np.ndarray],
                        gram: Callable[[np.ndarray], np.ndarray],
                        solve_project: Callable[[np.ndarray, np.ndarray], np.ndarray],
                        other_local: np.ndarray, row0: int, t: int, world: int,
                        select: Callable[[np.ndarray, int], np.ndarray] = default_select) -> np.ndarray:
    """One half-step of Alg. 2 on this rank's slab.

    product_rows(O): this slab's rows of A^T O (or A O) from the full other
    factor O; gram(F): F^T F of a slab (FP64); solve_project(Y, G):
    max(Y G^-1, 0).  other_local is this rank's slab of the other factor.
    Returns this rank's enforced rows."""
    O = allgather_rows(other_local, world)
    G = allreduce_sum(gram(other_local))
    X = solve_project(product_rows(O), G)
    return global_topt(X, row0, t, world, select)


def sharded_measures(d2_local: float, u2_local: float, cross_local: float,
                     a2_local: float, G_U: np.ndarray, G_V: np.ndarray) -> tuple[float, float]:
    """R and E (Sec. 3.1) from per-slab sums: d2 = ||U_new - U_old||^2,
    u2 = ||U_new||^2, cross = <U, A V>, a2 = ||A||^2 over the slab's rows;
    E^2 ||A||^2 = ||A||^2 - 2 <U, A V> + <U^T U, V^T V>."""
    s = allreduce_sum(np.array([d2_local, u2_local, cross_local, a2_local], dtype=np.float64))
    d2, u2, cross, a2 = (float(v) for v in s)
    R = 0.0 if u2 == 0.0 and d2 == 0.0 else (float("inf") if u2 == 0.0 else float(np.sqrt(d2 / u2)))
    f = a2 - 2.0 * cross + float(np.sum(G_U * G_V))
    E = 0.0 if a2 == 0.0 else float(np.sqrt(max(f, 0.0)) / np.sqrt(a2))
    return R, E


__all__: Sequence[str] = ["slab", "allreduce_sum", "allgather_rows", "default_select",
                          "global_topt", "sharded_half_update", "sharded_measures"]
