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
    candidates (global row index and row values, gathered separately) are
    all-gathered in global row order, the same selection is run again on the
    union (identical on every rank), and each rank keeps those of its
    candidates that survive.  Ties go to the lower global row, as in the
    single-GPU selector, because the union is laid out in global row order.

The residual and the error need only sums of per-slab scalars (all-reduce)
and are finished with tensor operations on the same device.

Every function takes and returns torch tensors and keeps them on their
device: CUDA tensors with the NCCL backend on GPU ranks (no host round
trip), CPU tensors with gloo.  The local steps (sparse product, solve and
projection, selection) are passed in as functions: on GPU ranks they are the
library's kernels (the selection defaults to ``espnmf_enforce_topt_buffer``
on the device tensor); the collectives come from ``torch.distributed``.
"""
from __future__ import annotations

from typing import Callable, Sequence

import torch


def slab(total: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous share of `total` rows."""
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    return dist


def allreduce_sum(x: torch.Tensor) -> torch.Tensor:
    """Sum over ranks, on x's device and in x's dtype (a new tensor)."""
    t = x.contiguous().clone()
    _dist().all_reduce(t)
    return t


def allgather_rows(local: torch.Tensor, world: int) -> torch.Tensor:
    """Concatenation of every rank's rows, in rank order, on local's device."""
    dist = _dist()
    t = local.contiguous()
    dev = t.device
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([t.shape[0]], dtype=torch.int64, device=dev))
    counts = [int(s) for s in torch.cat(sizes).cpu()]   # world integers: the slab sizes
    cap = max(counts)
    pad = torch.zeros((cap,) + tuple(t.shape[1:]), dtype=t.dtype, device=dev)
    pad[: t.shape[0]] = t
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def default_select(X: torch.Tensor, t: int) -> torch.Tensor:
    """Per-column top-t of a projected candidate (rows x k CUDA tensor) with
    the library's selector, in place on the device (lower row wins ties)."""
    from . import binding as B
    B.espnmf_enforce_topt_buffer(X, t, B.TOPT_COLUMN)
    return X


def global_topt(X_local: torch.Tensor, row0: int, t: int, world: int,
                select: Callable[[torch.Tensor, int], torch.Tensor] = default_select) -> torch.Tensor:
    """Exact per-column top-t of the row-sharded projected candidate whose
    rows [row0, row0 + len) this rank holds; returns this rank's enforced
    rows."""
    mine = select(X_local.clone(), t)                    # local top-t (superset of the final)
    rows = torch.nonzero((mine != 0).any(dim=1)).flatten()
    grow = allgather_rows(rows + row0, world)            # global row order (slabs ascend)
    union = allgather_rows(mine[rows], world)
    kept = select(union.clone(), t)                      # the same on every rank
    out = torch.zeros_like(X_local)
    here = (grow >= row0) & (grow < row0 + X_local.shape[0])
    out[grow[here] - row0] = kept[here]
    return out


def sharded_half_update(product_rows: Callable[[torch.Tensor], torch.Tensor],
                        gram: Callable[[torch.Tensor], torch.Tensor],
                        solve_project: Callable[[torch.Tensor, torch.Tensor], torch.Tensor],
                        other_local: torch.Tensor, row0: int, t: int, world: int,
                        select: Callable[[torch.Tensor, int], torch.Tensor] = default_select
                        ) -> torch.Tensor:
    """One half-step of Alg. 2 on this rank's slab.

    product_rows(O): this slab's rows of A^T O (or A O) from the full other
    factor O; gram(F): F^T F of a slab (FP64); solve_project(Y, G):
    max(Y G^-1, 0).  other_local is this rank's slab of the other factor.
    Returns this rank's enforced rows."""
    O = allgather_rows(other_local, world)
    G = allreduce_sum(gram(other_local))
    X = solve_project(product_rows(O), G)
    return global_topt(X, row0, t, world, select)


def sharded_measures(sums_local: torch.Tensor, G_U: torch.Tensor,
                     G_V: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """R and E (Sec. 3.1) from per-slab FP64 sums [d2, u2, cross, a2]:
    d2 = ||U_new - U_old||^2, u2 = ||U_new||^2, cross = <U, A V>, a2 = ||A||^2
    over the slab's rows; E^2 ||A||^2 = ||A||^2 - 2 <U, A V> + <U^T U, V^T V>.
    Returns two 0-d tensors on the sums' device."""
    s = allreduce_sum(sums_local.to(torch.float64))
    d2, u2, cross, a2 = s[0], s[1], s[2], s[3]
    zero = torch.zeros((), dtype=torch.float64, device=s.device)
    inf = torch.full((), float("inf"), dtype=torch.float64, device=s.device)
    R = torch.where(u2 == 0, torch.where(d2 == 0, zero, inf),
                    torch.sqrt(d2 / torch.where(u2 == 0, torch.ones_like(u2), u2)))
    f = a2 - 2.0 * cross + torch.sum(G_U.to(torch.float64) * G_V.to(torch.float64))
    E = torch.where(a2 == 0, zero,
                    torch.sqrt(torch.clamp(f, min=0.0)) / torch.sqrt(torch.where(a2 == 0, torch.ones_like(a2), a2)))
    return R, E


__all__: Sequence[str] = ["slab", "allreduce_sum", "allgather_rows", "default_select",
                          "global_topt", "sharded_half_update", "sharded_measures"]
