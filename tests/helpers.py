"""Shared test helpers: building a context from a gen.Corpus and comparing a
factor with the oracle's under the stated tolerances."""
import numpy as np

import paper_1510_05237_gb300 as E


def make_ctx(A, k, t_u, t_v, U0, mode=E.TOPT_COLUMN, compute=E.F64, device=True):
    import torch
    vals = A.val if compute == E.F64 else A.val.astype(np.float32)
    if device:
        rp = torch.from_numpy(np.ascontiguousarray(A.rowptr)).cuda()
        ci = torch.from_numpy(np.ascontiguousarray(A.colidx)).cuda()
        va = torch.from_numpy(np.ascontiguousarray(vals)).cuda()
        u0 = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
    else:
        rp, ci, va, u0 = A.rowptr, A.colidx, vals, np.ascontiguousarray(U0)
    return E.espnmf_init(rp, ci, va, A.n, A.m, k, t_u, t_v, mode, compute, u0)


def kth_positive(col: np.ndarray, t: int) -> float:
    pos = np.sort(col[col > 0])[::-1]
    if t <= 0:
        return np.inf
    return pos[t - 1] if len(pos) > t else 0.0


def compare_factor(gpu: np.ndarray, ref: np.ndarray, pre: np.ndarray, t: int, mode: int,
                   tol: float, what: str = "factor"):
    """Checks a GPU factor against the oracle's.

    gpu, ref: enforced factors; pre: the oracle's least-squares step before
    projection.  Per column (whole matrix in matrix mode) with scale = the
    largest oracle value of that column: values on the common support agree
    within tol*scale; the supports agree except where the oracle's projected
    value lies within tol*scale of the t-th largest (the threshold) or of 0.
    """
    assert gpu.shape == ref.shape
    proj = np.maximum(pre, 0.0)
    rows, k = ref.shape
    if mode == E.TOPT_MATRIX:
        groups = [np.arange(rows * k)]
        flat_g, flat_r, flat_p = gpu.reshape(-1), ref.reshape(-1), proj.reshape(-1)
        scale0 = max(np.abs(ref).max(), np.abs(proj).max(), 1e-300)
        taus = [kth_positive(flat_p, t)]
        scales = [scale0]
    else:
        flat_g, flat_r, flat_p = gpu.T.reshape(-1), ref.T.reshape(-1), proj.T.reshape(-1)
        groups = [np.arange(c * rows, (c + 1) * rows) for c in range(k)]
        scales = [max(np.abs(ref[:, c]).max(), np.abs(proj[:, c]).max(), 1e-300) for c in range(k)]
        taus = [kth_positive(proj[:, c], t) if mode == E.TOPT_COLUMN else 0.0 for c in range(k)]
    worst = 0.0
    for g, sc, tau in zip(groups, scales, taus):
        a, b, p = flat_g[g], flat_r[g], flat_p[g]
        both = (a != 0) & (b != 0)
        if both.any():
            worst = max(worst, float(np.abs(a[both] - b[both]).max() / sc))
        diff = (a != 0) != (b != 0)
        if diff.any():
            near = (np.abs(p[diff] - tau) <= tol * sc) | (p[diff] <= tol * sc)
            if not near.all():
                bad = np.flatnonzero(diff)[~near][:5]
                raise AssertionError(
                    f"{what}: support differs away from the threshold at {bad.tolist()} "
                    f"(gpu {a[bad]}, oracle {b[bad]}, projected {p[bad]}, tau {tau}, scale {sc})")
    assert worst <= tol, f"{what}: max normwise error {worst:.3e} > {tol:.1e}"
    return worst
