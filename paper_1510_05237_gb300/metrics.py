"""Document-clustering accuracy of a topic model (Sec. 3.2, Eq. 3 and 4).

A document belongs to topic c when its entry in column c of V is nonzero.
For a topic with n_D member documents drawn from n_J classes (journals in
the paper, planted topics in the synthetic corpora), the accuracy is

    Acc = (P - alpha) / (beta - alpha),

with P the number of member pairs that share a class, alpha the number of
such pairs when the members are spread as evenly as possible over the
classes (q = n_D // n_J, r = n_D % n_J: alpha = q (n_J (q - 1) / 2 + r)) and
beta = n_D (n_D - 1) / 2 the number of all pairs.  Acc is 1 when all members
share a class and 0 for an even spread.  A topic with at most one member has
Acc = 1 (as the paper sets it); so does one with beta == alpha (n_J == 1).

This is evaluation of a finished factor on the host, not a step of the
sweep: P is computed from the class histogram of the members,
sum_j c_j (c_j - 1) / 2.
"""
from __future__ import annotations

import numpy as np


def topic_accuracy(V, labels, n_classes: int) -> np.ndarray:
    """Accuracy of each column of V (rows = documents, dense m x k, numpy or
    torch); labels[i] in [0, n_classes) is document i's class."""
    if hasattr(V, "detach"):
        V = V.detach().cpu().numpy()
    V = np.asarray(V)
    labels = np.asarray(labels)
    if n_classes < 1:
        raise ValueError("n_classes must be >= 1")
    if V.ndim != 2 or V.shape[0] != labels.shape[0]:
        raise ValueError("V must be m x k with one label per row")
    acc = np.ones(V.shape[1])
    for c in range(V.shape[1]):
        lab = labels[V[:, c] != 0]
        n_d = lab.size
        if n_d <= 1:
            continue
        if lab.min() < 0 or lab.max() >= n_classes:
            raise ValueError("a member document's label is outside [0, n_classes)")
        counts = np.bincount(lab, minlength=n_classes).astype(np.float64)
        same = float((counts * (counts - 1.0) / 2.0).sum())
        q, r = divmod(n_d, n_classes)
        alpha = q * (n_classes * (q - 1) / 2.0 + r)
        beta = n_d * (n_d - 1) / 2.0
        if beta != alpha:
            acc[c] = (same - alpha) / (beta - alpha)
    return acc


def factor_dense(csc, rows: int, k: int) -> np.ndarray:
    """A factor exported as CSC (colptr, rowidx, values) as a dense rows x k array."""
    colptr, rowidx, vals = (np.asarray(x) for x in csc)
    out = np.zeros((rows, k), dtype=np.float64)
    for c in range(k):
        a, b = int(colptr[c]), int(colptr[c + 1])
        out[rowidx[a:b], c] = vals[a:b]
    return out
