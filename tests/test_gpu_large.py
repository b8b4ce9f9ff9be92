"""The large Zipf corpus (1M terms x 2M docs, Zipf(1.05), mean 200 terms per
document, ~400M nnz; k = 100, t = 5000 per column) against the oracle.

* A 1/100-scale copy (10k x 20k, ~1.2M nnz, k = 100, t = 50) is compared
  one half-step at a time in full, FP32 and FP64 forms (k > 64: the Gram
  inverse path).
* At full size, one sweep in the launch configuration the benchmark times
  (graph-replayed espnmf_iterate, FP32 form) is checked on sampled rows that
  the oracle computes one by one: the oracle's least-squares step for the
  sampled documents (V) and terms (U) from the GPU's own input iterate, on
  the sub-matrix those rows read.  A sampled entry the GPU kept must equal
  the oracle's value; one it dropped must lie at or below the column's
  threshold (its smallest kept value when t are kept, else 0).  Skipped when
  the host or the device lacks the memory the full-size context needs.
"""
import numpy as np
import pytest

import oracle
import paper_1510_05237_gb300 as E
from gen import uniform_init
from test_gpu_parity import step_parity

pytestmark = pytest.mark.gpu

K, T_FULL = 100, 5000


@pytest.mark.parametrize("compute", [E.F32, E.F64])
def test_step_parity_large_corpus_scaled(compute):
    from gen.device_corpus import zipf_1m_2m_device
    A = zipf_1m_2m_device(seed=3, scale=0.01).to_host()
    assert A.n == 10_000 and A.m == 20_000 and A.nnz > 1_000_000
    U0 = uniform_init(A.n, K, 3)
    step_parity(A, K, 50, 50, U0, E.TOPT_COLUMN, compute, "zipf 10k x 20k, k = 100")


def _mem_ok() -> bool:
    import torch
    avail = 0.0
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) / 2**20
    except OSError:
        pass
    return avail >= 64.0 and torch.cuda.mem_get_info()[0] / 2**30 >= 80.0


def _columns(rowptr, colidx, val, n, pick):
    """The sub-matrix A[:, pick] (pick ascending) as a host CSR over the n
    terms, columns renumbered 0 .. len(pick) - 1."""
    import torch
    from gen import Corpus
    pt = torch.as_tensor(pick, dtype=torch.int32, device=colidx.device)
    mask = torch.isin(colidx, pt)
    rows = torch.repeat_interleave(torch.arange(n, device=colidx.device), torch.diff(rowptr))[mask]
    cols = torch.searchsorted(pt, colidx[mask])
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(torch.bincount(rows, minlength=n).cpu().numpy(), out=rp[1:])
    return Corpus(n, len(pick), rp, cols.to(torch.int32).cpu().numpy(),
                  val[mask].double().cpu().numpy())


def _rows(rowptr, colidx, val, pick, docs):
    """The sub-matrix A[pick, docs] (docs ascending) as a host CSR,
    documents renumbered 0 .. len(docs) - 1; entries of other documents are
    left out."""
    from gen import Corpus
    rp_h = rowptr.cpu().numpy()
    ptr, cols, vals = [0], [], []
    for i in pick:
        c = colidx[rp_h[i]:rp_h[i + 1]].cpu().numpy()
        v = val[rp_h[i]:rp_h[i + 1]].double().cpu().numpy()
        pos = np.searchsorted(docs, c)
        ok = (pos < len(docs)) & (docs[np.minimum(pos, len(docs) - 1)] == c)
        cols.append(pos[ok].astype(np.int32))
        vals.append(v[ok])
        ptr.append(ptr[-1] + int(ok.sum()))
    return Corpus(len(pick), len(docs), np.array(ptr, dtype=np.int64),
                  np.concatenate(cols), np.concatenate(vals))


def _check_sampled(F, sample, pre, t, tol, what):
    """F: the GPU's enforced factor (dense, all rows); pre: the oracle's
    least-squares step for the sampled rows."""
    for c in range(F.shape[1]):
        col = F[:, c]
        kept = col > 0
        cnt = int(kept.sum())
        assert cnt <= t, (what, c, cnt)
        thr = col[kept].min() if cnt == t else 0.0
        scale = max(np.abs(pre[:, c]).max(), col.max(), 1e-300)
        g, o = col[sample], pre[:, c]
        on = g > 0
        assert np.all(np.abs(g[on] - o[on]) <= tol * scale), (what, c)
        assert np.all(o[~on] <= thr + tol * scale), (what, c)


def test_full_size_large_corpus_sampled_rows_fp32():
    import torch
    if not _mem_ok():
        pytest.skip("needs >= 64 GB available host memory and >= 80 GB free device memory")
    from gen.device_corpus import uniform_init_device, zipf_1m_2m_device
    A = zipf_1m_2m_device(seed=3)
    assert A.n == 1_000_000 and A.m == 2_000_000 and A.nnz > 300_000_000
    U0 = uniform_init_device(A.n, K, 3)
    ctx = E.espnmf_init(A.rowptr, A.colidx, A.val, A.n, A.m, K, T_FULL, T_FULL, E.TOPT_COLUMN,
                        E.F32, U0)
    R, Es = E.espnmf_iterate(ctx, 1)
    Vg = E.espnmf_get_factor(ctx, E.V)
    Ug = E.espnmf_get_factor(ctx, E.U)
    E.espnmf_destroy(ctx)
    assert np.isfinite(R[0]) and 0.0 < Es[0] < 1.0
    rng = np.random.default_rng(11)
    tol = 2e-5
    # V half: sampled documents (the longest one, the last one and random ones)
    lens = torch.bincount(A.colidx.long(), minlength=A.m)
    docs = np.unique(np.concatenate([rng.choice(A.m, 40, replace=False),
                                     [int(torch.argmax(lens)), A.m - 1]])).astype(np.int64)
    As = _columns(A.rowptr, A.colidx, A.val, A.n, docs)
    U0o = U0.double().cpu().numpy()
    _, preV = oracle.update_V(As, U0o, T_FULL, oracle.NONE, return_pre=True)
    _check_sampled(Vg, docs, preV, T_FULL, tol, "V")
    # U half: sampled terms (the most frequent one, the first one and random
    # ones); only documents with a nonzero V row contribute to A V and V^T V
    df = torch.diff(A.rowptr)
    terms = np.unique(np.concatenate([rng.choice(A.n, 40, replace=False),
                                      [int(torch.argmax(df)), 0]])).astype(np.int64)
    nzr = np.nonzero(Vg.any(axis=1))[0]
    Ar = _rows(A.rowptr, A.colidx, A.val, terms, nzr)
    _, preU = oracle.update_U(Ar, np.ascontiguousarray(Vg[nzr]), T_FULL, oracle.NONE,
                              return_pre=True)
    _check_sampled(Ug, terms, preU, T_FULL, tol, "U")
