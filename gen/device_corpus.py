"""Seeded synthetic term/document matrix generated on a CUDA device, for
corpora too large to build with the host generator (hundreds of millions of
nonzeros): the 1M-term x 2M-document Zipf corpus and scaled copies of it.

Input generation only -- no step of the factorisation.  The recipe is the
host generator's (``gen.corpus.zipf_corpus``), restated with torch tensor
operations:

* document lengths L_d (distinct terms) lognormal with the given mean and
  log-standard-deviation sigma, at least 1, at most n;
* each document draws ceil(1.6 L_d) + 2 term ranks from a finite Zipf(s) law
  over n terms (inverse CDF), mapped to term ids by a seeded permutation, and
  keeps its first L_d distinct terms in draw order (fewer if it drew fewer);
* raw counts Poisson(1) + 1 per kept term, values count * log(m / df),
  documents (columns) L2-normalised, stored as FP32.

Every step is deterministic for a seed on a given device and torch build
(counter-based random numbers, stable sorts, integer histograms and scans;
no floating-point atomics).  The result is CSR over terms, on the device:
rowptr int64[n+1], colidx int32[nnz] (sorted within each row), val
float32[nnz] (> 0).
"""
from __future__ import annotations

import dataclasses
import math


@dataclasses.dataclass
class DeviceCorpus:
    n: int
    m: int
    rowptr: "torch.Tensor"   # int64[n+1], device
    colidx: "torch.Tensor"   # int32[nnz], device
    val: "torch.Tensor"      # float32[nnz], device
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    def to_host(self):
        """The same matrix as a host ``gen.Corpus`` (float64 values that are
        exactly the FP32 ones)."""
        from .corpus import Corpus
        return Corpus(self.n, self.m, self.rowptr.cpu().numpy(), self.colidx.cpu().numpy(),
                      self.val.double().cpu().numpy(), name=self.name)


def zipf_corpus_device(n: int, m: int, mean_len: float, s: float, sigma: float, seed: int,
                       device="cuda", oversample: float = 1.6, name: str = "zipf-device"
                       ) -> DeviceCorpus:
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64, i64 = torch.float64, torch.int64
    # document lengths (distinct terms)
    mu = math.log(mean_len) - 0.5 * sigma * sigma
    z = torch.randn(m, dtype=f64, device=device, generator=g)
    lengths = torch.clamp(torch.round(torch.exp(mu + sigma * z)), 1, n).to(i64)
    draws = torch.ceil(lengths.to(f64) * oversample).to(i64) + 2
    total = int(draws.sum())
    dstart = torch.cumsum(draws, 0) - draws
    doc = torch.repeat_interleave(torch.arange(m, dtype=i64, device=device), draws)
    pos = torch.arange(total, dtype=i64, device=device) - dstart[doc]      # draw order in doc
    del dstart
    # Zipf(s) term ranks by inverse CDF, then term ids by a permutation
    w = 1.0 / torch.arange(1, n + 1, dtype=f64, device=device) ** s
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    u = torch.rand(total, dtype=f64, device=device, generator=g)
    rank = torch.clamp(torch.searchsorted(cdf, u, right=True), max=n - 1)
    del u, cdf, w
    perm = torch.randperm(n, device=device, generator=g)
    term = perm[rank]
    del rank, perm
    # first occurrence of every (doc, term) pair: the keys arrive in (doc,
    # draw) order, so a stable sort keeps the first draw first
    key, idx = torch.sort(doc * n + term, stable=True)
    del term
    first = torch.ones(total, dtype=torch.bool, device=device)
    first[1:] = key[1:] != key[:-1]
    starts = torch.nonzero(first).flatten()
    del first
    ukey = key[starts]
    upos = pos[idx[starts]]
    del key, idx, starts, pos, doc
    udoc = ukey // n
    # keep the first L_d distinct terms of each document, in draw order
    maxd = int(draws.max()) + 1
    o2 = torch.sort(udoc * maxd + upos, stable=True)[1]
    ukey, udoc = ukey[o2], udoc[o2]
    del o2, upos
    cnt = torch.bincount(udoc, minlength=m)
    cstart = torch.cumsum(cnt, 0) - cnt
    rank_in_doc = torch.arange(ukey.numel(), dtype=i64, device=device) - cstart[udoc]
    keep = rank_in_doc < lengths[udoc]
    ukey, udoc = ukey[keep], udoc[keep]
    del rank_in_doc, keep, cnt, cstart
    uterm = ukey % n
    del ukey
    # TF-IDF values, documents L2-normalised (entries are grouped by document)
    tf = torch.poisson(torch.ones(udoc.numel(), dtype=f64, device=device), generator=g) + 1.0
    df = torch.bincount(uterm, minlength=n).to(f64)
    val = tf * torch.log(m / torch.clamp(df[uterm], min=1.0))
    del tf, df
    ok = val > 0
    udoc, uterm, val = udoc[ok], uterm[ok], val[ok]
    cnt = torch.bincount(udoc, minlength=m)
    ends = torch.cumsum(cnt, 0)
    csum = torch.cumsum(val * val, 0)
    tot = torch.cat([csum.new_zeros(1), csum])
    nrm = torch.sqrt(tot[ends] - tot[ends - cnt])
    val = val / torch.where(nrm > 0, nrm, torch.ones_like(nrm))[udoc]
    del cnt, ends, csum, tot, nrm
    # CSR over terms, documents ascending within each row
    o3 = torch.sort(uterm * m + udoc, stable=True)[1]
    uterm, udoc, val = uterm[o3], udoc[o3], val[o3]
    del o3
    rowptr = torch.zeros(n + 1, dtype=i64, device=device)
    rowptr[1:] = torch.cumsum(torch.bincount(uterm, minlength=n), 0)
    return DeviceCorpus(n, m, rowptr, udoc.to(torch.int32), val.to(torch.float32), name=name)


def zipf_1m_2m_device(seed: int = 3, scale: float = 1.0, device="cuda") -> DeviceCorpus:
    """1M terms x 2M docs, Zipf(1.05) term ids, lognormal lengths with mean
    200 distinct terms (sigma 0.7), ~400M nnz.  ``scale`` shrinks n and m
    proportionally and the mean length by scale**0.25 (parity cases)."""
    n = max(64, int(1_000_000 * scale))
    m = max(64, int(2_000_000 * scale))
    mean = 200.0 * min(1.0, scale ** 0.25)
    return zipf_corpus_device(n, m, mean, 1.05, 0.7, seed, device=device,
                              name=f"zipf-{n}x{m}")


def uniform_init_device(n: int, k: int, seed: int, device="cuda"):
    """U0 ~ U[0, 1) (n x k, float32) on the device from a seeded generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.rand((n, k), dtype=torch.float32, device=device, generator=g)


__all__ = ["DeviceCorpus", "zipf_corpus_device", "zipf_1m_2m_device", "uniform_init_device"]
