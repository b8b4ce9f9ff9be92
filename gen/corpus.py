"""Seeded synthetic term/document matrices shaped like the paper's corpora.

The paper factors term/document matrices A (n terms x m documents, A >= 0)
built from Reuters-21578, a Wikipedia dump and PubMed abstracts (Sec. 3).
Those corpora are not available here, so these generators produce seeded
stand-ins with the same structure: Zipf-distributed term frequencies,
lognormal document lengths, optional planted topics, TF-IDF-like values and
L2-normalised document columns.

This module holds input generation only -- no step of the factorisation.
Both the CPU oracle and the CUDA path receive the same arrays from here.

Every matrix is returned in CSR over terms (rows = terms, columns = docs):
``rowptr`` int64[n+1], ``colidx`` int32[nnz] (sorted within each row) and
``val`` float64[nnz] (strictly positive).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Corpus:
    n: int                 # terms (rows of A)
    m: int                 # documents (columns of A)
    rowptr: np.ndarray     # int64[n+1]
    colidx: np.ndarray     # int32[nnz]
    val: np.ndarray        # float64[nnz], > 0
    name: str = ""
    labels: np.ndarray | None = None   # planted topic of each document, if any

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def dense(self) -> np.ndarray:
        """Dense n x m copy (tiny inputs only)."""
        A = np.zeros((self.n, self.m))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        A[rows, self.colidx] = self.val
        return A

    def astype(self, dtype) -> "Corpus":
        """Copy whose values are rounded to ``dtype`` and widened back to f64."""
        v = self.val.astype(dtype).astype(np.float64)
        return dataclasses.replace(self, val=v)

    def first_docs(self, m2: int) -> "Corpus":
        """The sub-corpus of documents 0..m2-1 (all terms kept)."""
        m2 = max(1, min(int(m2), self.m))
        keep = self.colidx < m2
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        counts = np.bincount(rows[keep], minlength=self.n)
        rowptr = np.zeros(self.n + 1, dtype=np.int64)
        np.cumsum(counts, out=rowptr[1:])
        labels = None if self.labels is None else self.labels[:m2].copy()
        return dataclasses.replace(self, m=m2, rowptr=rowptr,
                                   colidx=self.colidx[keep].copy(),
                                   val=self.val[keep].copy(),
                                   name=f"{self.name}[:{m2} docs]", labels=labels)


def _zipf_cdf(n: int, s: float) -> np.ndarray:
    w = 1.0 / np.arange(1, n + 1, dtype=np.float64) ** s
    c = np.cumsum(w)
    return c / c[-1]


def _draw(rng: np.random.Generator, cdf: np.ndarray, size: int) -> np.ndarray:
    u = rng.random(size)
    r = np.searchsorted(cdf, u, side="right")
    return np.minimum(r, len(cdf) - 1)


def _assemble(n: int, m: int, doc: np.ndarray, term: np.ndarray,
              lengths: np.ndarray | None, order: np.ndarray | None,
              tf: np.ndarray | None, rng: np.random.Generator,
              normalise: bool, weighting: str) -> Corpus:
    """Deduplicate (doc, term) tokens and build a TF-IDF CSR matrix.

    ``order`` is the draw position of each token; when ``lengths`` is given,
    only the first ``lengths[doc]`` distinct terms of each document (in draw
    order) are kept.  ``tf`` is the raw count per token (None: multiplicity).
    """
    key = doc.astype(np.int64) * n + term.astype(np.int64)
    if order is None:
        order = np.arange(len(key), dtype=np.int64)
    # first occurrence of every (doc, term) pair, with its multiplicity
    srt = np.lexsort((order, key))
    ks = key[srt]
    first = np.ones(len(ks), dtype=bool)
    first[1:] = ks[1:] != ks[:-1]
    starts = np.flatnonzero(first)
    mult = np.diff(np.append(starts, len(ks)))
    ukey = ks[starts]
    uorder = order[srt][starts]
    utf = None if tf is None else tf[srt][starts]
    udoc = ukey // n
    if lengths is not None:
        # keep the first lengths[d] distinct terms of each doc in draw order
        o2 = np.lexsort((uorder, udoc))
        d2 = udoc[o2]
        dstart = np.searchsorted(d2, np.arange(m))
        rank = np.arange(len(d2)) - dstart[d2]
        keep = np.zeros(len(ukey), dtype=bool)
        keep[o2[rank < lengths[d2]]] = True
        ukey, mult = ukey[keep], mult[keep]
        if utf is not None:
            utf = utf[keep]
    udoc = (ukey // n).astype(np.int64)
    uterm = (ukey % n).astype(np.int64)
    count = mult.astype(np.float64) if utf is None else utf.astype(np.float64)
    df = np.bincount(uterm, minlength=n).astype(np.float64)
    if weighting == "tfidf":
        val = count * np.log(m / np.maximum(df[uterm], 1.0))
    elif weighting == "rownnz":
        # Sec. 3 preprocessing: raw counts divided by the row's nonzero count
        val = count / np.maximum(df[uterm], 1.0)
    else:
        val = count
    ok = val > 0
    udoc, uterm, val = udoc[ok], uterm[ok], val[ok]
    if normalise:
        nrm = np.sqrt(np.bincount(udoc, weights=val * val, minlength=m))
        val = val / np.where(nrm > 0, nrm, 1.0)[udoc]
    # CSR over terms, columns sorted within each row
    srt = np.lexsort((udoc, uterm))
    uterm, udoc, val = uterm[srt], udoc[srt], val[srt]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(uterm, minlength=n), out=rowptr[1:])
    return Corpus(n, m, rowptr, udoc.astype(np.int32), val.astype(np.float64))


def zipf_corpus(n: int, m: int, mean_len: float, s: float, seed: int,
                sigma: float = 0.0, oversample: float = 1.6,
                weighting: str = "tfidf", name: str = "zipf") -> Corpus:
    """Documents whose term ids follow a finite Zipf(s) law over n terms.

    Document lengths (distinct terms) are ``mean_len`` (sigma == 0) or
    lognormal with that mean and log-standard-deviation ``sigma``.  Raw counts
    are Poisson(1)+1 and values are count * log(m/df); columns are
    L2-normalised.  Term ranks are mapped to ids by a seeded permutation.
    """
    rng = np.random.default_rng(seed)
    if sigma > 0:
        mu = math.log(mean_len) - 0.5 * sigma * sigma
        lengths = np.maximum(1, np.rint(rng.lognormal(mu, sigma, m))).astype(np.int64)
    else:
        lengths = np.full(m, int(round(mean_len)), dtype=np.int64)
    lengths = np.minimum(lengths, n)
    draws = np.ceil(lengths * oversample).astype(np.int64) + 2
    doc = np.repeat(np.arange(m, dtype=np.int64), draws)
    perm = rng.permutation(n)
    term = perm[_draw(rng, _zipf_cdf(n, s), len(doc))]
    tf = rng.poisson(1.0, len(doc)).astype(np.float64) + 1.0
    c = _assemble(n, m, doc, term, lengths, None, tf, rng, True, weighting)
    c.name = name
    return c


def planted_corpus(n: int, m: int, ntopics: int, topic_terms: int,
                   mean_len: float, sigma: float, alpha: float, noise: float,
                   seed: int, s: float = 1.1, oversample: float = 2.5,
                   name: str = "planted") -> Corpus:
    """Documents drawn from planted sparse topics.

    Each topic is a Zipf(s) distribution over a random subset of
    ``topic_terms`` terms.  Each document draws a mixture from
    Dirichlet(alpha) over the topics; a fraction ``noise`` of its tokens is
    uniform over all terms.  Document lengths (distinct terms) are lognormal
    with mean ``mean_len`` and log-sd ``sigma``.  Values are tf*log(m/df),
    documents L2-normalised.  ``labels`` holds each document's largest
    mixture component.
    """
    rng = np.random.default_rng(seed)
    mu = math.log(mean_len) - 0.5 * sigma * sigma
    lengths = np.maximum(1, np.rint(rng.lognormal(mu, sigma, m))).astype(np.int64)
    lengths = np.minimum(lengths, n)
    ntok = np.ceil(lengths * oversample).astype(np.int64) + 2
    theta = rng.dirichlet(np.full(ntopics, alpha), size=m)
    labels = np.argmax(theta, axis=1).astype(np.int32)
    nnoise = rng.binomial(ntok, noise)
    ntopic_tok = ntok - nnoise
    counts = rng.multinomial(ntopic_tok, theta)          # m x ntopics
    topic_vocab = np.stack([rng.choice(n, topic_terms, replace=False)
                            for _ in range(ntopics)])
    cdf = _zipf_cdf(topic_terms, s)
    docs, terms = [], []
    for z in range(ntopics):
        cz = counts[:, z]
        tot = int(cz.sum())
        if tot == 0:
            continue
        docs.append(np.repeat(np.arange(m, dtype=np.int64), cz))
        terms.append(topic_vocab[z][_draw(rng, cdf, tot)])
    docs.append(np.repeat(np.arange(m, dtype=np.int64), nnoise))
    terms.append(rng.integers(0, n, int(nnoise.sum())))
    doc = np.concatenate(docs)
    term = np.concatenate(terms).astype(np.int64)
    # random draw order so "first L distinct terms" does not favour a topic
    order = rng.permutation(len(doc)).astype(np.int64)
    c = _assemble(n, m, doc, term, lengths, order, None, rng, True, "tfidf")
    c.name = name
    c.labels = labels
    return c


def uniform_init(n: int, k: int, seed: int) -> np.ndarray:
    """Initial guess U0 ~ U[0,1), n x k, row-major float64."""
    return np.random.default_rng(seed + 7919).random((n, k))


def sparse_init(n: int, k: int, nnz_per_col: int, seed: int) -> np.ndarray:
    """Initial guess with ``nnz_per_col`` U[0,1) entries per column."""
    rng = np.random.default_rng(seed + 104729)
    U = np.zeros((n, k))
    for c in range(k):
        rows = rng.choice(n, min(nnz_per_col, n), replace=False)
        U[rows, c] = rng.random(len(rows)) + 1e-3
    return U


# ---------------------------------------------------------------------------
# The workloads, by what they are.

def small_zipf(seed: int = 1) -> Corpus:
    """2000 terms x 500 docs, ~50 distinct terms per doc, Zipf(1.1)."""
    return zipf_corpus(2000, 500, 50, 1.1, seed, name="zipf-2000x500")


def planted_50k_100k(seed: int = 2, scale: float = 1.0) -> Corpus:
    """50k terms x 100k docs, ~10M nnz, 50 planted topics of 500 terms.

    ``scale`` < 1 shrinks terms, documents and topic vocabularies together
    (used for parity cases the oracle finishes in seconds).
    """
    n = max(64, int(50_000 * scale))
    m = max(64, int(100_000 * scale))
    tt = max(8, int(500 * scale ** 0.5))
    return planted_corpus(n, m, 50, tt, 100.0 * min(1.0, scale ** 0.25), 0.7,
                          0.1, 0.05, seed, name=f"planted-{n}x{m}")


def zipf_100k_200k(seed: int = 5, scale: float = 1.0) -> Corpus:
    """100k terms x 200k docs, ~20M nnz, Zipf(1.1) (loss/gradient workload)."""
    n = max(64, int(100_000 * scale))
    m = max(64, int(200_000 * scale))
    return zipf_corpus(n, m, 100.0, 1.1, seed, sigma=0.7, name=f"zipf-{n}x{m}")


def batch_problems(count: int, seed: int = 4, max_scale: float = 1.0):
    """Uneven independent problems: n in [1k,20k], m in [500,10k], density in
    [0.1%, 2%] (all log-uniform), k uniform in [5, 40], t = 10% of the column
    length.  Returns a list of (Corpus, k, t_u, t_v)."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(math.exp(rng.uniform(math.log(1000), math.log(20000))) * max_scale)
        m = int(math.exp(rng.uniform(math.log(500), math.log(10000))) * max_scale)
        n, m = max(n, 16), max(m, 16)
        dens = math.exp(rng.uniform(math.log(0.001), math.log(0.02)))
        k = int(rng.integers(5, 41))
        k = min(k, n, m)
        c = zipf_corpus(n, m, max(1.0, dens * n), 1.1, seed * 1000 + p,
                        name=f"batch{p}")
        out.append((c, k, int(math.ceil(0.1 * n)), int(math.ceil(0.1 * m))))
    return out
