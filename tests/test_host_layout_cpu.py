"""The host-side layouts of A that espnmf_init builds (SELL part, the
frequent part's two tiers, the CSC transpose; csrc/host_layout.cuh),
checked on the CPU by tests/host_layout_check.cu, compiled here against the
library's own header:

* transpose_csr equals a serial transpose;
* the FP32 form's layouts built from FP32 values and from the same values
  widened to FP64 are bitwise equal (the set-up keeps FP32 input in FP32);
* every entry of A -- row, column and FP32 value -- and nothing else is
  recovered from each orientation's SELL part and frequent tiers, whose
  padding, row lists and work chunks are well formed;
* each product's frequent part has the size (h rows, h1 of them in shared
  memory) that its choice rule, restated here, gives;
* the factor export (pack_factor) matches a dense reference.

Corpora: the small Zipf corpus, a 60k x 40k Zipf corpus whose A^T U gets
both frequent tiers at k = 100, its transpose (both tiers in A V), the
widest padding (ld = 8), whole-matrix/none modes (no t per column), a
scaled planted corpus, and a matrix with explicit zeros, empty rows and
empty columns."""
import os
import re
import subprocess

import numpy as np
import pytest

from gen import Corpus, planted_50k_100k, small_zipf, zipf_corpus
from paper_1510_05237_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_05237_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    try:
        nvcc = B.nvcc_path()
    except RuntimeError:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("host_layout") / "host_layout_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", *B.ARCH, "-I", CSRC,
                    os.path.join(ROOT, "tests", "host_layout_check.cu"), "-o", exe],
                   check=True, timeout=900, capture_output=True)
    return exe


def _transpose(A: Corpus) -> Corpus:
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    order = np.lexsort((rows, A.colidx))
    rowptr = np.zeros(A.m + 1, dtype=np.int64)
    np.cumsum(np.bincount(A.colidx, minlength=A.m), out=rowptr[1:])
    return Corpus(A.m, A.n, rowptr, rows[order].astype(np.int32), A.val[order].copy())


def _with_zeros(seed: int) -> Corpus:
    """3000 x 2000, Zipf-skewed columns, a tenth of the values exactly 0,
    every fifth row and the last 100 columns empty."""
    rng = np.random.default_rng(seed)
    n, m = 3000, 1900
    ptr, cols = [0], []
    w = 1.0 / np.arange(1, m + 1) ** 1.1
    w /= w.sum()
    for r in range(n):
        k = 0 if r % 5 == 0 else int(rng.integers(1, 60))
        c = np.unique(rng.choice(m, size=k, p=w)) if k else np.zeros(0, dtype=np.int64)
        cols.append(c)
        ptr.append(ptr[-1] + len(c))
    colidx = np.concatenate(cols).astype(np.int32)
    val = rng.random(len(colidx)).astype(np.float32).astype(np.float64)
    val[rng.random(len(val)) < 0.1] = 0.0
    return Corpus(n, m + 100, np.array(ptr, dtype=np.int64), colidx, val)


_ZIPF = {}


def _zipf():
    if "z" not in _ZIPF:
        _ZIPF["z"] = zipf_corpus(60000, 40000, 60.0, 1.05, 7, sigma=0.7)
    return _ZIPF["z"]


CASES = {
    # name: (corpus, ld, t_u, t_v)
    "small_zipf": (lambda: small_zipf(3), 12, 40, 40),
    "zipf_two_tiers_AtU": (_zipf, 112, 1200, 400),
    "zipf_two_tiers_AV": (lambda: _transpose(_zipf()), 112, 400, 1200),
    "zipf_pad_32": (_zipf, 8, 300, 300),
    "zipf_no_t_per_column": (_zipf, 52, 0, 0),
    "planted_scaled": (lambda: planted_50k_100k(seed=2, scale=0.2), 52, 200, 200),
    "zeros_and_empty": (lambda: _with_zeros(5), 16, 200, 200),
}


def expected_frequent(weights: np.ndarray, nnz: int, ld: int, t_rows: int):
    """(h, h1) of a product's frequent part by its stated rule: candidates are
    the gathered rows referenced at least max(16, 4 x mean) times, by
    decreasing weight; the shared-memory tier takes as many as fit 200 KB
    (at most 65535); with t_rows = t (column mode) the part takes up to t
    candidates (and at most 16 MB of table) when that adds at least 256 rows
    beyond the first tier; the part is kept only if it covers a tenth of
    the entries."""
    ng = len(weights)
    if ng == 0 or nnz == 0:
        return 0, 0
    cap1 = min(200 * 1024 // (ld * 4), 65535)
    cap_all = min((16 << 20) // (ld * 4), 65535)
    floor_w = max(16.0, 4.0 * nnz / ng)
    order = sorted(np.nonzero(weights >= floor_w)[0], key=lambda g: (-weights[g], g))
    want = min(len(order), t_rows, cap_all)
    cap = want if want - cap1 >= 256 else cap1
    order = order[:cap]
    if not order or int(weights[order].sum()) * 10 < nnz:
        return 0, 0
    return len(order), min(len(order), cap1)


@pytest.mark.parametrize("name", list(CASES))
def test_host_layouts(checker, tmp_path, name):
    make, ld, t_u, t_v = CASES[name]
    A = make()
    pre = str(tmp_path / name)
    np.ascontiguousarray(A.rowptr, dtype=np.int64).tofile(pre + "_rp.bin")
    np.ascontiguousarray(A.colidx, dtype=np.int32).tofile(pre + "_ci.bin")
    np.ascontiguousarray(A.val, dtype=np.float32).tofile(pre + "_vf.bin")
    r = subprocess.run([checker, pre, str(A.n), str(A.m), str(ld), str(t_u), str(t_v)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith(": ok"), r.stdout
    if name.startswith("zipf_two_tiers"):
        assert "h=1200 (h1=457" in r.stdout, r.stdout      # both tiers present
    # the frequent parts of A V (gathered: documents, weights = their
    # lengths) and A^T U (gathered: terms, weights = their frequencies)
    doc_len = np.bincount(A.colidx, minlength=A.m)
    term_freq = np.diff(A.rowptr)
    got = re.findall(r"h=(\d+) \(h1=(\d+)", r.stdout)
    assert got == [tuple(str(x) for x in expected_frequent(doc_len, A.nnz, ld, t_v)),
                   tuple(str(x) for x in expected_frequent(term_freq, A.nnz, ld, t_u))], r.stdout
