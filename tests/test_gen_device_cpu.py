"""The large-corpus generator (gen.device_corpus), run with torch on the CPU
at a small scale: a valid CSR over terms (rows ascending, documents strictly
increasing within each row, positive values), L2-normalised documents,
lengths near the requested mean, Zipf-skewed document frequencies, and the
same matrix for the same seed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from gen.device_corpus import zipf_1m_2m_device, zipf_corpus_device  # noqa: E402


@pytest.fixture(scope="module")
def small():
    return zipf_1m_2m_device(seed=3, scale=0.005, device="cpu")


def test_csr_is_valid(small):
    A = small.to_host()
    assert A.n == 5000 and A.m == 10000
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz and np.all(np.diff(A.rowptr) >= 0)
    assert A.colidx.min() >= 0 and A.colidx.max() < A.m
    for r in range(0, A.n, 7):
        assert np.all(np.diff(A.colidx[A.rowptr[r]:A.rowptr[r + 1]]) > 0)
    assert np.all(A.val > 0)


def test_documents_are_unit_norm_and_lengths_follow_the_mean(small):
    A = small.to_host()
    norm2 = np.bincount(A.colidx, weights=A.val * A.val, minlength=A.m)
    assert np.all(norm2 > 0)
    np.testing.assert_allclose(norm2, 1.0, rtol=2e-6)       # FP32 values
    mean = 200.0 * 0.005 ** 0.25
    lens = np.bincount(A.colidx, minlength=A.m)
    assert 0.9 * mean < lens.mean() < 1.05 * mean


def test_term_frequencies_are_zipf_skewed(small):
    A = small.to_host()
    df = np.sort(np.diff(A.rowptr))[::-1]
    # the most frequent terms appear in most documents (a document counts a
    # term once, which flattens the head) and the frequencies fall off by
    # about a decade per decade of rank further down
    assert df[0] > 0.5 * A.m
    assert df[0] > 8 * df[99] and df[99] > 5 * df[999]


def test_same_seed_same_matrix_other_seed_other_matrix():
    a = zipf_corpus_device(2000, 3000, 40.0, 1.05, 0.7, 7, device="cpu")
    b = zipf_corpus_device(2000, 3000, 40.0, 1.05, 0.7, 7, device="cpu")
    c = zipf_corpus_device(2000, 3000, 40.0, 1.05, 0.7, 8, device="cpu")
    assert torch.equal(a.rowptr, b.rowptr) and torch.equal(a.colidx, b.colidx)
    assert torch.equal(a.val, b.val)
    assert not (a.colidx.numel() == c.colidx.numel() and torch.equal(a.colidx, c.colidx))
