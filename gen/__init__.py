"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path."""
from .corpus import (Corpus, zipf_corpus, planted_corpus, uniform_init,
                     sparse_init, small_zipf, planted_50k_100k,
                     zipf_100k_200k, batch_problems)

__all__ = ["Corpus", "zipf_corpus", "planted_corpus", "uniform_init",
           "sparse_init", "small_zipf", "planted_50k_100k", "zipf_100k_200k",
           "batch_problems"]
