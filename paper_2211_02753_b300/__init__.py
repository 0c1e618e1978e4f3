"""Tensor Data Platform hot path on B300 (sm_103a).

Relational operators over columnar tensors (filter with stream compaction,
group-by aggregation, hash equi-join, top-k, radix sort) and the
differentiable soft filter / soft aggregation of trainable queries, plus the
glyph-CNN trainable query, all behind the C ABI in include/tdp.h
(``libtdp.so``).  ``ops`` holds the tensor-level wrappers, ``autograd`` the
torch.autograd.Function wrappers of the soft operators, ``plans`` the query
plans of the benchmark workloads, ``cnn`` the trainable glyph query.
"""
from ._lib import TdpError  # noqa: F401
