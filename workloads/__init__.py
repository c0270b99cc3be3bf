"""Seeded synthetic inputs for the hash-table path and its oracle.

This package is the only code that both the CUDA path's tests/benchmarks and
the CPU oracle's tests use.  It draws key streams and state-space model
tables from seeded generators and holds none of the hash-table method's
arithmetic (no hash family, no probing, no successor semantics).
"""
from .keys import (EMPTY32, KEY_MASK63, distinct_keys, fill_stream, lookup_batch,
                   mix32_perm, mix63_perm)
from .statespace import (DMAX, LMAX, CMAX, PMAX, Model, random_model,
                         config3_model, batched_models)

__all__ = [
    "EMPTY32", "KEY_MASK63", "distinct_keys", "fill_stream", "lookup_batch",
    "mix32_perm", "mix63_perm", "DMAX", "LMAX", "CMAX", "PMAX", "Model",
    "random_model", "config3_model", "batched_models",
]
