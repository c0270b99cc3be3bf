"""Multiplicity sequences, the shape of the paper's random-data experiment
(Section 5.2, Fig. 5): random 32-bit keys drawn from a value range of n/m
values, so each value occurs m times on average, the whole sequence found or
inserted in ONE ht_find_or_put call into a table of 1.25x its distinct
values (load 0.8).  Both schemes, at m = 1, 50 and 1000, against the oracle:
per distinct key the same number of is_new flags (exactly one), and the
exported set equal to the oracle's, element by element after sorting.  At
m = 1000 about 2^22 / 1000 values share the whole call, so the in-batch
duplicate handling (Section 5.1.1) is what is tested."""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import device_keys as dk

from gpu_util import assert_flags_per_key, assert_same_set, keys_np, to_np

pytestmark = pytest.mark.gpu

N = 1 << 22


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


@pytest.fixture(scope="module")
def sequences(oracle_lib):
    out = {}
    for m in (1, 50, 1000):
        keys_d = dk.multiplicity_sequence_dev(N, m, seed=29 + m, device="cuda")
        kn = to_np(keys_d, np.uint32)
        orc = oracle_lib.OracleTable()
        exp = orc.find_or_put(kn)
        out[m] = (keys_d, kn, exp, np.sort(orc.export()[0].astype(np.uint64)))
    return out


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
@pytest.mark.parametrize("m", [1, 50, 1000])
def test_whole_sequence_in_one_call_matches_oracle(sequences, scheme, m):
    keys_d, kn, exp, oracle_set = sequences[m]
    distinct = len(oracle_set)
    assert abs(N / distinct - m) < 0.5 * m + 1          # the sequence has the intended multiplicity
    t = ht.HashTable(int(np.ceil(distinct * 1.25)), scheme, 32)
    flags = torch.empty(N, dtype=torch.uint8, device="cuda")
    ht.ht_find_or_put(t.handle, keys_d, flags)
    got = to_np(flags)
    assert int(got.sum()) == distinct
    assert_flags_per_key(kn, got, exp)
    assert t.sync() == 0 and t.size() == distinct
    k, _ = t.export()
    assert_same_set(keys_np(k, 32), oracle_set)
    # A second pass over the same sequence finds every key: no flag at all.
    ht.ht_find_or_put(t.handle, keys_d, flags)
    assert int(flags.sum()) == 0 and t.size() == distinct
