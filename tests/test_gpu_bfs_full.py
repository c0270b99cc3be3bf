"""Full-size state-space BFS (12 components x 32 local states, 4 sync pairs,
about 10^8 reachable states) against the oracle's stored levels.

The oracle run takes minutes, so tests/golden/statespace_config3.json holds
its per-level sizes and set digests (written by
tests/golden/make_statespace_fixtures.py, which calls only the oracle).  The
CUDA exploration must reproduce every level's size and digest, the total
state count and the number of successors generated.
"""
import json
import os
import sys

import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import statespace as ss

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
from digest import digest  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


@pytest.mark.parametrize("scheme,fused", [("bucket", False), ("bucket", True), ("cuckoo", False)],
                         ids=["bucket", "bucket_fused", "cuckoo"])
def test_config3_bfs_matches_stored_oracle_levels(scheme, fused):
    gold = json.load(open(os.path.join(GOLDEN, "statespace_config3.json")))
    m = ss.config3_model(seed=gold["model"]["seed"], p_sync=gold["model"]["p_sync"])
    hm = ht.make_model(m.C, m.bits, m.deg, m.tgt, m.lab, m.pairs)
    t = ht.HashTable(int(gold["states"] / 0.8), scheme, 64)
    states = torch.empty(gold["states"] + 1024, dtype=torch.int64, device="cuda")
    res, sizes = ht.ht_bfs(t.handle, hm, 0, 4096, states, fused=fused)
    assert res.complete == 1
    assert res.states == gold["states"]
    assert res.successors == gold["successors"]
    assert sizes == [lev[0] for lev in gold["levels"]]
    host = states[:res.states].cpu().numpy().view(np.uint64)
    off = 0
    for d, lev in enumerate(gold["levels"]):
        assert digest(host[off:off + lev[0]])[1:] == lev[1:3], "level %d differs" % d
        off += lev[0]
    assert t.size() == gold["states"]
