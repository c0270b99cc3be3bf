"""Autotuner bookkeeping (CPU) and one real tuning run (GPU)."""
import json

import pytest

from paper_1712_09494_gb300 import autotune as at


def test_class_key_rounds_capacity_load_and_repeats():
    k1 = at.class_key("GB300", "bucket", 64, 1_000_000, 0.8, 0.25)
    k2 = at.class_key("GB300", "bucket", 64, 1 << 20, 0.79, 0.26)
    assert k1 == k2 == "GB300|bucket|64|2^20|lf0.8|d0.3"
    assert at.class_key("GB300", "bucket", 64, 5, 0.8, 0.0).split("|")[3] == "2^10"


def test_pick_takes_the_fastest_exact_candidate():
    res = [(dict(a=1), 0.5), (dict(a=2), None), (dict(a=3), 0.2), (dict(a=4), 0.3)]
    assert at.pick(res) == dict(a=3)
    assert at.pick([(dict(a=1), None)]) is None


def test_tune_measures_once_then_uses_the_cache(tmp_path):
    path = str(tmp_path / "cache.json")
    calls = []

    def fake(p):
        calls.append(p)
        return None if p["num_hashes"] == 3 else 1.0 / (p["num_hashes"] * p["max_evictions"])

    best = at.tune("cuckoo", 64, 1 << 20, cache_path=path, measure=fake, device_name="dev")
    assert best == dict(num_hashes=5, max_evictions=1024)
    assert len(calls) == len(at.CANDIDATES["cuckoo"])
    again = at.tune("cuckoo", 64, 1 << 20, cache_path=path, measure=fake, device_name="dev")
    assert again == best and len(calls) == len(at.CANDIDATES["cuckoo"])
    stored = json.load(open(path))
    assert list(stored) == ["dev|cuckoo|64|2^20|lf0.8|d0.3"]
    with pytest.raises(RuntimeError):
        at.tune("cuckoo", 64, 1 << 12, cache_path=path, measure=lambda p: None, device_name="dev")


@pytest.mark.gpu
@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_tuned_parameters_fill_exactly(tmp_path, scheme, oracle_lib):
    import numpy as np
    import torch
    import paper_1712_09494_gb300 as ht
    from paper_1712_09494_gb300 import _build
    from workloads import keys as wk
    _build.build()
    cands = at.CANDIDATES[scheme][:4]
    best = at.tune(scheme, 64, 1 << 16, cache_path=str(tmp_path / "c.json"), candidates=cands)
    assert best in cands
    t = ht.HashTable(1 << 16, scheme, 64, best)
    keys = wk.distinct_keys(50_000, 64, seed=3)
    got = t.find_or_put(torch.from_numpy(keys.view(np.int64)).cuda()).cpu().numpy()
    assert got.sum() == 50_000 and t.size() == 50_000


def test_flags_exact_rejects_a_lost_or_doubled_key():
    import torch
    fresh = [torch.tensor([5, 9, 2]), torch.tensor([7])]
    batches = [torch.tensor([9, 5, 5, 2, 9]), torch.tensor([2, 7, 7, 5])]
    good = [torch.tensor([1, 0, 1, 1, 0], dtype=torch.uint8), torch.tensor([0, 0, 1, 0], dtype=torch.uint8)]
    assert at.flags_exact(batches, good, fresh)
    lost = [good[0].clone(), torch.tensor([0, 0, 0, 0], dtype=torch.uint8)]
    assert not at.flags_exact(batches, lost, fresh)
    doubled = [torch.tensor([1, 1, 1, 1, 0], dtype=torch.uint8), good[1]]
    assert not at.flags_exact(batches, doubled, fresh)
    old_flagged = [good[0], torch.tensor([1, 1, 0, 0], dtype=torch.uint8)]   # 2 was stored before
    assert not at.flags_exact(batches, old_flagged, fresh)
