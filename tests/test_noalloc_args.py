"""The allocation-free entry point's Python wrapper checks its tensors on the
host before any pointer reaches the device (no GPU needed): a keys tensor of
the wrong width, a short state block or a short flag buffer would otherwise
make the kernels read or write past a caller's allocation."""
import pytest
import torch

import paper_1712_09494_gb300 as ht


def _ok():
    return dict(slots=torch.empty(64, dtype=torch.int64), state=torch.empty(ht.NOALLOC_STATE_BYTES, dtype=torch.uint8),
                keys=torch.zeros(10, dtype=torch.int64), is_new=torch.empty(10, dtype=torch.uint8))


@pytest.mark.parametrize("bad", [
    dict(keys=torch.zeros(10, dtype=torch.int32)),                      # 32-bit keys: 4n bytes, not 8n
    dict(keys=torch.zeros((5, 2), dtype=torch.int64)),                  # not 1-D
    dict(state=torch.empty(ht.NOALLOC_STATE_BYTES - 1, dtype=torch.uint8)),
    dict(is_new=torch.empty(9, dtype=torch.uint8)),                     # shorter than the batch
    dict(is_new=torch.empty(10, dtype=torch.int32)),
    dict(slots=torch.empty(64, dtype=torch.int32)),
    dict(slots=torch.empty(0, dtype=torch.int64)),
    dict(keys=torch.zeros(ht.NOALLOC_MAX_BATCH + 1, dtype=torch.int64)),
])
def test_wrapper_rejects_malformed_tensors(bad):
    a = _ok()
    a.update(bad)
    with pytest.raises(ValueError):
        ht._noalloc_args(a["slots"], a["state"], a["keys"], a["is_new"])
    with pytest.raises(ValueError):
        ht.ht_cuckoo_find_or_put_noalloc(a["slots"], a["state"], 1, a["keys"], a["is_new"])


def test_wrapper_accepts_well_formed_tensors():
    a = _ok()
    assert ht._noalloc_args(a["slots"], a["state"], a["keys"], a["is_new"]) == 10
    assert ht._noalloc_args(a["slots"], a["state"], a["keys"], None) == 10
    # uint64 keys and a state block given as int64 words are fine too.
    st = torch.empty(ht.NOALLOC_STATE_BYTES // 8, dtype=torch.int64)
    assert ht._noalloc_args(a["slots"], st, torch.zeros(3, dtype=torch.uint64), None) == 3
