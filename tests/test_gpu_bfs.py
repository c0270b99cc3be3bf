"""Parity of the CUDA successor generator and BFS with the CPU oracle.

BFS levels are unique as sets, so each level of the GPU exploration must
equal the oracle's level exactly (order inside a level is free).  Successor
generation is compared as a multiset.
"""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import statespace as ss

from gpu_util import keys_np, to_dev, to_np

pytestmark = pytest.mark.gpu
SCHEMES = ["bucket", "cuckoo"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


def hmodel(m):
    return ht.make_model(m.C, m.bits, m.deg, m.tgt, m.lab, m.pairs)


MODELS = [
    dict(seed=1, C=3, L=8, R=5, P=0, p_sync=0.0),
    dict(seed=2, C=4, L=[4, 8, 5, 6], R=[3, 6, 5, 2], P=2, p_sync=0.5),
    dict(seed=3, C=6, L=16, R=6, P=3, p_sync=0.3),
    dict(seed=4, C=8, L=32, R=5, P=4, p_sync=0.25),
    dict(seed=5, C=12, L=32, R=[3] * 12, P=4, p_sync=0.3),      # 60-bit vectors
]


@pytest.mark.parametrize("spec", MODELS)
def test_successors_match_oracle(oracle_lib, spec):
    m = ss.random_model(spec["seed"], C=spec["C"], L=spec["L"], R=spec["R"], p_sync=spec["p_sync"], P=spec["P"])
    kw = m.key_width
    ref = oracle_lib.bfs(m, max_states=50_000)
    rng = np.random.default_rng(0)
    states = ref.states[rng.integers(0, len(ref.states), size=3001)]
    dt = np.uint32 if kw == 32 else np.uint64
    d_states = to_dev(states.astype(dt))
    cap = 3001 * 200
    succ = torch.empty(cap, dtype=torch.int32 if kw == 32 else torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ht.ht_successors(hmodel(m), d_states, succ, cnt)
    c = int(cnt.item())
    exp = np.concatenate([oracle_lib.successors(m, int(s)) for s in states])
    assert c == len(exp)
    np.testing.assert_array_equal(np.sort(keys_np(succ[:c], kw).astype(np.uint64)), np.sort(exp))


_REF = {}


def _oracle_bfs(oracle_lib, m):
    key = (m.meta.get("seed"), m.C, m.total_bits, m.P, m.deg.tobytes(), m.tgt.tobytes(), m.lab.tobytes())
    if key not in _REF:
        _REF[key] = oracle_lib.bfs(m, max_states=1 << 22)
    return _REF[key]


# BFS forms: (scheme, fused successor generation + find-or-put).
FORMS = [("bucket", False), ("bucket", True), ("cuckoo", False)]
FORM_IDS = ["bucket", "bucket_fused", "cuckoo"]


def _check_bfs(oracle_lib, m, scheme, params=None, fused=False):
    ref = _oracle_bfs(oracle_lib, m)
    assert ref.rc == 0
    kw = m.key_width
    t = ht.HashTable(max(64, int(ref.total / 0.7)), scheme, kw, params)
    states = torch.empty(ref.total + 16, dtype=torch.int32 if kw == 32 else torch.int64, device="cuda")
    res, sizes = ht.ht_bfs(t.handle, hmodel(m), 0, 4096, states, fused=fused)
    assert res.complete == 1
    assert res.states == ref.total
    assert res.successors == int(ref.level_succ.sum())
    np.testing.assert_array_equal(np.array(sizes), ref.level_sizes)
    got = keys_np(states[:res.states], kw).astype(np.uint64)
    off = 0
    for d, n_d in enumerate(sizes):
        np.testing.assert_array_equal(np.sort(got[off:off + n_d]), np.sort(ref.level(d)))
        off += n_d
    assert t.size() == ref.total
    return res


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("spec", MODELS)
def test_bfs_matches_oracle(oracle_lib, form, spec):
    m = ss.random_model(spec["seed"], C=spec["C"], L=spec["L"], R=spec["R"], p_sync=spec["p_sync"], P=spec["P"])
    _check_bfs(oracle_lib, m, form[0], fused=form[1])


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_bfs_medium_model_small_chunks(oracle_lib, form):
    # ~10^5-10^6 states; a small Cuckoo batch bound forces many chunks per level.
    scheme, fused = form
    m = ss.random_model(21, C=10, L=16, R=[4, 4, 4, 4, 3, 3, 3, 3, 4, 4], p_sync=0.2, P=3)
    params = dict(max_batch=1 << 12) if scheme == "cuckoo" else dict(bucket_slots=16, lanes_per_key=4)
    _check_bfs(oracle_lib, m, scheme, params, fused=fused)


@pytest.mark.parametrize("shape", [(8, 2), (32, 8), (16, 16)])
def test_bfs_fused_other_bucket_shapes(oracle_lib, shape):
    m = ss.random_model(33, C=9, L=32, R=3, p_sync=0.2, P=3)             # 45-bit vectors
    _check_bfs(oracle_lib, m, "bucket", dict(bucket_slots=shape[0], lanes_per_key=shape[1]), fused=True)


def test_bfs_fused_rejects_cuckoo():
    m = ss.random_model(1, C=3, L=8, R=5)
    t = ht.HashTable(1024, "cuckoo", 32)
    with pytest.raises(ht.HtError):
        ht.ht_bfs(t.handle, hmodel(m), 0, 16, torch.empty(1024, dtype=torch.int32, device="cuda"), fused=True)


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
def test_bfs_degenerate_models(oracle_lib, form):
    scheme, fused = form
    # Every transition synchronised with a partner that never matches: s0 only.
    L = [4, 4]
    bits = np.zeros(16, np.uint8)
    bits[:2] = 2
    deg = np.zeros((16, 32), np.uint8)
    tgt = np.zeros((16, 32, 4), np.uint8)
    lab = np.zeros((16, 32, 4), np.uint8)
    deg[0, :4] = 1
    tgt[0, :4, 0] = 1
    lab[0, :4, 0] = 1           # pair 0, but component 1 has no label-1 transitions
    m = ss.Model(C=2, L=np.array(L), bits=bits, deg=deg, tgt=tgt, lab=lab, pairs=np.array([[0, 1]], np.uint8))
    t = ht.HashTable(64, scheme, 32)
    res, sizes = ht.ht_bfs(t.handle, hmodel(m), 0, 16, torch.empty(8, dtype=torch.int32, device="cuda"), fused=fused)
    assert res.complete == 1 and sizes == [1] and res.successors == 0
    # A chain longer than max_levels stops incomplete.
    m2 = ss.random_model(1, C=1, L=32, R=32, deg_lo=1, deg_hi=1)
    t2 = ht.HashTable(64, scheme, 32)
    res2, sizes2 = ht.ht_bfs(t2.handle, hmodel(m2), 0, 5, torch.empty(64, dtype=torch.int32, device="cuda"),
                             fused=fused)
    assert res2.complete == 0 and sizes2 == [1] * 5


def test_bfs_rejects_bad_models():
    m = ss.random_model(1, C=3, L=8, R=5)
    hm = hmodel(m)
    hm.num_components = 17
    t = ht.HashTable(64, "bucket", 32)
    with pytest.raises(ht.HtError):
        ht.ht_bfs(t.handle, hm, 0, 16, torch.empty(64, dtype=torch.int32, device="cuda"))
    wide = ss.random_model(2, C=8, L=32, R=4)           # 40 bits do not fit 32-bit keys
    with pytest.raises(ht.HtError):
        ht.ht_bfs(t.handle, hmodel(wide), 0, 16, torch.empty(64, dtype=torch.int32, device="cuda"))
