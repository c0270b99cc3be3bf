"""Parity of the batched exploration form with the oracle, in every mode.

Each exploration's BFS levels must equal the oracle's levels as sets, whether
the explorations run together (one persistent launch, per-step launches or a
per-step graph) or one after another, with bucket or Cuckoo tables.
"""
import json
import os

import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import statespace as ss

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


def hmodel(m):
    return ht.make_model(m.C, m.bits, m.deg, m.tgt, m.lab, m.pairs)


def _run_and_check(oracle_lib, models, params=None, modes=(0, 1, 2, 3), schemes=None):
    refs = [oracle_lib.bfs(m, max_states=1 << 22) for m in models]
    caps = [max(256, int(r.total / 0.7)) for r in refs]
    mx = ht.MultiExploration([hmodel(m) for m in models], [0] * len(models), caps, params=params, schemes=schemes)
    for mode in modes:
        mx.reset()
        steps = mx.run(mode=mode)
        assert steps >= 1
        for i, (m, r) in enumerate(zip(models, refs)):
            res = mx.result(i, with_states=True, key_width=m.key_width)
            assert res["complete"] == 1, (mode, i)
            assert res["states"] == r.total, (mode, i)
            assert res["successors"] == int(r.level_succ.sum()), (mode, i)
            np.testing.assert_array_equal(res["level_sizes"], r.level_sizes)
            got = res["states_host"].astype(np.uint64)
            off = 0
            for d, n_d in enumerate(res["level_sizes"]):
                np.testing.assert_array_equal(np.sort(got[off:off + n_d]), np.sort(r.level(d)))
                off += n_d
    mx.close()


def test_multi_matches_oracle(oracle_lib):
    models = ss.batched_models(24, seed=7)
    _run_and_check(oracle_lib, models)


def test_multi_cuckoo_matches_oracle(oracle_lib):
    # Cuckoo tables in the persistent launch (probe, barrier, insert per
    # step) and in the one-at-a-time baseline.
    models = ss.batched_models(24, seed=8)
    _run_and_check(oracle_lib, models, modes=(0, 2), schemes="cuckoo")


def test_multi_mixed_schemes_and_cuckoo_parameters(oracle_lib):
    # Bucket and Cuckoo explorations in one run (separate groups), Cuckoo
    # with k = 3 / 5 and short eviction bounds, and a Cuckoo table capped by
    # its claim set (max_batch smaller than the table): several steps per
    # level for it.
    models = ss.batched_models(16, seed=9)
    schemes = ["bucket" if i % 2 else "cuckoo" for i in range(len(models))]
    params = [None if i % 2 else dict(num_hashes=3 + 2 * (i % 4 == 0), max_evictions=16 + i, max_batch=1 << 10)
              for i in range(len(models))]
    _run_and_check(oracle_lib, models, params=params, modes=(0, 2), schemes=schemes)


def test_persistent_run_reports_steps_and_rejects_cuckoo_in_step_modes(oracle_lib):
    models = ss.batched_models(4, seed=10)
    refs = [oracle_lib.bfs(m, max_states=1 << 22) for m in models]
    caps = [max(256, int(r.total / 0.7)) for r in refs]
    mx = ht.MultiExploration([hmodel(m) for m in models], [0] * 4, caps, schemes="cuckoo")
    steps = mx.run(mode=0)
    assert steps >= max(len(r.level_sizes) for r in refs) - 1
    for mode in (1, 3):
        mx.reset()
        with pytest.raises(ht.HtError) as e:
            mx.run(mode=mode)
        assert e.value.status == 1
    # A step limit stops every exploration early, with the levels done so far exact.
    mx.reset()
    mx.run(mode=0, max_steps=2)
    for i, r in enumerate(refs):
        res = mx.result(i)
        assert res["complete"] == 0 or len(r.level_sizes) <= 3
        assert res["level_sizes"][:1] == [1]
    mx.close()


def test_multi_mixed_key_widths_and_shapes(oracle_lib):
    small = [ss.random_model(s, C=4, L=8, R=[3, 5, 4, 2], p_sync=0.3, P=2) for s in range(6)]     # 12-bit vectors
    wide = [ss.random_model(100 + s, C=9, L=32, R=3, p_sync=0.2, P=3) for s in range(5)]        # 45-bit vectors
    models = small + wide
    assert {m.key_width for m in models} == {32, 64}
    shapes = [dict(bucket_slots=16, lanes_per_key=2), dict(bucket_slots=8, lanes_per_key=4),
              dict(bucket_slots=32, lanes_per_key=8)]
    params = [shapes[i % 3] for i in range(len(models))]
    _run_and_check(oracle_lib, models, params=params, modes=(0, 2, 3))


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_multi_uneven_sizes_share_the_successor_budget(oracle_lib, scheme):
    # One large exploration next to many tiny ones: the large one needs several
    # steps per level while the tiny ones finish early.
    big = ss.random_model(55, C=10, L=16, R=[4, 4, 4, 4, 4, 3, 3, 3, 3, 4], p_sync=0.1, P=2)
    tiny = [ss.random_model(60 + s, C=2, L=4, R=[2, 3], P=0) for s in range(20)]
    _run_and_check(oracle_lib, [big] + tiny, modes=(0,), schemes=scheme)


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_multi_full_batched_workload_against_stored_levels(scheme):
    path = os.path.join(GOLDEN, "statespace_batched.json")
    if not os.path.exists(path):
        pytest.skip("stored batched levels not generated")
    import sys
    sys.path.insert(0, GOLDEN)
    from digest import digest
    gold = json.load(open(path))
    models = ss.batched_models(gold["model"]["count"], seed=gold["model"]["seed"])
    caps = [max(256, int(g["states"] / 0.7)) for g in gold["explorations"]]
    mx = ht.MultiExploration([hmodel(m) for m in models], [0] * len(models), caps, schemes=scheme)
    mx.run(mode=0)
    for i, (m, g) in enumerate(zip(models, gold["explorations"])):
        res = mx.result(i, with_states=True, key_width=m.key_width)
        assert res["complete"] == 1 and res["states"] == g["states"], i
        assert res["successors"] == g["successors"], i
        got = res["states_host"].astype(np.uint64)
        off = 0
        for d, lev in enumerate(g["levels"]):
            n_d = lev[0]
            assert res["level_sizes"][d] == n_d
            assert digest(got[off:off + n_d])[1:] == lev[1:3], (i, d)
            off += n_d
    mx.close()


@pytest.mark.parametrize("mode,scheme", [(0, "bucket"), (2, "bucket"), (3, "bucket"), (0, "cuckoo"), (2, "cuckoo")])
def test_multi_reports_a_table_too_small_for_its_exploration(oracle_lib, mode, scheme):
    # Exploration 1's table (256 slots + stash + overflow set, ~1400 keys)
    # cannot hold its ~20000 reachable states: the run reports HT_ERR_FULL
    # instead of returning an inexact exploration.
    ok = ss.random_model(3, C=4, L=8, R=[3, 5, 4, 2], p_sync=0.3, P=2)
    big = ss.random_model(55, C=10, L=16, R=[4, 4, 4, 4, 4, 3, 3, 3, 3, 4], p_sync=0.1, P=2)
    r_ok, r_big = oracle_lib.bfs(ok, max_states=1 << 22), oracle_lib.bfs(big, max_states=1 << 22)
    assert r_big.total > 10_000
    mx = ht.MultiExploration([hmodel(ok), hmodel(big)], [0, 0], [max(256, int(r_ok.total / 0.7)), 256],
                             schemes=scheme)
    with pytest.raises(ht.HtError) as e:
        mx.run(mode=mode)
    assert e.value.status == 3
    mx.close()


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_persistent_barrier_wait_runs_out_and_reports_timeout(oracle_lib, scheme):
    """A block of the persistent launch leaves before its first grid barrier,
    as a block that died would: every other block's bounded wait (50 ms here)
    runs out, the launch ends, and the run returns HT_ERR_TIMEOUT.  The device
    stays usable: with the hooks cleared and the tables reset, the next run
    is exact."""
    import time
    models = ss.batched_models(6, seed=11)
    refs = [oracle_lib.bfs(m, max_states=1 << 22) for m in models]
    caps = [max(256, int(r.total / 0.7)) for r in refs]
    mx = ht.MultiExploration([hmodel(m) for m in models], [0] * 6, caps, schemes=scheme)
    mx.test_hooks(barrier_timeout_ns=50_000_000, absent_block=1)
    t0 = time.time()
    with pytest.raises(ht.HtError) as e:
        mx.run(mode=0)
    assert e.value.status == 5
    assert time.time() - t0 < 30
    mx.test_hooks()
    mx.reset()
    mx.run(mode=0)
    for i, r in enumerate(refs):
        res = mx.result(i)
        assert res["complete"] == 1 and res["states"] == r.total
        np.testing.assert_array_equal(res["level_sizes"], r.level_sizes)
    mx.close()
