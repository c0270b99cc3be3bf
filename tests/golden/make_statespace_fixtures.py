"""Writes the stored oracle results for the large state-space workloads.

Runs only the CPU oracle (oracle/) on models drawn by workloads/statespace.py
and stores, per BFS level, the level size and an order-independent digest of
the level's states (tests/golden/digest.py).  Outputs:
  statespace_config3.json   12 components x 32 local states, 4 sync pairs
                            (about 10^8 reachable states; several minutes and
                            ~8 GB of host memory)
  statespace_batched.json   the 256 explorations of the batched workload
Usage: python tests/golden/make_statespace_fixtures.py [config3] [batched]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from workloads import statespace as ss  # noqa: E402
from digest import digest  # noqa: E402


def explore(m, max_states):
    t0 = time.time()
    r = oracle.bfs(m, max_states=max_states, max_levels=4096, keep_states=True)
    assert r.rc == 0, "exploration exceeded its limits"
    levels = []
    for d in range(len(r.level_sizes)):
        levels.append([int(r.level_sizes[d])] + digest(r.level(d))[1:] + [int(r.level_succ[d])])
    return dict(states=int(r.total), successors=int(r.level_succ.sum()), levels=levels,
                oracle_seconds=round(time.time() - t0, 1))


def main(which):
    if "config3" in which:
        m = ss.config3_model()
        out = dict(model=dict(generator="workloads.statespace.config3_model", seed=3, p_sync=0.25),
                   level_fields=["size", "sum_mix", "xor_mix", "successors_generated"], **explore(m, 200_000_000))
        with open(os.path.join(HERE, "statespace_config3.json"), "w") as f:
            json.dump(out, f)
        print("config3", out["states"], len(out["levels"]), out["oracle_seconds"], flush=True)
    if "batched" in which:
        models = ss.batched_models(256, seed=4)
        res = []
        for i, m in enumerate(models):
            res.append(explore(m, 1 << 22))
        out = dict(model=dict(generator="workloads.statespace.batched_models", count=256, seed=4),
                   level_fields=["size", "sum_mix", "xor_mix", "successors_generated"], explorations=res)
        with open(os.path.join(HERE, "statespace_batched.json"), "w") as f:
            json.dump(out, f)
        print("batched", sum(r["states"] for r in res), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["config3", "batched"])
