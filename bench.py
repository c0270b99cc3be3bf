"""Benchmark: batched find-or-put into both hash-table schemes on one GB300.

A step is the paper's timed quantity (Section 5: the time to find-or-insert
every element of a sequence) on the random-key workload at load 0.8: an
empty table of ceil(n/0.8) slots is filled with n distinct uniformly random
64-bit keys by find-or-put batches of 2^24 keys, 25% of each batch repeats of
keys already issued; once with the bucket scheme and once with Cuckoo
hashing.  `value` = find-or-put keys processed per second over the whole
step, both schemes.

Prints one JSON line.  Under torchrun each rank runs its own replica (the
path has no exchange step) and rank 0 reports the whole-job throughput.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "find-or-put Mops/s per scheme at load 0.8; % HBM random-access roofline; p99 lat"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--no-sweep", action="store_true", help="skip the config-2 parameter sweep")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--schemes", default="bucket,cuckoo")
    ap.add_argument("--n-log2", type=int, default=27)
    ap.add_argument("--lf", type=float, default=0.8)
    ap.add_argument("--batch-log2", type=int, default=24)
    ap.add_argument("--dup", type=float, default=0.25)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-bfs", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--only", default="",
                    help="comma list: of the sections after the headline fill run only these (small, sweep, replay, "
                         "wide, long, wide_bfs, bfs, batched, serving)")
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-rate", type=float, default=40000.0, help="Poisson arrivals per second")
    ap.add_argument("--serve-deadline", type=float, default=120.0, help="seconds before a serving run gives up")
    return ap.parse_args()


def workload_config(a, schemes):
    n = 1 << a.n_log2
    return {
        "workload": "random 64-bit keys, fill to load %.2f: n=2^%d distinct, find-or-put batches of 2^%d, "
                    "%d%% repeats; schemes %s" % (a.lf, a.n_log2, a.batch_log2, round(a.dup * 100), "+".join(schemes)),
        "n_distinct": n,
        "capacity_slots": int(np.ceil(n / a.lf)),
        "load": a.lf,
        "batch": 1 << a.batch_log2,
        "dup_rate": a.dup,
        "key_width": 64,
        "schemes": schemes,
        "l2": "inputs larger than L2 (table %.2f GB, keys %.2f GB, L2 129 MB); no flush needed"
              % (np.ceil(n / a.lf) * 8 / 1e9, n / (1 - a.dup) * 8 / 1e9),
    }


# ----------------------------------------------------------------- helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value, device):
    """The largest `value` over all ranks (the job's step time is the slowest
    rank's); the identity when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mops(units_per_rank, world, ms_per_step_max):
    """Whole-job throughput: every rank processes units_per_rank per step
    (replicas; weak scaling), timed by the slowest rank."""
    return units_per_rank * world / (ms_per_step_max / 1e3) / 1e6


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def section_wanted(only, section, off):
    """Whether an optional section runs: with --only, exactly the sections it
    names; otherwise every section whose --no-* flag is not set."""
    return section in only if only else not off


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    kernel's source has not changed since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    for m in re.finditer(r"^traffic\s+(\S+)\s+(\S+)\s+(\d+)\s+(\w+)\s*$", text, re.M):
        name, src, nbytes, sha = m.groups()
        if name != kernel:
            continue
        # The sources the kernel is compiled from (comma-separated), hashed
        # together in the order given.
        h = hashlib.sha256()
        try:
            for f in src.split(","):
                h.update(open(os.path.join(ROOT, f), "rb").read())
        except OSError:
            return None, None
        if h.hexdigest()[:16] == sha:
            return int(nbytes), src
    return None, None


def new_key_load(fs, nslots):
    """Mean table load seen by the fill's new keys, each batch's taken at the
    batch's midpoint."""
    before, acc, tot = 0, 0.0, 0
    for f in fs.fresh_counts:
        acc += f * (before + f / 2) / nslots
        tot += f
        before += f
    return acc / max(1, tot)


def cuckoo_miss_probes(fs, table):
    """Mean slots a Cuckoo probe reads for a key absent from the table: h_1,
    and h_2..h_k only when h_1 is occupied, which for a uniform h_1 happens
    with probability equal to the table load."""
    if table is None:
        return 4.0
    info = table.info()
    return 1 + new_key_load(fs, info["slots"]) * (info["num_hashes"] - 1)


def random_access_roofline(scheme, fs, table, stats, ms_per_fill, probe):
    """Lower bound on a fill's time from the measured random-access rates:
    the lines a scheme must only read at the random-read rate plus the lines
    it must claim in at the random read-modify-write rate.  Bucket: one line
    per key, read-only for repeats, claimed for new keys.  Cuckoo: every slot
    its probes read (counted on the device, `stats`), except one per new key
    -- the slot its chain starts at, which the insert claims -- and every
    exchange its insertion chains made (counted), each a claimed line.  In-
    batch repeats that miss and the dedup set (kept in L2) are not counted,
    so the bound is optimistic and the fraction conservative."""
    if not probe or "rmw_line" not in probe:
        return None
    r_rmw = probe["rmw_line"]["gaccess_per_s"] * 1e9
    n_new = fs.n_distinct
    n_rep = fs.n_issued - fs.n_distinct
    if scheme == "bucket":
        r_read = probe["128B"]["gaccess_per_s"] * 1e9
        reads, claims = n_rep, n_new
    else:
        r_read = probe["8B"]["gaccess_per_s"] * 1e9
        if stats.get("probes"):
            reads = max(0, stats["probes"] - n_new)
        else:                       # the model: h_1, then h_2..h_k when h_1 is occupied
            info = table.info()
            reads = n_rep + n_new * new_key_load(fs, info["slots"]) * (info["num_hashes"] - 1)
        # every table atomic of the insertions: the probe's CASes into the
        # first empty slot, then the chains' exchanges
        claims = max(n_new, stats.get("probe_cas", 0) + stats["exchanges"])
    t_min = reads / r_read + claims / r_rmw
    return {"min_ms_per_fill": round(t_min * 1e3, 3), "frac": round(t_min * 1e3 / ms_per_fill, 3),
            "lines_read_per_key": round(reads / fs.n_issued, 3),
            "lines_claimed_per_key": round(claims / fs.n_issued, 3),
            "read_gaccess_per_s": round(r_read / 1e9, 2), "rmw_gaccess_per_s": round(r_rmw / 1e9, 2)}


def lower_bound_roofline(scheme, fs, ms_per_fill, probe, copy_gbs):
    """The stable lower-bound variant of a fill's algorithmic bytes per key:
    one probe unit (a 128-byte bucket, or one 32-byte Cuckoo slot sector) at
    the random-gather rate of its granularity, a 32-byte claimed sector per
    new key at the 32-byte gather rate, and the streamed key read and flag
    write (9 bytes) at the copy rate.  Independent of counted probes and
    chain lengths, so it moves only with the measured rates."""
    if not probe or "32B" not in probe or "128B" not in probe:
        return None
    p_new = fs.n_distinct / fs.n_issued
    unit, r_unit = (128, probe["128B"]["requested_gbs"]) if scheme == "bucket" else (32, probe["32B"]["requested_gbs"])
    r32 = probe["32B"]["requested_gbs"]
    s_per_key = unit / (r_unit * 1e9) + p_new * 32 / (r32 * 1e9) + 9 / (copy_gbs * 1e9)
    t_min_ms = s_per_key * fs.n_issued * 1e3
    return {"bytes_per_key": round(unit + p_new * 32 + 9, 1), "min_ms_per_fill": round(t_min_ms, 3),
            "mops_bound": round(1 / s_per_key / 1e6, 1), "frac": round(t_min_ms / ms_per_fill, 3)}


def cpu_host():
    """The host's core count and CPU model (from /proc/cpuinfo: the model
    name, or on Arm the implementer and part numbers)."""
    info = {"nproc": os.cpu_count(), "machine": os.uname().machine}
    try:
        txt = open("/proc/cpuinfo").read()
    except OSError:
        return info
    m = re.search(r"^model name\s*:\s*(.+)$", txt, re.M)
    if m:
        info["cpu"] = m.group(1).strip()
    else:
        imp = re.search(r"^CPU implementer\s*:\s*(\S+)", txt, re.M)
        part = re.search(r"^CPU part\s*:\s*(\S+)", txt, re.M)
        if imp and part:
            known = {("0x41", "0xd4f"): "Arm Neoverse-V2"}
            info["cpu"] = known.get((imp.group(1), part.group(1)), "implementer %s part %s" % (imp.group(1), part.group(1)))
    return info


def kernel_random_access(name, k, fs, tables, stats, probe, steps):
    """The dominant kernel against the measured random-access rates: its
    minimum time per launch (lines it must read at the random-read rate +
    lines it must claim in at the random-claim rate, as in
    random_access_roofline) over its measured average launch time."""
    r_read = probe["128B" if name == "bucket_find_or_put" else "8B"]["gaccess_per_s"] * 1e9
    r_rmw = probe["rmw_line"]["gaccess_per_s"] * 1e9
    n_new, n_rep = fs.n_distinct, fs.n_issued - fs.n_distinct
    if name == "bucket_find_or_put":
        reads, claims = n_rep, n_new
    elif name == "cuckoo_probe":
        if stats["cuckoo"].get("probes"):
            reads = stats["cuckoo"]["probes"]          # every slot the probes read, counted
        else:
            info = tables["cuckoo"].info()
            reads = n_rep + n_new * (1 + new_key_load(fs, info["slots"]) * (info["num_hashes"] - 1))
        claims = stats["cuckoo"].get("probe_cas", 0)
    elif name == "cuckoo_insert":
        reads, claims = 0, stats["cuckoo"]["exchanges"]
    else:
        return None
    per_launch_s = (reads / r_read + claims / r_rmw) * steps / k["launches"]
    return {"frac": round(per_launch_s / (k["avg_ms"] / 1e3), 3),
            "lines_read_per_launch": int(reads * steps / k["launches"]),
            "lines_claimed_per_launch": int(claims * steps / k["launches"]),
            "read_gaccess_per_s": round(r_read / 1e9, 2), "rmw_gaccess_per_s": round(r_rmw / 1e9, 2)}


# ----------------------------------------------------------------- our arm
def run_ours(a, rank, world, local):
    import torch
    import paper_1712_09494_gb300 as ht
    from workloads import keys as wk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    schemes = [s for s in a.schemes.split(",") if s]
    n = 1 << a.n_log2
    B = 1 << a.batch_log2
    fs = wk.fill_stream(n, B, a.dup, 64, seed=a.seed + rank)
    keys_h = torch.from_numpy(fs.keys.view(np.int64))
    keys_d = keys_h.to(dev)
    offs = fs.offsets.tolist()
    is_new_d = torch.empty(B, dtype=torch.uint8, device=dev)
    cap = int(np.ceil(n / a.lf))
    tables = {s: ht.HashTable(cap, s, 64) for s in schemes}
    stream = torch.cuda.current_stream(dev)
    n_ops = fs.n_issued * len(schemes)

    def fill(t, last=None):
        ht.ht_clear(t.handle)
        for b in range(fs.n_batches):
            if last is not None and b == fs.n_batches - 1:
                last[0].record(stream)
            ht.ht_find_or_put(t.handle, keys_d[offs[b]:offs[b + 1]], is_new_d[:offs[b + 1] - offs[b]])
        if last is not None:
            last[1].record(stream)

    ev = {s: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for s in schemes}
    per_ms = {s: 0.0 for s in schemes}
    for _ in range(a.warmup):
        for s in schemes:
            fill(tables[s])
    torch.cuda.synchronize()
    for s in schemes:
        rc = tables[s].sync()
        if rc != 0 or tables[s].size() != n:
            raise RuntimeError("warm-up fill of %s ended with status %d, size %d" % (s, rc, tables[s].size()))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    ht.ht_prof_reset()
    ht.ht_prof_enable(True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms_each = {s: [] for s in schemes}
    last_each = {s: [] for s in schemes}        # the last batch of each fill ("at load")
    barrier()
    clocks.start()
    t0.record(stream)
    for _ in range(a.steps):
        for s in schemes:
            ev[s][0].record(stream)
            last = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            fill(tables[s], last)
            last_each[s].append(last)
            ev[s][1].record(stream)
            step_ms_each[s].append((ev[s][0], ev[s][1]))
            ev[s] = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    ht.ht_prof_enable(False)
    kern = ht.ht_prof_read()
    ms_total = t0.elapsed_time(t1)
    med_ms = {}
    for s in schemes:
        each = [e0.elapsed_time(e1) for e0, e1 in step_ms_each[s]]
        per_ms[s] = sum(each) / a.steps
        med_ms[s] = statistics.median(each)
    ms_step = reduce_max(ms_total / a.steps, dev)
    for s in schemes:
        if tables[s].sync() != 0 or tables[s].size() != n:
            raise RuntimeError("timed fill of %s did not end exact" % s)
    fill_stats = {s: tables[s].stats() for s in schemes}      # of the last timed fill
    value = whole_job_mops(n_ops, world, ms_step)

    # Roofline of the dominant kernel: algorithmic bytes per launch / event time.
    p_new = fs.n_distinct / fs.n_issued
    miss_probes = cuckoo_miss_probes(fs, tables.get("cuckoo"))
    # Slots a Cuckoo probe reads per key: counted on the device over the last
    # timed fill when available, else the model (one h_1 read per repeat,
    # 1 + a(k-1) per new key).
    probes_model = (1 - p_new) * 1 + p_new * miss_probes
    probes_counted = (fill_stats["cuckoo"]["probes"] / fs.n_issued
                      if "cuckoo" in fill_stats and fill_stats["cuckoo"].get("probes") else None)
    probes_per_key = probes_counted if probes_counted is not None else probes_model
    cuckoo_exchanges_per_new = (fill_stats["cuckoo"]["exchanges"] / fs.n_distinct) if "cuckoo" in fill_stats else 1.0
    # The probe's CASes of absent keys into the first empty slot they saw
    # (an insertion's first step, taken in the probe kernel).
    cuckoo_cas_per_key = (fill_stats["cuckoo"].get("probe_cas", 0) / fs.n_issued) if "cuckoo" in fill_stats else 0.0
    # Algorithmic bytes per unit, as the method defines them (the per-unit
    # figures of the hot-path measurement plan): a Cuckoo hit moves the
    # sectors of the slots up to the one holding the key (E_hit, counted); a
    # miss the sectors of all k slots, whatever this kernel's early exit
    # saves; an insertion one 32-byte sector of read-modify-write per
    # exchange (counted), its first step a CAS in the probe kernel unless all
    # k slots were full, plus its record.  A bucket key moves one 128-byte bucket and,
    # when new, the claimed sector.  Every unit adds its 8-byte key and its
    # 1-byte flag.
    cs = fill_stats.get("cuckoo", {})
    k_cuckoo = tables["cuckoo"].info()["num_hashes"] if "cuckoo" in tables else 4
    miss_reads = cs.get("probe_miss_reads", 0)
    n_miss = cs.get("probe_misses", 0)
    if cs.get("probes") and n_miss:
        probe_slots_method = (cs["probes"] - miss_reads + n_miss * k_cuckoo) / fs.n_issued
    else:
        probe_slots_method = probes_per_key
    per_key = {
        "bucket_find_or_put": 8 + 1 + 128 + p_new * 32,
        "cuckoo_probe": 8 + 1 + probe_slots_method * 32 + cuckoo_cas_per_key * 32 + p_new * 16,
        "cuckoo_insert": 16 + 32 * cuckoo_exchanges_per_new,
    }
    # The same with the work this implementation does: the slots its probes
    # actually read (counted), and a sector read and written per exchange.
    per_key_done = dict(per_key)
    per_key_done["cuckoo_probe"] = 8 + 1 + probes_per_key * 32 + cuckoo_cas_per_key * 64 + p_new * 16
    per_key_done["cuckoo_insert"] = 16 + 64 * cuckoo_exchanges_per_new
    # units over the timed region; divided by each kernel's launch count below
    units_total = {"bucket_find_or_put": fs.n_issued * a.steps,
                   "cuckoo_probe": fs.n_issued * a.steps,
                   "cuckoo_insert": fs.n_distinct * a.steps}
    peak, peak_src = measured_peaks()
    kernels = {}
    for name, (launches, tot) in kern.items():
        entry = {"launches": launches, "total_ms": round(tot, 3), "avg_ms": round(tot / launches, 4)}
        if name in per_key:
            alg = per_key[name] * units_total[name] / launches
            entry["alg_bytes_per_launch"] = int(alg)
            entry["achieved_gbs"] = round(alg / (tot / launches / 1e3) / 1e9, 1)
            entry["frac_of_" + peak_src] = round(entry["achieved_gbs"] / peak, 3)
            done = per_key_done[name] * units_total[name] / launches
            entry["frac_of_" + peak_src + "_work_done"] = round(done / (tot / launches / 1e3) / 1e9 / peak, 3)
        kernels[name] = entry
    dom = max((k for k in kernels if k in per_key), key=lambda k: kernels[k]["total_ms"])
    traffic, _ = recorded_traffic(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["achieved_gbs"], "peak": peak,
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, copy burst)" if peak_src == "measured"
                else "fallback 6.8 TB/s",
                "unit": "GB/s", "frac": round(kernels[dom]["achieved_gbs"] / peak, 3),
                "frac_of_nominal_7900": round(kernels[dom]["achieved_gbs"] / 7900.0, 3),
                "traffic": traffic, "alg_bytes_per_key": round(per_key[dom], 1),
                "alg_bytes": "the method's per-unit figures: Cuckoo hit E_hit x 32 B, miss k x 32 B, "
                             "32 B per insertion CAS (probe) or exchange (insert); bucket one 128-byte bucket + "
                             "32 B per new key; + key and flag",
                "frac_work_done": kernels[dom].get("frac_of_" + peak_src + "_work_done"),
                "alg_bytes_per_key_work_done": round(per_key_done[dom], 1),
                "cuckoo_slots_per_key_method": round(probe_slots_method, 3),
                "cuckoo_probes_per_key": round(probes_per_key, 3), "cuckoo_probes_per_key_model": round(probes_model, 3),
                "cuckoo_probes_counted": probes_counted is not None,
                "cuckoo_exchanges_per_new_key": round(cuckoo_exchanges_per_new, 3),
                "cuckoo_probe_cas_per_new_key": round(cuckoo_cas_per_key * fs.n_issued / fs.n_distinct, 3)}

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "Mops/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(a, schemes),
        "per_scheme": {s: {"ms_per_fill": round(per_ms[s], 3), "median_ms_per_fill": round(med_ms[s], 3),
                           "mops": round(fs.n_issued / (per_ms[s] / 1e3) / 1e6, 1),
                           "at_load_mops": round((offs[-1] - offs[-2]) / (statistics.median(
                               [e0.elapsed_time(e1) for e0, e1 in last_each[s]]) / 1e3) / 1e6, 1)}
                       for s in schemes},
        "roofline": roofline, "kernels": kernels, "clocks": clk,
        "gpu_launches": int(sum(v[0] for v in kern.values())),
    }

    # End to end through the C ABI from pinned host buffers.
    if not a.no_e2e:
        out["e2e"] = run_e2e(a, ht, torch, dev, fs, tables, schemes, world)
    if not a.no_probe and rank == 0:
        out["random_read_roofline"] = run_probe(ht, torch, dev)
        for s in schemes:
            out["per_scheme"][s]["random_access_roofline"] = random_access_roofline(
                s, fs, tables[s], fill_stats[s], per_ms[s], out["random_read_roofline"])
            out["per_scheme"][s]["lower_bound_roofline"] = lower_bound_roofline(
                s, fs, per_ms[s], out["random_read_roofline"], peak)
        out["roofline"]["random_access"] = kernel_random_access(
            dom, kernels[dom], fs, tables, fill_stats, out["random_read_roofline"], a.steps)
    for t in tables.values():
        t.close()
    tables = {}
    only = {x for x in a.only.split(",") if x}

    def want(section, off):
        return section_wanted(only, section, off)

    if want("small", a.no_small):
        out["small_map_config1"] = run_small_map(ht, torch, dev, schemes)
        out["many_tables_one_call"] = run_multi_table(ht, torch, dev)
    if want("sweep", a.no_sweep):
        out["sweep_config2"] = run_sweep(ht, torch, dev)
    if want("replay", a.no_sweep):
        out["replay_multiplicity"] = run_replay(ht, torch, dev)
    if want("wide", a.no_sweep):
        out["wide_keys_128"] = run_wide(ht, torch, dev)
    if want("long", a.no_sweep):
        out["long_keys_256_512"] = run_long(ht, torch, dev)
    if want("wide_bfs", a.no_sweep):
        out["wide_bfs_80bit"] = run_wide_bfs(ht, torch, dev)
    if want("bfs", a.no_bfs):
        out["bfs_config3"] = run_bfs(ht, torch, dev, schemes)
    if want("batched", a.no_batched):
        out["batched_config4"] = run_batched(ht, torch)
    if want("serving", a.no_serving):
        out["serving_config5"] = run_serving(ht, a)
    for t in tables.values():
        t.close()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return out


def run_e2e(a, ht, torch, dev, fs, tables, schemes, world, nbuf=3):
    """Same step through the public API with the keys in pinned host memory
    and the is_new flags returned to pinned host memory, every copy inside
    the timed region.  Copies overlap the kernels as a user would arrange
    it: keys are copied in on one stream up to nbuf - 1 batches ahead of the
    find-or-put calls and flags copied out on another, through nbuf device
    buffers used round robin across batches, fills and steps (events guard
    their reuse), so the copy of a fill's first batch overlaps the previous
    fill's last kernels.  Reported beside the rate: the host link's measured
    rate, the time the find-or-put calls kept the device busy, and the rest
    of the step (copies or gaps the kernels waited on)."""
    B = 1 << a.batch_log2
    keys_h = torch.from_numpy(fs.keys.view(np.int64)).pin_memory()
    out_h = torch.empty(fs.n_issued, dtype=torch.uint8).pin_memory()
    kbuf = [torch.empty(B, dtype=torch.int64, device=dev) for _ in range(nbuf)]
    fbuf = [torch.empty(B, dtype=torch.uint8, device=dev) for _ in range(nbuf)]
    offs = fs.offsets.tolist()
    comp = torch.cuda.current_stream(dev)
    h2d = torch.cuda.Stream(dev)
    d2h = torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()
    k_free = [ev() for _ in range(nbuf)]     # kernel done reading kbuf[i]
    f_free = [ev() for _ in range(nbuf)]     # copy-out done reading fbuf[i]
    k_full = [ev() for _ in range(nbuf)]
    f_full = [ev() for _ in range(nbuf)]
    for i in range(nbuf):
        k_free[i].record(comp)
        f_free[i].record(comp)
    seq = [0]                                # batches issued so far (round-robin buffer index)
    busy = []                                # (start, end) events around each find-or-put call

    def step(record=False):
        for s in schemes:
            t = tables[s]
            ht.ht_clear(t.handle)
            for b in range(fs.n_batches):
                i = seq[0] % nbuf
                seq[0] += 1
                m = offs[b + 1] - offs[b]
                h2d.wait_event(k_free[i])
                with torch.cuda.stream(h2d):
                    kbuf[i][:m].copy_(keys_h[offs[b]:offs[b + 1]], non_blocking=True)
                k_full[i].record(h2d)
                comp.wait_event(k_full[i])
                comp.wait_event(f_free[i])
                if record:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(comp)
                ht.ht_find_or_put(t.handle, kbuf[i][:m], fbuf[i][:m], stream=comp)
                if record:
                    e1.record(comp)
                    busy.append((e0, e1))
                k_free[i].record(comp)
                f_full[i].record(comp)
                d2h.wait_event(f_full[i])
                with torch.cuda.stream(d2h):
                    out_h[offs[b]:offs[b + 1]].copy_(fbuf[i][:m], non_blocking=True)
                f_free[i].record(d2h)
        # the step ends when the last flags are on the host
        comp.wait_stream(d2h)

    for _ in range(max(1, a.warmup)):
        step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(comp)
    for _ in range(a.steps):
        step(record=True)
    t1.record(comp)
    torch.cuda.synchronize()
    ms = reduce_max(t0.elapsed_time(t1) / a.steps, dev)
    busy_ms = sum(e0.elapsed_time(e1) for e0, e1 in busy) / a.steps
    # the last step's flags must count exactly the distinct keys
    if int(out_h.sum()) != fs.n_distinct:
        raise RuntimeError("e2e flags do not count the distinct keys")
    for t in tables.values():
        if t.sync() != 0:
            raise RuntimeError("e2e fill did not end exact")
    # The host link's own rate: pinned host -> device copies of one batch of
    # keys into a device buffer, timed alone on one stream (best of five);
    # the step cannot beat its bytes at this rate.  Then every batch of the
    # stream copied alone once: the whole buffer's rate, which shows pages
    # of the pinned buffer that copy slower than the first batch's.
    m = offs[1] - offs[0]
    rates = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(comp)
        kbuf[0][:m].copy_(keys_h[:m], non_blocking=True)
        e1.record(comp)
        torch.cuda.synchronize()
        rates.append(m * 8 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    h2d_gbs = max(rates)
    per_batch = []
    for b in range(fs.n_batches):
        mb = offs[b + 1] - offs[b]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(comp)
        kbuf[0][:mb].copy_(keys_h[offs[b]:offs[b + 1]], non_blocking=True)
        e1.record(comp)
        torch.cuda.synchronize()
        per_batch.append(mb * 8 / (e0.elapsed_time(e1) / 1e3) / 1e9)
    all_ms = sum((offs[b + 1] - offs[b]) * 8 / (r * 1e9) for b, r in enumerate(per_batch)) * 1e3
    h2d_bytes = fs.n_issued * 8 * len(schemes)
    return {"value": round(fs.n_issued * len(schemes) * world / (ms / 1e3) / 1e6, 1), "unit": "Mops/s",
            "ms_per_step": round(ms, 3), "h2d_bytes_per_step": int(h2d_bytes),
            "d2h_bytes_per_step": int(fs.n_issued * len(schemes)),
            "overlap": "3 streams (copy-in, kernels, copy-out), %d device buffers round robin" % nbuf,
            "h2d_gbs_measured": round(h2d_gbs, 1),
            "link_bound_ms_per_step": round(h2d_bytes / (h2d_gbs * 1e9) * 1e3, 2),
            "h2d_gbs_every_batch_min_median": [round(min(per_batch), 1), round(statistics.median(per_batch), 1)],
            "link_bound_ms_per_step_every_batch": round(all_ms * len(schemes), 2),
            "find_or_put_busy_ms_per_step": round(busy_ms, 3),
            "kernel_stream_waiting_ms_per_step": round(ms - busy_ms, 3)}


def run_probe(ht, torch, dev):
    """Random-access rates over a 4 GiB buffer (>> L2), best of 5 launches:
    8-byte slot probes, 32-byte reads and 128-byte lines read by 8-lane
    groups; and random claims (8-byte atomic adds, one per random line).  On
    GB300 each random read costs a whole 128-byte line of DRAM traffic, so
    the line rate is the ceiling for both schemes' probes; a claim adds the
    write-back of the dirtied sector."""
    buf = torch.empty(1 << 29, dtype=torch.int64, device=dev)
    buf.fill_(1)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    res = {"buffer_gib": 4}

    def best_ms(launch, reps=5):
        launch(0)
        times = []
        for r in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            launch(r + 1)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return min(times)

    for gran in (8, 32, 128):
        n_acc = (1 << 33) // 128          # the same number of accesses for every size
        ms = best_ms(lambda r: ht.ht_probe_random_read(buf, gran, n_acc, 11 + r, sink))
        res["%dB" % gran] = {"gaccess_per_s": round(n_acc / (ms / 1e3) / 1e9, 2),
                             "requested_gbs": round(n_acc * gran / (ms / 1e3) / 1e9, 1),
                             "line_gbs": round(n_acc * 128 / (ms / 1e3) / 1e9, 1)}
    n_acc = (1 << 33) // 128
    ms = best_ms(lambda r: ht.ht_probe_random_rmw(buf, n_acc, 21 + r))
    res["rmw_line"] = {"gaccess_per_s": round(n_acc / (ms / 1e3) / 1e9, 2),
                       "line_read_gbs": round(n_acc * 128 / (ms / 1e3) / 1e9, 1)}
    del buf
    return res


# ----------------------------------------------------------------- other rows
def _hmodel(ht, m):
    return ht.make_model(m.C, m.bits, m.deg, m.tgt, m.lab, m.pairs)


def run_bfs(ht, torch, dev, schemes, warmup=1, reps=3):
    """Config 3: full BFS of the 12 x 32 model (~10^8 states), per scheme:
    states/s and find-or-put ops/s (successors/s); levels checked against the
    stored oracle levels."""
    from workloads import statespace as ss
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "statespace_config3.json")))
    m = ss.config3_model(seed=gold["model"]["seed"], p_sync=gold["model"]["p_sync"])
    hm = _hmodel(ht, m)
    states = torch.empty(gold["states"] + 1024, dtype=torch.int64, device=dev)
    out = {"workload": "12 components x 32 local states, 4 sync pairs, from the all-zero state: %d states, "
                       "%d levels, %d successors" % (gold["states"], len(gold["levels"]), gold["successors"])}
    forms = [(sch, False) for sch in schemes] + ([("bucket", True)] if "bucket" in schemes else [])
    for sch, fused in forms:
        t = ht.HashTable(int(gold["states"] / 0.8), sch, 64)
        times = []
        for r in range(warmup + reps):
            ht.ht_clear(t.handle)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res, sizes = ht.ht_bfs(t.handle, hm, 0, 4096, states, fused=fused)
            torch.cuda.synchronize()
            if r >= warmup:
                times.append(time.perf_counter() - t0)
        ok = (res.complete == 1 and res.states == gold["states"] and res.successors == gold["successors"]
              and sizes == [lv[0] for lv in gold["levels"]])
        sec = statistics.median(times)
        # One more run with the library's kernel timer on: where the time goes.
        ht.ht_clear(t.handle)
        torch.cuda.synchronize()
        ht.ht_prof_reset()
        ht.ht_prof_enable(True)
        ht.ht_bfs(t.handle, hm, 0, 4096, states, fused=fused)
        torch.cuda.synchronize()
        ht.ht_prof_enable(False)
        kern = {k: round(v[1], 2) for k, v in ht.ht_prof_read().items() if k != "clear"}
        out[sch + ("_fused" if fused else "")] = {"seconds": round(sec, 4), "states_per_s_M": round(res.states / sec / 1e6, 1),
                    "find_or_put_mops": round(res.successors / sec / 1e6, 1),
                    "levels_match_oracle": bool(ok), "host_syncs": len(sizes) + 2, "kernel_ms": kern,
                    "multiplicity": round(res.successors / max(1, res.states), 2)}
        t.close()
    del states
    return out


def run_batched(ht, torch):
    """Config 4: 256 explorations (6-10 components, 8-32 local states,
    2^10..2^20 states each), bucket and Cuckoo tables: the persistent launch
    (one cooperative kernel per table kind runs every level of every
    exploration), the per-step graph and per-step launches (bucket), and one
    exploration at a time (the baseline), same tables; every run's levels
    checked against the stored oracle levels.  Then the same with each
    exploration's table parameters picked by the autotuner."""
    from workloads import statespace as ss
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "statespace_batched.json")))
    models = ss.batched_models(gold["model"]["count"], seed=gold["model"]["seed"])
    caps = [max(256, int(g["states"] / 0.7)) for g in gold["explorations"]]
    tot = sum(g["successors"] for g in gold["explorations"])
    res = {"workload": "%d explorations, %d states, %d successors in total" % (
        len(models), sum(g["states"] for g in gold["explorations"]), tot)}

    def exact(mx):
        return all(mx.result(i)["states"] == g["states"] and
                   mx.result(i)["level_sizes"] == [lv[0] for lv in g["levels"]]
                   for i, g in enumerate(gold["explorations"]))

    def timed(mx, mode, reps=3):
        times, steps = [], 0
        for r in range(reps):
            mx.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps = mx.run(mode=mode)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        sec = min(times[1:])
        return {"seconds": round(sec, 4), "steps": steps, "find_or_put_mops": round(tot / sec / 1e6, 1),
                "levels_match_oracle": bool(exact(mx))}

    runs = {"bucket": ((0, "batched_persistent"), (3, "batched_graph"), (1, "batched_launches"),
                       (2, "one_table_at_a_time")),
            "cuckoo": ((0, "batched_persistent"), (2, "one_table_at_a_time"))}
    for scheme, modes in runs.items():
        mx = ht.MultiExploration([_hmodel(ht, m) for m in models], [0] * len(models), caps, schemes=scheme)
        r = {name: timed(mx, mode) for mode, name in modes}
        r["speedup_persistent_vs_per_table"] = round(r["one_table_at_a_time"]["seconds"] /
                                                     r["batched_persistent"]["seconds"], 2)
        mx.close()
        # Autotuned: each exploration's capacity class tuned once (bucket:
        # width, lanes, hash functions; Cuckoo: hash functions, eviction
        # bound) for a BFS-like repeat rate, then the persistent run.
        import tempfile
        from paper_1712_09494_gb300 import autotune
        t0 = time.perf_counter()
        with tempfile.TemporaryDirectory() as d:
            cache = os.path.join(d, "autotune.json")
            params = [autotune.tune(scheme, m.key_width, c, load=0.7, dup=0.9, cache_path=cache)
                      for m, c in zip(models, caps)]
            n_classes = len(json.load(open(cache)))
        tune_s = time.perf_counter() - t0
        mx = ht.MultiExploration([_hmodel(ht, m) for m in models], [0] * len(models), caps, params=params,
                                 schemes=scheme)
        r["batched_persistent_autotuned"] = dict(timed(mx, 0), tuning_seconds=round(tune_s, 2),
                                                 classes_tuned=n_classes,
                                                 chosen=sorted({json.dumps(p, sort_keys=True) for p in params}))
        mx.close()
        res[scheme] = r
    return res


def run_sweep(ht, torch, dev, reps=3):
    """Config 2 beyond the headline point: fills of random 64-bit keys over
    load (0.5-0.9), size (2^24-2^27), batch size (2^20-2^24) and repeat rate
    (0-0.5), for the bucket scheme and Cuckoo with k = 3 and 4 (stash 101).
    Streams are drawn on the device (workloads.device_keys).  Per point: the
    median of `reps` whole fills (keys issued / time) and the rate of the
    last batch, the one that takes the table to its load ("at load"); every
    fill must end with exactly n keys stored."""
    from workloads import device_keys as dk
    base = dict(n_log2=27, lf=0.8, batch_log2=24, dup=0.25)
    points = [dict(base, lf=lf) for lf in (0.5, 0.7, 0.8, 0.9)]
    points += [dict(base, n_log2=nl) for nl in (24, 25, 26)]
    points += [dict(base, batch_log2=bl) for bl in (20, 22)]
    points += [dict(base, dup=d) for d in (0.0, 0.5)]
    schemes = [("bucket", None), ("cuckoo", 3), ("cuckoo", 4)]
    out = []
    for pt in points:
        n = 1 << pt["n_log2"]
        batches, _ = dk.fill_batches_dev(n, 1 << pt["batch_log2"], pt["dup"], seed=11 + pt["n_log2"], device=dev)
        issued = sum(b.numel() for b in batches)
        flags = torch.empty(max(b.numel() for b in batches), dtype=torch.uint8, device=dev)
        cap = int(np.ceil(n / pt["lf"]))
        for sch, k in schemes:
            rec = dict(pt, scheme=sch if k is None else "cuckoo_k%d" % k)
            t = ht.HashTable(cap, sch, 64, None if k is None else dict(num_hashes=k))
            fills, lasts = [], []
            for r in range(reps + 1):
                ht.ht_clear(t.handle)
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record()
                for b in batches[:-1]:
                    ht.ht_find_or_put(t.handle, b, flags[:b.numel()])
                e[1].record()
                ht.ht_find_or_put(t.handle, batches[-1], flags[:batches[-1].numel()])
                e[2].record()
                torch.cuda.synchronize()
                if r:
                    fills.append(e[0].elapsed_time(e[2]))
                    lasts.append(e[1].elapsed_time(e[2]))
            st = t.sync()
            rec["exact"] = st == 0 and t.size() == n
            rec["mops"] = round(issued / (statistics.median(fills) / 1e3) / 1e6, 1)
            rec["at_load_mops"] = round(batches[-1].numel() / (statistics.median(lasts) / 1e3) / 1e6, 1)
            if st:
                rec["status"] = st
            t.close()
            out.append(rec)
        del batches, flags
        torch.cuda.empty_cache()
    return {"workload": "random 64-bit keys; one parameter varied at a time around n=2^27, load 0.8, "
                        "batches 2^24, 25% repeats; bucket 16x2/k16 and Cuckoo k=3/4 (stash 101)",
            "points": out, "all_exact": all(p["exact"] for p in out)}


def run_replay(ht, torch, dev, n=100_000_000, mults=(1, 2, 5, 10, 50, 100, 200, 450, 700, 1000), reps=2):
    """The shape of the paper's random-data experiment (Section 5.2, Fig. 5):
    sequences of 10^8 32-bit integers whose value range sets the mean
    multiplicity, each found-or-inserted as one whole sequence into a table
    of 1.25 x its distinct values (load 0.8), both schemes.  Synthetic
    stand-in for the paper's files; exact when the table ends with exactly
    the sequence's distinct values and the last timed call flagged exactly
    that many keys new (the per-key comparison with the oracle is the
    replay test's)."""
    from workloads import device_keys as dk
    flags = torch.empty(n, dtype=torch.uint8, device=dev)
    pts = []
    for m in mults:
        keys = dk.multiplicity_sequence_dev(n, m, seed=29 + m, device=dev)
        uniq = int(torch.unique(keys).numel())
        rec = {"multiplicity_range": m, "distinct": uniq, "mean_multiplicity": round(n / uniq, 2)}
        for sch in ("bucket", "cuckoo"):
            t = ht.HashTable(int(np.ceil(uniq * 1.25)), sch, 32)
            times = []
            for r in range(reps + 1):
                ht.ht_clear(t.handle)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ht.ht_find_or_put(t.handle, keys, flags)
                e1.record()
                torch.cuda.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            nflag = int(flags.sum())
            rec[sch] = {"ms": round(ms, 2), "mops": round(n / (ms / 1e3) / 1e6, 1),
                        "exact": t.sync() == 0 and t.size() == uniq and nflag == uniq}
            t.close()
        rec["cuckoo_time_over_bucket"] = round(rec["cuckoo"]["ms"] / rec["bucket"]["ms"], 2)
        pts.append(rec)
        del keys
    return {"workload": "10^8 random 32-bit keys per sequence, value range n/m for mean multiplicity ~m, "
                        "table 1.25 x distinct (load 0.8), whole sequence in one find-or-put call",
            "points": pts, "all_exact": all(p["bucket"]["exact"] and p["cuckoo"]["exact"] for p in pts)}


def run_wide(ht, torch, dev, n_log2=26, batch_log2=24, dup=0.25, lf=0.8, reps=3):
    """128-bit keys (state vectors wider than 64 bits), both schemes: a fill
    of 2^26 random keys to load 0.8 in batches of 2^24 with 25% repeats (two
    independent 63-bit streams as the words); exact when the table ends with
    exactly 2^26 keys."""
    from workloads import device_keys as dk
    n = 1 << n_log2
    batches, _ = dk.fill_batches_dev(n, 1 << batch_log2, dup, seed=91, device=dev)
    out = {"workload": "2^%d random 128-bit keys to load %.1f, batches 2^%d, %d%% repeats" % (
        n_log2, lf, batch_log2, int(dup * 100))}
    # The high word is a bijection of the low word (another seed of the same
    # permutation), so distinct low words give distinct keys and repeats repeat.
    pairs = [torch.stack([b, dk.mix63_perm_dev(b, 92)], dim=1).contiguous() for b in batches]
    issued = sum(p.shape[0] for p in pairs)
    flags = torch.empty(max(p.shape[0] for p in pairs), dtype=torch.uint8, device=dev)
    for name, sch, params in (("bucket_lanes2", "bucket", dict(lanes_per_key=2)),
                              ("bucket_lanes4", "bucket", dict(lanes_per_key=4)), ("cuckoo", "cuckoo", None)):
        t = ht.HashTable(int(np.ceil(n / lf)), sch, 128, params)
        times = []
        for r in range(reps + 1):
            ht.ht_clear(t.handle)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for p in pairs:
                ht.ht_find_or_put(t.handle, p, flags[:p.shape[0]])
            e1.record()
            torch.cuda.synchronize()
            if r:
                times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        out[name] = {"ms_per_fill": round(ms, 2), "mops": round(issued / (ms / 1e3) / 1e6, 1),
                     "exact": t.sync() == 0 and t.size() == n}
        t.close()
    return out


def run_long(ht, torch, dev, n_log2=25, batch_log2=23, dup=0.25, lf=0.8, reps=2):
    """Keys of 4 and 8 64-bit words (256 and 512 bits), both schemes: a fill of
    2^25 random keys to load 0.8 in batches of 2^23 with 25% repeats, then a
    lookup of 2^23 stored and 2^23 absent keys.  Word 0 is a 63-bit stream
    key and the others bijections of it, so distinct stream keys give
    distinct keys; exact when the table ends with exactly 2^25 keys and the
    lookups find exactly the stored half."""
    from workloads import device_keys as dk
    n = 1 << n_log2
    batches, _ = dk.fill_batches_dev(n, 1 << batch_log2, dup, seed=93, device=dev)
    issued = sum(b.numel() for b in batches)
    out = {"workload": "2^%d random keys of 4 and 8 words to load %.1f, batches 2^%d, %d%% repeats; lookups of "
                       "2^%d present + 2^%d absent" % (n_log2, lf, batch_log2, int(dup * 100), batch_log2, batch_log2)}
    q_in = batches[0][: 1 << batch_log2]
    for w in (4, 8):
        def widen(b):
            return torch.stack([b] + [dk.mix63_perm_dev(b, 95 + j) for j in range(w - 1)], dim=1).contiguous()
        rows = [widen(b) for b in batches]
        # Absent keys: stored keys with the last word's low bit flipped (a
        # stored key's last word is fixed by its first).
        absent = widen(q_in)
        absent[:, w - 1] ^= 1
        q = torch.cat([widen(q_in), absent])
        flags = torch.empty(max(r.shape[0] for r in rows), dtype=torch.uint8, device=dev)
        found = torch.empty(q.shape[0], dtype=torch.uint8, device=dev)
        for sch in ("bucket", "cuckoo"):
            t = ht.HashTable(int(np.ceil(n / lf)), sch, 64 * w)
            times, ltimes = [], []
            for r in range(reps + 1):
                ht.ht_clear(t.handle)
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record()
                for b in rows:
                    ht.ht_find_or_put(t.handle, b, flags[:b.shape[0]])
                e1.record()
                ht.ht_lookup(t.handle, q, None, found)
                e2.record()
                torch.cuda.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
                    ltimes.append(e1.elapsed_time(e2))
            ms, lms = statistics.median(times), statistics.median(ltimes)
            half = q.shape[0] // 2
            exact = (t.sync() == 0 and t.size() == n and bool(found[:half].all()) and not bool(found[half:].any()))
            out["w%d_%s" % (w, sch)] = {"key_bits": 64 * w, "ms_per_fill": round(ms, 2),
                                        "mops": round(issued / (ms / 1e3) / 1e6, 1),
                                        "lookup_mops": round(q.shape[0] / (lms / 1e3) / 1e6, 1), "exact": exact}
            t.close()
        del rows, q
    return out


def run_wide_bfs(ht, torch, dev, reps=2):
    """BFS over 80-bit state vectors (16 components x 32 local states, windows
    of 3, no synchronisation: 3^16 = 43 M states) in a 128-bit bucket table.
    Without synchronisation the level sizes have a closed form -- the
    convolution of the components' BFS-distance histograms -- which checks
    the run exactly."""
    from collections import deque
    from workloads import statespace as ss
    R = [3] * 16
    m = ss.random_model(47, C=16, L=32, R=R, p_sync=0.0, P=0)
    poly = np.array([1], dtype=np.int64)
    for c in range(m.C):
        dist = {0: 0}
        q = deque([0])
        while q:
            u = q.popleft()
            for j in range(int(m.deg[c, u])):
                v = int(m.tgt[c, u, j])
                if v not in dist:
                    dist[v] = dist[u] + 1
                    q.append(v)
        poly = np.convolve(poly, np.bincount(list(dist.values())))
    total = int(np.prod(R))
    hm = _hmodel(ht, m)
    states = torch.empty((total + 1024, 2), dtype=torch.int64, device=dev)
    t = ht.HashTable(int(total / 0.8), "bucket", 128)
    times = []
    for r in range(reps + 1):
        ht.ht_clear(t.handle)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, sizes = ht.ht_bfs(t.handle, hm, 0, 4096, states)
        torch.cuda.synchronize()
        if r:
            times.append(time.perf_counter() - t0)
    sec = statistics.median(times)
    ok = res.complete == 1 and res.states == total and sizes == poly.tolist() and t.size() == total
    t.close()
    del states
    return {"workload": "16 components x 32 local states (80-bit vectors), windows of 3, no sync: %d states, "
                        "%d levels, %d successors" % (total, len(sizes), res.successors),
            "seconds": round(sec, 4), "states_per_s_M": round(total / sec / 1e6, 1),
            "find_or_put_mops": round(res.successors / sec / 1e6, 1), "levels_match_closed_form": bool(ok)}


def run_multi_table(ht, torch, dev, n_tables=1024, keys_per=4096, rounds=8):
    """Many small tables: every round gives each of 1024 bucket tables (2^16
    slots) 4096 keys (25% repeats of its earlier keys); one
    ht_multi_find_or_put call per round against one ht_find_or_put per table.
    Results are checked equal (per table, the stored-key counts)."""
    from workloads import keys as wk
    rng = np.random.default_rng(17)
    fresh_per = keys_per * 3 // 4
    batches = []
    for r in range(rounds):
        per = []
        for t in range(n_tables):
            k = wk.distinct_keys(keys_per, 64, seed=2000 + t, start=r * fresh_per)
            if r:
                k[fresh_per:] = wk.distinct_keys(r * fresh_per, 64, seed=2000 + t)[
                    rng.integers(0, r * fresh_per, size=keys_per - fresh_per)]
            per.append(k)
        batches.append(torch.from_numpy(np.stack(per).view(np.int64)).to(dev))
    flags = torch.empty(n_tables, keys_per, dtype=torch.uint8, device=dev)
    out = {"workload": "%d bucket tables of 2^16 slots, %d rounds of %d keys per table (25%% repeats)" % (
        n_tables, rounds, keys_per)}
    sizes = {}
    for mode in ("packed", "per_table"):
        tabs = [ht.HashTable(1 << 16, "bucket", 64) for _ in range(n_tables)]
        handles = [t.handle for t in tabs]

        def run():
            for b in batches:
                if mode == "packed":
                    ht.ht_multi_find_or_put(handles, [(i, b[i], flags[i]) for i in range(n_tables)])
                else:
                    for i in range(n_tables):
                        ht.ht_find_or_put(handles[i], b[i], flags[i])

        run()                                            # warm-up (and exactness check below)
        torch.cuda.synchronize()
        for t in tabs:
            t.clear()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run()
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        sizes[mode] = [t.size() for t in tabs]
        out[mode] = {"seconds": round(sec, 4), "mops": round(n_tables * keys_per * rounds / sec / 1e6, 1)}
        for t in tabs:
            t.close()
    out["exact"] = sizes["packed"] == sizes["per_table"] == [fresh_per * rounds] * n_tables
    out["speedup_packed_vs_per_table"] = round(out["per_table"]["seconds"] / out["packed"]["seconds"], 2)
    return out


def run_small_map(ht, torch, dev, schemes, reps=10):
    """Config 1: 2^20 distinct random 32-bit keys with 32-bit values into a
    map of 2^21 slots (16 MB, load 0.5, L2-sized), then a lookup of 2^20 keys
    (half present); with and without the L2 persisting window."""
    from workloads import keys as wk
    n = 1 << 20
    keys = torch.from_numpy(wk.distinct_keys(n, 32, seed=1).view(np.int32)).to(dev)
    vals = torch.arange(n, dtype=torch.int32, device=dev)
    q, present = wk.lookup_batch(n, n, 32, seed=1)
    qd = torch.from_numpy(q.view(np.int32)).to(dev)
    found = torch.empty(n, dtype=torch.uint8, device=dev)
    out_v = torch.empty(n, dtype=torch.int32, device=dev)
    res = {"workload": "2^20 random 32-bit keys + values into 2^21 slots (16 MB), then 2^20 lookups, 50% present"}
    for sch in schemes:
        for persist in (0, 1):
            t = ht.HashTable(1 << 21, sch, 32, dict(l2_persist=persist))
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ins, look = [], []
            for r in range(reps + 2):
                ht.ht_clear(t.handle)
                e[0].record()
                ht.ht_insert(t.handle, keys, vals)
                e[1].record()
                ht.ht_lookup(t.handle, qd, out_v, found)
                e[2].record()
                torch.cuda.synchronize()
                if r >= 2:
                    ins.append(e[0].elapsed_time(e[1]))
                    look.append(e[1].elapsed_time(e[2]))
            ok = bool(np.array_equal(found.cpu().numpy(), present)) and t.size() == n
            res["%s_l2persist%d" % (sch, persist)] = {
                "insert_mops": round(n / (statistics.median(ins) / 1e3) / 1e6, 1),
                "lookup_mops": round(n / (statistics.median(look) / 1e3) / 1e6, 1), "exact": ok}
            t.close()
    # The table fits in L2, so its bound is L2's random-access rate, not HBM's:
    # the same random-read probe over a 16 MB buffer.
    buf = torch.ones(1 << 21, dtype=torch.int64, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    l2 = {}
    for gran in (8, 128):
        n_acc = 1 << 28
        ht.ht_probe_random_read(buf, gran, n_acc, 3, sink)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ht.ht_probe_random_read(buf, gran, n_acc, 4, sink)
        e1.record()
        torch.cuda.synchronize()
        l2["%dB_gaccess_per_s" % gran] = round(n_acc / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    res["l2_random_read"] = dict(l2, bound="L2: the 16 MB table fits the L2 cache, HBM roofline not binding")
    return res


def serving_trace(n_req, rate, seed=5, n_tables=1024):
    """Poisson arrivals of find-or-put batches over up to 1024 tables of
    2^12..2^30 slots (log-uniform); batch sizes log-uniform in 1..2^20; each
    table lives for a contiguous session of the trace (opened before its
    first request, closed after its last), so admission by free memory
    matters; keys are random 64-bit with repeats of the table's earlier keys
    (serving_keys), never more distinct keys than 0.8 of a table's slots."""
    rng = np.random.default_rng(seed)
    caps = np.exp2(rng.uniform(12, 30, size=n_tables)).astype(np.int64)
    pos = np.sort(rng.uniform(0, n_tables, size=n_req))
    table = np.minimum(n_tables - 1, (pos + rng.uniform(-8, 8, size=n_req)).clip(0)).astype(np.int64)
    sizes = np.exp(rng.uniform(0, np.log(2 ** 20), size=n_req)).astype(np.int64).clip(1, 2 ** 20)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    return caps, table, sizes, arrivals


def serving_keys(trace, load=0.8, seed=6):
    """Per request: a quarter repeats of its table's earlier keys (once it has
    some), the rest fresh keys of the table -- until the table holds `load` x
    its capacity distinct keys; from then on the request's other keys are
    repeats too, so no table is filled past that load."""
    from workloads import keys as wk
    rng = np.random.default_rng(seed)
    caps, table, sizes, arrivals = trace
    issued, keys = {}, []
    for i in range(len(sizes)):
        t, n = int(table[i]), int(sizes[i])
        base = issued.get(t, 0)
        room = max(0, int(load * caps[t]) - base)
        fresh = min(n - (min(n // 4, base)), room)
        if base + fresh == 0:
            fresh = 1                                   # a table's first key
        rep = n - fresh
        k = np.empty(n, dtype=np.uint64)
        k[:fresh] = wk.distinct_keys(fresh, 64, seed=1000 + t, start=base)
        if rep:
            idx = rng.integers(0, base + fresh, size=rep).astype(np.uint64)
            k[fresh:] = wk.mix63_perm(idx, 1000 + t)
        issued[t] = base + fresh
        keys.append(k[rng.permutation(n)])
    return keys


def run_serving_once(ht, a, pack, inflight, trace, keys, schemes=None):
    import threading
    caps, table, sizes, arrivals = trace
    n_req = len(sizes)
    srv = ht.Server(pack=pack, max_inflight=inflight, batch_key_budget=1 << 22,
                    hbm_reserve_bytes=8 << 30)
    last = {}
    for i, t in enumerate(table):
        last[int(t)] = i
    tid = {}
    rids = [None] * n_req
    done_lat = [None] * n_req
    errors = []

    deadline = time.perf_counter() + a.serve_deadline

    def completer():
        for i in range(n_req):
            while rids[i] is None:
                time.sleep(0.0001)
            left_ms = max(1, int((deadline - time.perf_counter()) * 1000))
            st, lat, _ = srv.wait(rids[i], timeout_ms=left_ms)
            if st != 0:
                errors.append(st)
                if st == 5:                       # deadline passed: stop waiting
                    break
            done_lat[i] = lat
            t = int(table[i])
            if last[t] == i:
                srv.close_table(tid[t])

    th = threading.Thread(target=completer)
    th.start()
    t0 = time.perf_counter()
    for i in range(n_req):
        t = int(table[i])
        if t not in tid:
            tid[t] = srv.open_table(int(caps[t]), schemes[t] if schemes is not None else "bucket")
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        rids[i] = srv.submit(tid[t], keys[i])
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    if errors:
        srv.close()
        return {"error": "%d requests failed or missed the %.0f s deadline (first status %d)" % (
            len(errors), a.serve_deadline, errors[0])}
    srv.close()
    lat = np.array(done_lat)
    # Where the wall time goes: the worker thread's own work (admission --
    # allocating tables and launching their clears --, packing keys into
    # staging, finishing -- results out), and the time with at least one
    # batch in flight on the device.  The worker's host work and the
    # in-flight time are each a share of the wall; the device-side work
    # behind them is estimated from the bytes moved at measured rates
    # (table clears at the copy peak, keys over the host link).
    shares = {"worker_admission": st["admit_seconds"] / wall, "worker_packing": st["pack_seconds"] / wall,
              "worker_finishing": st["finish_seconds"] / wall,
              "batch_in_flight": st["inflight_seconds"] / wall}
    worker = (st["admit_seconds"] + st["pack_seconds"] + st["finish_seconds"]) / wall
    return {"p50_us": round(float(np.percentile(lat, 50)), 1), "p99_us": round(float(np.percentile(lat, 99)), 1),
            "mean_us": round(float(lat.mean()), 1), "sustained_mops": round(float(sizes.sum()) / wall / 1e6, 1),
            "wall_s": round(wall, 3), "batches": int(st["batches"]), "errors": len(errors),
            "worker": {"admit_s": round(st["admit_seconds"], 3), "pack_s": round(st["pack_seconds"], 3),
                       "finish_s": round(st["finish_seconds"], 3), "batch_us_mean": round(st["batch_us_mean"], 1),
                       "batch_gpu_us_mean": round(st["batch_gpu_us_mean"], 1),
                       "tables_created": int(st["tables_created"]),
                       "table_gb_cleared": round(st["table_bytes_created"] / 1e9, 1),
                       "clear_ms_at_copy_peak": round(st["table_bytes_created"] / (measured_peaks()[0] * 1e9) * 1e3, 1),
                       "share_of_wall": {k: round(v, 3) for k, v in shares.items()},
                       "worker_busy_share": round(worker, 3),
                       "limiter": "worker thread (host)" if worker > shares["batch_in_flight"] else "device batches"}}


def run_serving(ht, a):
    trace = serving_trace(a.serve_requests, a.serve_rate)
    caps, table, sizes, arrivals = trace
    out = {"workload": "%d requests over %d tables (2^12..2^30 slots, sessions), batch 1..2^20 keys log-uniform "
                       "(mean %d), Poisson %.0f req/s offered" % (len(sizes), len(set(table.tolist())),
                                                                  int(sizes.mean()), a.serve_rate)}
    import torch
    # Request keys live in page-locked host memory, as a serving front end
    # that receives them into pinned buffers would hold them.
    pinned = [torch.from_numpy(k.view(np.int64)).pin_memory() for k in serving_keys(trace)]
    keys = [p.numpy().view(np.uint64) for p in pinned]
    out["continuous_batching"] = run_serving_once(ht, a, pack=1, inflight=4, trace=trace, keys=keys)
    # Packing alone: the same four batch slots in flight, one launch per request.
    out["per_request_launches_inflight4"] = run_serving_once(ht, a, pack=0, inflight=4, trace=trace, keys=keys)
    out["per_request_launches"] = run_serving_once(ht, a, pack=0, inflight=1, trace=trace, keys=keys)
    out["packing_speedup_at_inflight4"] = round(
        out["continuous_batching"].get("sustained_mops", 0) /
        max(1e-9, out["per_request_launches_inflight4"].get("sustained_mops", 0)), 2)
    # Cuckoo tables in the same trace: every other table is a Cuckoo table
    # (its requests run the probe / insert kernels; bucket tables share the
    # packed kernel).
    mixed = ["cuckoo" if t % 2 else "bucket" for t in range(len(caps))]
    out["continuous_batching_mixed_schemes"] = run_serving_once(ht, a, pack=1, inflight=4, trace=trace, keys=keys,
                                                                schemes=mixed)
    out["per_request_launches_mixed_schemes"] = run_serving_once(ht, a, pack=0, inflight=4, trace=trace, keys=keys,
                                                                 schemes=mixed)
    # Offered rate swept towards saturation (continuous batching; the same
    # requests, only the arrival times change).
    sweep = []
    for rate in (10000.0, 160000.0, 640000.0):
        tr = serving_trace(a.serve_requests, rate)
        r = run_serving_once(ht, a, pack=1, inflight=4, trace=tr, keys=keys)
        sweep.append({"offered_req_per_s": rate, "p50_us": r.get("p50_us"), "p99_us": r.get("p99_us"),
                      "sustained_mops": r.get("sustained_mops"), "errors": r.get("errors", r.get("error"))})
    out["continuous_batching_rate_sweep"] = sweep
    return out


# ----------------------------------------------------------------- CPU legs
def run_cpu_oracle(a, sample_batches=4):
    """The oracle (single-threaded std::unordered_map) on the first batches of
    the same stream; returns (Mops/s, description)."""
    import oracle
    from workloads import keys as wk
    n = 1 << a.n_log2
    B = 1 << a.batch_log2
    per_batch_fresh = max(1, int(round(B * (1.0 - a.dup))))
    total_batches = -(-n // per_batch_fresh)
    fs = wk.fill_stream(n, B, a.dup, 64, seed=a.seed, max_batches=sample_batches)
    nb = fs.n_batches
    keys = fs.keys[:fs.offsets[nb]]
    t = oracle.OracleTable(reserve=n)
    t0 = time.perf_counter()
    t.find_or_put(keys)
    dt = time.perf_counter() - t0
    return len(keys) / dt / 1e6, "first %d of %d batches of the stream (%d keys, one scheme-free set)" % (
        nb, total_batches, len(keys))


def run_reference(a, rank, world):
    if rank != 0:
        return None
    schemes = [s for s in a.schemes.split(",") if s]
    vals = []
    desc = None
    for _ in range(a.warmup):
        run_cpu_oracle(a, sample_batches=1)
    t_start = time.perf_counter()
    for _ in range(a.steps):
        v, desc = run_cpu_oracle(a, sample_batches=1)
        vals.append(v)
    wall = time.perf_counter() - t_start
    v = statistics.median(vals)
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": "Mops/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(wall / a.steps * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": workload_config(a, schemes),
        "cpu_baseline": {"value": round(v, 2), "unit": "Mops/s", "cores": 1, "kind": "oracle", "sample": desc,
                         "host": cpu_host()},
        "e2e": {"value": round(v, 2), "unit": "Mops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    a = parse()
    rank, world, local = dist_env()
    if a.impl == "reference":
        out = run_reference(a, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out = run_ours(a, rank, world, local)
    if rank == 0:
        if not a.no_cpu and world == 1:
            v, desc = run_cpu_oracle(a)
            out["cpu_baseline"] = {"value": round(v, 2), "unit": "Mops/s", "cores": 1, "kind": "oracle",
                                   "sample": desc, "host": cpu_host()}
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
