"""Autotuner for the table parameters: bucket width, lanes per key, number of
hash functions (bucket scheme); hash functions and eviction bound (Cuckoo).

For a workload class -- scheme, key width, capacity (rounded to a power of
two), target load and repeat rate -- it fills a table of that class with
synthetic keys under every candidate parameter set, keeps only candidates
whose fill is exact (every key new to the table flagged exactly once in its
batch, no other key flagged, every distinct key stored), and caches the fastest
in a JSON file keyed by device name and class.  The timing runs the library's
own kernels; only the bookkeeping is Python.
"""
import json
import math
import os

CANDIDATES = {
    "bucket": [dict(bucket_slots=bs, lanes_per_key=g, num_hashes=k)
               for (bs, g) in [(8, 2), (8, 4), (16, 2), (16, 4), (16, 8), (32, 4), (32, 8)]
               for k in (8, 16)],
    "cuckoo": [dict(num_hashes=k, max_evictions=e) for k in (3, 4, 5) for e in (64, 256, 1024)],
}


def default_cache_path():
    root = os.environ.get("HT_AUTOTUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                                "paper_1712_09494_gb300")
    return os.path.join(root, "autotune.json") if not root.endswith(".json") else root


def class_key(device_name, scheme, key_width, capacity, load, dup):
    """Workload class: capacity to the nearest power of two (at least 2^10),
    load and repeat rate to one decimal."""
    c = max(10, int(round(math.log2(max(1, capacity)))))

    def tenth(x):                      # to one decimal, halves up
        return math.floor(x * 10 + 0.5) / 10

    return "%s|%s|%d|2^%d|lf%.1f|d%.1f" % (device_name, scheme, key_width, c, tenth(load), tenth(dup))


def load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path, cache):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(results):
    """Fastest exact candidate: results = [(params, seconds or None when not exact)]."""
    ok = [(sec, i, p) for i, (p, sec) in enumerate(results) if sec is not None]
    if not ok:
        return None
    return min(ok)[2]


def measure_fill(params, scheme, key_width, capacity, load, dup, trials=3, seed=7, max_keys=1 << 22):
    """Seconds to fill a table of `capacity` (capped so that at most max_keys
    distinct keys are inserted) to `load` with batches of 2^20 keys; None if
    the fill is not exact."""
    import torch
    from . import HashTable, ht_clear, ht_find_or_put
    dev = torch.device("cuda", torch.cuda.current_device())
    cap = int(capacity)
    n = int(min(max_keys, cap * load))
    if n < 1:
        return None
    cap = int(math.ceil(n / load))
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    hi = 2 ** 31 - 2 if key_width == 32 else 2 ** 62
    dt = torch.int32 if key_width == 32 else torch.int64
    fresh = torch.unique(torch.randint(0, hi, (n + n // 8 + 16,), device=dev, generator=g))[:n]
    n = fresh.numel()
    B = 1 << 20
    per = max(1, int(B * (1 - dup)))
    batches, fresh_of, issued = [], [], 0
    while issued < n:
        nf = min(per, n - issued)
        nd = int(nf * dup / max(1e-9, 1 - dup))
        dups = fresh[torch.randint(0, issued + nf, (nd,), device=dev, generator=g)] if nd else fresh[:0]
        b = torch.cat([fresh[issued:issued + nf], dups]).to(dt)
        batches.append(b[torch.randperm(b.numel(), device=dev, generator=g)])
        fresh_of.append(fresh[issued:issued + nf].to(dt))
        issued += nf
    try:
        t = HashTable(cap, scheme, key_width, params)
    except Exception:
        return None
    flags = [torch.empty(b.numel(), dtype=torch.uint8, device=dev) for b in batches]
    times = []
    for r in range(trials + 1):
        ht_clear(t.handle)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for b, f in zip(batches, flags):
            ht_find_or_put(t.handle, b, f)
        e1.record()
        torch.cuda.synchronize()
        if r:
            times.append(e0.elapsed_time(e1) / 1e3)
    exact = t.sync() == 0 and t.size() == n and flags_exact(batches, flags, fresh_of)
    t.close()
    return min(times) if exact else None


def flags_exact(batches, flags, fresh_of):
    """Per key, for the last fill: in every batch the keys flagged new are
    exactly that batch's fresh keys, each once (sorted flagged keys == sorted
    fresh keys), so a candidate that loses or doubles a key is rejected."""
    import torch
    for b, f, fr in zip(batches, flags, fresh_of):
        got = torch.sort(b[f.bool()]).values
        if got.numel() != fr.numel() or not torch.equal(got, torch.sort(fr).values):
            return False
    return True


def tune(scheme, key_width, capacity, load=0.8, dup=0.25, cache_path=None, candidates=None, measure=None,
         device_name=None, refresh=False):
    """Returns the cached or newly measured best parameters (a dict) for the
    workload class; `measure(params) -> seconds or None` may be supplied
    (tests); by default measure_fill runs on the current CUDA device."""
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    path = cache_path or default_cache_path()
    key = class_key(device_name, scheme, key_width, capacity, load, dup)
    cache = load_cache(path)
    if not refresh and key in cache:
        return dict(cache[key]["params"])
    cands = candidates if candidates is not None else CANDIDATES[scheme]
    if measure is None:
        def measure(p):
            return measure_fill(p, scheme, key_width, capacity, load, dup)
    results = [(dict(p), measure(dict(p))) for p in cands]
    best = pick(results)
    if best is None:
        raise RuntimeError("no candidate filled the table exactly for class %s" % key)
    cache[key] = {"params": best, "seconds": {json.dumps(p, sort_keys=True): s for p, s in results}}
    save_cache(path, cache)
    return dict(best)
