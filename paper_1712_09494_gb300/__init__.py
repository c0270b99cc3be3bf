"""GPU hash set/map for state-space exploration on GB300 (sm_103a).

A thin Python binding over the C ABI in include/ht.h.  Each ``ht_*`` function
here has the C function's name and only marshals arguments (tensor data
pointers, the current CUDA stream); every step of every operation runs in
the CUDA kernels of libht.so.  There is no CPU fallback: if the library is
missing, importing the functions raises.

The schemes are the two compared by Cassee & Wijs (GaM 2017): the
GPUexplore bucket table (Section 4.2) and Cuckoo hashing after Alcantara et
al. (Section 4.1); the operations follow Section 5's find-or-insert.
"""
import ctypes

import torch

from ._lib import (HT_BUCKET, HT_CUCKOO, HtBfsResult, HtError, HtModel, HtParams, HtServerConfig,
                   HtServerStats, HtTableStats, HtWork, load)

__all__ = [
    "HT_BUCKET", "HT_CUCKOO", "HtError", "HtParams", "HashTable", "load",
    "ht_default_params", "ht_create", "ht_destroy", "ht_find_or_put", "ht_find_or_put_append",
    "ht_insert", "ht_lookup", "ht_sync", "ht_size", "ht_export", "ht_clear", "ht_info",
    "ht_compact", "ht_table_words", "ht_prof_enable", "ht_prof_reset", "ht_prof_read", "ht_prof_kernels",
    "ht_probe_random_read", "ht_probe_random_rmw", "ht_stats", "ht_grow", "ht_multi_find_or_put", "ht_cuckoo_find_or_put_noalloc", "NOALLOC_STATE_BYTES",
    "NOALLOC_MAX_BATCH", "scheme_of", "HtModel", "HtBfsResult", "make_model", "ht_successors", "ht_bfs",
    "MultiExploration", "Server", "HtServerConfig", "HtServerStats",
]

NOALLOC_STATE_BYTES = 2048      # HT_NOALLOC_STATE_BYTES
NOALLOC_MAX_BATCH = 1 << 18     # HT_NOALLOC_MAX_BATCH

_KEY_DTYPES = {32: (torch.int32, torch.uint32), 64: (torch.int64, torch.uint64)}


def scheme_of(name):
    if isinstance(name, int):
        return name
    return {"bucket": HT_BUCKET, "cuckoo": HT_CUCKOO}[name]


def _check(status, where):
    if status != 0:
        raise HtError(status, where)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dptr(t, what):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    return ctypes.c_void_p(t.data_ptr())


def _key_width(keys):
    """32 or 64 for a 1-D int32/int64 tensor; 64*W for an (n, W) int64
    tensor of W words per key (W = 2: (low word, high word) pairs; W = 3..8:
    long keys)."""
    es = keys.element_size()
    if es == 8 and keys.dim() == 2 and 2 <= keys.shape[1] <= 8:
        return 64 * keys.shape[1]
    if es not in (4, 8):
        raise ValueError("keys must be 32- or 64-bit integers")
    return es * 8


def _nkeys(keys):
    return keys.shape[0] if _key_width(keys) >= 128 else keys.numel()


def _params(params, scheme):
    if params is None:
        return None
    if isinstance(params, HtParams):
        return params
    p = ht_default_params(scheme)
    for k, v in dict(params).items():
        setattr(p, k, v)
    return p


# ----------------------------------------------------------------- C ABI
def ht_default_params(scheme):
    p = HtParams()
    _check(load().ht_default_params(scheme_of(scheme), ctypes.byref(p)), "ht_default_params")
    return p


def ht_create(capacity, scheme, key_width, params=None, stream=None):
    scheme = scheme_of(scheme)
    if int(key_width) == 128 and isinstance(params, dict):
        # 16-byte slots: 8 per 128-byte bucket unless given.
        params = dict(dict(bucket_slots=8), **params)
    p = _params(params, scheme)
    out = ctypes.c_void_p()
    _check(load().ht_create(int(capacity), scheme, int(key_width),
                            ctypes.byref(p) if p is not None else None, _stream(stream),
                            ctypes.byref(out)), "ht_create")
    return out


def ht_destroy(table):
    _check(load().ht_destroy(table), "ht_destroy")


def ht_find_or_put(table, keys, is_new=None, stream=None):
    _check(load().ht_find_or_put(table, _dptr(keys, "keys"), _nkeys(keys), _dptr(is_new, "is_new"),
                                 _stream(stream)), "ht_find_or_put")


def ht_find_or_put_append(table, keys, new_keys, new_count, is_new=None, stream=None):
    _check(load().ht_find_or_put_append(table, _dptr(keys, "keys"), _nkeys(keys), _dptr(is_new, "is_new"),
                                        _dptr(new_keys, "new_keys"), _dptr(new_count, "new_count"),
                                        _stream(stream)), "ht_find_or_put_append")


def ht_insert(table, keys, values=None, stream=None):
    _check(load().ht_insert(table, _dptr(keys, "keys"), _dptr(values, "values"), _nkeys(keys),
                            _stream(stream)), "ht_insert")


def ht_lookup(table, keys, values=None, found=None, stream=None):
    _check(load().ht_lookup(table, _dptr(keys, "keys"), _nkeys(keys), _dptr(values, "values"),
                            _dptr(found, "found"), _stream(stream)), "ht_lookup")


def ht_sync(table, stream=None):
    return load().ht_sync(table, _stream(stream))


def ht_size(table, stream=None):
    n = ctypes.c_uint64()
    _check(load().ht_size(table, ctypes.byref(n), _stream(stream)), "ht_size")
    return n.value


def ht_export(table, keys_out, values_out=None, stream=None):
    n = ctypes.c_uint64()
    _check(load().ht_export(table, _dptr(keys_out, "keys_out"), _dptr(values_out, "values_out"),
                            _nkeys(keys_out), ctypes.byref(n), _stream(stream)), "ht_export")
    return n.value


def ht_clear(table, stream=None):
    _check(load().ht_clear(table, _stream(stream)), "ht_clear")


def ht_info(table):
    s, k, r = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().ht_info(table, ctypes.byref(s), ctypes.byref(k), ctypes.byref(r)), "ht_info")
    return dict(slots=s.value, num_hashes=k.value, rebuilds=r.value)


def ht_table_words(table):
    """(device address, bytes) of the table's slot array."""
    ptr, nbytes = ctypes.c_void_p(), ctypes.c_uint64()
    _check(load().ht_table_words(table, ctypes.byref(ptr), ctypes.byref(nbytes)), "ht_table_words")
    return ptr.value, nbytes.value


def ht_multi_find_or_put(tables, items, stream=None):
    """find-or-put over many tables in one call: `tables` a list of handles,
    `items` a list of (table index, keys tensor, is_new uint8 tensor or None)."""
    import numpy as np
    n = len(tables)
    arr_t = (ctypes.c_void_p * max(1, n))(*[getattr(t, "value", t) for t in tables])
    w = np.zeros(max(1, len(items)), dtype=_WORK_DTYPE)
    for i, (ti, keys, is_new) in enumerate(items):
        if not (keys.is_cuda and keys.is_contiguous()):
            raise ValueError("keys of item %d must be a contiguous CUDA tensor" % i)
        if is_new is not None and not (is_new.is_cuda and is_new.is_contiguous()):
            raise ValueError("is_new of item %d must be a contiguous CUDA tensor" % i)
        w[i] = (ti, 0, keys.data_ptr() if keys.numel() else 0, keys.numel(),
                is_new.data_ptr() if is_new is not None and is_new.numel() else 0)
    _check(load().ht_multi_find_or_put(arr_t, n, w.ctypes.data_as(ctypes.c_void_p), len(items), _stream(stream)),
           "ht_multi_find_or_put")


# numpy layout of ht_work (include/ht.h), checked against the ctypes struct.
def _work_dtype():
    import numpy as np
    dt = np.dtype([("table", "<u4"), ("reserved_", "<u4"), ("d_keys", "<u8"), ("n", "<u8"), ("d_is_new", "<u8")])
    assert dt.itemsize == ctypes.sizeof(HtWork)
    assert all(dt.fields[f][1] == getattr(HtWork, f).offset for f, _ in HtWork._fields_)
    return dt


_WORK_DTYPE = _work_dtype()


def ht_grow(table, new_capacity, stream=None):
    _check(load().ht_grow(table, int(new_capacity), _stream(stream)), "ht_grow")


def ht_stats(table, stream=None):
    """Counters since the last clear or rebuild (synchronises the stream)."""
    st = HtTableStats()
    _check(load().ht_stats(table, ctypes.byref(st), _stream(stream)), "ht_stats")
    return {f: getattr(st, f) for f, _ in HtTableStats._fields_ if f != "reserved_"}


def ht_compact(keys, flags, out, count, stream=None):
    _check(load().ht_compact(_dptr(keys, "keys"), _dptr(flags, "flags"), keys.numel(), _key_width(keys),
                             _dptr(out, "out"), _dptr(count, "count"), _stream(stream)), "ht_compact")


def ht_prof_enable(on=True):
    _check(load().ht_prof_enable(1 if on else 0), "ht_prof_enable")


def ht_prof_reset():
    _check(load().ht_prof_reset(), "ht_prof_reset")


def ht_prof_kernels():
    lib = load()
    return [lib.ht_prof_kernel_name(i).decode() for i in range(lib.ht_prof_num_kernels())]


def ht_prof_read():
    """{kernel name: (launches, total_ms)} over the launches since the last reset."""
    lib = load()
    out = {}
    for i, name in enumerate(ht_prof_kernels()):
        n, ms = ctypes.c_uint64(), ctypes.c_double()
        _check(lib.ht_prof_read(i, ctypes.byref(n), ctypes.byref(ms)), "ht_prof_read")
        if n.value:
            out[name] = (n.value, ms.value)
    return out


def ht_probe_random_read(buf, gran, n_access, seed, sink, stream=None):
    _check(load().ht_probe_random_read(_dptr(buf, "buf"), buf.numel() * buf.element_size(), int(gran),
                                       int(n_access), int(seed), _dptr(sink, "sink"), _stream(stream)),
           "ht_probe_random_read")


def ht_probe_random_rmw(buf, n_access, seed, stream=None):
    _check(load().ht_probe_random_rmw(_dptr(buf, "buf"), buf.numel() * buf.element_size(), int(n_access),
                                      int(seed), _stream(stream)), "ht_probe_random_rmw")


def _noalloc_args(slots, state, keys, is_new):
    """Checks the tensors of ht_cuckoo_find_or_put_noalloc before any pointer
    reaches the device: a wrong dtype or a short buffer would make the kernels
    read or write past the end of a caller's allocation."""
    if slots.dtype not in (torch.int64, torch.uint64) or slots.dim() != 1 or slots.numel() == 0:
        raise ValueError("slots must be a non-empty 1-D int64/uint64 tensor")
    if state.numel() * state.element_size() < NOALLOC_STATE_BYTES:
        raise ValueError("state must hold at least %d bytes" % NOALLOC_STATE_BYTES)
    if keys.dtype not in (torch.int64, torch.uint64) or keys.dim() != 1:
        raise ValueError("keys must be a 1-D int64/uint64 tensor")
    n = keys.numel()
    if n > NOALLOC_MAX_BATCH:
        raise ValueError("at most %d keys per call" % NOALLOC_MAX_BATCH)
    if is_new is not None and (is_new.dtype != torch.uint8 or is_new.numel() < n):
        raise ValueError("is_new must be a uint8 tensor of at least %d entries" % n)
    devs = {t.device for t in (slots, state, keys, is_new) if t is not None}
    if len(devs) != 1:
        raise ValueError("slots, state, keys and is_new must be on one CUDA device")
    return n


def ht_cuckoo_find_or_put_noalloc(slots, state, seed, keys, is_new=None, reset=False, stream=None):
    """Find-or-put into a Cuckoo set held in caller tensors (``slots``: int64
    table words, ``state``: NOALLOC_STATE_BYTES bytes); allocates nothing.
    Raises ValueError on a malformed tensor and HtError on a non-OK status.
    Reserved keys, overflow use and dropped keys are reported only in the
    state block's status word (bytes 24..27), which the call does not read."""
    n = _noalloc_args(slots, state, keys, is_new)
    _check(load().ht_cuckoo_find_or_put_noalloc(
        _dptr(slots, "slots"), slots.numel(), _dptr(state, "state"), int(seed) & (2**64 - 1),
        _dptr(keys, "keys"), n, _dptr(is_new, "is_new"), 1 if reset else 0, _stream(stream)),
        "ht_cuckoo_find_or_put_noalloc")


def make_model(num_components, bits, deg, tgt, lab, pairs):
    """Pack model tables (array-likes shaped like ht_model's fields) into an HtModel."""
    import numpy as np
    m = HtModel()
    m.num_components = int(num_components)
    pairs = np.asarray(pairs, dtype=np.uint8).reshape(-1, 2)
    m.num_pairs = int(pairs.shape[0])

    def put(field, arr, size):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.uint8).ravel()[:size])
        ctypes.memmove(field, a.ctypes.data, a.nbytes)

    put(m.bits, bits, 16)
    c1 = np.zeros(8, dtype=np.uint8)
    c2 = np.zeros(8, dtype=np.uint8)
    c1[:m.num_pairs] = pairs[:, 0]
    c2[:m.num_pairs] = pairs[:, 1]
    put(m.pair_c1, c1, 8)
    put(m.pair_c2, c2, 8)
    put(m.deg, deg, 16 * 32)
    put(m.tgt, tgt, 16 * 32 * 4)
    put(m.lab, lab, 16 * 32 * 4)
    return m


def ht_successors(model, states, succ, count, stream=None):
    _check(load().ht_successors(ctypes.byref(model), _key_width(states), _dptr(states, "states"), _nkeys(states),
                                _dptr(succ, "succ"), _nkeys(succ), _dptr(count, "count"), _stream(stream)),
           "ht_successors")


def ht_bfs(table, model, s0=0, max_levels=4096, states=None, states_cap=0, stream=None, fused=False):
    """Returns (HtBfsResult, level sizes list); `states` (optional tensor)
    receives every reachable state in level order.  fused=True runs
    ht_bfs_fused (bucket-scheme tables)."""
    sizes = (ctypes.c_uint64 * max_levels)()
    res = HtBfsResult()
    cap = _nkeys(states) if states is not None else int(states_cap)
    name = "ht_bfs_fused" if fused else "ht_bfs"
    _check(getattr(load(), name)(table, ctypes.byref(model), int(s0), int(max_levels), sizes,
                                 _dptr(states, "states"), cap, ctypes.byref(res), _stream(stream)), name)
    return res, [int(sizes[i]) for i in range(res.levels)]


class MultiExploration:
    """Many explorations advanced together (ht_multi_*).  `schemes`: None
    (all bucket), one scheme for all, or one per exploration.  run(mode):
    0 persistent launch, 1 per-step launches, 2 one exploration at a time,
    3 per-step graph replay."""

    def __init__(self, models, s0, capacities, params=None, max_levels=4096, stream=None, schemes=None):
        n = len(models)
        arr_m = (HtModel * n)(*models)
        arr_s0 = (ctypes.c_uint64 * n)(*[int(x) for x in s0])
        arr_c = (ctypes.c_uint64 * n)(*[int(x) for x in capacities])
        if schemes is None:
            sch = [HT_BUCKET] * n
        elif isinstance(schemes, (str, int)):
            sch = [scheme_of(schemes)] * n
        else:
            sch = [scheme_of(x) for x in schemes]
        arr_s = (ctypes.c_int32 * n)(*sch)
        arr_p = None
        if params is not None:
            arr_p = (HtParams * n)(*[_params(p, sc) if p is not None else ht_default_params(sc)
                                    for p, sc in zip(params, sch)])
        out = ctypes.c_void_p()
        _check(load().ht_multi_create_ex(n, arr_m, arr_s0, arr_c, arr_s, arr_p, int(max_levels), _stream(stream),
                                         ctypes.byref(out)), "ht_multi_create_ex")
        self._h = out
        self.count = n
        self.max_levels = int(max_levels)
        self._keepalive = (arr_m, arr_s0, arr_c, arr_p, arr_s)

    def reset(self, stream=None):
        _check(load().ht_multi_reset(self._h, _stream(stream)), "ht_multi_reset")

    def test_hooks(self, barrier_timeout_ns=0, absent_block=-1):
        """Failure-detection test hooks of the persistent mode (ht_multi_test_hooks)."""
        _check(load().ht_multi_test_hooks(self._h, int(barrier_timeout_ns), int(absent_block)),
               "ht_multi_test_hooks")

    def run(self, mode=0, max_steps=0, stream=None):
        _check(load().ht_multi_run(self._h, int(mode), int(max_steps), _stream(stream)), "ht_multi_run")
        return int(load().ht_multi_steps(self._h))

    def result(self, i, with_states=False, key_width=64):
        """Counts and level sizes of exploration i; with_states=True also
        returns its states (numpy, level order) copied to the host."""
        import numpy as np
        lv, st, gen = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        comp = ctypes.c_int32()
        sizes = (ctypes.c_uint64 * self.max_levels)()
        ptr = ctypes.c_void_p()
        _check(load().ht_multi_result(self._h, int(i), ctypes.byref(lv), ctypes.byref(st), ctypes.byref(gen),
                                      ctypes.byref(comp), sizes, ctypes.byref(ptr), None, 0), "ht_multi_result")
        out = dict(levels=lv.value, states=st.value, successors=gen.value, complete=comp.value,
                   level_sizes=[int(sizes[j]) for j in range(lv.value)], states_ptr=ptr.value)
        if with_states:
            arr = np.empty(st.value, dtype=np.uint32 if key_width == 32 else np.uint64)
            _check(load().ht_multi_result(self._h, int(i), None, None, None, None, None, None,
                                          arr.ctypes.data_as(ctypes.c_void_p), st.value), "ht_multi_result")
            out["states_host"] = arr
        return out

    def close(self):
        if self._h is not None and self._h.value:
            load().ht_multi_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving loop (ht_server_*): keys are uint64 numpy arrays in host memory."""

    def __init__(self, **cfg):
        c = HtServerConfig()
        _check(load().ht_server_default_config(ctypes.byref(c)), "ht_server_default_config")
        for k, v in cfg.items():
            if k == "table_params":
                c.table_params = _params(v, HT_BUCKET)
            else:
                setattr(c, k, v)
        out = ctypes.c_void_p()
        _check(load().ht_server_create(ctypes.byref(c), ctypes.byref(out)), "ht_server_create")
        self._h = out
        self._live = {}

    def open_table(self, capacity, scheme="bucket"):
        tid = ctypes.c_uint32()
        _check(load().ht_server_open_table(self._h, int(capacity), scheme_of(scheme), ctypes.byref(tid)),
               "ht_server_open_table")
        return tid.value

    def close_table(self, table_id):
        _check(load().ht_server_close_table(self._h, int(table_id)), "ht_server_close_table")

    def table_state(self, table_id):
        adm, size = ctypes.c_int32(), ctypes.c_uint64()
        _check(load().ht_server_table_state(self._h, int(table_id), ctypes.byref(adm), ctypes.byref(size)),
               "ht_server_table_state")
        return adm.value, size.value

    def submit(self, table_id, keys, out=None):
        """Queues a find-or-put; `keys` (uint64) and `out` (uint8) must stay alive
        until the request is waited for (the server holds references)."""
        import numpy as np
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        if out is None:
            out = np.empty(len(keys), dtype=np.uint8)
        rid = ctypes.c_uint64()
        _check(load().ht_server_submit(self._h, int(table_id), keys.ctypes.data_as(ctypes.c_void_p), len(keys),
                                       out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rid)), "ht_server_submit")
        self._live[rid.value] = (keys, out)
        return rid.value

    def wait(self, request_id, timeout_ms=60000):
        """Returns (status, latency_us, flags); status 5 (HT_ERR_TIMEOUT) keeps it queued."""
        lat = ctypes.c_double()
        st = load().ht_server_wait(self._h, int(request_id), int(timeout_ms), ctypes.byref(lat))
        if st == 5:
            return st, None, None
        keys, out = self._live.pop(request_id, (None, None))
        return st, lat.value, out

    def stats(self, reset=False):
        s = HtServerStats()
        _check(load().ht_server_get_stats(self._h, ctypes.byref(s), 1 if reset else 0), "ht_server_get_stats")
        return {f: getattr(s, f) for f, _ in HtServerStats._fields_}

    def close(self):
        if self._h is not None and self._h.value:
            load().ht_server_destroy(self._h)
        self._h = None
        self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- helper
class HashTable:
    """Owns one table; methods allocate their outputs with torch on the keys' device."""

    def __init__(self, capacity, scheme="bucket", key_width=64, params=None, stream=None):
        self.scheme = scheme_of(scheme)
        self.key_width = int(key_width)
        self._h = ht_create(capacity, self.scheme, self.key_width, params, stream)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            ht_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _keys(self, keys):
        if _key_width(keys) != self.key_width:
            raise ValueError("table has %d-bit keys" % self.key_width)
        return keys.contiguous()

    def find_or_put(self, keys, stream=None):
        keys = self._keys(keys)
        is_new = torch.empty(_nkeys(keys), dtype=torch.uint8, device=keys.device)
        ht_find_or_put(self._h, keys, is_new, stream)
        return is_new

    def insert(self, keys, values=None, stream=None):
        keys = self._keys(keys)
        ht_insert(self._h, keys, None if values is None else values.contiguous(), stream)

    def lookup(self, keys, stream=None):
        keys = self._keys(keys)
        found = torch.empty(_nkeys(keys), dtype=torch.uint8, device=keys.device)
        values = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device) if self.key_width == 32 else None
        ht_lookup(self._h, keys, values, found, stream)
        return found, values

    def sync(self, stream=None):
        return ht_sync(self._h, stream)

    def size(self, stream=None):
        return ht_size(self._h, stream)

    def export(self, stream=None):
        n = self.size(stream)
        dt = torch.int32 if self.key_width == 32 else torch.int64
        dev = torch.device("cuda", torch.cuda.current_device())
        shape = (max(n, 1), self.key_width // 64) if self.key_width >= 128 else (max(n, 1),)
        keys = torch.empty(shape, dtype=dt, device=dev)
        vals = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if self.key_width == 32 else None
        got = ht_export(self._h, keys, vals, stream)
        return keys[:got], (vals[:got] if vals is not None else None)

    def clear(self, stream=None):
        ht_clear(self._h, stream)

    def info(self):
        return ht_info(self._h)

    def stats(self, stream=None):
        return ht_stats(self._h, stream)

    def grow(self, new_capacity, stream=None):
        ht_grow(self._h, new_capacity, stream)

    # Checkpoint / resume: the stored keys (and values) with the table's
    # shape, written with numpy; load re-creates the table and inserts them.
    def save(self, path, stream=None):
        import numpy as np
        keys, vals = self.export(stream)
        info = self.info()
        np.savez(path, keys=keys.cpu().numpy(), values=(vals.cpu().numpy() if vals is not None else np.empty(0)),
                 scheme=int(self.scheme), key_width=self.key_width, slots=info["slots"])

    @classmethod
    def load(cls, path, params=None, stream=None):
        import numpy as np
        z = np.load(path)
        t = cls(int(z["slots"]), int(z["scheme"]), int(z["key_width"]), params, stream)
        keys = z["keys"]
        if len(keys):
            dev = torch.device("cuda", torch.cuda.current_device())
            k = torch.from_numpy(keys).to(dev)
            v = torch.from_numpy(z["values"]).to(dev) if t.key_width == 32 and len(z["values"]) else None
            t.insert(k, v, stream)
        return t
