"""ctypes loader for libht.so: declares every C-ABI signature of include/ht.h."""
import ctypes
import os

from . import _build

HT_BUCKET, HT_CUCKOO = 0, 1
STATUS = {0: "HT_OK", 1: "HT_ERR_INVALID", 2: "HT_ERR_OOM", 3: "HT_ERR_FULL",
          4: "HT_ERR_CUDA", 5: "HT_ERR_TIMEOUT"}


class HtParams(ctypes.Structure):
    _fields_ = [
        ("num_hashes", ctypes.c_uint32), ("max_evictions", ctypes.c_uint32),
        ("stash_slots", ctypes.c_uint32), ("bucket_slots", ctypes.c_uint32),
        ("lanes_per_key", ctypes.c_uint32), ("max_rebuilds", ctypes.c_uint32),
        ("max_batch", ctypes.c_uint64), ("seed", ctypes.c_uint64),
        ("l2_persist", ctypes.c_int32), ("grow_load_permille", ctypes.c_uint32),
        ("digest_bits", ctypes.c_uint32), ("cuckoo_chain_h1", ctypes.c_uint32),
        ("publish_wait_polls", ctypes.c_uint32), ("reserved_", ctypes.c_uint32),
    ]


class HtModel(ctypes.Structure):
    _fields_ = [
        ("num_components", ctypes.c_int32), ("num_pairs", ctypes.c_int32),
        ("bits", ctypes.c_uint8 * 16),
        ("pair_c1", ctypes.c_uint8 * 8), ("pair_c2", ctypes.c_uint8 * 8),
        ("deg", ctypes.c_uint8 * (16 * 32)),
        ("tgt", ctypes.c_uint8 * (16 * 32 * 4)),
        ("lab", ctypes.c_uint8 * (16 * 32 * 4)),
    ]


class HtBfsResult(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_uint64), ("states", ctypes.c_uint64),
                ("successors", ctypes.c_uint64), ("complete", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]


class HtServerConfig(ctypes.Structure):
    _fields_ = [
        ("max_inflight", ctypes.c_uint32), ("max_requests_per_batch", ctypes.c_uint32),
        ("batch_key_budget", ctypes.c_uint64), ("hbm_reserve_bytes", ctypes.c_uint64),
        ("fake_free_bytes", ctypes.c_uint64), ("pack", ctypes.c_int32), ("reserved_", ctypes.c_int32 * 3),
        ("table_params", HtParams),
    ]


class HtServerStats(ctypes.Structure):
    _fields_ = [
        ("requests", ctypes.c_uint64), ("keys", ctypes.c_uint64), ("batches", ctypes.c_uint64),
        ("seconds", ctypes.c_double), ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
        ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double), ("admitted_bytes", ctypes.c_uint64),
        ("tables_admitted", ctypes.c_uint32), ("status", ctypes.c_int32),
        ("admit_seconds", ctypes.c_double), ("pack_seconds", ctypes.c_double),
        ("finish_seconds", ctypes.c_double), ("batch_us_mean", ctypes.c_double),
        ("batch_gpu_us_mean", ctypes.c_double),
        ("tables_created", ctypes.c_uint64), ("inflight_seconds", ctypes.c_double),
        ("table_bytes_created", ctypes.c_uint64),
    ]


class HtTableStats(ctypes.Structure):
    _fields_ = [
        ("size", ctypes.c_uint64), ("dropped", ctypes.c_uint64), ("exchanges", ctypes.c_uint64),
        ("stash_used", ctypes.c_uint32), ("overflow_used", ctypes.c_uint32),
        ("rebuilds", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("probes", ctypes.c_uint64),
        ("probe_misses", ctypes.c_uint64), ("probe_miss_reads", ctypes.c_uint64), ("probe_cas", ctypes.c_uint64),
    ]


class HtWork(ctypes.Structure):
    _fields_ = [
        ("table", ctypes.c_uint32), ("reserved_", ctypes.c_uint32), ("d_keys", ctypes.c_void_p),
        ("n", ctypes.c_uint64), ("d_is_new", ctypes.c_void_p),
    ]


class HtError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s" % (where, STATUS.get(status, status)))


_VP, _U64, _U32, _I32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
_P = ctypes.POINTER

# name -> (restype, argtypes); mirrors include/ht.h.
SIGNATURES = {
    "ht_default_params": (_I32, [_I32, _P(HtParams)]),
    "ht_create": (_I32, [_U64, _I32, _U32, _P(HtParams), _VP, _P(_VP)]),
    "ht_destroy": (_I32, [_VP]),
    "ht_find_or_put": (_I32, [_VP, _VP, _U64, _VP, _VP]),
    "ht_find_or_put_append": (_I32, [_VP, _VP, _U64, _VP, _VP, _VP, _VP]),
    "ht_insert": (_I32, [_VP, _VP, _VP, _U64, _VP]),
    "ht_lookup": (_I32, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "ht_sync": (_I32, [_VP, _VP]),
    "ht_size": (_I32, [_VP, _P(_U64), _VP]),
    "ht_export": (_I32, [_VP, _VP, _VP, _U64, _P(_U64), _VP]),
    "ht_clear": (_I32, [_VP, _VP]),
    "ht_info": (_I32, [_VP, _P(_U64), _P(_U32), _P(_U32)]),
    "ht_table_words": (_I32, [_VP, _P(_VP), _P(_U64)]),
    "ht_stats": (_I32, [_VP, _P(HtTableStats), _VP]),
    "ht_grow": (_I32, [_VP, _U64, _VP]),
    "ht_multi_find_or_put": (_I32, [_VP, _U32, _VP, _U32, _VP]),
    "ht_status_str": (ctypes.c_char_p, [_I32]),
    "ht_compact": (_I32, [_VP, _VP, _U64, _U32, _VP, _VP, _VP]),
    "ht_prof_enable": (_I32, [ctypes.c_int]),
    "ht_prof_reset": (_I32, []),
    "ht_prof_num_kernels": (_U32, []),
    "ht_prof_kernel_name": (ctypes.c_char_p, [_U32]),
    "ht_prof_read": (_I32, [_U32, _P(_U64), _P(ctypes.c_double)]),
    "ht_probe_random_read": (_I32, [_VP, _U64, _U32, _U64, _U64, _VP, _VP]),
    "ht_probe_random_rmw": (_I32, [_VP, _U64, _U64, _U64, _VP]),
    "ht_cuckoo_find_or_put_noalloc": (_I32, [_VP, _U64, _VP, _U64, _VP, _U64, _VP, ctypes.c_int, _VP]),
    "ht_successors": (_I32, [_P(HtModel), _U32, _VP, _U64, _VP, _U64, _VP, _VP]),
    "ht_bfs": (_I32, [_VP, _P(HtModel), _U64, _U32, _VP, _VP, _U64, _P(HtBfsResult), _VP]),
    "ht_bfs_fused": (_I32, [_VP, _P(HtModel), _U64, _U32, _VP, _VP, _U64, _P(HtBfsResult), _VP]),
    "ht_multi_create": (_I32, [_U32, _VP, _VP, _VP, _VP, _U32, _VP, _P(_VP)]),
    "ht_multi_create_ex": (_I32, [_U32, _VP, _VP, _VP, _VP, _VP, _U32, _VP, _P(_VP)]),
    "ht_multi_reset": (_I32, [_VP, _VP]),
    "ht_multi_run": (_I32, [_VP, ctypes.c_int, _U64, _VP]),
    "ht_multi_result": (_I32, [_VP, _U32, _P(_U64), _P(_U64), _P(_U64), _P(ctypes.c_int32), _VP, _P(_VP), _VP,
                               _U64]),
    "ht_multi_steps": (_U64, [_VP]),
    "ht_multi_destroy": (_I32, [_VP]),
    "ht_multi_test_hooks": (_I32, [_VP, _U64, ctypes.c_int32]),
    "ht_server_default_config": (_I32, [_P(HtServerConfig)]),
    "ht_server_create": (_I32, [_P(HtServerConfig), _P(_VP)]),
    "ht_server_destroy": (_I32, [_VP]),
    "ht_server_open_table": (_I32, [_VP, _U64, _I32, _P(_U32)]),
    "ht_server_close_table": (_I32, [_VP, _U32]),
    "ht_server_table_state": (_I32, [_VP, _U32, _P(ctypes.c_int32), _P(_U64)]),
    "ht_server_submit": (_I32, [_VP, _U32, _VP, _U64, _VP, _P(_U64)]),
    "ht_server_wait": (_I32, [_VP, _U64, _U32, _P(ctypes.c_double)]),
    "ht_server_get_stats": (_I32, [_VP, _P(HtServerStats), ctypes.c_int]),
}

_lib = None


def lib_path():
    return _build.LIB


def load():
    """Loads the in-tree libht.so.  Raises if it has not been built: there is
    no fallback implementation of any operation."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError("libht.so is missing (%s); run __graft_entry__.build() or "
                          "python paper_1712_09494_gb300/_build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
