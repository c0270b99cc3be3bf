"""The C-ABI library builds, loads and exports every function include/ht.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\*?\s*(ht_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1712_09494_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_1712_09494_gb300 import _lib
    names = _declared("ht.h")
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, "binding lacks %s" % n


def test_default_params(lib):
    from paper_1712_09494_gb300 import HT_BUCKET, HT_CUCKOO, HtParams
    p = HtParams()
    assert lib.ht_default_params(HT_BUCKET, ctypes.byref(p)) == 0
    assert (p.num_hashes, p.bucket_slots, p.stash_slots) == (16, 16, 101)
    assert lib.ht_default_params(HT_CUCKOO, ctypes.byref(p)) == 0
    assert (p.num_hashes, p.max_evictions) == (4, 256)
    assert lib.ht_default_params(7, ctypes.byref(p)) == 1


@pytest.mark.parametrize("cap,scheme,kw,field,val", [
    (0, 0, 64, None, None),
    (1 << 41, 0, 64, None, None),
    (1024, 0, 48, None, None),
    (1024, 5, 64, None, None),
    (1024, 0, 160, None, None),            # not a multiple of 64
    (1024, 1, 576, None, None),            # more than 8 words
    (1024, 0, 64, "digest_bits", 8),       # a long-key knob only
    (1024, 1, 256, "digest_bits", 65),
    (1024, 0, 256, "bucket_slots", 8),     # long-key buckets are 16 headers
    (1024, 0, 64, "bucket_slots", 12),
    (1024, 0, 64, "num_hashes", 17),
    (1024, 0, 64, "lanes_per_key", 3),
    (1024, 1, 64, "num_hashes", 9),
    (1024, 1, 64, "max_evictions", 5000),
    (1024, 1, 32, "stash_slots", 5000),
])
def test_create_rejects_bad_arguments_before_any_cuda_call(lib, cap, scheme, kw, field, val):
    from paper_1712_09494_gb300 import HtParams
    p = HtParams()
    lib.ht_default_params(scheme if scheme in (0, 1) else 0, ctypes.byref(p))
    if field:
        setattr(p, field, val)
    out = ctypes.c_void_p(123)
    assert lib.ht_create(cap, scheme, kw, ctypes.byref(p), None, ctypes.byref(out)) == 1
    assert not out.value


def test_key_width_of_tensors():
    # The binding reads the key width from the tensor's shape: 1-D 32/64-bit,
    # or (n, W) int64 words for W = 2..8.
    import torch
    from paper_1712_09494_gb300 import _key_width, _nkeys
    assert _key_width(torch.empty(5, dtype=torch.int32)) == 32
    assert _key_width(torch.empty(5, dtype=torch.int64)) == 64
    for w in range(2, 9):
        t = torch.empty((5, w), dtype=torch.int64)
        assert _key_width(t) == 64 * w and _nkeys(t) == 5
    with pytest.raises(ValueError):
        _key_width(torch.empty(5, dtype=torch.int16))


def test_null_arguments_are_invalid(lib):
    assert lib.ht_find_or_put(None, None, 0, None, None) == 1
    assert lib.ht_lookup(None, None, 0, None, None, None) == 1
    assert lib.ht_size(None, None, None) == 1
    assert lib.ht_compact(None, None, 5, 64, None, None, None) == 1
    assert lib.ht_compact(None, None, 0, 48, None, None, None) == 1
    assert lib.ht_probe_random_read(None, 0, 32, 1, 1, None, None) == 1
    assert lib.ht_probe_random_rmw(None, 0, 1, 1, None) == 1
    assert lib.ht_stats(None, None, None) == 1
    assert lib.ht_multi_find_or_put(None, 0, None, 3, None) == 1
    assert lib.ht_multi_find_or_put(None, 0, None, 0, None) == 0
    assert lib.ht_destroy(None) == 0
    assert lib.ht_status_str(3) == b"table full: keys could not be placed"


def test_profiler_names(lib):
    from paper_1712_09494_gb300 import ht_prof_kernels
    names = ht_prof_kernels()
    assert "bucket_find_or_put" in names and "cuckoo_insert" in names
    assert len(set(names)) == len(names)
