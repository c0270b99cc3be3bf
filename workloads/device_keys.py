"""The key streams of ``workloads.keys`` drawn on a torch device, for
measurement runs whose streams are too large to build quickly on the host.

``distinct_keys_dev`` computes the same 63-bit bijection as
``keys.mix63_perm`` (so the same seed and index range give the same keys);
``fill_batches_dev`` follows ``keys.fill_stream``'s recipe -- each batch
(1-d)*B fresh keys plus repeats drawn uniformly from every key issued so far,
shuffled -- with torch's generator for the draws, so its repeats differ from
the host stream's.  Only 64-bit keys.
"""
import torch

_M63 = (1 << 63) - 1


def _wrap(v):
    """A 64-bit constant as the int64 with the same bits."""
    return v - (1 << 64) if v >= 1 << 63 else v


def mix63_perm_dev(x, seed=0):
    """keys.mix63_perm on an int64 tensor of indices (< 2^63)."""
    s = (seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & _M63
    z = (x + s) & _M63
    # int64 products wrap mod 2^64 like the uint64 ones; after the 63-bit
    # mask the words are non-negative, so >> is the logical shift.
    z = (z * _wrap(0xD6E8FEB86659FD93)) & _M63
    z = z ^ (z >> 29)
    z = (z * _wrap(0xA0761D6478BD642F)) & _M63
    z = z ^ (z >> 32)
    z = (z * _wrap(0xE7037ED1A0B428DB)) & _M63
    z = z ^ (z >> 29)
    return z


def distinct_keys_dev(n, seed, start=0, device="cpu"):
    idx = torch.arange(start, start + n, dtype=torch.int64, device=device)
    return mix63_perm_dev(idx, seed)


def fill_batches_dev(n_distinct, batch, dup_rate, seed, device):
    """(list of int64 key tensors, list of fresh counts) filling an empty
    table with exactly n_distinct keys."""
    if not 0.0 <= dup_rate < 1.0:
        raise ValueError("dup_rate must be in [0, 1)")
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    fresh = distinct_keys_dev(n_distinct, seed, device=device)
    per = max(1, int(round(batch * (1.0 - dup_rate))))
    out, counts, issued = [], [], 0
    while issued < n_distinct:
        nf = min(per, n_distinct - issued)
        nd = batch - nf if nf == per else int(round(nf * dup_rate / (1.0 - dup_rate)))
        end = issued + nf
        parts = [fresh[issued:end]]
        if nd:
            parts.append(fresh[torch.randint(0, end, (nd,), device=device, generator=g)])
        b = torch.cat(parts)
        out.append(b[torch.randperm(b.numel(), device=device, generator=g)])
        counts.append(nf)
        issued = end
    return out, counts


_M32 = 0xFFFFFFFF


def _perm32_once_dev(z, s):
    z = (z + s) & _M32
    z = (z * 0x7FEB352D) & _M32
    z = z ^ (z >> 15)
    z = (z * 0x846CA68B) & _M32
    z = z ^ (z >> 16)
    return z


def mix32_perm_dev(x, seed=0):
    """keys.mix32_perm on an int64 tensor of indices in [0, 2^32 - 1):
    the 32-bit permutation, re-applied while the result is the reserved
    0xFFFFFFFF (cycle walking)."""
    s = (seed * 0x9E3779B9 + 0x85EBCA6B) & _M32
    z = _perm32_once_dev(x & _M32, s)
    bad = z == _M32
    while bool(bad.any()):
        z = torch.where(bad, _perm32_once_dev(z, s), z)
        bad = z == _M32
    return z


def multiplicity_sequence_dev(n, mult, seed, device):
    """n 32-bit keys (int32 tensor with the keys' bits) drawn uniformly from a
    value range of round(n / mult) values, so a value occurs `mult` times on
    average among those drawn: the shape of the paper's random sequences
    (Section 5.2, mean multiplicity 1..1000)."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rng = max(1, int(round(n / mult)))
    v = torch.randint(0, rng, (n,), device=device, generator=g, dtype=torch.int64)
    k = mix32_perm_dev(v, seed)
    return (k - ((k >> 31) << 32)).to(torch.int32)      # same 32 bits, as int32
