"""The random-access probes that give the bench its roofline denominators:
they must touch exactly what they claim to (n_access accesses, at random
lines of the buffer, nothing outside it)."""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


@pytest.mark.parametrize("lines,n_access", [(1, 1000), (777, 123_457), (1 << 16, 3_000_001)])
def test_rmw_probe_adds_once_per_access_at_line_starts(lines, n_access):
    buf = torch.zeros(lines * 16 + 16, dtype=torch.int64, device="cuda")   # one guard line
    ht.ht_probe_random_rmw(buf[:lines * 16], n_access, 9)
    got = buf.cpu().numpy().reshape(-1, 16)
    assert got[:, 1:].sum() == 0                  # only the first word of a line
    assert got[lines:].sum() == 0                 # nothing past the buffer
    assert got[:lines, 0].sum() == n_access       # every access exactly once
    if lines > 1:
        # Uniform over lines: no line takes more than a few times its share.
        assert got[:lines, 0].max() < max(50, 8 * n_access / lines)


def test_read_probe_leaves_buffer_and_rejects_bad_grain():
    buf = torch.arange(1 << 12, dtype=torch.int64, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    for gran in (8, 32, 128):
        ht.ht_probe_random_read(buf, gran, 100_000, 3, sink)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(buf.cpu().numpy(), np.arange(1 << 12))
    with pytest.raises(ht.HtError):
        ht.ht_probe_random_read(buf, 16, 10, 3, sink)
    with pytest.raises(ht.HtError):
        ht.ht_probe_random_rmw(buf[1:], 10, 3)    # not 128-byte aligned
