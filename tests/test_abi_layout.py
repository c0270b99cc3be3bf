"""The ctypes mirrors of the C ABI's structs have the C layout: a small C
program compiled against include/ht.h prints sizeof and every field's
offsetof, and they must equal the ctypes sizes and offsets (no GPU)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1712_09494_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "ht_params": _lib.HtParams,
    "ht_table_stats": _lib.HtTableStats,
    "ht_model": _lib.HtModel,
    "ht_bfs_result": _lib.HtBfsResult,
    "ht_work": _lib.HtWork,
    "ht_server_config": _lib.HtServerConfig,
    "ht_server_stats": _lib.HtServerStats,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ht.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        s, f, v = line.split()
        out[(s, f)] = int(v)
    return out


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_ctypes_mirror_matches_c_layout(c_layout, cname):
    py = STRUCTS[cname]
    assert ctypes.sizeof(py) == c_layout[(cname, "sizeof")], cname
    for f in py._fields_:
        assert getattr(py, f[0]).offset == c_layout[(cname, f[0])], (cname, f[0])
