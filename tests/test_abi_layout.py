"""The C ABI from C (no GPU): the ctypes mirrors of its structs have the C
layout (a small C program prints sizeof and every field's offsetof), and a C
program linked against libht.so calls the entry points that answer without
touching CUDA."""
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


def test_a_c_program_links_and_calls_the_host_entry_points(tmp_path):
    # The boundary used from plain C: link libht.so, read the defaults, name
    # a status, and have ht_create reject bad arguments before any CUDA call.
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_1712_09494_gb300 import _build
    lib = _build.build()
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "ht.h"
int main(void) {
    ht_params p;
    if (ht_default_params(HT_CUCKOO, &p) != HT_OK) return 1;
    if (p.num_hashes != 4 || p.max_evictions != 256 || p.digest_bits != 0) return 2;
    if (strcmp(ht_status_str(HT_ERR_FULL), "table full: keys could not be placed") != 0) return 3;
    ht_table* t = (ht_table*)0x1;
    if (ht_create(0, HT_BUCKET, 64, NULL, NULL, &t) != HT_ERR_INVALID || t != NULL) return 4;
    if (ht_create(1024, HT_BUCKET, 160, NULL, NULL, &t) != HT_ERR_INVALID) return 5;
    p.digest_bits = 8;
    if (ht_create(1024, HT_CUCKOO, 64, &p, NULL, &t) != HT_ERR_INVALID) return 6;
    if (ht_destroy(NULL) != HT_OK) return 7;
    printf("ok\n");
    return 0;
}
''')
    exe = tmp_path / "use"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), lib,
                           "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)
