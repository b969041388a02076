"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a and loads, it exports every function include/chimera.h declares,
the ctypes structures match the C layout, and the error paths that need no
device behave as documented."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chimera.h")


@pytest.fixture(scope="module")
def chim():
    from paper_2504_02034_b300 import build
    build.build()
    import paper_2504_02034_b300 as pkg
    pkg.lib()
    return pkg


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chimera_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(chim):
    names = _declared()
    assert len(names) >= 19
    L = C.CDLL(chim.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(chim.ABI), set(names) ^ set(chim.ABI)


def test_only_abi_is_exported(chim):
    out = subprocess.run(["nm", "-D", "--defined-only", chim.LIB_PATH], capture_output=True, text=True).stdout
    syms = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert syms and all(s.startswith("chimera_") for s in syms), syms


def test_struct_layout_matches_header(chim, tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "chimera.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(chimera_catalog_desc),
         offsetof(chimera_catalog_desc, n_gal_total), offsetof(chimera_catalog_desc, n_inj_total),
         offsetof(chimera_catalog_desc, kde_mode), offsetof(chimera_catalog_desc, gal_storage));
  printf("%zu %zu\n", sizeof(chimera_catalog_info_t), offsetof(chimera_catalog_info_t, device_bytes));
  printf("%zu %zu\n", sizeof(chimera_serve_stats_t), offsetof(chimera_serve_stats_t, p99_ms));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    a, b, c = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)]).decode().splitlines()]
    D = chim.CatalogDesc
    assert a == [C.sizeof(D), D.n_gal_total.offset, D.n_inj_total.offset, D.kde_mode.offset,
                 D.gal_storage.offset]
    assert b == [C.sizeof(chim.CatalogInfo), chim.CatalogInfo.device_bytes.offset]
    assert c == [C.sizeof(chim.ServeStats), chim.ServeStats.p99_ms.offset]


def test_strerror_names(chim):
    assert chim.chimera_strerror(0) == "ok"
    assert chim.chimera_strerror(chim.CHIMERA_ERR_ADMISSION) == "HBM budget exceeded"
    assert chim.chimera_strerror(12345) == "unknown error"


def test_null_arguments_rejected(chim):
    L = chim.lib()
    assert L.chimera_create(None, 0, 0) == chim.CHIMERA_ERR_INVALID_ARG
    assert L.chimera_loglike(None, 0, 1, None, 0, None, None, None) == chim.CHIMERA_ERR_INVALID_ARG
    assert L.chimera_serve_stats(None, None) == chim.CHIMERA_ERR_INVALID_ARG
    assert L.chimera_serve_reset_stats(None) == chim.CHIMERA_ERR_INVALID_ARG
    L.chimera_destroy(None)


def test_no_cpu_fallback_without_gpu(chim):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(chim.ChimeraError) as e:
        chim.chimera_create(0)
    assert e.value.code == chim.CHIMERA_ERR_CUDA


def test_every_field_offset_matches_header(chim, tmp_path):
    """Each ctypes mirror of a header struct has the header's fields at the
    header's offsets, field by field."""
    structs = [("chimera_catalog_desc", chim.CatalogDesc), ("chimera_catalog_info_t", chim.CatalogInfo),
               ("chimera_serve_stats_t", chim.ServeStats)]
    lines = []
    for cname, py in structs:
        for f in py._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (cname, f[0]))
        lines.append('  printf("%%zu\\n", sizeof(%s));' % cname)
    prog = tmp_path / "fields.c"
    prog.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"chimera.h\"\nint main(void) {\n"
                    + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "fields"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = list(map(int, subprocess.check_output([str(exe)]).decode().split()))
    want = []
    for _, py in structs:
        want += [getattr(py, f[0]).offset for f in py._fields_] + [C.sizeof(py)]
    assert got == want
