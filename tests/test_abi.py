"""CPU-side checks of the C ABI: the library loads and exports every function
declared in include/rhseg.h, and the ctypes structures match the header's
layouts.  No compute call is made (there may be no GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rhseg.h")


def _declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(rhseg_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def so_path():
    from paper_2106_12942_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["rhseg_create", "rhseg_create_device", "rhseg_run", "rhseg_get_level", "rhseg_get_log",
              "rhseg_get_stats", "rhseg_destroy", "rhseg_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(so_path):
    out = subprocess.run(["nm", "-D", "--defined-only", so_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(rhseg_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header(so_path):
    from paper_2106_12942_b300 import _abi
    assert sorted(_abi.SIGNATURES) == _declared_functions()
    L = C.CDLL(so_path)
    for n in _declared_functions():
        assert hasattr(L, n)


def test_struct_layouts_match_header(so_path):
    # compile a tiny C program against the header and compare sizes/offsets
    from paper_2106_12942_b300 import _abi
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "rhseg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(rhseg_params), offsetof(rhseg_params, spclust_wght),
         offsetof(rhseg_params, precision), sizeof(rhseg_merge), offsetof(rhseg_merge, key));
  printf("%zu %zu %zu\n", sizeof(rhseg_stats), offsetof(rhseg_stats, stalled_sections), offsetof(rhseg_stats, run_ms));
  return 0;
}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
        a, b = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    a = list(map(int, a.split()))
    b = list(map(int, b.split()))
    assert a == [C.sizeof(_abi.Params), _abi.Params.spclust_wght.offset, _abi.Params.precision.offset,
                 C.sizeof(_abi.Merge), _abi.Merge.key.offset]
    assert b == [C.sizeof(_abi.Stats), _abi.Stats.stalled_sections.offset, _abi.Stats.run_ms.offset]


def test_every_field_offset_matches_header(so_path):
    # every field of the three structures, by name, against offsetof() in C
    from paper_2106_12942_b300 import _abi
    structs = [("rhseg_params", _abi.Params), ("rhseg_merge", _abi.Merge), ("rhseg_stats", _abi.Stats)]
    lines = []
    want = []
    for cname, py in structs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(C.sizeof(py))
        for f, _ in py._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
            want.append(getattr(py, f).offset)
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"rhseg.h\"\nint main(void) {\n" + \
          "\n".join(lines) + "\n  return 0;\n}\n"
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
        got = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    assert got == want


def test_strerror_is_host_only(so_path):
    from paper_2106_12942_b300 import _abi
    L = _abi.load(so_path)
    assert L.rhseg_strerror(0) == b"ok"
    assert L.rhseg_strerror(-7) == b"output buffer too small"


def test_param_validation_needs_no_device(so_path):
    from paper_2106_12942_b300 import _abi
    from paper_2106_12942_b300.rhseg import make_params
    L = _abi.load(so_path)
    h = C.c_void_p()
    img = (C.c_uint16 * 4)()
    for bad in [dict(spclust_wght=1.5), dict(connectivity=6), dict(rnb_levels=0), dict(rnb_levels=7),
                dict(precision=9), dict(conv_nregions=0), dict(incremental=1, precision=1),
                dict(multi_merge=2), dict(multi_merge=1, incremental=1, precision=3),
                dict(wait_cycles=-1), dict(screen_group=9), dict(screen_pair=2), dict(adjacency=2),
                dict(adjacency=1, incremental=1, precision=3)]:
        p = make_params(**bad)
        assert L.rhseg_create(img, 2, 2, 1, None, C.byref(p), None, C.byref(h)) == _abi.RHSEG_EINVAL
