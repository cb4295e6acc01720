"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/dbg.h declares."""
import ctypes
import os
import re

from paper_1003_1940_gb300 import build_lib, dbg

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dbg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(dbg_\w+)\s*\(", text))
    # typedef'd function pointer types are not entry points
    return sorted(n for n in names if not n.endswith("_fn"))


def test_library_exports_every_declared_symbol():
    path = build_lib.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert len(declared_functions()) >= 20


def test_binding_covers_every_symbol():
    bound = {name for name, _, _ in dbg._SIGNATURES}
    assert set(declared_functions()) <= bound


def test_options_init_without_gpu():
    lib = dbg.load(build=True)
    opt = dbg.dbg_options()
    lib.dbg_options_init(ctypes.byref(opt))
    assert opt.struct_size == ctypes.sizeof(dbg.dbg_options)
    assert opt.device == -1


def test_sort_variant_tables_fit_the_autotune_report():
    """Every sort kind's variant table fits the per-kind stride of the
    autotune report (DBG_MAX_SORT_VARIANTS), and each variant has a name."""
    dbg.load(build=True)
    stride = int(re.search(r"#define DBG_MAX_SORT_VARIANTS (\d+)", open(HEADER).read()).group(1))
    assert stride == dbg.MAX_SORT_VARIANTS
    for kd in range(4):
        count = dbg.dbg_sort_variant_count(kd)
        assert 1 <= count <= stride
        names = [dbg.dbg_sort_variant_name(kd, v) for v in range(count)]
        assert all(names) and len(set(names)) == count
