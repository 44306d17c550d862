"""The C-ABI library builds, loads on a machine without a GPU, and exports
every entry point that include/gff.h declares (no compute call is made)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gff.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gff_status|void|const char\s*\*)\s*(gff_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gff_create", "gff_apply_operator", "gff_project", "gff_step", "gff_run_history",
                     "gff_get_fips", "gff_save_state", "gff_load_state"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1806_10599_gb300 import build

    if not os.path.exists(build.LIB):
        build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_1806_10599_gb300 import build

    if not os.path.exists(build.LIB):
        build.build()
    from paper_1806_10599_gb300 import gff

    for n in declared_functions():
        assert n in gff._SIGS, n
        assert callable(getattr(gff, n)), n


def test_options_default_is_host_only():
    from paper_1806_10599_gb300 import build

    if not os.path.exists(build.LIB):
        build.build()
    from paper_1806_10599_gb300 import gff

    o = gff.gff_options_default()
    assert o.newton_tol == 1e-8 and o.cg_max == 2000 and o.projection == gff.GFF_PROJ_CONTINUOUS
