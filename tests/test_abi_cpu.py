"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/omss.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_1411_4356_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "omss.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(om_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    assert sorted(_lib.SIGNATURES) == header_functions()


def test_status_strings_and_einval_without_gpu():
    lib = _lib.load()
    assert lib.om_status_str(0) == b"OM_OK"
    assert b"OM_ENOCONV" in lib.om_status_str(-5)
    # NULL arguments are rejected before any CUDA call
    st = lib.om_build_liouvillian(None, None, None, None)
    assert st == -1
    assert b"NULL" in lib.om_last_error()


def test_oracle_is_not_linked_into_the_library():
    """The product library shares no code with the oracle."""
    out = os.popen(f"nm -D {build.LIB}").read()
    assert "oracle_" not in out


def test_set_allocator_argument_checks_without_gpu():
    lib = _lib.load()
    assert lib.om_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None) == 0
    only_alloc = _lib.ALLOC_FN(lambda n, s, c: None)
    assert lib.om_set_allocator(only_alloc, _lib.FREE_FN(), None) == -1
    assert lib.om_allocator_hook_calls() >= 0
