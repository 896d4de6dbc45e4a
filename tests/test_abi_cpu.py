"""Host-only checks of the C ABI: the library builds, loads and exports every declared symbol.

No compute call is made (this machine may have no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swiftcl.h")


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(swcl_\w+)\s*\(", txt, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2505_22718_gb300 import _lib
    return _lib.load()


def test_header_declares_the_abi():
    syms = declared_symbols()
    for s in ("swcl_create", "swcl_destroy", "swcl_set_grids", "swcl_set_tracers", "swcl_set_windows",
              "swcl_set_power", "swcl_compute_cl", "swcl_vjp", "swcl_last_error", "swcl_strerror"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_signatures_cover_the_header(lib):
    from paper_2505_22718_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)


def test_strerror_is_host_only(lib):
    assert lib.swcl_strerror(0) == b"ok"
    assert lib.swcl_strerror(-3) == b"memory budget exceeded"
    assert lib.swcl_strerror(12345) == b"unknown status"


def test_null_context_is_rejected_without_a_gpu(lib):
    assert lib.swcl_destroy(None) == 0
    assert lib.swcl_sync(None) == -1
    assert lib.swcl_set_grids(None, 1.0, 2.0, 64, None, 0, None, 0, None, 0) == -1
