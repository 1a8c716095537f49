"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/aaag.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aaag.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(aaag_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2504_12811_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("aaag_preprocess", "aaag_cull", "aaag_sort", "aaag_render",
                     "aaag_workspace_bytes", "aaag_workspace_init", "aaag_get_stats"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_2504_12811_gb300 import aaag
    bound = {name for name, _, _ in aaag.SIGNATURES}
    assert set(declared_functions()) <= bound
    aaag.lib()      # loads and sets every signature


def test_host_argument_checks_without_gpu(libpath):
    """Pure host-side paths: sizes and argument validation."""
    from paper_2504_12811_gb300 import aaag
    assert aaag.aaag_workspace_bytes(-1, 16, 16, 10) == 0
    b1 = aaag.aaag_workspace_bytes(1000, 128, 128, 4096)
    b2 = aaag.aaag_workspace_bytes(2000, 128, 128, 4096)
    assert 0 < b1 < b2
    with pytest.raises(aaag.AaagError):
        aaag.aaag_workspace_init(None, b1, 1000, 128, 128, 4096)
    assert aaag.aaag_radix_sort_scratch_bytes(0) > 0
