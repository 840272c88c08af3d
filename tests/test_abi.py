"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol that include/vsie.h declares (no GPU work)."""
import os
import re
import subprocess

import pytest

from paper_2206_12409_gb300 import vsie as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vsie.h")).read()
    return sorted(set(re.findall(r"VSIE_API\s+[\w\s\*]+?\b(vsie_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(V.LIB_PATH):
        from paper_2206_12409_gb300 import build
        build.build(verbose=False)
    return V.load_library()


def test_header_declares_expected_symbols():
    assert _declared() == sorted(V.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", V.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\sT\s(vsie_\w+)", out))
    assert set(_declared()) <= exported
    for name in _declared():
        assert hasattr(lib, name)


def test_version_and_null_context_errors(lib):
    assert "libvsie" in V.vsie_version()
    with pytest.raises(V.VsieError) as e:
        V.vsie_sizes(None)
    assert e.value.status == V.VSIE_EINVAL


def test_struct_layouts_match_header():
    import ctypes as C
    # sizes computed from the C declarations (LP64): padding included
    assert C.sizeof(V.vsie_grid) == 4 * 3 + 4 + 8 + 24
    assert C.sizeof(V.vsie_mesh) == 48
    assert C.sizeof(V.vsie_options) == 4 * 8 + 8 * 3 + 4 * 2 + 4 * 2 + 8 + 4 * 2
    assert C.sizeof(V.vsie_solve_opts) == 4 * 3 + 4 + 8 + 4 + 4
