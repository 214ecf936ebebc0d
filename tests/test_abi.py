"""The C-ABI library loads without a GPU and exports every symbol that
include/*.h declares; host-only entry points answer without a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("mond_pm.h", "mond_fno.h")]


def declared_functions():
    names = set()
    for hdr in HEADERS:
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(mond_(?:pm|fno)_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2312_02968_gb300 import binding

    return binding.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2312_02968_gb300 import binding

    assert set(binding.SIGNATURES) == set(declared_functions())


def test_workspace_bytes_host_only(lib):
    from paper_2312_02968_gb300 import binding as B

    n256 = B.workspace_bytes(256, 1, 1.5, 1_000_000)
    assert 1.0e9 < n256 < 3.0e9
    assert B.workspace_bytes(64, 2, 2.0, 2) > B.workspace_bytes(64, 1, 2.0, 2)
    for bad in [(100, 1, 1.0), (256, 3, 1.0), (256, 1, 0.5), (1024, 1, 1.0)]:
        with pytest.raises(B.MondError):
            B.workspace_bytes(bad[0], bad[1], bad[2], 10)


def test_increment_workspace_bytes_host_only(lib):
    # the base deposit (int64) and two float32 vector fields, plus alignment slack
    from paper_2312_02968_gb300 import binding as B

    n = ctypes.c_size_t()
    for side, pad in ((256, 1), (64, 2), (96, 1)):
        assert lib.mond_pm_increment_workspace_bytes(B.Grid(side, pad), ctypes.byref(n)) == 0
        n3 = (side * pad) ** 3
        assert 32 * n3 <= n.value <= 32 * n3 + 1024
    for bad in ((100, 1), (256, 3), (1024, 1), (0, 1)):
        assert lib.mond_pm_increment_workspace_bytes(B.Grid(*bad), ctypes.byref(n)) == -1
    assert lib.mond_pm_increment_workspace_bytes(B.Grid(64, 1), None) == -1
    assert lib.mond_pm_set_increment_workspace(None, None, 0) == -1


def test_create_rejects_bad_arguments_without_touching_the_device(lib):
    from paper_2312_02968_gb300 import binding as B

    h = ctypes.c_void_p()
    rc = lib.mond_pm_create(B.Grid(100, 1), 1.0, 1.0, 1.0, 0, 1.0, None, None, 0, 10, ctypes.byref(h))
    assert rc == -1 and not h.value
    assert b"unsupported" in lib.mond_pm_last_error(None)
    rc = lib.mond_pm_create(B.Grid(64, 1), 64.0, 1.0, 1.0, 0, 1.0, None, ctypes.c_void_p(4096 + 8), 1 << 30, 10,
                            ctypes.byref(h))
    assert rc == -1  # misaligned workspace
