"""The C-ABI library builds, loads without a GPU, and exports every entry point the header declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(nedf_compose_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2308_04669_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_entry_points()
    assert len(names) >= 18
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native
    assert declared_entry_points() <= set(native.EXPORTS)


def test_last_error_without_handle_is_empty_or_text():
    from paper_2308_04669_gb300 import build
    build.build()
    from paper_2308_04669_gb300 import native
    assert isinstance(native._lib.nedf_compose_last_error(None), bytes)
