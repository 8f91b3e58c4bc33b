"""The CUDA library builds for sm_103a and exports every entry point declared in include/css.h.

No compute call is made here (no GPU needed)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib_path():
    from paper_2605_20918_gb300 import build
    return build.build()


def declared_symbols():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        names |= set(re.findall(r"CSS_API[^;(]*?\b(css_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("css_create", "css_destroy", "css_color", "css_color_graph", "css_color_check", "css_color_update",
                 "css_probes", "css_density",
                 "css_density_batch", "css_pbuild", "css_get_info", "css_status_str", "css_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(str(lib_path))
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(str(lib_path))
    lib.css_status_str.restype = ctypes.c_char_p
    lib.css_status_str.argtypes = [ctypes.c_int]
    assert lib.css_status_str(0) == b"CSS_OK"
    assert lib.css_status_str(6) == b"CSS_WARN_BREAKDOWN"


def test_binding_refuses_missing_library(tmp_path):
    import paper_2605_20918_gb300 as css
    with pytest.raises(RuntimeError, match="not found"):
        css.load_library(tmp_path / "nope.so")


def test_binding_constants_match_the_header():
    """The Python binding's precision and flag values are the header's (the C-ABI passes them as
    plain integers)."""
    import paper_2605_20918_gb300 as css
    text = (ROOT / "include" / "css.h").read_text()
    enum = dict(re.findall(r"\b(CSS_(?:FP64|MIXED_FP32|MIXED_3XTF32|FP64_SPLIT))\s*=\s*(\d+)", text))
    assert set(enum) == {"CSS_FP64", "CSS_MIXED_FP32", "CSS_MIXED_3XTF32", "CSS_FP64_SPLIT"}
    for name, val in enum.items():
        assert getattr(css, name) == int(val), name
    for name, val in re.findall(r"#define\s+(CSS_[A-Z_0-9]+)\s+(\d+)u\b", text):
        if hasattr(css, name):
            assert getattr(css, name) == int(val), name


def test_info_struct_matches_the_header():
    """css_get_info writes the header's css_info into the caller's memory: the binding's ctypes
    structure has the same fields, in the same order, with the same C types."""
    from paper_2605_20918_gb300 import _Info
    text = (ROOT / "include" / "css.h").read_text()
    end = text.index("} css_info;")
    body = text[text.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for ctype, names in re.findall(r"(int32_t|int64_t|double)\s+([^;]+);", body):
        for n in names.split(","):
            fields.append((n.strip(), ctype))
    ct = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double}
    assert [(n, ct[t]) for n, t in fields] == [(n, t) for n, t in _Info._fields_]
