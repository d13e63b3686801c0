"""The C ABI library loads and exports every entry point include/*.h declares (CPU only, no compute)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(?:tc_status|const char\s*\*|uint64_t|void|int)\s+\**\s*(tc_\w+)\s*\(", text):
            syms.add(m.group(1))
    return syms


@pytest.fixture(scope="module")
def lib():
    import paper_2401_01607_gb300 as pkg
    path = pkg.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("tc_open_stream", "tc_set_ir", "tc_push_block", "tc_close", "tc_flush", "tc_set_ir_at"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in sorted(declared_symbols()) if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2401_01607_gb300 import capi
    missing = [s for s in sorted(declared_symbols()) if not hasattr(capi, s)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    lib.tc_status_str.restype = ctypes.c_char_p
    assert lib.tc_status_str(0) == b"TC_OK"
    assert lib.tc_status_str(5) == b"TC_ETIMEOUT"


def test_null_arguments_are_rejected_without_gpu(lib):
    # Argument checks run before any CUDA call.
    lib.tc_last_error.restype = ctypes.c_char_p
    assert lib.tc_open_stream(ctypes.c_size_t(0), ctypes.c_size_t(64), None) == 1
    assert lib.tc_push_block(None, None, ctypes.c_size_t(1), None) == 1
    assert lib.tc_close(None) == 0


def test_inject_hook_arguments_without_gpu(lib):
    # Arming and disarming the test hook touches no device.
    assert lib.tc_test_inject(99, 1) == 1
    assert lib.tc_test_inject(1, -1) == 1
    assert lib.tc_test_inject(1, 2) == 0 and lib.tc_test_inject(1, 0) == 0
    assert lib.tc_test_inject(2, 0) == 0


def test_product_package_never_reaches_the_oracle():
    # The library's Python side (binding, build, generators) imports, loads or runs nothing under oracle/.
    import ast
    pkg_dir = os.path.join(ROOT, "paper_2401_01607_gb300")
    for path in glob.glob(os.path.join(pkg_dir, "*.py")):
        tree = ast.parse(open(path).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
            if isinstance(node, ast.ImportFrom):
                assert "oracle" not in (node.module or ""), path
                assert not any(a.name == "oracle" for a in node.names), path
        assert "liboracle" not in open(path).read(), path
    for path in glob.glob(os.path.join(pkg_dir, "csrc", "*")):
        assert "oracle" not in open(path).read().lower(), path


def test_binding_raises_when_the_library_is_missing(monkeypatch, tmp_path):
    # No CPU fallback: without libtaches.so every entry point fails loudly.
    from paper_2401_01607_gb300 import capi
    monkeypatch.setattr(capi, "_lib", None)
    monkeypatch.setattr(capi, "lib_path", lambda: str(tmp_path / "libtaches.so"))
    with pytest.raises(RuntimeError, match="not built"):
        capi.tc_open_stream(1000, 64)
    with pytest.raises(RuntimeError, match="not built"):
        capi.tc_status_str(0)
