"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/ws_prox.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ws_prox.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:ws_status|void|const char\*)\s+(ws_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ws_prox", "ws_prox_batched", "ws_prox_backward", "ws_prox_backward_batched",
                     "ws_plan_create", "ws_ctx_create", "ws_get_status"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2311_03096_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2311_03096_gb300 import ws
    with pytest.raises(RuntimeError):
        ws.Context(0)


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2311_03096_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "ws_oracle" not in text, f
