"""The C-ABI library loads without a GPU and exports every entry point that
include/gmapp.h declares; the Python binding binds all of them."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        # function declarations: <type> <name>(...);  (not typedefs)
        for m in re.finditer(r"^\s*(?!typedef)[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;",
                             src, flags=re.M):
            names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for core in ("filter_cloud", "rollout_agents", "score_and_select", "gmapp_create",
                 "gmapp_destroy", "gmapp_sync"):
        assert core in names


def test_library_exports_every_declared_symbol():
    from paper_2606_12579_b300 import _abi, build
    build.build()
    lib = ctypes.CDLL(_abi.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2606_12579_b300 import _abi
    assert set(_declared()) == set(_abi.PROTOTYPES), set(_declared()) ^ set(_abi.PROTOTYPES)
    _abi.load()


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2606_12579_b300 as gm
    with pytest.raises(RuntimeError):
        gm.Context(0)
