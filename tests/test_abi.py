"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declares.  Host-only calls (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2603_12292_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(sr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("sr_create", "sr_destroy", "sr_eval", "sr_predict", "sr_sync"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    assert sorted(binding.EXPORTS) == declared_functions()


def test_status_strings(lib):
    for s, text in [(0, b"ok"), (1, b"invalid argument"), (3, b"device wait timed out")]:
        assert lib.sr_status_string(s) == text


def test_null_context_is_rejected(lib):
    assert lib.sr_eval(None, None, None, None, 1, 8, 0, None, None, 1, 4, 4, 0, None, None) == binding.SR_EINVAL
    assert lib.sr_predict(None, None, None, None, 1, 8, 0, None, 1, 4, 4, None, 4, None) == binding.SR_EINVAL
    assert lib.sr_sync(None) == binding.SR_EINVAL
    assert lib.sr_destroy(None) == binding.SR_OK
    h = ctypes.c_void_p()
    assert lib.sr_create(None, 0, None) == binding.SR_EINVAL
    assert lib.sr_create(ctypes.byref(h), -1, None) == binding.SR_EINVAL
