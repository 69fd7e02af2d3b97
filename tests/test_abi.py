"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
that include/vv10.h declares (no compute calls are made here)."""
import os
import re
import subprocess

import pytest

from paper_2208_14639_gb300 import build, vv10

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vv10.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vv10_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    return build.build()


def test_header_declares_the_binding_names():
    assert sorted(vv10.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vv10_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing


def test_library_loads_and_reports_status_strings(lib_path):
    lib = vv10.load()
    assert vv10.vv10_status_string(vv10.VV10_OK) == "ok"
    assert "invalid" in vv10.vv10_status_string(vv10.VV10_ERR_INVALID_ARG)
    assert vv10.vv10_last_error(None) == "null handle"
    assert lib is vv10.load()


def test_create_fails_cleanly_without_gpu(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(vv10.VV10Error) as ei:
        vv10.vv10_create(0)
    assert ei.value.status in (vv10.VV10_ERR_CUDA, vv10.VV10_ERR_INVALID_ARG)
