"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "odwf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|double|const char\*)\s+(\w+)\s*\(", src, re.M)))


def test_header_matches_binding_exports():
    from paper_1710_09621_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_library_builds_and_exports_every_symbol():
    from paper_1710_09621_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    import ctypes
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1710_09621_gb300 import binding
    with pytest.raises(RuntimeError):
        binding._lib = None
        binding.load_library(str(tmp_path / "missing.so"))
    binding._lib = None
