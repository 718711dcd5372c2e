"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, and exports every entry
point that include/usrt.h declares (no compute call: there is no GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2604_15017_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "usrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(us_\w+)\s*\(", src, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = cuda_build.build()
    lib = ctypes.CDLL(path)
    names = declared_entry_points()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_2604_15017_gb300 import usrt

    assert sorted(usrt.EXPORTS) == names


def test_binding_refuses_without_gpu():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2604_15017_gb300 import usrt

    with pytest.raises(Exception):
        usrt.Context(0)
