"""The C-ABI library builds, loads and exports every function its header declares.

Runs without a GPU: only symbol lookup, no compute call.
"""
import ctypes
import os

import pytest

from paper_1704_06258_gb300 import binding, build as _build


@pytest.fixture(scope="module")
def built():
    return _build.build()


def test_every_declared_function_is_exported(built):
    names = set()
    for f in os.listdir(os.path.join(_build.ROOT, "include")):
        if f.endswith(".h"):
            names |= set(binding.header_functions(os.path.join(_build.ROOT, "include", f)))
    assert "usaphmp_create" in names and "usaphmp_solve" in names and "usaphmp_eval" in names
    L = ctypes.CDLL(built)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_every_header_function(built):
    names = set(binding.header_functions())
    assert names <= set(binding._SIGS), sorted(names - set(binding._SIGS))
