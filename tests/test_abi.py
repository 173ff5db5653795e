"""The C-ABI library loads without a GPU and exports every function that
include/sqsm.h declares; argument errors are reported before any CUDA work."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sqsm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(sqsm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    path = os.path.join(ROOT, "paper_2207_00426_gb300", "libsqsm.so")
    if not os.path.exists(path):
        import __graft_entry__
        __graft_entry__.build()
    from paper_2207_00426_gb300 import binding
    return binding


def test_header_declarations_found():
    names = _declared()
    assert "sqsm_lgssm_smooth" in names and "sqsm_ipls_smooth" in names
    assert len(names) >= 8


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib.lib, name), name
    assert sorted(lib.EXPORTED) == _declared()


def test_null_context_is_rejected(lib):
    assert lib.lib.sqsm_lgssm_smooth(None, 0, 4, 2, 10, *([None, 0] * 6), None, None, None,
                                     None, None, None, None, None, None) == lib.ERR_INVALID_ARG
    assert lib.lib.sqsm_destroy(None) == lib.OK
    assert lib.lib.sqsm_last_error(None) == b""


def test_supported_shapes(lib):
    assert lib.supported_shape(5, 2) and lib.supported_shape(4, 2)
    assert not lib.supported_shape(7, 7)
