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


def test_enum_values_match_the_header(lib):
    """Every enum constant of include/sqsm.h that the binding mirrors has the
    header's value."""
    src = open(os.path.join(ROOT, "include", "sqsm.h")).read()
    values = {k: int(v) for k, v in re.findall(r"\bSQSM_([A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    assert {"OK", "CUBATURE", "MODEL_CT_BEARINGS_R"} <= set(values)
    mirrored = [k for k in values if hasattr(lib, k)]
    assert len(mirrored) >= 15
    for k in mirrored:
        assert getattr(lib, k) == values[k], k


def test_ct_model_from_theta_length(lib):
    """Three CT parameters select the shared-noise model, four the model with
    one noise level per sensor; other lengths are refused on the host."""
    import numpy as np
    sensors = np.array([[-1.5, 0.5], [1.0, 1.0]])
    m3, t3 = lib._ct_model(np.log([0.05, 0.01, 0.1]), 0.01, sensors)
    m4, t4 = lib._ct_model(np.log([0.03, 0.01, 0.1, 0.08]), 0.01, sensors)
    assert m3.kind == lib.MODEL_CT_BEARINGS and len(t3) == 3
    assert m4.kind == lib.MODEL_CT_BEARINGS_R and len(t4) == 4
    assert abs(t4[3] - np.log(0.08)) == 0.0 and m4.dt == 0.01
    assert list(m4.sensors) == [-1.5, 0.5, 1.0, 1.0]
    for bad in ([0.0, 0.0], [0.0] * 5):
        with pytest.raises(ValueError):
            lib._ct_model(bad, 0.01, sensors)
