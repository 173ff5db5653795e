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


def test_noalloc_argument_errors_before_any_cuda_call(lib):
    """The no-allocation smoother validates its arguments on the host before
    any CUDA call (so this runs without a GPU): a pointer that is not a
    multiple of its element size, a negative stride, a null output, n < 1
    and an unknown dtype are refused."""
    f = lib.lib.sqsm_lgssm_smooth_noalloc
    good = 0x10000                      # never dereferenced: validation fails first
    ptrs = [good] * 13

    def call(dtype=0, n=10, ptrs=ptrs, strides=(25, 5, 25, 10, 2, 4), ll=good):
        args = []
        for p, s in zip(ptrs[:6], strides):
            args += [p, s]
        return f(dtype, 5, 2, n, *args, *ptrs[6:9], *ptrs[9:13], ll, None)

    for i in range(13):
        bad = list(ptrs)
        bad[i] = good + 2               # misaligned for float and double
        assert call(ptrs=bad) == lib.ERR_INVALID_ARG, i
        assert call(dtype=1, ptrs=bad) == lib.ERR_INVALID_ARG, i
    bad = list(ptrs)
    bad[0] = good + 4                   # aligned for float, not for double
    assert call(dtype=1, ptrs=bad) == lib.ERR_INVALID_ARG
    assert call(ll=good + 4) == lib.ERR_INVALID_ARG
    assert call(strides=(25, 5, 25, 10, 2, -4)) == lib.ERR_INVALID_ARG
    nul = list(ptrs)
    nul[10] = None                      # Nf
    assert call(ptrs=nul) == lib.ERR_INVALID_ARG
    assert call(n=0) == lib.ERR_INVALID_ARG
    assert call(dtype=2) == lib.ERR_INVALID_ARG
    assert f(0, 7, 7, 10, *([good, 0] * 6), *([good] * 7), good, None) == lib.ERR_UNSUPPORTED
