"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/pasm.h declares, and the host-side validation rejects malformed
inputs before any device work."""
import ctypes

import numpy as np
import pytest
import scipy.sparse as sp

import meshgen as mg


@pytest.fixture(scope="module")
def capi():
    from paper_1908_10251_gb300 import build, capi
    build.build()
    capi.load_library()
    return capi


def test_header_symbols_exported(capi):
    names = capi.header_symbols()
    assert "pasm_setup" in names and "pasm_step" in names and "pasm_solve" in names
    lib = ctypes.CDLL(capi.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name


def test_default_opts(capi):
    o = capi.pasm_default_opts()
    assert o.omega == pytest.approx(2.0 / 3.0)
    assert (o.nu_pre, o.nu_post, o.cycles_per_step) == (2, 2, 2)
    assert o.precision == capi.PASM_FP64 and o.score_norm == capi.PASM_SCORE_A


def test_opts_layout_matches_the_header(capi):
    """pasm_default_opts writes exactly the binding's pasm_opts: bytes past it
    stay untouched, and every field after the integer block, the trailing
    float64 res_tol included, has its documented default."""
    size = ctypes.sizeof(capi.pasm_opts)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    capi.load_library().pasm_default_opts(ctypes.cast(buf, ctypes.POINTER(capi.pasm_opts)))
    assert all(b == 0xAB for b in bytes(buf)[size:])
    o = capi.pasm_opts.from_buffer_copy(bytes(buf)[:size])
    assert o.autotune == 1 and o.res_tol == 0.0 and abs(o.omega - 2.0 / 3.0) < 1e-15


def test_strerror(capi):
    assert capi.pasm_strerror(0) == "success"
    assert "coarse" in capi.pasm_strerror(capi.PASM_EK_TOO_BIG)
    assert capi.pasm_strerror(999) == "unknown status"


def _levels():
    H = mg.build_hierarchy(2, 16, 4)
    return [lv.A.copy() for lv in H.levels], [lv.M.copy() for lv in H.levels], [P.copy() for P in H.P]


@pytest.mark.parametrize("case", ["col_out_of_range", "row_ptr_decreasing", "shape_mismatch", "zero_diagonal",
                                  "p_shape"])
def test_setup_rejects_malformed_hierarchy(capi, case):
    """Malformed CSR or inconsistent shapes return PASM_EINVAL from host-side
    validation, before any CUDA call."""
    A, M, P = _levels()
    if case == "col_out_of_range":
        A[1].indices[3] = A[1].shape[1] + 5
    elif case == "row_ptr_decreasing":
        A[2].indptr[5], A[2].indptr[6] = A[2].indptr[6], A[2].indptr[5]
    elif case == "shape_mismatch":
        M[1] = sp.csr_matrix(M[1].toarray()[:-1, :-1])
    elif case == "zero_diagonal":
        A[0] = A[0].tolil(); A[0][2, 2] = 0.0; A[0] = A[0].tocsr()
    elif case == "p_shape":
        P[0] = sp.csr_matrix(P[0].toarray()[:, :-1])
    with pytest.raises(capi.PasmError) as ei:
        capi.pasm_setup(A, M, P)
    assert ei.value.code == capi.PASM_EINVAL


def test_setup_rejects_bad_options(capi):
    A, M, P = _levels()
    for field, val in (("omega", 0.0), ("cycles_per_step", 0), ("precision", 7), ("nu_pre", -1)):
        with pytest.raises(capi.PasmError) as ei:
            capi.pasm_setup(A, M, P, capi.pasm_default_opts(**{field: val}))
        assert ei.value.code == capi.PASM_EINVAL


def test_binding_rejects_wrong_dtype(capi):
    with pytest.raises(TypeError):
        capi._ptr(np.zeros(3, dtype=np.float32))
    with pytest.raises(TypeError):
        capi._ptr(np.zeros((4, 4))[:, ::2])
