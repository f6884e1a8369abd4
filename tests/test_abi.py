"""The C ABI: every function declared in include/zolo.h is exported, and the host-side
argument checks return the documented status codes (no GPU needed)."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import paper_1701_08935_gb300 as Z
import synth

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "zolo.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zolo_[a-z_]+)\s*\(", src)))


def test_every_declared_function_is_exported():
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(Z.lib, n), n
    assert set(names) == set(Z.EXPORTED)


def test_version_and_strerror():
    assert Z.lib.zolo_version() >= 100
    for s in range(9):
        assert Z.lib.zolo_strerror(s)


def test_non_hermitian_rejected_before_any_device_work():
    p = synth.pencil_2d_real(6, seed=1)
    A = p.A.tolil()
    A[0, 1] = A[0, 1] + 0.5
    f = Z.Filter(0.0, 0.5, 1.0, 1.5, 2, 2)
    with pytest.raises(Z.ZoloError) as e:
        Z.Factor(A.tocsr(), p.B, f, opts=Z.default_opts(grid=(6, 6)), stream=0)
    assert e.value.status == Z.ENOTHERM


def test_bad_csr_rejected():
    p = synth.pencil_2d_real(6, seed=1)
    A = p.A.copy()
    A.indices = A.indices.copy()
    A.indices[0] = 99
    with pytest.raises(Z.ZoloError) as e:
        Z.Symbolic(A, p.B, Z.default_opts(grid=(6, 6)))
    assert e.value.status == Z.EINVAL
    A = p.A.copy()
    A.data = A.data.copy()
    A.data[3] = np.nan
    with pytest.raises(Z.ZoloError):
        Z.Symbolic(A, p.B, Z.default_opts(grid=(6, 6)))


def test_missing_diagonal_rejected():
    A = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 2.0]]))
    A.eliminate_zeros()
    B = sp.identity(2, format="csr")
    with pytest.raises(Z.ZoloError):
        Z.Symbolic(A, B, Z.default_opts())


def test_bad_tensor_core_policy_rejected_before_any_device_work():
    p = synth.pencil_2d_real(6, seed=1)
    f = Z.Filter(0.0, 0.5, 1.0, 1.5, 2, 2)
    for bad in (-1, 3):
        with pytest.raises(Z.ZoloError) as e:
            Z.Factor(p.A, p.B, f, opts=Z.default_opts(grid=(6, 6), precision=Z.PREC_MIXED, tensor_core=bad),
                     stream=0)
        assert e.value.status == Z.EINVAL


def test_slices_reject_bad_bounds_before_any_device_work():
    import ctypes as C
    p = synth.pencil_2d_real(6, seed=1)
    hA, hB = Z.HostCsr(p.A), Z.HostCsr(p.B)
    o = Z.default_opts(grid=(6, 6))
    for bounds in ([0.5, 0.5, 1.0], [0.0, float("nan"), 1.0], [1.0, 0.5]):
        bd = np.asarray(bounds, dtype=np.float64)
        ev = np.zeros(4)
        nf = C.c_int64(0)
        rc = Z.lib.zolo_eigs_slices(C.byref(hA.s), C.byref(hB.s), len(bd) - 1, bd.ctypes.data, C.byref(o),
                                    ev.ctypes.data, C.c_void_p(1), 4, 4, C.byref(nf), None, None, None, None)
        assert rc == Z.EINVAL


def test_short_blocks_refused_before_any_launch():
    """The binding checks block shapes itself (the C ABI receives bare pointers)."""
    Z.check_block((10, 3), "X", 10)
    Z.check_block((10, 3), "out", 10, 3)
    for shape, k in (((9, 3), None), ((10, 2), 3), ((10, 0), None), ((10,), None)):
        with pytest.raises(ValueError):
            Z.check_block(shape, "X", 10, k)
