"""GPU parity of the paths the benchmark takes at full size and of the boundary's options:
real blocks of real pencils (one solve per pole), GMRES column chunks, split inner
extents in the solve products, locking in Algorithm 1, the ZOLO_EGAP check, the one-call
driver zolo_eigs without gaps, CSR input in device memory and with complex64 values, and
the contour-integral filters -- all through the C ABI against the oracle."""
import ctypes as C

import numpy as np
import pytest

import paper_1701_08935_gb300 as Z
from oracle import apply as AP
from oracle import eigs as E
from oracle import factor as FA
from oracle import filter as F
from gpu_common import case, colrel, dev, host, need_gpu
import synth

pytestmark = pytest.mark.gpu


def _fac(name, r=(2, 2), prec=Z.PREC_FP64, **kw):
    pen, leaf, gaps, lam = case(name)
    flt = Z.Filter(*gaps, *r)
    opts = Z.default_opts(grid=pen.dims, leaf_max=leaf, precision=prec, **kw)
    return pen, gaps, lam, flt, Z.Factor(pen.A, pen.B, flt, opts=opts)


@pytest.mark.parametrize("prec", [Z.PREC_FP64, Z.PREC_MIXED])
def test_real_block_of_real_pencil(prec):
    """Real X of a real pencil: K^-H B x = conj(K^-1 B x) (eq. solve), so the library runs one
    solve per pole and returns a real block; it must equal the complex-arithmetic path and
    the oracle's exact partial fractions."""
    need_gpu()
    pen, gaps, lam, flt, fac = _fac("real2d_40", prec=prec)
    X = synth.random_block(pen.n, 24, 3, complex_=False).astype(np.complex128)
    Yd, st = fac.apply(dev(X))
    Y = host(Yd)
    assert np.all(Y.imag == 0.0)
    ref = AP.apply_exact(pen.A, pen.B, X, F.ZoloFilter(*gaps, 2, 2))
    assert colrel(Y, ref) < 1e-9
    cols_real = fac.stats()["solve_cols"]
    _, _, _, _, fac2 = _fac("real2d_40", prec=prec, real_block=0)
    Y2 = host(fac2.apply(dev(X))[0])
    assert colrel(Y2, ref) < 1e-9
    assert fac2.stats()["solve_cols"] >= 1.9 * cols_real          # two instances per pole there


@pytest.mark.parametrize("prec", [Z.PREC_FP64, Z.PREC_MIXED])
def test_gmres_column_chunks(prec):
    """The benchmark's k = 300 runs GMRES in column chunks, each with its own step count:
    force three chunks of at most 16 columns on k = 40."""
    need_gpu()
    pen, gaps, lam, flt, fac = _fac("cplx3d_12", (2, 3), prec, gmres_chunk=16)
    X = synth.random_block(pen.n, 40, 12)
    Y = host(fac.apply(dev(X))[0])
    assert colrel(Y, AP.apply_exact(pen.A, pen.B, X, F.ZoloFilter(*gaps, 2, 3))) < 1e-9


@pytest.mark.parametrize("prec,tc", [(Z.PREC_FP64, Z.TC_AUTO), (Z.PREC_MIXED, Z.TC_ALWAYS), (Z.PREC_MIXED, Z.TC_OFF)])
def test_split_inner_extent(prec, tc):
    """Solve products whose inner extent is split over several CTAs (atomic accumulation,
    including empty trailing slices): split_k_min = 32 forces it at test size, for the
    complex128 FMA kernel, the tensor-core kernel and the complex64 FMA kernels."""
    need_gpu()
    pen, gaps, lam, flt, fac = _fac("cplx3d_12", prec=prec, split_k_min=32, tensor_core=tc)
    Bk = synth.random_block(pen.n, 19, 5)
    for j, s in enumerate(flt.sigma_hat):
        ref = FA.Solver(pen.A, pen.B, s)
        for herm in (False, True):
            X = host(fac.solve(j, dev(Bk), herm=herm))
            assert colrel(X, ref.solve(Bk, herm=herm)) < 1e-10, (j, herm)


def test_locking_same_pairs_fewer_solves():
    """Locking (footnote of Algorithm 1): the same eigenpairs with fewer solve columns.  The
    composite Zolotarev filter is flat on (a, b), so its Ritz pairs converge together; a
    Gauss-Legendre contour filter is not (R ~ 1/2 near a and b), so pairs near the middle
    converge iterations earlier and are locked (on the oracle: 13 of 20 after 4 iterations)."""
    need_gpu()
    pen, leaf, gaps, lam = case("real2d_40")
    a, b = 0.5 * (gaps[0] + gaps[1]), 0.5 * (gaps[2] + gaps[3])
    out = {}
    for lock in (0, 1):
        flt = Z.ContourFilter(Z.FILTER_CIGQ, a, b, 8)
        fac = Z.Factor(pen.A, pen.B, flt, opts=Z.default_opts(grid=pen.dims, leaf_max=leaf, n_iter_max=10, lock=lock))
        ev, V, res, st, rc = fac.eigs(a, b, 32, X0=dev(synth.random_block(pen.n, 32, 21)))
        assert rc == Z.OK
        inside = lam[(lam > a) & (lam < b)]
        assert np.allclose(ev, inside, rtol=1e-10, atol=1e-12)
        assert np.max(res) <= 1e-10
        Vh = host(V)
        assert np.allclose(Vh.conj().T @ (pen.B @ Vh), np.eye(len(ev)), atol=1e-10)
        out[lock] = (st["n_iter"], fac.stats()["solve_cols"])
    assert out[0][0] >= 3
    assert out[1][1] < out[0][1], out


def test_egap_when_a_gap_holds_an_eigenvalue():
    """Gaps declared around a spot that holds an eigenvalue: the eigenvalue is filtered with
    R ~ 1/2, converges, and ZOLO_EGAP is returned (with the pairs in (a, b) still filled)."""
    need_gpu()
    pen = synth.pencil_2d_real(12, seed=1)
    lam, _ = E.dense_eigs(pen.A, pen.B)
    # true gaps around numbers 20 and 36, then the lower gap widened over eigenvalue 20
    am, ap = lam[18] + 0.5 * (lam[19] - lam[18]), lam[20] - 0.2 * (lam[20] - lam[19])
    bm, bp = lam[35] + 0.3 * (lam[36] - lam[35]), lam[36] - 0.3 * (lam[36] - lam[35])
    assert am < lam[19] < ap
    f = Z.Filter(am, ap, bm, bp, 2, 3)
    fac = Z.Factor(pen.A, pen.B, f, opts=Z.default_opts(grid=pen.dims, leaf_max=8, n_iter_max=4))
    a, b = 0.5 * (am + ap), 0.5 * (bm + bp)
    ev, V, res, st, rc = fac.eigs(a, b, 28)
    assert rc == Z.EGAP
    am2, ap2 = lam[19] + 0.3 * (lam[20] - lam[19]), lam[20] - 0.3 * (lam[20] - lam[19])
    ok = Z.Filter(am2, ap2, bm, bp, 2, 3)
    fac2 = Z.Factor(pen.A, pen.B, ok, opts=Z.default_opts(grid=pen.dims, leaf_max=8, n_iter_max=4))
    ev2, _, _, _, rc2 = fac2.eigs(0.5 * (am2 + ap2), b, 28)
    assert rc2 == Z.OK


def _eigs_call(Acsr, Bcsr, a, b, n_est, spec, opts, n):
    import torch
    cap = 64
    evals, resid = np.zeros(cap), np.zeros(cap)
    V = torch.zeros((n, cap), dtype=torch.complex128, device="cuda")
    nf = C.c_int64(0)
    st = Z.Stats()
    rc = Z.lib.zolo_eigs(C.byref(Acsr), C.byref(Bcsr), a, b, n_est, spec, C.byref(opts), evals.ctypes.data,
                         C.c_void_p(V.data_ptr()), cap, cap, C.byref(nf), resid.ctypes.data, C.byref(st), None)
    m = int(nf.value)
    return rc, evals[:m], resid[:m], V[:, :m]


def test_zolo_eigs_one_call_without_gaps():
    """zolo_eigs with spec = NULL: gaps of gap_rel (b - a) outside (a, b) (the library's gap
    rule); (a, b) placed mid-way in wide spacings of the brute-force spectrum."""
    need_gpu()
    pen = synth.pencil_2d_real(40, seed=1)
    lam, _ = E.dense_eigs(pen.A, pen.B)
    sp = np.diff(lam)
    p = 100 + int(np.argmax(sp[100:110]))
    q = 120 + int(np.argmax(sp[120:130]))
    a, b = 0.5 * (lam[p] + lam[p + 1]), 0.5 * (lam[q] + lam[q + 1])
    g = 1e-2 * (b - a)
    assert lam[p] < a - g and b + g < lam[q + 1]
    hA, hB = Z.HostCsr(pen.A), Z.HostCsr(pen.B)
    opts = Z.default_opts(grid=pen.dims, leaf_max=32, n_iter_max=5, r1=2, r2=3)
    rc, ev, res, V = _eigs_call(hA.s, hB.s, a, b, q - p, None, opts, pen.n)
    assert rc == Z.OK, Z.lib.zolo_last_error()
    inside = lam[(lam > a) & (lam < b)]
    assert len(ev) == len(inside) == q - p
    assert np.allclose(ev, inside, rtol=1e-10)
    assert np.max(E.residuals(pen.A, pen.B, ev, host(V))) <= 1e-10


def _dev_csr(M, dtype):
    """A zolo_csr over device arrays (torch tensors kept alive by the returned tuple)."""
    import torch
    M = M.tocsr()
    M.sort_indices()
    rp = torch.from_numpy(M.indptr.astype(np.int64)).cuda()
    ci = torch.from_numpy(M.indices.astype(np.int32)).cuda()
    if dtype == Z.C64:
        v = torch.from_numpy(M.data.astype(np.complex64)).cuda()
    elif dtype == Z.C128:
        v = torch.from_numpy(M.data.astype(np.complex128)).cuda()
    else:
        v = torch.from_numpy(M.data.real.astype(np.float64)).cuda()
    s = Z.Csr(M.shape[0], M.nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), dtype, Z.DEVICE)
    return s, (rp, ci, v)


@pytest.mark.parametrize("dtype", ["C128", "C64", "R64"])
def test_device_csr_input(dtype):
    """The same pencil given in device memory (complex128, complex64 or double values) gives
    the same eigenpairs as the host CSR of the same values."""
    need_gpu()
    pen, leaf, gaps, lam = case("cplx3d_9" if dtype != "R64" else "real2d_12")
    A, B = pen.A, pen.B
    if dtype == "C64":                   # values exactly representable in complex64
        A = A.astype(np.complex64).astype(np.complex128)
        B = B.astype(np.complex64).astype(np.complex128)
        lam, _ = E.dense_eigs(A, B)
        win = (40, 70)
        gaps = (lam[win[0] - 1], lam[win[0]], lam[win[1] - 1], lam[win[1]])
    a, b = 0.5 * (gaps[0] + gaps[1]), 0.5 * (gaps[2] + gaps[3])
    spec = Z.FilterSpec(*gaps, 2, 3, 0.0)
    opts = Z.default_opts(grid=pen.dims, leaf_max=leaf, n_iter_max=6)
    n_est = int(np.sum((lam > a) & (lam < b)))
    dA, keepA = _dev_csr(A, getattr(Z, dtype))
    dB, keepB = _dev_csr(B, getattr(Z, dtype))
    rc, ev, res, V = _eigs_call(dA, dB, a, b, n_est, C.byref(spec), opts, pen.n)
    assert rc == Z.OK, Z.lib.zolo_last_error()
    hA, hB = Z.HostCsr(A), Z.HostCsr(B)
    rc2, ev2, res2, V2 = _eigs_call(hA.s, hB.s, a, b, n_est, C.byref(spec), opts, pen.n)
    assert rc2 == Z.OK
    assert np.allclose(ev, ev2, rtol=1e-13)
    assert np.allclose(ev, lam[(lam > a) & (lam < b)], rtol=1e-10)


@pytest.mark.parametrize("kind", ["CITZ", "CIGQ"])
def test_contour_filter_apply(kind):
    """Contour-integral filters run through the factored-pole path (no GMRES)."""
    need_gpu()
    pen, leaf, gaps, lam = case("cplx3d_9")
    a, b = 0.5 * (gaps[0] + gaps[1]), 0.5 * (gaps[2] + gaps[3])
    flt = Z.ContourFilter(getattr(Z, "FILTER_" + kind), a, b, 8)
    fac = Z.Factor(pen.A, pen.B, flt, opts=Z.default_opts(grid=pen.dims, leaf_max=leaf))
    X = synth.random_block(pen.n, 21, 2)
    Y = host(fac.apply(dev(X))[0])
    ref = AP.apply_contour(pen.A, pen.B, X, F.ContourFilter(kind, a, b, 8))
    assert colrel(Y, ref) < 1e-10
    assert colrel(Y, AP.apply_dense(pen.A, pen.B, X, F.ContourFilter(kind, a, b, 8))) < 1e-9


def test_contour_filter_eigs():
    """Algorithm 1 with a CIGQ(16) filter (FEAST-like poles through the same kernels)
    finds the same eigenpairs as the brute force."""
    need_gpu()
    pen, leaf, gaps, lam = case("real2d_12")
    a, b = 0.5 * (gaps[0] + gaps[1]), 0.5 * (gaps[2] + gaps[3])
    flt = Z.ContourFilter(Z.FILTER_CIGQ, a, b, 16)
    fac = Z.Factor(pen.A, pen.B, flt, opts=Z.default_opts(grid=pen.dims, leaf_max=leaf, n_iter_max=12))
    ev, V, res, st, rc = fac.eigs(a, b, 28)
    assert rc == Z.OK
    assert np.allclose(ev, lam[(lam > a) & (lam < b)], rtol=1e-10)
    assert np.max(res) <= 1e-10


@pytest.mark.parametrize("prec", [Z.PREC_FP64, Z.PREC_MIXED])
def test_example1_hamiltonian_smallest_88(prec):
    """Example 1 of Section 3.1 at N = 12^3: the smallest 88 eigenpairs of the Gaussian-well
    Hamiltonian with a- = -inf, a+ = lam_1, b- = lam_88, b+ = lam_89 (the true eigenvalues as
    input), r = (4, 4), subspace dimension 89 and tolerance 1e-8 reach every pair in ONE
    subspace iteration (n_iter = 1 in Table 1) when GMRES runs to 1e-12 (the paper's errors of
    ~1e-15 after one iteration imply a GMRES run to near machine precision); the eigenvalues
    match the dense eigensolver and n_solv = r n_ss n_iter n_gmres (Section 3)."""
    need_gpu()
    pen = synth.hamiltonian_wells(12, 2)
    lam = np.linalg.eigvalsh(pen.A.toarray())
    l1, l88, l89 = lam[0], lam[87], lam[88]
    assert 1e-4 <= (l89 - l88) / (l88 - l1) <= 1e-3      # the paper's selection rule holds for this seed
    flt = Z.Filter(-np.inf, l1, l88, l89, 4, 4)
    opts = Z.default_opts(grid=pen.dims, leaf_max=32, precision=prec, tol=1e-8, gmres_tol=1e-12,
                          gmres_m_max=100, n_iter_max=1)
    fac = Z.Factor(pen.A, pen.B, flt, opts=opts)
    a, b = l1 - 0.5 * (l88 - l1), 0.5 * (l88 + l89)
    ev, V, res, st, rc = fac.eigs(a, b, 89)
    assert rc == Z.OK and st["n_iter"] == 1
    assert len(ev) == 88
    assert np.allclose(np.sort(ev), lam[:88], rtol=1e-10, atol=0)
    assert np.max(res) <= 1e-8 and st["relerr"] <= 1e-8
    assert st["n_solv"] == 4 * 89 * st["n_gmres"]
