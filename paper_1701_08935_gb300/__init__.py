"""GB300 Zolotarev-filter interior eigensolver: Python binding of libzolo.so.

A thin ctypes layer over the C ABI declared in ``include/zolo.h`` (Li & Yang,
arXiv:1701.08935): it converts arguments (scipy CSR matrices, torch CUDA tensors,
streams) and returns results.  Every step of the computation runs in the library's
own CUDA kernels (or, for the filter coefficients and the ordering, in its host
C++ code).  There is no Python or CPU fallback: importing this package fails if
the compiled library is missing -- build it with ``python paper_1701_08935_gb300/build.py``.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libzolo.so")
if not os.path.exists(_LIBPATH):
    raise ImportError(f"{_LIBPATH} is missing: build it with `python paper_1701_08935_gb300/build.py` "
                      "(the package has no fallback path)")
lib = C.CDLL(_LIBPATH)

OK, EINVAL, ENOTHERM, ENOMEM, ESINGULAR, ENOCONV, ETIMEOUT, ECUDA, EGAP = range(9)
FILTER_ZOLO, FILTER_CITZ, FILTER_CIGQ = 0, 1, 2
R64, C128, C64 = 1, 2, 3
HOST, DEVICE = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
TC_AUTO, TC_OFF, TC_ALWAYS = 0, 1, 2
MAX_R = 16

_i32, _i64, _u64, _dbl, _vp = C.c_int32, C.c_int64, C.c_uint64, C.c_double, C.c_void_p


class ZoloError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib.zolo_last_error().decode()
        super().__init__(f"{where}: {lib.zolo_strerror(status).decode()} ({status}): {msg}")


class Csr(C.Structure):
    _fields_ = [("n", _i64), ("nnz", _i64), ("row_ptr", _vp), ("col_idx", _vp), ("val", _vp),
                ("dtype", _i32), ("mem", _i32)]


class FilterSpec(C.Structure):
    _fields_ = [("a_minus", _dbl), ("a_plus", _dbl), ("b_minus", _dbl), ("b_plus", _dbl),
                ("r1", _i32), ("r2", _i32), ("eps", _dbl)]


class FilterInfo(C.Structure):
    _fields_ = [("alpha", _dbl), ("beta", _dbl), ("gamma", _dbl), ("ell1", _dbl), ("ell2", _dbl),
                ("delta1", _dbl), ("delta0", _dbl), ("r1", _i32), ("r2", _i32), ("M_hat", _dbl),
                ("const_hat", _dbl), ("a_hat", _dbl * MAX_R), ("c_hat", _dbl * MAX_R),
                ("sigma_hat", _dbl * (2 * MAX_R)), ("w_hat", _dbl * (2 * MAX_R)), ("M", _dbl),
                ("a", _dbl * MAX_R), ("c", _dbl * MAX_R), ("gap", _dbl * 4), ("kind", _i32), ("npoles", _i32)]


class Opts(C.Structure):
    _fields_ = [("grid", _i32 * 3), ("leaf_max", _i32), ("precision", _i32), ("gmres_m_max", _i32),
                ("gmres_tol", _dbl), ("refine_max", _i32), ("refine_tol", _dbl), ("n_iter_max", _i32),
                ("tol", _dbl), ("drop_tol", _dbl), ("k", _i32), ("r1", _i32), ("r2", _i32),
                ("gap_rel", _dbl), ("seed", _u64), ("verbose", _i32), ("tensor_core", _i32),
                ("gmres_chunk", _i32), ("split_k_min", _i32), ("real_block", _i32), ("lock", _i32)]


class Stats(C.Structure):
    _fields_ = [("n_iter", _i32), ("n_gmres", _i32), ("n_solv", _i64), ("n_refine_max", _i32),
                ("n_found", _i32), ("gmres_res", _dbl), ("max_resid", _dbl), ("relerr", _dbl),
                ("t_factor_ms", _dbl), ("t_apply_ms", _dbl), ("t_rr_ms", _dbl), ("t_total_ms", _dbl),
                ("min_pivot", _dbl), ("flops_factor", _dbl), ("flops_solve", _dbl), ("solve_cols", _i64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SymInfo(C.Structure):
    _fields_ = [("n", _i64), ("nnodes", _i64), ("nlevels", _i64), ("nnz_factor", _i64),
                ("front_entries", _i64), ("update_rows", _i64), ("max_front", _i32),
                ("max_pivots", _i32), ("flops_lu", _dbl)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_P = C.POINTER
_sig("zolo_strerror", C.c_char_p, [C.c_int])
_sig("zolo_last_error", C.c_char_p, [])
_sig("zolo_version", C.c_int, [])
_sig("zolo_opts_default", None, [_P(Opts)])
_sig("zolo_filter_build", C.c_int, [_P(FilterSpec), _P(_vp)])
_sig("zolo_filter_get_info", C.c_int, [_vp, _P(FilterInfo)])
_sig("zolo_filter_eval", C.c_int, [_vp, _i64, _vp, _vp])
_sig("zolo_filter_destroy", None, [_vp])
_sig("zolo_filter_table", C.c_int, [_P(FilterSpec), _i32, _vp])
_sig("zolo_filter_build_contour", C.c_int, [_i32, _dbl, _dbl, _i32, _P(_vp)])
_sig("zolo_analyze", C.c_int, [_P(Csr), _P(Csr), _P(Opts), _P(_vp)])
_sig("zolo_symbolic_get_info", C.c_int, [_vp, _P(SymInfo)])
_sig("zolo_symbolic_export", C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp])
_sig("zolo_symbolic_destroy", None, [_vp])
_sig("zolo_factor", C.c_int, [_P(Csr), _P(Csr), _vp, _vp, _P(Opts), _vp, _P(_vp)])
_sig("zolo_refactor", C.c_int, [_vp, _vp])
_sig("zolo_inertia", C.c_int, [_P(Csr), _P(Csr), _vp, _P(Opts), _i32, _vp, _vp, _vp])
_sig("zolo_profile_begin", C.c_int, [_i32])
_sig("zolo_profile_end", C.c_int, [_vp, _P(_i64), _P(_i64), _P(_dbl), _P(_dbl)])
_sig("zolo_profile_tc", C.c_int, [_P(_i64), _P(_dbl), _P(_dbl)])
_sig("zolo_profile_bytes", C.c_int, [_P(_dbl), _P(_dbl)])
_sig("zolo_factor_destroy", None, [_vp])
_sig("zolo_factor_get_stats", C.c_int, [_vp, _P(Stats)])
_sig("zolo_solve", C.c_int, [_vp, _i32, _i32, _i64, _vp, _i64, _vp, _i64, _vp])
_sig("zolo_solve_noalloc", C.c_int, [_vp, _i32, _i32, _i64, _vp, _i64, _vp, _i64, _vp])
_sig("zolo_matmul", C.c_int, [_vp, _i32, _i64, _vp, _i64, _vp, _i64, _vp])
_sig("zolo_apply_inner", C.c_int, [_vp, _i64, _vp, _i64, _vp, _i64, _vp])
_sig("zolo_apply", C.c_int, [_vp, _i64, _vp, _i64, _vp, _i64, _P(Stats), _vp])
_sig("zolo_eigs_factored", C.c_int, [_vp, _dbl, _dbl, _i64, _vp, _vp, _vp, _i64, _i64, _P(_i64), _vp,
                                     _P(Stats), _vp])
_sig("zolo_eigs", C.c_int, [_P(Csr), _P(Csr), _dbl, _dbl, _i64, _P(FilterSpec), _P(Opts), _vp, _vp, _i64,
                            _i64, _P(_i64), _vp, _P(Stats), _vp])
_sig("zolo_eigs_slices", C.c_int, [_P(Csr), _P(Csr), C.c_int32, _vp, _P(Opts), _vp, _vp, _i64, _i64, _P(_i64), _vp,
                                   _vp, _P(Stats), _vp])

EXPORTED = ["zolo_opts_default", "zolo_strerror", "zolo_last_error", "zolo_version", "zolo_filter_build",
            "zolo_filter_table", "zolo_filter_build_contour",
            "zolo_filter_get_info", "zolo_filter_eval", "zolo_filter_destroy", "zolo_analyze",
            "zolo_symbolic_get_info", "zolo_symbolic_export", "zolo_symbolic_destroy", "zolo_factor",
            "zolo_refactor", "zolo_inertia", "zolo_solve_noalloc", "zolo_profile_begin", "zolo_profile_end",
            "zolo_profile_tc", "zolo_profile_bytes", "zolo_factor_destroy", "zolo_factor_get_stats", "zolo_solve", "zolo_matmul",
            "zolo_apply_inner", "zolo_apply", "zolo_eigs_factored", "zolo_eigs", "zolo_eigs_slices"]


def _check(st, where):
    if st != OK:
        raise ZoloError(st, where)


def default_opts(**kw):
    o = Opts()
    lib.zolo_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "grid":
            g = list(v) + [1] * (3 - len(v))
            o.grid[0], o.grid[1], o.grid[2] = int(g[0]), int(g[1]), int(g[2])
        else:
            setattr(o, k, v)
    return o


class HostCsr:
    """Keeps the numpy arrays of a scipy CSR matrix alive and exposes a zolo_csr."""

    def __init__(self, M):
        M = M.tocsr()
        M.sort_indices()
        self.rp = np.ascontiguousarray(M.indptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(M.indices, dtype=np.int32)
        if np.iscomplexobj(M.data):
            self.val = np.ascontiguousarray(M.data, dtype=np.complex128)
            dt = C128
        else:
            self.val = np.ascontiguousarray(M.data, dtype=np.float64)
            dt = R64
        self.s = Csr(M.shape[0], len(self.ci), self.rp.ctypes.data, self.ci.ctypes.data, self.val.ctypes.data, dt, 0)


class Filter:
    """R_ab of eq. R2 with every constant of Algorithm 2's filter-construction steps (host-built)."""

    def __init__(self, a_minus, a_plus, b_minus, b_plus, r1=2, r2=2, eps=0.0):
        spec = FilterSpec(a_minus, a_plus, b_minus, b_plus, r1, r2, eps)
        h = _vp()
        _check(lib.zolo_filter_build(C.byref(spec), C.byref(h)), "zolo_filter_build")
        self._init_from(h)

    def _init_from(self, h):
        self.h = h
        inf = FilterInfo()
        _check(lib.zolo_filter_get_info(h, C.byref(inf)), "zolo_filter_get_info")
        self.info = inf
        r1, r2 = inf.r1, inf.r2
        self.r1, self.r2 = r1, r2
        self.sigma_hat = np.array(inf.sigma_hat[:2 * r1:2]) + 1j * np.array(inf.sigma_hat[1:2 * r1:2])
        self.w_hat = np.array(inf.w_hat[:2 * r1:2]) + 1j * np.array(inf.w_hat[1:2 * r1:2])
        self.a_hat = np.array(inf.a_hat[:r1])
        self.c_hat = np.array(inf.c_hat[:r1])
        self.a = np.array(inf.a[:r2])
        self.c = np.array(inf.c[:r2])

    def __call__(self, x):
        x = np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64)))
        out = np.empty_like(x)
        _check(lib.zolo_filter_eval(self.h, len(x), x.ctypes.data, out.ctypes.data), "zolo_filter_eval")
        return out

    def __del__(self):
        if getattr(self, "h", None):
            lib.zolo_filter_destroy(self.h)
            self.h = None


def filter_table(a_minus, a_plus, b_minus, b_plus, rmax):
    """delta0 of R_ab for every order pair: table[r1 - 1, r2 - 1] (Remark after Algorithm 2)."""
    spec = FilterSpec(a_minus, a_plus, b_minus, b_plus, 0, 0, 0.0)
    out = np.zeros(rmax * rmax)
    _check(lib.zolo_filter_table(C.byref(spec), int(rmax), out.ctypes.data), "zolo_filter_table")
    return out.reshape(rmax, rmax)


class ContourFilter(Filter):
    """Contour-integral filter (eq. contourintegral) on the circle through a and b:
    kind FILTER_CITZ (trapezoidal rule) or FILTER_CIGQ (Gauss-Legendre), npoles points."""

    def __init__(self, kind, a, b, npoles):
        h = _vp()
        _check(lib.zolo_filter_build_contour(int(kind), float(a), float(b), int(npoles), C.byref(h)),
               "zolo_filter_build_contour")
        self._init_from(h)


class Symbolic:
    """Nested-dissection ordering and front structures (host)."""

    def __init__(self, A, B, opts=None):
        self._A, self._B = HostCsr(A), HostCsr(B)
        o = opts if opts is not None else default_opts()
        h = _vp()
        _check(lib.zolo_analyze(C.byref(self._A.s), C.byref(self._B.s), C.byref(o), C.byref(h)), "zolo_analyze")
        self.h = h
        inf = SymInfo()
        _check(lib.zolo_symbolic_get_info(h, C.byref(inf)), "zolo_symbolic_get_info")
        self.info = inf.as_dict()

    def export(self):
        n, nn = self.info["n"], self.info["nnodes"]
        perm = np.empty(n, np.int32)
        first = np.empty(nn, np.int32)
        npiv = np.empty(nn, np.int32)
        parent = np.empty(nn, np.int32)
        uptr = np.empty(nn + 1, np.int64)
        _check(lib.zolo_symbolic_export(self.h, perm.ctypes.data, first.ctypes.data, npiv.ctypes.data,
                                        parent.ctypes.data, uptr.ctypes.data, None), "zolo_symbolic_export")
        urows = np.empty(int(uptr[-1]), np.int32)
        _check(lib.zolo_symbolic_export(self.h, None, None, None, None, None, urows.ctypes.data),
               "zolo_symbolic_export")
        return {"perm": perm, "first": first, "npiv": npiv, "parent": parent, "uptr": uptr, "urows": urows}

    def __del__(self):
        if getattr(self, "h", None):
            lib.zolo_symbolic_destroy(self.h)
            self.h = None


def inertia(A, B, shifts, sym=None, opts=None, stream=None):
    """Number of eigenvalues of (A, B) below each real shift (Sylvester's law of inertia)."""
    hA, hB = HostCsr(A), HostCsr(B)
    sh = np.ascontiguousarray(np.atleast_1d(np.asarray(shifts, dtype=np.float64)))
    out = np.zeros(len(sh), dtype=np.int64)
    o = opts if opts is not None else default_opts()
    _check(lib.zolo_inertia(C.byref(hA.s), C.byref(hB.s), sym.h if sym is not None else None, C.byref(o),
                            len(sh), sh.ctypes.data, out.ctypes.data, _stream(stream)), "zolo_inertia")
    return out


def eigs_slices(A, B, bounds, opts=None, cap=None, stream=None):
    """Eigenpairs in every slice (bounds[s], bounds[s+1]) (zolo_eigs_slices): returns
    (evals, V (device, n x found), resid, slice_of, stats, status)."""
    import torch
    hA, hB = HostCsr(A), HostCsr(B)
    bd = np.ascontiguousarray(np.asarray(bounds, dtype=np.float64))
    o = opts if opts is not None else default_opts()
    n = A.shape[0]
    if cap is None:
        cnt = inertia(A, B, bd[[0, -1]], opts=o, stream=stream)
        cap = int(cnt[1] - cnt[0])
    evals, resid = np.zeros(max(cap, 1)), np.zeros(max(cap, 1))
    sl = np.zeros(max(cap, 1), dtype=np.int32)
    V = torch.zeros((n, max(cap, 1)), dtype=torch.complex128, device="cuda")
    nf = _i64(0)
    st = Stats()
    rc = lib.zolo_eigs_slices(C.byref(hA.s), C.byref(hB.s), len(bd) - 1, bd.ctypes.data, C.byref(o),
                              evals.ctypes.data, _vp(V.data_ptr()), max(cap, 1), cap, C.byref(nf),
                              resid.ctypes.data, sl.ctypes.data, C.byref(st), _stream(stream))
    if rc not in (OK, ENOCONV):
        _check(rc, "zolo_eigs_slices")
    m = int(nf.value)
    return evals[:m], V[:, :m], resid[:m], sl[:m], st.as_dict(), rc


def profile_begin(gemm_events=0):
    """Start counting the library's kernel launches (and time GEMM launches: 1 = complex64,
    2 = complex128, 3 = both)."""
    _check(lib.zolo_profile_begin(int(gemm_events)), "zolo_profile_begin")


def profile_end(stream=None):
    n, ng, ms, fl = _i64(0), _i64(0), _dbl(0), _dbl(0)
    _check(lib.zolo_profile_end(_stream(stream), C.byref(n), C.byref(ng), C.byref(ms), C.byref(fl)),
           "zolo_profile_end")
    tn, tms, tfl = _i64(0), _dbl(0), _dbl(0)
    _check(lib.zolo_profile_tc(C.byref(tn), C.byref(tms), C.byref(tfl)), "zolo_profile_tc")
    gb, tb = _dbl(0), _dbl(0)
    _check(lib.zolo_profile_bytes(C.byref(gb), C.byref(tb)), "zolo_profile_bytes")
    return {"launches": n.value, "gemm_launches": ng.value, "gemm_ms": ms.value, "gemm_flops": fl.value,
            "tc_launches": tn.value, "tc_ms": tms.value, "tc_flops": tfl.value, "gemm_bytes": gb.value,
            "tc_bytes": tb.value}


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    return _vp(int(stream))


def check_block(shape, name, n, k=None):
    """Row and column counts of a block passed to the C ABI, which gets raw pointers and
    cannot check sizes: a block with fewer rows or columns than the call reads or writes
    is refused here, before any launch."""
    if len(shape) != 2 or shape[1] < 1:
        raise ValueError(f"{name}: need a non-empty 2-D block, got shape {tuple(shape)}")
    if shape[0] != n:
        raise ValueError(f"{name}: has {shape[0]} rows, the pencil has n = {n}")
    if k is not None and shape[1] != k:
        raise ValueError(f"{name}: has {shape[1]} columns, expected {k}")


def _blk(t, name, n, k=None):
    """Pointer, width and row stride of an (n, k) CUDA complex128 block."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.dim() == 2
            and t.stride(1) == 1):
        raise ValueError(f"{name}: need a CUDA complex128 tensor (n, k) with unit column stride")
    check_block(tuple(t.shape), name, n, k)
    return _vp(t.data_ptr()), t.shape[1], t.stride(0)


class Factor:
    """Device factorisations of K_j = A - sigma_hat_j B (j < r1) plus the uploaded pencil."""

    def __init__(self, A, B, flt, sym=None, opts=None, stream=None):
        self._A, self._B = HostCsr(A), HostCsr(B)
        self.n = A.shape[0]
        self.flt = flt
        self.opts = opts if opts is not None else default_opts()
        h = _vp()
        _check(lib.zolo_factor(C.byref(self._A.s), C.byref(self._B.s), flt.h, sym.h if sym is not None else None,
                               C.byref(self.opts), _stream(stream), C.byref(h)), "zolo_factor")
        self.h = h

    def stats(self):
        s = Stats()
        _check(lib.zolo_factor_get_stats(self.h, C.byref(s)), "zolo_factor_get_stats")
        return s.as_dict()

    def refactor(self, stream=None):
        _check(lib.zolo_refactor(self.h, _stream(stream)), "zolo_refactor")

    def solve(self, pole, B, herm=False, out=None, stream=None):
        import torch
        pb, k, ldb = _blk(B, "B", self.n)
        out = out if out is not None else torch.empty_like(B)
        px, _, ldx = _blk(out, "out", self.n, k)
        _check(lib.zolo_solve(self.h, pole, 1 if herm else 0, k, pb, ldb, px, ldx, _stream(stream)), "zolo_solve")
        return out

    def solve_noalloc(self, pole, B, out, herm=False, stream=None):
        """zolo_solve through the fixed no-allocation workspace (see include/zolo.h)."""
        pb, k, ldb = _blk(B, "B", self.n)
        px, _, ldx = _blk(out, "out", self.n, k)
        _check(lib.zolo_solve_noalloc(self.h, pole, 1 if herm else 0, k, pb, ldb, px, ldx, _stream(stream)),
               "zolo_solve_noalloc")
        return out

    def matmul(self, which, X, out=None, stream=None):
        import torch
        px, k, ldx = _blk(X, "X", self.n)
        out = out if out is not None else torch.empty_like(X)
        py, _, ldy = _blk(out, "out", self.n, k)
        _check(lib.zolo_matmul(self.h, 0 if which in ("A", 0) else 1, k, px, ldx, py, ldy, _stream(stream)),
               "zolo_matmul")
        return out

    def apply_inner(self, X, out=None, stream=None):
        import torch
        px, k, ldx = _blk(X, "X", self.n)
        out = out if out is not None else torch.empty_like(X)
        py, _, ldy = _blk(out, "out", self.n, k)
        _check(lib.zolo_apply_inner(self.h, k, px, ldx, py, ldy, _stream(stream)), "zolo_apply_inner")
        return out

    def apply(self, X, out=None, stream=None):
        import torch
        px, k, ldx = _blk(X, "X", self.n)
        out = out if out is not None else torch.empty_like(X)
        py, _, ldy = _blk(out, "out", self.n, k)
        st = Stats()
        _check(lib.zolo_apply(self.h, k, px, ldx, py, ldy, C.byref(st), _stream(stream)), "zolo_apply")
        return out, st.as_dict()

    def eigs(self, a, b, k0, X0=None, cap=None, stream=None, host_vectors=False):
        import torch
        cap = cap if cap is not None else k0
        evals = np.zeros(cap)
        resid = np.zeros(cap)
        V = torch.zeros((self.n, cap), dtype=torch.complex128, device="cuda")
        nf = _i64(0)
        st = Stats()
        x0 = _vp(X0.data_ptr()) if X0 is not None else None
        if X0 is not None:
            _blk(X0, "X0", self.n, k0)
        rc = lib.zolo_eigs_factored(self.h, a, b, k0, x0, evals.ctypes.data, _vp(V.data_ptr()), cap, cap,
                                    C.byref(nf), resid.ctypes.data, C.byref(st), _stream(stream))
        if rc not in (OK, ENOCONV, EGAP):       # these still return the pairs found
            _check(rc, "zolo_eigs_factored")
        m = int(nf.value)
        return evals[:m], V[:, :m], resid[:m], st.as_dict(), rc

    def __del__(self):
        if getattr(self, "h", None):
            lib.zolo_factor_destroy(self.h)
            self.h = None
