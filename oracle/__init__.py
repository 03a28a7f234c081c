"""ctypes binding of the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` are its only users.  The product path
(``paper_2504_04989_gb300``) never imports it.

Arrays follow the oracle's layout: a real tensor of size n1 x n2 x n3 is a
float64 numpy array of shape (n3, n1, n2) (frontal slices contiguous); a half
spectrum is complex128 of shape (h, n1, n2) with h = n3 // 2 + 1.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

MODES = {"canonical": 0, "literal": 1, "alg1": 2, "exact": 3, "qtrunc": 4}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        u32p = C.POINTER(C.c_uint32)
        i = C.c_int
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_gaussian.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_long, dp]
        L.orc_dft_mode3.argtypes = [dp, i, i, i, ip, i, dp]
        L.orc_idft_mode3.argtypes = [dp, i, i, i, dp]
        L.orc_tprod.argtypes = [dp, dp, i, i, i, i, dp]
        L.orc_tprod_bcirc.argtypes = [dp, dp, i, i, i, i, dp]
        L.orc_ttranspose.argtypes = [dp, i, i, i, dp]
        L.orc_tprod_backward.argtypes = [dp, dp, dp, i, i, i, i, dp, dp]
        L.orc_tproj_backward.argtypes = [dp, dp, dp, i, i, i, i, dp, dp]
        L.orc_householder_qr.argtypes = [i, i, dp, dp, dp]
        L.orc_jacobi_svd.argtypes = [i, i, dp, dp, dp, dp]
        L.orc_rtsvd_fourier.argtypes = [dp, i, i, i, i, i, i, i, dp, C.c_uint64, ip, i, dp, dp, dp, dp, ip]
        L.orc_range_basis_fourier.argtypes = [dp, i, i, i, i, i, i, i, dp, C.c_uint64, ip, i, dp]
        L.orc_rtsvd.argtypes = [dp, i, i, i, i, i, i, i, dp, C.c_uint64, dp, dp, dp, dp]
        L.orc_reconstruct.argtypes = [dp, dp, dp, i, i, i, i, dp]
        L.orc_rtsvd_hat.argtypes = [dp, dp, i, i, i, i, i, i, i, dp, dp, dp, dp, ip]
        L.orc_fill_in.argtypes = [dp, dp, C.POINTER(C.c_ubyte), dp, C.c_long]
        L.orc_fill_in.restype = C.c_double
        L.orc_psnr.argtypes = [dp, dp, C.c_long, C.c_double]
        L.orc_psnr.restype = C.c_double
        L.orc_tqr.argtypes = [dp, i, i, i, dp, dp]
        L.orc_tpinv.argtypes = [dp, i, i, i, dp]
        L.orc_num_threads.argtypes = []
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(rc, what):
    if rc < 0:
        raise ValueError("oracle %s rejected its arguments (rc=%d)" % (what, rc))
    return rc


def num_threads():
    return lib().orc_num_threads()


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    out = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, out)
    return [int(x) for x in out]


def gaussian(seed, n, stream=0, tensor_id=0):
    out = np.empty(int(n), dtype=np.float64)
    lib().orc_gaussian(C.c_uint64(int(seed)), stream, tensor_id, int(n), _dp(out))
    return out


def dft_mode3(X, slices=None):
    X = _f64(X)
    n3, n1, n2 = X.shape
    h = n3 // 2 + 1
    if slices is None:
        sl, ns, slp = None, h, None
    else:
        sl = np.ascontiguousarray(slices, dtype=np.int32)
        ns, slp = len(sl), sl.ctypes.data_as(C.POINTER(C.c_int))
    out = np.empty((ns, n1, n2), dtype=np.complex128)
    _check(lib().orc_dft_mode3(_dp(X), n1, n2, n3, slp, ns, _dp(out)), "dft_mode3")
    return out


def idft_mode3(Xhat, n3):
    Xhat = _c128(Xhat)
    h, n1, n2 = Xhat.shape
    assert h == n3 // 2 + 1
    out = np.empty((n3, n1, n2), dtype=np.float64)
    _check(lib().orc_idft_mode3(_dp(Xhat), n1, n2, n3, _dp(out)), "idft_mode3")
    return out


def tprod(A, B):
    A, B = _f64(A), _f64(B)
    n3, n1, n2 = A.shape
    n3b, n2b, n4 = B.shape
    assert n3 == n3b and n2 == n2b
    out = np.empty((n3, n1, n4))
    _check(lib().orc_tprod(_dp(A), _dp(B), n1, n2, n4, n3, _dp(out)), "tprod")
    return out


def tprod_bcirc(A, B):
    A, B = _f64(A), _f64(B)
    n3, n1, n2 = A.shape
    n4 = B.shape[2]
    out = np.empty((n3, n1, n4))
    _check(lib().orc_tprod_bcirc(_dp(A), _dp(B), n1, n2, n4, n3, _dp(out)), "tprod_bcirc")
    return out


def ttranspose(A):
    A = _f64(A)
    n3, n1, n2 = A.shape
    out = np.empty((n3, n2, n1))
    _check(lib().orc_ttranspose(_dp(A), n1, n2, n3, _dp(out)), "ttranspose")
    return out


def tprod_backward(A, B, dC):
    A, B, dC = _f64(A), _f64(B), _f64(dC)
    n3, n1, n2 = A.shape
    n4 = B.shape[2]
    dA = np.empty_like(A)
    dB = np.empty_like(B)
    _check(lib().orc_tprod_backward(_dp(A), _dp(B), _dp(dC), n1, n2, n4, n3, _dp(dA), _dp(dB)), "tprod_backward")
    return dA, dB


def tproj_backward(Q, A, dY):
    Q, A, dY = _f64(Q), _f64(A), _f64(dY)
    n3, n1, m = Q.shape
    n2 = A.shape[2]
    dQ = np.empty_like(Q)
    dA = np.empty_like(A)
    _check(lib().orc_tproj_backward(_dp(Q), _dp(A), _dp(dY), n1, m, n2, n3, _dp(dQ), _dp(dA)), "tproj_backward")
    return dQ, dA


def householder_qr(X):
    X = _c128(X)
    M, N = X.shape
    Q = np.empty((M, N), dtype=np.complex128)
    R = np.empty((N, N), dtype=np.complex128)
    _check(lib().orc_householder_qr(M, N, _dp(X), _dp(Q), _dp(R)), "householder_qr")
    return Q, R


def jacobi_svd(X):
    """X (M x N, M >= N) = W diag(s) V^H; returns (W, s, V, sweeps)."""
    X = _c128(X)
    M, N = X.shape
    W = np.empty((M, N), dtype=np.complex128)
    s = np.empty(N)
    V = np.empty((N, N), dtype=np.complex128)
    sweeps = _check(lib().orc_jacobi_svd(M, N, _dp(X), _dp(W), _dp(s), _dp(V)), "jacobi_svd")
    return W, s, V, sweeps


def rtsvd_fourier(X, R, P=0, q=0, mode="canonical", omega=None, seed=0, slices=None):
    """Randomized (or exact) truncated T-SVD on the chosen Fourier slices.

    Returns dict with Uhat (ns, n1, R), sig (ns, R), Vhat (ns, n2, R),
    err2 (ns,) = ||Xhat_k - Uhat diag(sig) Vhat^H||_F^2 and m (ns,) basis sizes.
    """
    X = _f64(X)
    n3, n1, n2 = X.shape
    h = n3 // 2 + 1
    b = R + P
    if slices is None:
        ns, slp = h, None
    else:
        sl = np.ascontiguousarray(slices, dtype=np.int32)
        ns, slp = len(sl), sl.ctypes.data_as(C.POINTER(C.c_int))
    om = None
    if omega is not None:
        om = _f64(omega)
        assert om.shape == (n3, n2, b), om.shape
    Uh = np.empty((ns, n1, R), dtype=np.complex128)
    sg = np.empty((ns, R))
    Vh = np.empty((ns, n2, R), dtype=np.complex128)
    e2 = np.empty(ns)
    mu = np.empty(ns, dtype=np.int32)
    _check(lib().orc_rtsvd_fourier(_dp(X), n1, n2, n3, R, P, q, MODES[mode], _dp(om) if om is not None else None,
                                   C.c_uint64(int(seed)), slp, ns, _dp(Uh), _dp(sg), _dp(Vh), _dp(e2),
                                   mu.ctypes.data_as(C.POINTER(C.c_int))), "rtsvd_fourier")
    return {"Uhat": Uh, "sig": sg, "Vhat": Vh, "err2": e2, "m": mu}


def rtsvd_hat(Xhat, Omhat, R, P=0, q=0, mode="canonical"):
    """Alg. 2 on given Fourier slices Xhat (ns, n1, n2) with test blocks Omhat
    (ns, n2, R+P); returns the dict of rtsvd_fourier."""
    Xhat, Omhat = _c128(Xhat), _c128(Omhat)
    ns, n1, n2 = Xhat.shape
    assert Omhat.shape == (ns, n2, R + P), Omhat.shape
    Uh = np.empty((ns, n1, R), dtype=np.complex128)
    sg = np.empty((ns, R))
    Vh = np.empty((ns, n2, R), dtype=np.complex128)
    e2 = np.empty(ns)
    mu = np.empty(ns, dtype=np.int32)
    _check(lib().orc_rtsvd_hat(_dp(Xhat), _dp(Omhat), ns, n1, n2, R, P, q, MODES[mode], _dp(Uh), _dp(sg), _dp(Vh),
                               _dp(e2), mu.ctypes.data_as(C.POINTER(C.c_int))), "rtsvd_hat")
    return {"Uhat": Uh, "sig": sg, "Vhat": Vh, "err2": e2, "m": mu}


def range_basis(X, R, P=0, q=0, mode="canonical", omega=None, seed=0, slices=None):
    """Orthonormal range basis Qhat (ns, n1, m) of the chosen mode per Fourier slice."""
    X = _f64(X)
    n3, n1, n2 = X.shape
    h = n3 // 2 + 1
    b = R + P
    if slices is None:
        ns, slp = h, None
    else:
        sl = np.ascontiguousarray(slices, dtype=np.int32)
        ns, slp = len(sl), sl.ctypes.data_as(C.POINTER(C.c_int))
    om = None
    if omega is not None:
        om = _f64(omega)
        assert om.shape == (n3, n2, b), om.shape
    mmax = min((1 if mode == "alg1" else q + 1) * b, n1, n2)
    Qh = np.empty((ns, n1, mmax), dtype=np.complex128)
    m = _check(lib().orc_range_basis_fourier(_dp(X), n1, n2, n3, R, P, q, MODES[mode],
                                             _dp(om) if om is not None else None, C.c_uint64(int(seed)),
                                             slp, ns, _dp(Qh)), "range_basis")
    assert m == mmax
    return Qh


def rtsvd(X, R, P=0, q=0, mode="canonical", omega=None, seed=0):
    """Spatial factors: U (n3,n1,R), S tubes (n3,R), V (n3,n2,R), sig_hat (h,R)."""
    X = _f64(X)
    n3, n1, n2 = X.shape
    h = n3 // 2 + 1
    b = R + P
    om = None
    if omega is not None:
        om = _f64(omega)
        assert om.shape == (n3, n2, b), om.shape
    U = np.empty((n3, n1, R))
    S = np.empty((n3, R))
    V = np.empty((n3, n2, R))
    sh = np.empty((h, R))
    _check(lib().orc_rtsvd(_dp(X), n1, n2, n3, R, P, q, MODES[mode], _dp(om) if om is not None else None,
                           C.c_uint64(int(seed)), _dp(U), _dp(S), _dp(V), _dp(sh)), "rtsvd")
    return U, S, V, sh


def reconstruct(U, S, V):
    U, S, V = _f64(U), _f64(S), _f64(V)
    n3, n1, R = U.shape
    n2 = V.shape[1]
    out = np.empty((n3, n1, n2))
    _check(lib().orc_reconstruct(_dp(U), _dp(S), _dp(V), n1, n2, n3, R, _dp(out)), "reconstruct")
    return out


def rel_error(X, Xr):
    """Relative error e = ||X - Xr||_F / ||X||_F (Sec. 5)."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.linalg.norm((X - Xr).ravel()) / np.linalg.norm(X.ravel()))


def tqr(X):
    """Alg. TQR: X = Q * R; returns Q (n3, n1, p), R (n3, p, n2), p = min(n1, n2)."""
    X = _f64(X)
    n3, n1, n2 = X.shape
    p = min(n1, n2)
    Q = np.empty((n3, n1, p))
    R = np.empty((n3, p, n2))
    _check(lib().orc_tqr(_dp(X), n1, n2, n3, _dp(Q), _dp(R)), "tqr")
    return Q, R


def tpinv(X):
    """Alg. mp: the Moore-Penrose pseudoinverse (n3, n2, n1) of X (n3, n1, n2)."""
    X = _f64(X)
    n3, n1, n2 = X.shape
    out = np.empty((n3, n2, n1))
    _check(lib().orc_tpinv(_dp(X), n1, n2, n3, _dp(out)), "tpinv")
    return out


def fill_in(Cm, M, T, X):
    """Ex. 3 fill-in: returns (C_new, sum (C_new - C_old)^2)."""
    Cn = _f64(Cm).copy()
    M, X = _f64(M), _f64(X)
    T = np.ascontiguousarray(T, dtype=np.uint8)
    ch = lib().orc_fill_in(_dp(Cn), _dp(M), T.ctypes.data_as(C.POINTER(C.c_ubyte)), _dp(X), Cn.size)
    return Cn, ch


def psnr(X, Y, peak=255.0):
    X, Y = _f64(X), _f64(Y)
    return lib().orc_psnr(_dp(X), _dp(Y), X.size, float(peak))
