"""Pins for the oracle's T-QR (Alg. TQR) and Moore-Penrose pseudoinverse
(Alg. mp), Sec. 2, against things other than the oracle: LAPACK per Fourier
slice (numpy qr / pinv), the block-circulant definition of the t-product built
here, tensor orthogonality, triangular structure and the four Penrose
conditions.  CPU only."""
import numpy as np
import pytest

from paper_2504_04989_gb300 import workloads as wl

rng = np.random.default_rng(4321)


def _bcirc(X):
    n3, n1, n2 = X.shape
    M = np.zeros((n1 * n3, n2 * n3))
    for r in range(n3):
        for c in range(n3):
            M[r * n1:(r + 1) * n1, c * n2:(c + 1) * n2] = X[(r - c) % n3]
    return M


def _tp(A, B):
    """t-product by its definition fold(bcirc(A) unfold(B)) (Sec. 2)."""
    n3, n1, _ = A.shape
    n4 = B.shape[2]
    return (_bcirc(A) @ B.reshape(-1, n4)).reshape(n3, n1, n4)


def _tt(A):
    """tensor transpose by its definition: transpose every frontal slice, then
    reverse the order of slices 2..n3 (Sec. 2)."""
    T = np.swapaxes(A, 1, 2)
    return np.concatenate([T[:1], T[1:][::-1]], axis=0)


def _identity(n3, n):
    I = np.zeros((n3, n, n))
    I[0] = np.eye(n)
    return I


def _lapack_qr(Xk):
    """Economy QR of one slice with diag(R) real and >= 0 (the convention fixed by the oracle)."""
    n1, n2 = Xk.shape
    p = min(n1, n2)
    Q, Rl = np.linalg.qr(Xk[:, :p])
    d = np.diagonal(Rl)
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1), 1)
    Q = Q * ph[None, :]
    return Q, Q.conj().T @ Xk


SHAPES = [(7, 5, 6), (5, 7, 5), (6, 6, 1), (9, 4, 4), (3, 8, 7)]


@pytest.mark.parametrize("n1,n2,n3", SHAPES)
def test_tqr_against_lapack_per_slice(orc, n1, n2, n3):
    X = rng.standard_normal((n3, n1, n2))
    Q, R = orc.tqr(X)
    p = min(n1, n2)
    assert Q.shape == (n3, n1, p) and R.shape == (n3, p, n2)
    Xh, Qh, Rh = (np.fft.rfft(T, axis=0) for T in (X, Q, R))
    for k in range(n3 // 2 + 1):
        Qn, Rn = _lapack_qr(Xh[k])
        np.testing.assert_allclose(Qh[k], Qn, atol=1e-12)
        np.testing.assert_allclose(Rh[k], Rn, atol=1e-12)


@pytest.mark.parametrize("n1,n2,n3", SHAPES)
def test_tqr_definitions(orc, n1, n2, n3):
    """X = Q * R, Q^T * Q = I, and every frontal slice of R upper triangular."""
    X = rng.standard_normal((n3, n1, n2))
    Q, R = orc.tqr(X)
    p = min(n1, n2)
    np.testing.assert_allclose(_tp(Q, R), X, atol=1e-12)
    np.testing.assert_allclose(_tp(_tt(Q), Q), _identity(n3, p), atol=1e-12)
    low = np.tril(np.ones((p, n2), dtype=bool), -1)
    assert np.abs(R[:, low]).max(initial=0.0) < 1e-13


def test_tqr_single_slice_is_matrix_qr(orc):
    X = rng.standard_normal((1, 8, 5))
    Q, R = orc.tqr(X)
    Qn, Rn = _lapack_qr(X[0])
    np.testing.assert_allclose(Q[0], Qn.real, atol=1e-13)
    np.testing.assert_allclose(R[0], Rn.real, atol=1e-13)
    assert np.all(np.diagonal(R[0]) > 0)


@pytest.mark.parametrize("n1,n2,n3", SHAPES)
def test_tpinv_against_lapack_per_slice(orc, n1, n2, n3):
    X = rng.standard_normal((n3, n1, n2))
    Xp = orc.tpinv(X)
    assert Xp.shape == (n3, n2, n1)
    Xh, Ph = np.fft.rfft(X, axis=0), np.fft.rfft(Xp, axis=0)
    for k in range(n3 // 2 + 1):
        np.testing.assert_allclose(Ph[k], np.linalg.pinv(Xh[k]), atol=1e-11)


@pytest.mark.parametrize("n1,n2,n3", SHAPES)
def test_tpinv_penrose_conditions(orc, n1, n2, n3):
    """The four conditions of the definition of the MP inverse (Sec. 2), with
    the t-product and transpose built from their definitions here."""
    A = rng.standard_normal((n3, n1, n2))
    X = orc.tpinv(A)
    AX, XA = _tp(A, X), _tp(X, A)
    np.testing.assert_allclose(_tp(AX, A), A, atol=1e-11)
    np.testing.assert_allclose(_tp(XA, X), X, atol=1e-10)
    np.testing.assert_allclose(_tt(AX), AX, atol=1e-11)
    np.testing.assert_allclose(_tt(XA), XA, atol=1e-11)


def test_tpinv_rank_deficient_and_projectors(orc):
    """Tubal rank 3 in a 9 x 7 x 5 tensor: the pseudoinverse keeps only the
    nonzero singular values (LAPACK pinv per slice, same relative cut-off),
    and A * A^dagger = U * U^T, the projector onto the range (Sec. 2)."""
    A, parts = wl.low_tubal_rank(9, 7, 5, [3.0, 2.0, 1.0], seed=3, return_parts=True)
    X = orc.tpinv(A)
    Xh, Ph = np.fft.rfft(A, axis=0), np.fft.rfft(X, axis=0)
    for k in range(3):
        np.testing.assert_allclose(Ph[k], np.linalg.pinv(Xh[k], rcond=1e-10), atol=1e-12)
        U = parts["Uhat"][k]
        np.testing.assert_allclose(Xh[k] @ Ph[k], U @ U.conj().T, atol=1e-12)
    np.testing.assert_allclose(_tp(_tp(A, X), A), A, atol=1e-12)


def test_tpinv_of_invertible_tensor_is_inverse(orc):
    """A square tensor with invertible Fourier slices: A^dagger * A = I."""
    A = rng.standard_normal((4, 6, 6)) + 3 * _identity(4, 6)
    X = orc.tpinv(A)
    np.testing.assert_allclose(_tp(X, A), _identity(4, 6), atol=1e-12)
    np.testing.assert_allclose(_tp(A, X), _identity(4, 6), atol=1e-12)
