"""Pins for the FP64 CPU oracle, each against something other than the oracle
itself: library routines (numpy FFT / LAPACK), definitions evaluated a second
way (bcirc vs. Fourier t-product), closed forms (Eckart-Young), identities and
inequalities of the paper's Sec. 4, finite differences and published
known-answer vectors.  CPU only."""
import os

import numpy as np
import pytest

from paper_2504_04989_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(1234)


def rand(*shape):
    return rng.standard_normal(shape)


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers(orc):
    """Philox4x32-10 against the published known-answer vectors."""
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert orc.philox4x32_10(w[:4], w[4:6]) == w[6:10]
        n += 1
    assert n == 3


def test_gaussian_distribution(orc):
    from scipy import stats
    z = orc.gaussian(7, 400_000)
    assert abs(z.mean()) < 5e-3 and abs(z.var() - 1) < 1e-2
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different streams / tensor ids / seeds give different draws
    assert not np.allclose(orc.gaussian(7, 64, stream=1)[:8], z[:8])
    assert not np.allclose(orc.gaussian(7, 64, tensor_id=3)[:8], z[:8])
    assert not np.allclose(orc.gaussian(8, 64)[:8], z[:8])
    # a prefix of a longer draw is the shorter draw (counter based)
    np.testing.assert_array_equal(orc.gaussian(7, 10), z[:10])


# --------------------------------------------------------------------------- DFT
@pytest.mark.parametrize("n3", [1, 2, 3, 4, 5, 8, 16, 100])
def test_dft_against_numpy_fft(orc, n3):
    X = rand(n3, 3, 4)
    got = orc.dft_mode3(X)
    ref = np.fft.rfft(X, axis=0)  # library FFT, omega = exp(-2 pi i / n), unnormalised
    assert got.shape == ref.shape == (n3 // 2 + 1, 3, 4)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * max(1, n3))
    # requested subset of slices
    sl = [n3 // 2, 0]
    np.testing.assert_allclose(orc.dft_mode3(X, slices=sl), ref[sl], atol=1e-12 * max(1, n3))


@pytest.mark.parametrize("n3", [1, 2, 7, 8, 100])
def test_idft_inverse_and_parseval(orc, n3):
    X = rand(n3, 4, 3)
    Xh = orc.dft_mode3(X)
    np.testing.assert_allclose(orc.idft_mode3(Xh, n3), X, atol=1e-12)
    np.testing.assert_allclose(orc.idft_mode3(Xh, n3), np.fft.irfft(Xh, n=n3, axis=0), atol=1e-12)
    # Parseval (Sec. 2, the Parseval relation) over the full spectrum, i.e. half-spectrum weights 1, 2, .., (1)
    full = np.fft.fft(X, axis=0)
    assert np.isclose(np.sum(X ** 2), np.sum(np.abs(full) ** 2) / n3, rtol=1e-12)
    w = np.full(n3 // 2 + 1, 2.0)
    w[0] = 1.0
    if n3 % 2 == 0:
        w[-1] = 1.0
    assert np.isclose(np.sum(X ** 2), np.sum(w[:, None, None] * np.abs(Xh) ** 2) / n3, rtol=1e-12)


# --------------------------------------------------------------------------- t-algebra
@pytest.mark.parametrize("n3", [1, 2, 3, 4, 5, 8])
def test_tprod_fourier_equals_bcirc_definition(orc, n3):
    A, B = rand(n3, 3, 4), rand(n3, 4, 2)
    np.testing.assert_allclose(orc.tprod(A, B), orc.tprod_bcirc(A, B), atol=1e-12)


def test_tprod_bcirc_small_cases(orc):
    # n3 = 1: the t-product is the matrix product
    A, B = rand(1, 3, 5), rand(1, 5, 2)
    np.testing.assert_allclose(orc.tprod_bcirc(A, B)[0], A[0] @ B[0], atol=1e-14)
    # identity tensor (first slice I, other slices 0) is a two-sided unit
    I = np.zeros((4, 3, 3))
    I[0] = np.eye(3)
    A = rand(4, 3, 3)
    np.testing.assert_allclose(orc.tprod_bcirc(I, A), A, atol=1e-14)
    np.testing.assert_allclose(orc.tprod_bcirc(A, I), A, atol=1e-14)
    # a single nonzero slice shifts circularly: (e_s * B)^{(r)} = B^{(r-s mod n3)}
    n3 = 5
    E = np.zeros((n3, 2, 2))
    E[2] = np.eye(2)
    B = rand(n3, 2, 3)
    np.testing.assert_allclose(orc.tprod_bcirc(E, B), np.roll(B, 2, axis=0), atol=1e-14)


def _bcirc(X):
    """Block circulant matrix of the definition in Sec. 2, built independently."""
    n3, n1, n2 = X.shape
    M = np.zeros((n1 * n3, n2 * n3))
    for r in range(n3):
        for c in range(n3):
            M[r * n1:(r + 1) * n1, c * n2:(c + 1) * n2] = X[(r - c) % n3]
    return M


@pytest.mark.parametrize("n3", [1, 2, 5, 6])
def test_ttranspose_rules(orc, n3):
    X, Y = rand(n3, 3, 4), rand(n3, 4, 2)
    XT = orc.ttranspose(X)
    # bcirc(X^T) = bcirc(X)^T (Lemma on bcirc)
    np.testing.assert_allclose(_bcirc(XT), _bcirc(X).T, atol=0)
    # (X*Y)^T = Y^T * X^T
    np.testing.assert_allclose(orc.ttranspose(orc.tprod(X, Y)), orc.tprod(orc.ttranspose(Y), XT), atol=1e-12)
    np.testing.assert_allclose(orc.ttranspose(XT), X, atol=0)
    # Fourier slice of X^T is the conjugate transpose of the slice of X
    np.testing.assert_allclose(orc.dft_mode3(XT), np.conj(np.swapaxes(orc.dft_mode3(X), 1, 2)), atol=1e-12)


def test_tprod_matches_bcirc_matrix_product(orc):
    n3 = 4
    A, B = rand(n3, 3, 2), rand(n3, 2, 5)
    C = orc.tprod(A, B)
    unfoldB = B.reshape(n3 * 2, 5)
    np.testing.assert_allclose(C.reshape(n3 * 3, 5), _bcirc(A) @ unfoldB, atol=1e-12)


# --------------------------------------------------------------------------- QR / SVD
@pytest.mark.parametrize("M,N", [(6, 6), (9, 4), (30, 7), (5, 1)])
def test_householder_qr(orc, M, N):
    X = rand(M, N) + 1j * rand(M, N)
    Q, R = orc.householder_qr(X)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(N), atol=1e-13)
    np.testing.assert_allclose(Q @ R, X, atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0)
    _, Rl = np.linalg.qr(X)  # LAPACK: |R_ii| is unique
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=1e-12)


def test_householder_qr_rank_deficient(orc):
    X = np.zeros((8, 4), dtype=complex)
    X[:, 0] = rand(8)
    X[:, 2] = 2 * X[:, 0]  # rank 1 plus two zero columns
    Q, R = orc.householder_qr(X)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(4), atol=1e-13)
    np.testing.assert_allclose(Q @ R, X, atol=1e-13)


@pytest.mark.parametrize("M,N", [(5, 5), (12, 7), (40, 3), (3, 1)])
def test_jacobi_svd_against_lapack(orc, M, N):
    X = rand(M, N) + 1j * rand(M, N)
    W, s, V, sweeps = orc.jacobi_svd(X)
    assert sweeps > 0
    np.testing.assert_allclose(s, np.linalg.svd(X, compute_uv=False), rtol=1e-13)
    np.testing.assert_allclose((W * s) @ V.conj().T, X, atol=1e-13)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(N), atol=1e-13)
    np.testing.assert_allclose(W.conj().T @ W, np.eye(N), atol=1e-12)
    assert np.all(np.diff(s) <= 0)


def test_jacobi_svd_graded_and_deficient(orc):
    # graded singular values keep high relative accuracy (one-sided Jacobi)
    n = 8
    U, _ = np.linalg.qr(rand(n, n) + 1j * rand(n, n))
    V, _ = np.linalg.qr(rand(n, n) + 1j * rand(n, n))
    s0 = 10.0 ** -np.arange(n)
    X = (U * s0) @ V.conj().T
    _, s, _, _ = orc.jacobi_svd(X)
    np.testing.assert_allclose(s[:5], s0[:5], rtol=1e-10)
    # exact zero singular values come out as zeros, V stays unitary
    X = np.outer(rand(6), rand(3)).astype(complex)
    W, s, V, _ = orc.jacobi_svd(X)
    assert s[1] < 1e-14 * s[0] and s[2] < 1e-14 * s[0]
    np.testing.assert_allclose(V.conj().T @ V, np.eye(3), atol=1e-13)


# --------------------------------------------------------------------------- Alg. 2 / Alg. 1
def _fourier_err2_total(err2, n3):
    """||X - X_R||_F^2 from per-slice Fourier errors (Parseval, half-spectrum weights)."""
    w = np.full(len(err2), 2.0)
    w[0] = 1.0
    if n3 % 2 == 0:
        w[-1] = 1.0
    return float(np.sum(w * err2) / n3)


def test_exact_tsvd_eckart_young_closed_form(orc):
    """Exact truncated T-SVD: per-slice singular values equal the construction's,
    and the error equals the closed form sum_{i>R} sigma_i^2."""
    sig = np.array([5.0, 3.0, 2.0, 1.0, 0.5, 0.25])
    X = wl.low_tubal_rank(10, 8, 6, sig, seed=3)
    R = 3
    out = orc.rtsvd_fourier(X, R, mode="exact")
    np.testing.assert_allclose(out["sig"], np.tile(sig[:R], (4, 1)), rtol=1e-12)
    e2 = _fourier_err2_total(out["err2"], 6)
    assert np.isclose(e2, wl.optimal_error2(sig, R), rtol=1e-10)
    # and the spatial reconstruction agrees (idft + t-products of the oracle)
    U, S, V, _ = orc.rtsvd(X, R, mode="exact")
    Xr = orc.reconstruct(U, S, V)
    assert np.isclose(np.sum((X - Xr) ** 2), wl.optimal_error2(sig, R), rtol=1e-9)


def test_exact_tsvd_against_lapack_per_slice(orc):
    X = rand(5, 7, 9)
    out = orc.rtsvd_fourier(X, 4, mode="exact")
    ref = np.linalg.svd(np.fft.rfft(X, axis=0), compute_uv=False)[:, :4]
    np.testing.assert_allclose(out["sig"], ref, rtol=1e-12)


@pytest.mark.parametrize("mode", ["canonical", "literal"])
def test_alg2_exact_recovery_low_tubal_rank(orc, mode):
    """Noise-free tubal rank r <= R: the Krylov space contains range(X), the
    error is at rounding level (Thm. 3 with A_{k,perp} = 0)."""
    sig = np.linspace(4, 1, 5)
    X = wl.low_tubal_rank(20, 16, 8, sig, seed=4)
    U, S, V, sh = orc.rtsvd(X, 5, P=3, q=1, mode=mode, omega=wl.omega(16, 8, 8, seed=1))
    assert orc.rel_error(X, orc.reconstruct(U, S, V)) < 1e-12
    np.testing.assert_allclose(sh, np.tile(sig, (5, 1)), rtol=1e-12)


def test_alg2_full_basis_is_exact_tsvd(orc):
    """m = (q+1)(R+P) >= min(n1,n2): span(K) is the whole column space, so Alg. 2
    returns the exact truncated T-SVD."""
    X = rand(7, 12, 10)
    R = 4
    a = orc.rtsvd_fourier(X, R, P=2, q=1, mode="canonical", seed=5)
    e = orc.rtsvd_fourier(X, R, mode="exact")
    assert np.all(a["m"] == 10)  # min(n1, n2)
    np.testing.assert_allclose(a["sig"], e["sig"], rtol=1e-12)
    np.testing.assert_allclose(a["err2"], e["err2"], rtol=1e-10)


def test_canonical_matches_literal_when_well_conditioned(orc):
    """The block-orthonormalised Krylov basis spans the same space as the raw
    K = [K_0, .., K_q] of Alg. 2: results agree on a well-conditioned case."""
    sig = np.linspace(3.0, 1.0, 24)
    X = wl.low_tubal_rank(30, 28, 5, sig, noise_std=1e-2, seed=6)
    om = wl.omega(28, 6, 5, seed=2)
    c = orc.rtsvd_fourier(X, 4, P=2, q=1, mode="canonical", omega=om)
    l = orc.rtsvd_fourier(X, 4, P=2, q=1, mode="literal", omega=om)
    np.testing.assert_allclose(c["sig"], l["sig"], rtol=1e-10)
    np.testing.assert_allclose(c["err2"], l["err2"], rtol=1e-8)
    Qc = orc.range_basis(X, 4, P=2, q=1, mode="canonical", omega=om)
    Ql = orc.range_basis(X, 4, P=2, q=1, mode="literal", omega=om)
    for k in range(Qc.shape[0]):  # same projector
        np.testing.assert_allclose(Qc[k] @ Qc[k].conj().T, Ql[k] @ Ql[k].conj().T, atol=1e-9)


def test_basis_orthogonal_tensor(orc):
    """Q^T * Q = I (orthogonal tensor, Sec. 2) for the spatial basis tensor
    built from the per-slice bases (conjugate mirror + inverse DFT)."""
    X = rand(6, 9, 7)
    Qh = orc.range_basis(X, 2, P=1, q=1, seed=11)
    m = Qh.shape[2]
    Q = orc.idft_mode3(Qh, 6)
    QtQ = orc.tprod(orc.ttranspose(Q), Q)
    I = np.zeros((6, m, m))
    I[0] = np.eye(m)
    np.testing.assert_allclose(QtQ, I, atol=1e-13)


def test_alg2_monotone_in_q_and_beats_alg1(orc):
    """With a fixed Omega the Krylov spaces are nested in q, and the Rayleigh-Ritz
    result is the best rank-R approximation from range(Q) (Sec. 4, best approximation within range(Q)), so the
    error cannot grow with q and Alg. 2 is never worse than Alg. 1."""
    X = wl.low_tubal_rank(40, 36, 6, np.arange(1, 37) ** -1.0, seed=7)
    R, P = 5, 2
    om = wl.omega(36, R + P, 6, seed=3)
    errs = []
    for q in range(0, 4):
        e2 = _fourier_err2_total(orc.rtsvd_fourier(X, R, P, q, omega=om)["err2"], 6)
        e1 = _fourier_err2_total(orc.rtsvd_fourier(X, R, P, q, mode="alg1", omega=om)["err2"], 6)
        assert e2 <= e1 * (1 + 1e-10)
        errs.append(e2)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-10) for i in range(len(errs) - 1))
    assert errs[-1] < errs[0]
    opt = wl.optimal_error2(np.arange(1, 37) ** -1.0, R)
    assert errs[-1] >= opt * (1 - 1e-10)


def test_nested_krylov_bases(orc):
    X = rand(6, 30, 25)
    om = wl.omega(25, 4, 6, seed=4)
    Q1 = orc.range_basis(X, 3, P=1, q=1, omega=om)
    Q2 = orc.range_basis(X, 3, P=1, q=2, omega=om)
    for k in range(Q1.shape[0]):  # span(Q1) is inside span(Q2)
        resid = Q1[k] - Q2[k] @ (Q2[k].conj().T @ Q1[k])
        assert np.linalg.norm(resid) < 1e-10


def test_projection_lemma_and_theorems(orc):
    """Sec. 4, the projection lemma: the output equals the projection U_k U_k^H A (i.e.
    Q (Q^H A)_k); Thm. 3 (Frobenius) and Thm. 1 (spectral) bounds, per slice."""
    sig = np.arange(1, 21) ** -0.7
    X = wl.low_tubal_rank(24, 20, 5, sig, noise_std=1e-3, seed=8)
    R, P, q = 4, 2, 1
    om = wl.omega(20, R + P, 5, seed=5)
    out = orc.rtsvd_fourier(X, R, P, q, omega=om)
    Qh = orc.range_basis(X, R, P, q, omega=om)
    Xh = np.fft.rfft(X, axis=0)
    for k in range(Xh.shape[0]):
        A, U = Xh[k], out["Uhat"][k]
        approx = (U * out["sig"][k]) @ out["Vhat"][k].conj().T
        np.testing.assert_allclose(approx, U @ (U.conj().T @ A), atol=1e-12)
        Q = Qh[k]
        C = Q.conj().T @ A
        u, s, vh = np.linalg.svd(C)
        Ck = (u[:, :R] * s[:R]) @ vh[:R]
        np.testing.assert_allclose(approx, Q @ Ck, atol=1e-11)  # A - U U^H A = A - Q (Q^H A)_k
        ua, sa, vha = np.linalg.svd(A)
        Ak = (ua[:, :R] * sa[:R]) @ vha[:R]
        lhs = np.linalg.norm(A - approx) ** 2
        rhs = np.linalg.norm(Ak - Q @ (Q.conj().T @ Ak)) ** 2 + np.sum(sa[R:] ** 2)
        assert lhs <= rhs * (1 + 1e-10)  # Thm. 3
        # Thm. 1 (per Fourier slice): ||(I - QQ^H) A||_2 <= ||(I - QQ^H) Z||_2^{1/(2q+1)},
        # Z = [A, (A A^H) A, .., (A A^H)^q A]
        blocks, Bk = [A], A
        for _ in range(q):
            Bk = A @ (A.conj().T @ Bk)
            blocks.append(Bk)
        Z = np.concatenate(blocks, axis=1)
        Pz = Z - Q @ (Q.conj().T @ Z)
        assert np.linalg.norm(A - Q @ C, 2) <= np.linalg.norm(Pz, 2) ** (1.0 / (2 * q + 1)) * (1 + 1e-10)
        # Sec. 4, the projected power inequality: ||P M P||^r <= ||P M^r P|| for PSD M and an orthogonal projector P
        Pm = np.eye(A.shape[0]) - Q @ Q.conj().T
        M = A @ A.conj().T
        r = 2 * q + 1
        assert np.linalg.norm(Pm @ M @ Pm, 2) ** r <= np.linalg.norm(Pm @ np.linalg.matrix_power(M, r) @ Pm, 2) * (1 + 1e-9) + 1e-14


# --------------------------------------------------------------------------- gradients
def test_tprod_backward_finite_differences(orc):
    A, B, dC = rand(5, 3, 4), rand(5, 4, 2), rand(5, 3, 2)
    dA, dB = orc.tprod_backward(A, B, dC)
    L = lambda A_, B_: np.sum(dC * orc.tprod_bcirc(A_, B_))
    for _ in range(3):
        E, F = rand(*A.shape), rand(*B.shape)
        eps = 1e-3
        fd_a = (L(A + eps * E, B) - L(A - eps * E, B)) / (2 * eps)
        fd_b = (L(A, B + eps * F) - L(A, B - eps * F)) / (2 * eps)
        assert np.isclose(fd_a, np.sum(dA * E), rtol=1e-9)
        assert np.isclose(fd_b, np.sum(dB * F), rtol=1e-9)


def test_tproj_backward_finite_differences(orc):
    Q, A, dY = rand(4, 5, 2), rand(4, 5, 3), rand(4, 5, 3)
    dQ, dA = orc.tproj_backward(Q, A, dY)

    def L(Q_, A_):
        return np.sum(dY * orc.tprod_bcirc(Q_, orc.tprod_bcirc(orc.ttranspose(Q_), A_)))
    for _ in range(3):
        E, F = rand(*Q.shape), rand(*A.shape)
        eps = 1e-3  # L is quadratic in Q, linear in A: central differences are exact
        fd_q = (L(Q + eps * E, A) - L(Q - eps * E, A)) / (2 * eps)
        fd_a = (L(Q, A + eps * F) - L(Q, A - eps * F)) / (2 * eps)
        assert np.isclose(fd_q, np.sum(dQ * E), rtol=1e-9)
        assert np.isclose(fd_a, np.sum(dA * F), rtol=1e-9)


def test_philox_drawn_omega_path(orc):
    """Omega = NULL draws the test tensor from the Philox stream (seed, stream 0)."""
    X = rand(4, 10, 9)
    R, P = 2, 2
    om = orc.gaussian(3, 4 * 9 * (R + P)).reshape(4, 9, R + P)
    a = orc.rtsvd_fourier(X, R, P, 1, seed=3)
    b = orc.rtsvd_fourier(X, R, P, 1, omega=om)
    np.testing.assert_array_equal(a["sig"], b["sig"])


def test_argument_errors(orc):
    X = rand(4, 5, 6)
    with pytest.raises(ValueError):
        orc.rtsvd_fourier(X, 7)  # R > min(n1, n2)
    with pytest.raises(ValueError):
        orc.dft_mode3(X, slices=[5])


# --------------------------------------------------------------------------- Alg. 1 pin
def _alg1_numpy(Xk, Omk, R, q):
    """Alg. 1 (Sec. 3) on one Fourier slice, written with numpy / LAPACK only:
    Y = (X X^H)^q X Om, Q = qr(Y), and the rank-R SVD of Q^H X."""
    Y = Xk @ Omk
    for _ in range(q):
        Y = Xk @ (Xk.conj().T @ Y)
    Q, _ = np.linalg.qr(Y)
    s = np.linalg.svd(Q.conj().T @ Xk, compute_uv=False)
    return Q, s[:R]


@pytest.mark.parametrize("q", [0, 1, 2])
def test_alg1_against_numpy_power_iteration(orc, q):
    """The oracle's Alg. 1 mode against a numpy/LAPACK restatement on small
    well-conditioned slices (spectrum 1..0.4, so (X X^H)^q X Om stays well
    conditioned without intermediate orthonormalisation): the range projector
    Q Q^H to 1e-10 and the top-R singular values of Q^H X to 1e-12.  A missing
    power step, X in place of X^H, or Omega's rows taken from n1 all fail."""
    n3, n1, n2, R, P = 5, 14, 11, 3, 2
    sig = np.linspace(1.0, 0.4, 11)
    X = wl.low_tubal_rank(n1, n2, n3, sig, noise_std=1e-2, seed=21)
    om = wl.omega(n2, R + P, n3, seed=22)
    Xh = np.fft.rfft(X, axis=0)
    Omh = np.fft.rfft(om, axis=0)
    Qo = orc.range_basis(X, R, P, q, mode="alg1", omega=om)
    ro = orc.rtsvd_fourier(X, R, P, q, mode="alg1", omega=om)
    for k in range(n3 // 2 + 1):
        Qn, sn = _alg1_numpy(Xh[k], Omh[k], R, q)
        np.testing.assert_allclose(Qo[k] @ Qo[k].conj().T, Qn @ Qn.conj().T, atol=1e-10)
        np.testing.assert_allclose(ro["sig"][k], sn, rtol=1e-12, atol=0)


def test_alg1_full_basis_is_exact_tsvd(orc):
    """Degenerate case R + P >= min(n1, n2): the Alg. 1 basis spans the whole
    column space, so its singular values are the exact per-slice ones (LAPACK)."""
    n3, n1, n2, R, P = 4, 9, 6, 4, 3   # b = 7 > n2 = 6
    X = rand(n3, n1, n2)
    om = wl.omega(n2, R + P, n3, seed=5)
    ro = orc.rtsvd_fourier(X, R, P, 1, mode="alg1", omega=om)
    Xh = np.fft.rfft(X, axis=0)
    for k in range(n3 // 2 + 1):
        s = np.linalg.svd(Xh[k], compute_uv=False)[:R]
        np.testing.assert_allclose(ro["sig"][k], s, rtol=1e-12)
        assert ro["m"][k] == n2


# --------------------------------------------------------------------------- Ex. 1 truncated basis
def test_qtrunc_against_numpy_sketch(orc):
    """The Q-truncated variant of Alg. 2 (Ex. 1, Sec. 5: Q cut to its leading
    R + P columns before the projection) against numpy/LAPACK: the leading
    R + P columns of the Krylov basis span X Omega, so the result is the
    rank-R SVD of Q_0^H X with Q_0 = qr(X Omega), whatever q is."""
    n3, n1, n2, R, P, q = 5, 30, 26, 4, 3, 2
    X = wl.low_tubal_rank(n1, n2, n3, np.arange(1, 27) ** -2.0, noise_std=1e-3, seed=31)
    om = wl.omega(n2, R + P, n3, seed=32)
    ro = orc.rtsvd_fourier(X, R, P, q, mode="qtrunc", omega=om)
    assert np.all(ro["m"] == R + P)
    Xh, Omh = np.fft.rfft(X, axis=0), np.fft.rfft(om, axis=0)
    for k in range(n3 // 2 + 1):
        Q0, _ = np.linalg.qr(Xh[k] @ Omh[k])
        s = np.linalg.svd(Q0.conj().T @ Xh[k], compute_uv=False)[:R]
        np.testing.assert_allclose(ro["sig"][k], s, rtol=1e-12)
    full = orc.rtsvd_fourier(X, R, P, q, omega=om)  # the full basis is at least as good (nested spans)
    assert np.all(full["err2"] <= ro["err2"] * (1 + 1e-12))


# --------------------------------------------------------------------------- Ex. 3 fill-in and PSNR
def test_fill_in_invariants(orc):
    """C <- T .* M + (1 - T) .* X: observed entries equal M, the others X,
    applying it twice changes nothing, and the reported change is the squared
    distance of the old and new C (checked on entries chosen by hand)."""
    r = np.random.default_rng(5)
    M, X, C0 = r.standard_normal(200), r.standard_normal(200), r.standard_normal(200)
    T = (r.random(200) < 0.3).astype(np.uint8)
    C1, ch = orc.fill_in(C0, M, T, X)
    assert np.array_equal(C1[T == 1], M[T == 1]) and np.array_equal(C1[T == 0], X[T == 0])
    C2, ch2 = orc.fill_in(C1, M, T, X)
    assert np.array_equal(C2, C1) and ch2 == 0.0
    Cz, chz = orc.fill_in(np.zeros(3), np.array([1.0, 2.0, 3.0]), np.array([1, 0, 1], np.uint8),
                          np.array([7.0, -2.0, 9.0]))
    assert np.array_equal(Cz, [1.0, -2.0, 3.0]) and chz == 1.0 + 4.0 + 9.0


def test_psnr_closed_forms(orc):
    """PSNR of Sec. 5: a constant offset d gives 10 log10(255^2 / d^2); equal
    images give +inf; scaling the error by 10 lowers the PSNR by 20 dB."""
    X = np.random.default_rng(6).uniform(0, 255, (3, 8, 8))
    assert abs(orc.psnr(X, X + 2.0) - 10 * np.log10(255.0 ** 2 / 4.0)) < 1e-12
    assert orc.psnr(X, X) == np.inf
    E = np.random.default_rng(7).standard_normal(X.shape)
    assert abs(orc.psnr(X, X + E) - orc.psnr(X, X + 10 * E) - 20.0) < 1e-9
