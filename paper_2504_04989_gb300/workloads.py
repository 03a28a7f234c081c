"""Seeded synthetic workloads shaped like the paper's image / video / hyperspectral
data (arXiv 2504.04989, Sec. 5), and the Gaussian test tensor Omega.

This module is the one input generator shared by the CUDA path, its tests and
the CPU oracle.  It holds none of the method's arithmetic: tensors are built in
the Fourier domain from numpy's own FFT and QR library routines and a numpy
PCG64 stream, so neither side under test can bias its inputs.

Layout: a real n1 x n2 x n3 tensor is a float64 array of shape (n3, n1, n2).

The paper's own datasets (Kodak images, etc.) are not reproduced; these tensors
stand in for them with the stated spectra.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(salt)])


def omega(n2: int, b: int, n3: int, seed: int = 0) -> np.ndarray:
    """Real Gaussian test tensor B = randn(n2, R+P, n3) (Alg. 2, first line;
    rows = n2 so that X * B is defined).  Shape (n3, n2, b)."""
    return _rng(seed, 1).standard_normal((n3, n2, b))


def haar_fourier_factor(n: int, r: int, n3: int, rng: np.random.Generator) -> np.ndarray:
    """Half spectrum (h, n, r) of a t-factor with orthonormal columns per
    Fourier slice: complex Haar (QR of a complex Gaussian, phases fixed) on the
    interior slices, real Haar on the DC and (even n3) Nyquist slices, so the
    spatial tensor is real."""
    h = n3 // 2 + 1
    out = np.empty((h, n, r), dtype=np.complex128)
    for k in range(h):
        real_slice = (k == 0) or (n3 % 2 == 0 and k == n3 // 2)
        if real_slice:
            G = rng.standard_normal((n, r))
        else:
            G = (rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r))) / np.sqrt(2.0)
        Q, Rf = np.linalg.qr(G)
        d = np.diagonal(Rf)
        ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
        out[k] = Q * ph[None, :]
    return out


def reflector_fourier_factor(n: int, n3: int, rng: np.random.Generator, nref: int = 4):
    """A cheap random unitary per Fourier slice for large n: product of `nref`
    random Householder reflectors and a random diagonal phase (real +-1 on the
    DC / Nyquist slices).  Returned as (vs, phases) to be applied, not formed."""
    h = n3 // 2 + 1
    vs, phs = [], []
    for k in range(h):
        real_slice = (k == 0) or (n3 % 2 == 0 and k == n3 // 2)
        if real_slice:
            V = rng.standard_normal((nref, n))
            ph = np.sign(rng.standard_normal(n)) + 0j
        else:
            V = rng.standard_normal((nref, n)) + 1j * rng.standard_normal((nref, n))
            ph = np.exp(2j * np.pi * rng.random(n))
        V /= np.linalg.norm(V, axis=1, keepdims=True)
        vs.append(V)
        phs.append(ph)
    return vs, phs


def _apply_reflectors_left(vs: np.ndarray, ph: np.ndarray, M: np.ndarray) -> np.ndarray:
    """(H_1 ... H_r D) M with H_j = I - 2 v_j v_j^H, D = diag(ph)."""
    M = ph[:, None] * M
    for v in vs[::-1]:
        M = M - 2.0 * np.outer(v, v.conj() @ M)
    return M


def tensor_from_fourier(Xhat: np.ndarray, n3: int) -> np.ndarray:
    """Real spatial tensor (n3, n1, n2) from its half spectrum (library irfft)."""
    try:
        import scipy.fft as sf
        return sf.irfft(Xhat, n=n3, axis=0, workers=-1)
    except ImportError:
        return np.fft.irfft(Xhat, n=n3, axis=0)


def low_tubal_rank(n1: int, n2: int, n3: int, sigma, noise_std: float = 0.0, seed: int = 0,
                   return_parts: bool = False):
    """X = U * S * V^T + noise with Haar t-factors and the same singular values
    `sigma` (length r) on every Fourier slice (Ex. 1 style construction)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    r = len(sigma)
    rng = _rng(seed, 2)
    Uh = haar_fourier_factor(n1, r, n3, rng)
    Vh = haar_fourier_factor(n2, r, n3, rng)
    Xh = np.einsum("kir,r,kjr->kij", Uh, sigma, Vh.conj())
    X = tensor_from_fourier(Xh, n3)
    if noise_std > 0:
        X = X + noise_std * rng.standard_normal(X.shape)
    if return_parts:
        return X, {"Uhat": Uh, "Vhat": Vh, "sigma": sigma}
    return X


def _reflected_diagonal(d, uvs, uph, vvs, vph):
    """U diag(d) V^H for U = H_1..H_r diag(uph), V = H'_1..H'_r diag(vph)
    (H = I - 2 v v^H), kept as diag(d') + L R^H while the reflectors are
    applied (each adds one column to L and R), then formed by one n x 2r x n
    product.  Same matrix as applying the reflectors to the dense product."""
    n = d.shape[0]
    dd = (uph * d).astype(np.complex128)            # diag(uph) diag(d)
    L = np.zeros((n, 0), dtype=np.complex128)
    Rm = np.zeros((n, 0), dtype=np.complex128)
    for v in uvs[::-1]:                             # M <- H M: M - 2 v (M^H v)^H
        w = dd.conj() * v + Rm @ (L.conj().T @ v)
        L = np.concatenate([L, -2.0 * v[:, None]], axis=1)
        Rm = np.concatenate([Rm, w[:, None]], axis=1)
    dd = dd * vph.conj()                            # M <- M diag(vph)^H
    Rm = Rm * vph[:, None]
    for v in vvs[::-1]:                             # M <- M H': M - 2 (M v) v^H
        mv = dd * v + L @ (Rm.conj().T @ v)
        L = np.concatenate([L, -2.0 * mv[:, None]], axis=1)
        Rm = np.concatenate([Rm, v[:, None]], axis=1)
    M = L @ Rm.conj().T
    M[np.arange(n), np.arange(n)] += dd
    return M


def power_law_reflector(n1: int, n2: int, n3: int, sigma, noise_rel: float = 0.0, seed: int = 0,
                        dtype=np.float64):
    """Large full-spectrum tensor: Xhat_k = U_k diag(sigma) V_k^H with U_k, V_k
    random reflector products (exact singular values sigma on every slice),
    plus Gaussian noise of std noise_rel x RMS of the noise-free entries.
    Square slices (n1 == n2) with len(sigma) == n1."""
    sigma = np.asarray(sigma, dtype=np.float64)
    assert n1 == n2 == len(sigma)
    rng = _rng(seed, 3)
    h = n3 // 2 + 1
    uvs, uph = reflector_fourier_factor(n1, n3, rng)
    vvs, vph = reflector_fourier_factor(n2, n3, rng)
    Xh = np.empty((h, n1, n2), dtype=np.complex128)
    for k in range(h):
        Xh[k] = _reflected_diagonal(sigma, uvs[k], uph[k], vvs[k], vph[k])
    X = tensor_from_fourier(Xh, n3)
    del Xh
    if noise_rel > 0:
        rms = float(np.sqrt(np.mean(X * X)))
        X += noise_rel * rms * rng.standard_normal(X.shape, dtype=np.float32)
    return X.astype(dtype, copy=False)


def optimal_error2(sigma, R: int) -> float:
    """Eckart-Young closed form for the constructions above (no noise):
    ||X - X_R||_F^2 = (1/n3) sum_k sum_{i>R} sigma_i^2 = sum_{i>R} sigma_i^2,
    by Parseval (Sec. 2, the Parseval relation of the mode-3 DFT) and the per-slice matrix Eckart-Young theorem."""
    s = np.asarray(sigma, dtype=np.float64)
    return float(np.sum(s[R:] ** 2))


# ---------------------------------------------------------------------------
# Configurations (synthetic stand-ins; seeds fixed)
# ---------------------------------------------------------------------------
CONFIGS = {
    "c1": dict(name="plain-fp64 64x64x16 tubal-rank-10 + noise 1e-3", n1=64, n2=64, n3=16, R=10, P=5, q=2,
               precision="fp64"),
    "c2": dict(name="image-like fp32 512x512x64 sigma_i=i^-1.5", n1=512, n2=512, n3=64, R=50, P=10, q=4,
               precision="fp32"),
    "c3": dict(name="video-like mixed 2048x2048x128 sigma_i=1/i + 1e-4 noise", n1=2048, n2=2048, n3=128, R=100,
               P=20, q=3, precision="tf32"),
    "c5": dict(name="completion 256x256x100 tubal-rank-20, Bernoulli(0.3) mask", n1=256, n2=256, n3=100, R=20,
               P=10, q=2, precision="fp32"),
}


def make_c1(seed: int = 0) -> np.ndarray:
    return low_tubal_rank(64, 64, 16, np.linspace(10.0, 1.0, 10), noise_std=1e-3, seed=seed)


def c2_sigma(n: int = 512) -> np.ndarray:
    return np.arange(1, n + 1, dtype=np.float64) ** -1.5


def make_c2(seed: int = 0) -> np.ndarray:
    return low_tubal_rank(512, 512, 64, c2_sigma(512), noise_std=0.0, seed=seed)


def make_c3(seed: int = 0, n: int = 2048, n3: int = 128, dtype=np.float32) -> np.ndarray:
    sig = 1.0 / np.arange(1, n + 1, dtype=np.float64)
    return power_law_reflector(n, n, n3, sig, noise_rel=1e-4, seed=seed, dtype=dtype)


def make_c5(seed: int = 0):
    """Tubal-rank-20 256x256x100 tensor and a Bernoulli(0.3) observation mask."""
    X = low_tubal_rank(256, 256, 100, np.linspace(10.0, 1.0, 20), noise_std=0.0, seed=seed)
    mask = (_rng(seed, 4).random(X.shape) < 0.3)
    return X, mask


def ex1_sigma(n: int, case: int) -> np.ndarray:
    """Ex. 1 (Sec. 5) singular values of every frontal slice: case 1
    sigma_m = m^-5, case 2 m^-6, case 3 0.5^m, m = 1..n."""
    m = np.arange(1, n + 1, dtype=np.float64)
    return {1: m ** -5.0, 2: m ** -6.0, 3: 0.5 ** m}[case]


def make_ex1(n: int, case: int, seed: int = 0) -> np.ndarray:
    """n x n x n tensor with the Ex. 1 spectrum on every Fourier slice (Haar
    t-factors, no noise)."""
    return low_tubal_rank(n, n, n, ex1_sigma(n, case), noise_std=0.0, seed=seed)


def make_c4(seed: int = 0, count: int = 256):
    """Batch of `count` uneven tensors: n1, n2 ~ U{32..512}, n3 ~ U{8,16,32,64},
    exact tubal rank r ~ U{5..40} (clamped to min(n1, n2)) plus noise 1e-3;
    R = r, P = 5, q = 2.  Returns a list of dicts (X, R, P, q)."""
    rng = _rng(seed, 5)
    items = []
    for t in range(count):
        n1 = int(rng.integers(32, 513))
        n2 = int(rng.integers(32, 513))
        n3 = int(rng.choice([8, 16, 32, 64]))
        r = min(int(rng.integers(5, 41)), n1, n2)
        X = low_tubal_rank(n1, n2, n3, np.linspace(10.0, 1.0, r), noise_std=1e-3, seed=seed * 100003 + t)
        items.append(dict(X=X, R=r, P=5, q=2))
    return items


# ---------------------------------------------------------------------------
# Completion (Sec. 5, Ex. 3 and Ex. 4): image-like tensors and missing-pixel
# masks.  The Kodak images are not reproduced; an image-like tensor is a
# full-spectrum tensor with slowly decaying singular values, shifted and
# scaled to the 0..255 range of 8-bit pixels (n3 = 3 colour channels).
# ---------------------------------------------------------------------------
def make_image(n1: int = 256, n2: int = 256, n3: int = 3, rank: int = 20, noise: float = 0.5,
               seed: int = 0) -> np.ndarray:
    """Image-like (n3, n1, n2) float64 tensor in [0, 255]: tubal rank `rank`
    (sigma = linspace(3, 1, rank) on every Fourier slice, Haar t-factors),
    shifted to mean 128 with RMS contrast 40, plus Gaussian pixel noise of
    std `noise`, clipped to 0..255."""
    X = low_tubal_rank(n1, n2, n3, np.linspace(3.0, 1.0, rank), seed=seed)
    X = 128.0 + 40.0 * (X - X.mean()) / X.std()
    if noise > 0:
        X = X + noise * _rng(seed, 9).standard_normal(X.shape)
    return np.clip(X, 0.0, 255.0)


def mask_random(shape, missing: float, seed: int = 0) -> np.ndarray:
    """Observation mask (uint8, 1 = observed) with each pixel missing with
    probability `missing` (Ex. 3: 70 %, Ex. 4: 80 %)."""
    return (_rng(seed, 6).random(shape) >= missing).astype(np.uint8)


def mask_lines(shape, spacing: int = 16, width: int = 2, seed: int = 0) -> np.ndarray:
    """Structured mask: horizontal and vertical line segments `width` pixels
    wide, about one every `spacing` pixels, each of random length (a quarter
    to three quarters of the image) and position, the same in every frontal
    slice (Ex. 3's line patterns; a smaller spacing is the denser variant).
    Rows or columns missing over their whole length would carry no
    information for any low-rank completion, hence segments."""
    n3, n1, n2 = shape
    rng = _rng(seed, 7)
    m = np.ones((n1, n2), dtype=np.uint8)
    for n, other, axis in ((n1, n2, 0), (n2, n1, 1)):
        for start in range(int(rng.integers(0, spacing)), n, spacing):
            lo = int(np.clip(start + rng.integers(-spacing // 4, spacing // 4 + 1), 0, n - 1))
            length = int(rng.integers(other // 4, 3 * other // 4 + 1))
            a = int(rng.integers(0, other - length + 1))
            if axis == 0:
                m[lo:lo + width, a:a + length] = 0
            else:
                m[a:a + length, lo:lo + width] = 0
    return np.broadcast_to(m, shape).copy()


def mask_circles(shape, count: int = 40, radius: float = 6.0, seed: int = 0) -> np.ndarray:
    """Structured mask: `count` discs of the given radius missing at random
    centres, the same in every frontal slice (Ex. 3's circle patterns; more
    or larger discs are the denser variants)."""
    n3, n1, n2 = shape
    rng = _rng(seed, 8)
    ii, jj = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    m = np.ones((n1, n2), dtype=np.uint8)
    for _ in range(count):
        ci, cj = rng.uniform(0, n1), rng.uniform(0, n2)
        m[(ii - ci) ** 2 + (jj - cj) ** 2 <= radius * radius] = 0
    return np.broadcast_to(m, shape).copy()
