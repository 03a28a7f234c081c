"""GPU parity of the randomized block Krylov truncated T-SVD (Alg. 2) against
the CPU oracle: Fourier-domain singular values element by element and the
reconstruction error, never the sign/phase-ambiguous factors."""
import numpy as np
import pytest

from paper_2504_04989_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# tolerances: singular values 1e-10 relative on the FP64 path, 1e-4 on the
# FP32 and mixed paths; reconstruction error within 1e-3 of the oracle's.
SIG_TOL = {"fp64": 1e-10, "fp32": 1e-4, "tf32": 1e-4, "bf16": 1e-4}
ERR_TOL = 1e-3


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2504_04989_gb300 import api as a
    return a


def dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def weights(n3):
    h = n3 // 2 + 1
    w = np.full(h, 2.0)
    w[0] = 1.0
    if n3 % 2 == 0:
        w[-1] = 1.0
    return w


def run_gpu(api, X, R, P, q, precision, omega=None, seed=0, fp64_qr=False):
    dt = torch.float64 if precision == "fp64" else torch.float32
    om = None if omega is None else dev(omega.astype(np.float32) if dt == torch.float32 else omega, dt)
    U, S, V, sig, info = api.rbk(dev(X, dt), R, P, q, seed=seed, precision=precision, omega=om, return_info=True,
                                 fp64_qr=fp64_qr)
    torch.cuda.synchronize()
    assert info["status"] == 0, info
    return U.double().cpu().numpy(), S.double().cpu().numpy(), V.double().cpu().numpy(), sig.cpu().numpy(), info


def check_against_oracle(api, orc, X, R, P, q, precision, omega=None, seed=0, sig_floor=0.0, fp64_qr=False):
    n3 = X.shape[0]
    Xin = X.astype(np.float32).astype(np.float64) if precision != "fp64" else X
    om_in = None
    if omega is not None:
        om_in = omega.astype(np.float32).astype(np.float64) if precision != "fp64" else omega
    U, S, V, sig, info = run_gpu(api, Xin, R, P, q, precision, om_in, seed, fp64_qr)
    ref = orc.rtsvd_fourier(Xin, R, P, q, omega=om_in, seed=seed)
    s_ref = ref["sig"]
    mask = s_ref > sig_floor * s_ref.max()
    rel = np.abs(sig - s_ref)[mask] / s_ref[mask]
    assert rel.max() < SIG_TOL[precision], (rel.max(), np.unravel_index(np.argmax(rel), rel.shape))
    e_orc = np.sqrt(np.sum(weights(n3) * ref["err2"]) / n3)
    Xr = orc.reconstruct(U, S, V)
    e_gpu = np.linalg.norm((Xin - Xr).ravel())
    nx = np.linalg.norm(Xin.ravel())
    assert abs(e_gpu - e_orc) <= ERR_TOL * e_orc + 1e-12 * nx, (e_gpu, e_orc)
    assert info["m_eff"] == min((q + 1) * (R + P), X.shape[1], X.shape[2])
    return sig, s_ref, e_gpu / nx, e_orc / nx, info


def test_c1_fp64_with_given_omega(api, orc):
    X = wl.make_c1(0)
    om = wl.omega(64, 15, 16, seed=0)
    check_against_oracle(api, orc, X, 10, 5, 2, "fp64", omega=om)


def test_c1_fp64_philox_omega(api, orc):
    """Omega drawn on each side from the same Philox stream (seed 0)."""
    X = wl.make_c1(0)
    check_against_oracle(api, orc, X, 10, 5, 2, "fp64", seed=0)
    check_against_oracle(api, orc, X, 10, 5, 2, "fp64", seed=12345)


@pytest.mark.parametrize("fp64_qr", [False, True])
def test_c1_fp32(api, orc, fp64_qr):
    X = wl.make_c1(0)
    om = wl.omega(64, 15, 16, seed=0)
    check_against_oracle(api, orc, X, 10, 5, 2, "fp32", omega=om, fp64_qr=fp64_qr)


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_c1_mixed_tensor_core(api, orc, precision):
    """Basis-building products X-hat Omega and X-hat Y_i on tcgen05 (TF32 /
    BF16 operands, FP32 accumulation); C = Q^H X-hat and everything after it
    as on the FP32 path.  Same sigma tolerance as the FP32 path."""
    X = wl.make_c1(0)
    om = wl.omega(64, 15, 16, seed=0)
    with api.profile() as pr:
        check_against_oracle(api, orc, X, 10, 5, 2, precision, omega=om)
    assert "krylov_gemm_tc" in pr.stages  # the tcgen05 kernel ran


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
@pytest.mark.parametrize("n1,n2,n3,R,P,q", [(65, 129, 7, 6, 4, 3), (130, 63, 4, 12, 4, 2)])
def test_mixed_ragged_shapes(api, orc, n1, n2, n3, R, P, q, precision):
    """Odd n2 (padded tensor-core rows), M and N not multiples of the 128 tiles."""
    X = wl.low_tubal_rank(n1, n2, n3, np.arange(1, min(n1, n2) + 1) ** -1.0, noise_std=1e-4, seed=n1 + n3)
    om = wl.omega(n2, R + P, n3, seed=3)
    check_against_oracle(api, orc, X, R, P, q, precision, omega=om, sig_floor=1e-6)


@pytest.mark.parametrize("n1,n2,n3,R,P,q,precision", [
    (480, 480, 32, 100, 20, 3, "fp32"),   # m = 480 on 17 slices: clusters of 8 CTAs
    (400, 410, 38, 90, 10, 3, "tf32"),    # m = 400 on 20 slices: clusters of 4
    (340, 340, 158, 75, 10, 3, "fp32"),   # m = 340 on 80 slices: one CTA per slice
])
def test_l2_row_tridiagonalisation_shapes(api, orc, n1, n2, n3, R, P, q, precision):
    """Eigen-problems whose packed rows do not fit in a cluster's shared memory:
    the one-sweep double-float reduction with the rows in L2, at three of the
    cluster sizes it takes (the 2048 x 2048 x 128 test covers clusters of 2),
    and bitwise the same on a second run (its sums have a fixed order)."""
    X = wl.low_tubal_rank(n1, n2, n3, np.arange(1, min(n1, n2) + 1) ** -1.0, noise_std=1e-4, seed=n1 + n3)
    om = wl.omega(n2, R + P, n3, seed=9)
    sig, _, _, _, _ = check_against_oracle(api, orc, X, R, P, q, precision, omega=om, sig_floor=1e-6)
    again = run_gpu(api, X.astype(np.float32).astype(np.float64), R, P, q, precision,
                    om.astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(again[3], sig)


@pytest.mark.parametrize("n1,n2,n3,R,P,q", [
    (70, 90, 1, 5, 3, 2),     # n3 = 1: the matrix block Krylov method
    (40, 33, 2, 4, 2, 1),     # only DC and Nyquist slices
    (65, 129, 7, 6, 4, 3),    # odd n3, ragged tiles, n1 < n2
    (150, 70, 5, 3, 0, 0),    # P = 0, q = 0: plain range finder
    (33, 40, 8, 10, 10, 4),   # (q+1)(R+P) > min(n1, n2): basis clamped to 33
    (20, 24, 6, 1, 2, 1),     # R = 1
])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_shapes_and_edge_cases(api, orc, n1, n2, n3, R, P, q, precision):
    X = wl.low_tubal_rank(n1, n2, n3, np.arange(1, min(n1, n2) + 1) ** -1.0, noise_std=1e-4, seed=n1 + n3)
    om = wl.omega(n2, R + P, n3, seed=3)
    check_against_oracle(api, orc, X, R, P, q, precision, omega=om, sig_floor=1e-6 if precision == "fp32" else 0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_exact_low_tubal_rank_recovery(api, orc, precision):
    """Noise-free tubal rank 6 < R + P: dependent Krylov columns are replaced
    (dead_columns > 0) and the tensor is recovered to rounding level."""
    sig = np.linspace(5, 1, 6)
    X = wl.low_tubal_rank(48, 40, 9, sig, seed=21)
    dt = torch.float64 if precision == "fp64" else torch.float32
    U, S, V, s, info = run_gpu(api, X if precision == "fp64" else X.astype(np.float32), 6, 4, 2, precision)
    if precision == "fp64":  # FP32 rounding noise keeps the extra directions alive
        assert info["dead_columns"] > 0
    np.testing.assert_allclose(s, np.tile(sig, (5, 1)), rtol=1e-12 if precision == "fp64" else 1e-5)
    Xr = orc.reconstruct(U, S, V)
    err = np.linalg.norm((X - Xr).ravel()) / np.linalg.norm(X.ravel())
    assert err < (1e-12 if precision == "fp64" else 1e-5)


def test_zero_tensor(api):
    for precision in ("fp64", "fp32"):
        X = np.zeros((4, 16, 12))
        U, S, V, s, info = run_gpu(api, X, 3, 2, 1, precision)
        assert np.all(s == 0) and np.all(np.isfinite(U)) and np.all(np.isfinite(V))
        assert np.all(S == 0)


@pytest.mark.parametrize("n1,n2,n3,R,P,q,precision", [
    (65, 129, 7, 6, 4, 3, "fp32"),       # ragged tiles
    (300, 410, 10, 40, 10, 3, "tf32"),   # m = 200
    (64, 4096, 2, 10, 5, 1, "fp32"),     # n2 = 4096: digit-product sums nearest 2^24
    (1100, 700, 4, 100, 20, 3, "tf32"),  # m = 480, tensor-core orthonormalisation
])
def test_sliced_gram_bitwise_equals_integer_gram(api, n1, n2, n3, R, P, q, precision):
    """The exact Gram in base-64 digits on the BF16 tensor cores gives the same G as
    the 64-bit integer kernel, so the whole T-SVD is bitwise the same."""
    X = wl.low_tubal_rank(n1, n2, n3, np.arange(1, min(n1, n2) + 1) ** -1.0, noise_std=1e-4, seed=n2 + n3)
    om = wl.omega(n2, R + P, n3, seed=11).astype(np.float32)
    Xd, od = dev(X, torch.float32), dev(om, torch.float32)
    a = api.rbk(Xd, R, P, q, precision=precision, omega=od)
    b = api.rbk(Xd, R, P, q, precision=precision, omega=od, gram_int=True)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_deterministic(api):
    X = wl.make_c1(1)
    a = run_gpu(api, X, 10, 5, 2, "fp64", seed=3)
    b = run_gpu(api, X, 10, 5, 2, "fp64", seed=3)
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)


def test_invariants_on_gpu_output(api, orc):
    """Alg. 2 output properties at any size: U^T*U = I, V^T*V = I (tensor
    orthogonality, Sec. 2), singular values descending, and the error never
    below the Eckart-Young optimum (closed form for this construction)."""
    sig = np.arange(1, 61) ** -1.2
    X = wl.low_tubal_rank(60, 60, 8, sig, seed=5)
    R = 8
    for precision, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        U, S, V, s, _ = run_gpu(api, X, R, 6, 2, precision)
        I = np.zeros((8, R, R))
        I[0] = np.eye(R)
        np.testing.assert_allclose(orc.tprod(orc.ttranspose(U), U), I, atol=tol * 10)
        np.testing.assert_allclose(orc.tprod(orc.ttranspose(V), V), I, atol=tol * 10)
        assert np.all(np.diff(s, axis=1) <= tol)
        err2 = np.sum((X - orc.reconstruct(U, S, V)) ** 2)
        assert err2 >= wl.optimal_error2(sig, R) * (1 - 1e-6)


def test_error_monotone_in_q(api, orc):
    X = wl.low_tubal_rank(80, 64, 6, np.arange(1, 65) ** -0.8, seed=9)
    om = wl.omega(64, 9, 6, seed=4)
    errs = []
    for q in range(4):
        U, S, V, _, _ = run_gpu(api, X, 6, 3, q, "fp64", omega=om)
        errs.append(np.sum((X - orc.reconstruct(U, S, V)) ** 2))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(3))


@pytest.mark.slow
def test_c2_full_size_fp32_sampled_slices(api, orc):
    """Image-like workload 512 x 512 x 64, sigma_i = i^-1.5, R=50, P=10, q=4 in
    the configuration bench.py times; the oracle computes sampled slices."""
    X = wl.make_c2(0).astype(np.float32)
    om = wl.omega(512, 60, 64, seed=0).astype(np.float32)
    U, S, V, sig, info = run_gpu(api, X.astype(np.float64), 50, 10, 4, "fp32", om.astype(np.float64))
    slices = [0, 1, 16, 32]
    ref = orc.rtsvd_fourier(X.astype(np.float64), 50, 10, 4, omega=om.astype(np.float64), slices=slices)
    rel = np.abs(sig[slices] - ref["sig"]) / ref["sig"]
    assert rel.max() < SIG_TOL["fp32"], rel.max()
    # global error vs the Eckart-Young optimum sum_{i>50} sigma_i^2 (closed form)
    e2 = np.sum((X.astype(np.float64) - orc.reconstruct(U, S, V)) ** 2)
    opt = wl.optimal_error2(wl.c2_sigma(512), 50)
    assert opt <= e2 * (1 + 1e-4)
    # per-slice Fourier errors of the oracle on the sampled slices, vs the GPU's (Parseval)
    Xh = np.fft.rfft(X.astype(np.float64), axis=0)[slices]
    Uh = np.fft.rfft(U, axis=0)[slices]
    Vh = np.fft.rfft(V, axis=0)[slices]
    for j in range(len(slices)):
        g = np.linalg.norm(Xh[j] - (Uh[j] * sig[slices[j]]) @ Vh[j].conj().T) ** 2
        assert abs(g - ref["err2"][j]) <= ERR_TOL * ref["err2"][j], (slices[j], g, ref["err2"][j])


@pytest.mark.slow
def test_c2_full_size_fp64_sampled_slices(api, orc):
    """The FP64 path on the 512 x 512 x 64 workload: sigma-hat on sampled
    Fourier slices (DC, interior, Nyquist) within 1e-10 of the oracle, and the
    per-slice Fourier errors within 1e-3 of the oracle's."""
    X = wl.make_c2(0).astype(np.float32).astype(np.float64)
    om = wl.omega(512, 60, 64, seed=0)
    U, S, V, sig, info = run_gpu(api, X, 50, 10, 4, "fp64", om)
    slices = [0, 11, 32]
    ref = orc.rtsvd_fourier(X, 50, 10, 4, omega=om, slices=slices)
    rel = np.abs(sig[slices] - ref["sig"]) / ref["sig"]
    assert rel.max() < SIG_TOL["fp64"], rel.max()
    Xh = np.fft.rfft(X, axis=0)[slices]
    Uh = np.fft.rfft(U, axis=0)[slices]
    Vh = np.fft.rfft(V, axis=0)[slices]
    for j in range(len(slices)):
        g = np.linalg.norm(Xh[j] - (Uh[j] * sig[slices[j]]) @ Vh[j].conj().T) ** 2
        assert abs(g - ref["err2"][j]) <= ERR_TOL * ref["err2"][j], (slices[j], g, ref["err2"][j])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n1,n2,n3,R,P,q", [(64, 64, 16, 10, 5, 2), (65, 129, 7, 6, 4, 3), (40, 33, 2, 4, 2, 1)])
def test_alg1_against_oracle(api, orc, n1, n2, n3, R, P, q, precision):
    """Alg. 1 (power iteration, orthonormalised after every step) with the
    same kernels: sigma-hat against the oracle's Alg. 1 mode, and the
    invariant err(Alg. 2) <= err(Alg. 1) for the same Omega (nested spans)."""
    X = wl.make_c1(0) if (n1, n2, n3) == (64, 64, 16) else \
        wl.low_tubal_rank(n1, n2, n3, np.arange(1, min(n1, n2) + 1) ** -1.0, noise_std=1e-4, seed=n1 + n3)
    om = wl.omega(n2, R + P, n3, seed=5)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Xin = X if precision == "fp64" else X.astype(np.float32).astype(np.float64)
    omi = om if precision == "fp64" else om.astype(np.float32).astype(np.float64)
    U1, S1, V1, s1, info = api.rbk(dev(Xin, dt), R, P, q, precision=precision, omega=dev(omi, dt), alg1=True,
                                   return_info=True)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["m_eff"] == min(R + P, n1, n2)
    ref = orc.rtsvd_fourier(Xin, R, P, q, mode="alg1", omega=omi)
    s1 = s1.cpu().numpy()
    mask = ref["sig"] > (1e-6 if precision == "fp32" else 0) * ref["sig"].max()
    rel = np.abs(s1 - ref["sig"])[mask] / ref["sig"][mask]
    assert rel.max() < SIG_TOL[precision], rel.max()
    U2, S2, V2, s2 = api.rbk(dev(Xin, dt), R, P, q, precision=precision, omega=dev(omi, dt))
    torch.cuda.synchronize()
    e1 = api.tsvd_error(dev(Xin, dt), U1, S1, V1).item()
    e2 = api.tsvd_error(dev(Xin, dt), U2, S2, V2).item()
    assert e2 <= e1 * (1 + (1e-10 if precision == "fp64" else 1e-4)), (e1, e2)


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_tensor_core_orthonormalisation_shapes(api, orc, precision):
    """From n1 = 1024 on, the FP32 block orthonormalisation runs its block Gram
    and W R^-1 on tcgen05 (split TF32): parity with the oracle on every slice
    of a 1040 x 300 x 6 tensor (ragged tiles: n1 not a multiple of 128,
    b = 30 and a last block of 30 columns)."""
    X = wl.low_tubal_rank(1040, 300, 6, np.arange(1, 301) ** -1.0, noise_std=1e-4, seed=77)
    om = wl.omega(300, 30, 6, seed=78)
    check_against_oracle(api, orc, X, 20, 10, 2, precision, omega=om, sig_floor=1e-6)
