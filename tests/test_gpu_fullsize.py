"""Full-size parity for the two large configurations, in the launch
configuration the library runs them in:

* video-like 2048 x 2048 x 128, sigma_i = 1/i with noise 1e-4 x RMS, R = 100,
  P = 20, q = 3: the mixed paths (basis products on tcgen05 in TF32 / BF16;
  TF32 with FP64 block orthonormalisation, as the configuration states it)
  and the FP64 path, against the FP64 oracle on four sampled Fourier slices
  (about half a minute per slice on one host core, run at once) and, on every
  slice, the bounds that hold at any size;
* the uneven batch of 256 tensors as one graph-captured batched call:
  bit-identical to separate calls, and the oracle on the smallest tensors."""
import numpy as np
import pytest

from paper_2504_04989_gb300 import workloads as wl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2504_04989_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def c3():
    return wl.make_c3(0)  # float32 (128, 2048, 2048)


C3_SLICES = [0, 21, 43, 64]  # DC, two interior slices, Nyquist


@pytest.fixture(scope="module")
def c3_oracle(orc, c3):
    """The FP64 oracle on the sampled Fourier slices of the 2048 x 2048 x 128
    workload (the Philox Omega of seed 0 on both sides)."""
    return orc.rtsvd_fourier(c3.astype(np.float64), 100, 20, 3, seed=0, slices=C3_SLICES)


def _slice_err2(api, Xd, U, S, V, sig, slices):
    """||X_k - U_k diag(sigma_k) V_k^H||_F^2 on Fourier slices, from the outputs (FP64 on the GPU)."""
    Xh = api.rfft3(Xd.double())[slices]
    Uh = api.rfft3(U.double())[slices]
    Vh = api.rfft3(V.double())[slices]
    s = sig[slices].to(Uh.dtype)
    Rk = Xh - (Uh * s[:, None, :]) @ Vh.conj().transpose(1, 2)
    return (Rk.abs() ** 2).sum(dim=(1, 2)).cpu().numpy()


@pytest.mark.parametrize("path", ["tf32", "bf16", "tf32+fp64_qr", "fp64"])
def test_c3_full_size_against_oracle(api, orc, c3, c3_oracle, path):
    """sigma-hat on the sampled slices within 1e-4 of the oracle's (mixed
    paths) or 1e-10 (FP64 path), per-slice Fourier errors within 1e-3 of the
    oracle's, and on every slice the bounds that hold at any size (Weyl: a Ritz
    value never exceeds the slice's singular value plus the noise's norm; the
    error never beats the truncation optimum of the noise-free part by more
    than the noise can explain)."""
    R, P, q = 100, 20, 3
    n3, n1, n2 = c3.shape
    precision = path.split("+")[0]
    Xd = torch.from_numpy(c3).cuda()
    if precision == "fp64":
        Xd = Xd.double()
    U, S, V, sig, info = api.rbk(Xd, R, P, q, seed=0, precision=precision, fp64_qr="fp64_qr" in path,
                                 return_info=True)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["m_eff"] == (q + 1) * (R + P)
    s = sig.cpu().numpy()
    ref = c3_oracle
    rel = np.abs(s[C3_SLICES] - ref["sig"]) / ref["sig"]
    assert rel.max() < (1e-10 if precision == "fp64" else 1e-4), rel.max()
    e_gpu = _slice_err2(api, Xd, U, S, V, sig, C3_SLICES)
    assert np.all(np.abs(e_gpu - ref["err2"]) <= 1e-3 * ref["err2"]), (e_gpu, ref["err2"])
    sigma = 1.0 / np.arange(1, R + 1)
    # noise: entries N(0, std^2) in space; per Fourier slice a complex Gaussian
    # matrix with entry variance std^2 n3, spectral norm <= std sqrt(n3)(sqrt(n1)+sqrt(n2)) (x1.2 margin)
    std = 1e-4 * np.sqrt(np.sum(sigma ** 2) / (n1 * n2))  # RMS of the noise-free entries (Parseval)
    eps = 1.2 * std * np.sqrt(n3) * (np.sqrt(n1) + np.sqrt(n2))
    tol = 1e-4 * sigma[0]
    assert np.all(s <= sigma[None, :] + eps + tol), np.max(s - sigma[None, :])
    assert np.all(s[:, :20] >= sigma[None, :20] * (1 - 1e-3) - eps), np.min(s[:, :20] / sigma[None, :20])
    e2 = api.tsvd_error(Xd.float() if precision != "fp64" else Xd, U, S, V).item()
    opt = wl.optimal_error2(1.0 / np.arange(1, n1 + 1), R)
    noise = std ** 2 * n1 * n2 * n3
    assert e2 <= 1.05 * (opt + noise), (e2, opt, noise)


def test_c4_full_batch(api, orc):
    items = wl.make_c4(0, 256)
    shapes = [(it["X"].shape[1], it["X"].shape[2], it["X"].shape[0]) for it in items]
    Rs = [it["R"] for it in items]
    xs = [torch.from_numpy(it["X"].astype(np.float32)).cuda() for it in items]
    plan = api.RbkBatchPlan(shapes, Rs, P=5, q=2, seed=0, precision="fp32", lanes=8, graph=True)
    U, S, V, sig = plan(xs)
    torch.cuda.synchronize()
    size = [np.prod(sh) for sh in shapes]
    order = np.argsort(size)
    for i in list(order[:2]) + [int(order[-1])]:  # two smallest and the largest: separate calls, bit-identical
        u, s_, v, sg = api.rbk(xs[i], Rs[i], 5, 2, seed=int(i), precision="fp32")
        torch.cuda.synchronize()
        assert torch.equal(sg, sig[i]) and torch.equal(u, U[i])
    for i in order[:2]:  # the oracle on the two smallest tensors (Omega from seed i on both sides)
        X = items[i]["X"].astype(np.float32).astype(np.float64)
        ref = orc.rtsvd_fourier(X, Rs[i], 5, 2, seed=int(i))
        s = sig[i].cpu().numpy()
        mask = ref["sig"] > 1e-6 * ref["sig"].max()
        rel = np.abs(s - ref["sig"])[mask] / ref["sig"][mask]
        assert rel.max() < 1e-4, (i, rel.max())
