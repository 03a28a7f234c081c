"""The per-rank step of the slice-sharded path on one GPU: tsvd_rbk_fourier
on sub-ranges of Fourier slices against tsvd_rbk on the whole tensor, the
exported transforms against the oracle's DFT, and the sharded driver at world
size 1 (its exchanges are then local) against tsvd_rbk."""
import numpy as np
import pytest

from paper_2504_04989_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2504_04989_gb300 import api as a
    return a


@pytest.mark.parametrize("n3", [7, 16])
def test_transforms_against_oracle(api, orc, n3):
    X = np.random.default_rng(3).standard_normal((n3, 9, 13))
    Xh = api.rfft3(torch.from_numpy(X).cuda())
    np.testing.assert_allclose(Xh.cpu().numpy(), orc.dft_mode3(X), atol=1e-12 * n3)
    back = api.irfft3(Xh, n3)
    np.testing.assert_allclose(back.cpu().numpy(), X, atol=1e-13)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fourier_slices_match_whole_tensor(api, precision):
    n1, n2, n3, R, P, q = 96, 80, 12, 6, 4, 2
    X = wl.low_tubal_rank(n1, n2, n3, np.arange(1, 41) ** -1.0, noise_std=1e-3, seed=9)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Xd = torch.from_numpy(X).to("cuda", dt)
    U0, _, V0, sig = api.rbk(Xd, R, P, q, seed=4, precision=precision)
    Ah = api.rfft3(Xd)
    U0h, V0h = api.rfft3(U0), api.rfft3(V0)
    tol = 1e-10 if precision == "fp64" else 1e-4

    def resid(Uh, s, Vh, A):
        return torch.linalg.vector_norm(A - (Uh * s.to(Uh.dtype)[:, None, :]) @ Vh.conj().transpose(1, 2)).item()

    for k0, k1 in ((0, 7), (2, 5), (6, 7)):
        Uh, Vh, sg, info = api.rbk_fourier(Ah[k0:k1], n3, k0, R, P, q, seed=4, precision=precision, return_info=True)
        torch.cuda.synchronize()
        assert info["status"] == 0
        rel = (sg - sig[k0:k1]).abs() / sig[k0:k1]
        assert rel.max().item() < tol
        # the slice factors leave the same residual as the whole-tensor call's factors
        e = resid(Uh, sg, Vh, Ah[k0:k1])
        e0 = resid(U0h[k0:k1], sig[k0:k1], V0h[k0:k1], Ah[k0:k1])
        assert abs(e - e0) <= (1e-8 if precision == "fp64" else 1e-3) * e0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sharded_world_one_matches_rbk(api, precision):
    from paper_2504_04989_gb300 import sharded
    n1, n2, n3, R, P, q = 64, 64, 16, 10, 5, 2
    X = wl.make_c1(0)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Xd = torch.from_numpy(X).to("cuda", dt)
    U, S, V, sig = sharded.rbk_sharded(Xd, n1, n2, n3, R, P, q, seed=2, steps=sharded.CudaSteps(precision))
    U0, S0, V0, sig0 = api.rbk(Xd, R, P, q, seed=2, precision=precision)
    torch.cuda.synchronize()
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert ((sig - sig0).abs() / sig0).max().item() < tol
    e = api.tsvd_error(Xd, U, S, V).item()
    e0 = api.tsvd_error(Xd, U0, S0, V0).item()
    assert abs(e - e0) <= 1e-6 * e0
