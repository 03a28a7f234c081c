"""Fused approximation-error evaluation ||X - U*S*V^T||_F^2 (Fourier domain,
Parseval over the half spectrum) against the FP64 oracle: element-exact
definition on random factors, the zero-factor case, and the Rayleigh-Ritz
identity ||X||^2 - sum w_k sigma_k^2 / n3 on the outputs of Alg. 2."""
import numpy as np
import pytest

from paper_2504_04989_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
rng = np.random.default_rng(2025)


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2504_04989_gb300 import api as a
    return a


def dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)


# ragged 64-wide tiles, R across 16-wide rank rounds, odd / even / unit n3
SHAPES = [(1, 1, 1, 1), (7, 9, 4, 3), (33, 70, 5, 10), (65, 31, 8, 40), (130, 64, 3, 17), (20, 129, 16, 1)]


@pytest.mark.parametrize("n1,n2,n3,R", SHAPES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_error_matches_oracle_definition(api, orc, n1, n2, n3, R, precision):
    X = rng.standard_normal((n3, n1, n2))
    U = rng.standard_normal((n3, n1, R))
    S = rng.standard_normal((n3, R))
    V = rng.standard_normal((n3, n2, R))
    if precision == "fp32":
        X, U, S, V = (a.astype(np.float32).astype(np.float64) for a in (X, U, S, V))
    dt = torch.float64 if precision == "fp64" else torch.float32
    got = api.tsvd_error(dev(X, dt), dev(U, dt), dev(S, dt), dev(V, dt)).item()
    ref = float(np.sum((X - orc.reconstruct(U, S, V)) ** 2))
    tol = 1e-12 if precision == "fp64" else 2e-5
    assert abs(got - ref) <= tol * ref, (got, ref)


def test_zero_factors_give_norm(api):
    X = rng.standard_normal((6, 40, 70))
    z = torch.zeros
    got = api.tsvd_error(dev(X, torch.float64), z((6, 40, 3), dtype=torch.float64, device="cuda"),
                         z((6, 3), dtype=torch.float64, device="cuda"),
                         z((6, 70, 3), dtype=torch.float64, device="cuda")).item()
    assert abs(got - np.sum(X ** 2)) <= 1e-13 * np.sum(X ** 2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_error_of_rbk_output(api, orc, precision):
    """On the 64x64x16 tubal-rank-10 workload: the fused error equals the
    oracle's reconstruction error of the same factors, and the Rayleigh-Ritz
    identity ||X - U S V^T||^2 = ||X||^2 - (1/n3) sum_k w_k sum_i sigma_ik^2."""
    X = wl.make_c1(0)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Xin = X if precision == "fp64" else X.astype(np.float32).astype(np.float64)
    Xd = dev(Xin, dt)
    U, S, V, sig = api.rbk(Xd, 10, 5, 2, precision=precision)
    got = api.tsvd_error(Xd, U, S, V).item()
    ref = float(np.sum((Xin - orc.reconstruct(U.double().cpu().numpy(), S.double().cpu().numpy(),
                                              V.double().cpu().numpy())) ** 2))
    assert abs(got - ref) <= (1e-10 if precision == "fp64" else 1e-4) * ref, (got, ref)
    n3 = X.shape[0]
    w = np.full(n3 // 2 + 1, 2.0)
    w[0] = 1.0
    if n3 % 2 == 0:
        w[-1] = 1.0
    s = sig.cpu().numpy()
    ident = np.sum(Xin ** 2) - np.sum(w[:, None] * s ** 2) / n3
    nx = np.sum(Xin ** 2)
    # FP32 path: the products forming C carry about 22 significant bits (split TF32 on the
    # tensor cores), so the identity holds to ~2^-22 sqrt(n) relative; the sigma tolerance
    # of the path (1e-4) would allow 2e-4
    assert abs(got - ident) <= (1e-12 if precision == "fp64" else 1e-5) * nx, (got, ident)
