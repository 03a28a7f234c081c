"""T-QR (Alg. TQR) and the Moore-Penrose pseudoinverse (Alg. mp) through the
C ABI against the FP64 CPU oracle: element by element (the QR with diag(R_k)
real and >= 0 is unique for full-rank slices), plus the defining identities
X = Q * R, Q^T * Q = I and the Penrose conditions on the GPU results.  Shapes
cover tall, wide and square slices, one Fourier slice, several column blocks
of the orthonormalisation (p > 128) and ragged triangular-inverse blocks."""
import numpy as np
import pytest

from paper_2504_04989_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(70, 45, 9), (40, 66, 8), (64, 64, 5), (33, 17, 1), (300, 200, 6), (150, 260, 4)]


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2504_04989_gb300 import api as a
    return a


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _input(n1, n2, n3, seed):
    X = np.random.default_rng(seed).standard_normal((n3, n1, n2))
    if n1 == n2:
        X[0] += 3 * np.eye(n1)  # keep square slices well conditioned
    return X


@pytest.mark.parametrize("n1,n2,n3", SHAPES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tqr_against_oracle(api, orc, n1, n2, n3, precision):
    X = _input(n1, n2, n3, 11)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Xd = torch.from_numpy(X).to("cuda", dt)
    Q, R, info = api.tqr(Xd, precision, return_info=True)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["dead_columns"] == 0
    Qo, Ro = orc.tqr(Xd.double().cpu().numpy())
    tol = 1e-10 if precision == "fp64" else 2e-4
    assert _rel(Q.double().cpu().numpy(), Qo) < tol
    assert _rel(R.double().cpu().numpy(), Ro) < tol
    # identities on the GPU result (FP64 t-products of the returned factors)
    p = min(n1, n2)
    Qg, Rg = Q.double(), R.double()
    QtQ = api.tprod(api.ttranspose(Qg), Qg, "fp64").cpu().numpy()
    I = np.zeros((n3, p, p))
    I[0] = np.eye(p)
    assert np.abs(QtQ - I).max() < (1e-12 if precision == "fp64" else 1e-5) * np.sqrt(p)
    assert _rel(api.tprod(Qg, Rg, "fp64").cpu().numpy(), Xd.double().cpu().numpy()) < tol


def test_tqr_rank_deficient_keeps_orthonormal_q(api):
    X = wl.low_tubal_rank(30, 20, 4, [3.0, 2.0, 1.0], seed=5)
    Xd = torch.from_numpy(X).cuda()
    Q, R, info = api.tqr(Xd, "fp64", return_info=True)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["dead_columns"] > 0
    QtQ = api.tprod(api.ttranspose(Q), Q, "fp64").cpu().numpy()
    I = np.zeros((4, 20, 20))
    I[0] = np.eye(20)
    assert np.abs(QtQ - I).max() < 1e-12
    assert _rel(api.tprod(Q, R, "fp64").cpu().numpy(), X) < 1e-12


@pytest.mark.parametrize("n1,n2,n3", SHAPES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tpinv_against_oracle(api, orc, n1, n2, n3, precision):
    X = _input(n1, n2, n3, 12)
    dt = torch.float64 if precision == "fp64" else torch.float32
    Xd = torch.from_numpy(X).to("cuda", dt)
    P, info = api.tpinv(Xd, precision, return_info=True)
    torch.cuda.synchronize()
    assert info["status"] == 0
    Po = orc.tpinv(Xd.double().cpu().numpy())
    assert _rel(P.double().cpu().numpy(), Po) < (1e-9 if precision == "fp64" else 1e-3)
    if precision == "fp64":  # the four Penrose conditions on the GPU result
        A, Pg = Xd, P
        AP, PA = api.tprod(A, Pg, "fp64"), api.tprod(Pg, A, "fp64")
        assert _rel(api.tprod(AP, A, "fp64").cpu().numpy(), X) < 1e-10
        assert _rel(api.tprod(PA, Pg, "fp64").cpu().numpy(), Po) < 1e-9
        assert _rel(api.ttranspose(AP).cpu().numpy(), AP.cpu().numpy()) < 1e-10
        assert _rel(api.ttranspose(PA).cpu().numpy(), PA.cpu().numpy()) < 1e-10


def test_tpinv_reports_rank_deficiency(api):
    X = wl.low_tubal_rank(30, 20, 4, [3.0, 2.0, 1.0], seed=6)
    _, info = api.tpinv(torch.from_numpy(X).cuda(), "fp64", return_info=True)
    assert info["status"] == -6 and info["dead_columns"] > 0
