"""GPU parity of the mode-3 transforms, the t-product, its adjoints and the
Philox stream, against the CPU oracle (element by element)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
rng = np.random.default_rng(99)


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as g
    g.build()
    from paper_2504_04989_gb300 import api as a
    return a


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


def rand(*s):
    return rng.standard_normal(s)


def test_philox_words_bit_exact(api, orc):
    key = (0x12345678, 0x9ABCDEF0)
    n = 1000
    got = api.philox_words(key, 7, 3, 11, n).cpu().numpy()
    for i in list(range(0, 20)) + [511, 999]:
        assert list(got[i]) == orc.philox4x32_10([i, 7, 3, 11], key)
    # the published known-answer vector with counter (0,0,0,0), key (0,0)
    w = api.philox_words((0, 0), 0, 0, 0, 1).cpu().numpy()[0]
    assert [int(x) for x in w] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


def test_gaussian_matches_oracle(api, orc):
    n = 100_003
    g = api.gaussian(5, n, stream_id=0, tensor_id=0).cpu().numpy()
    o = orc.gaussian(5, n)
    np.testing.assert_allclose(g, o, rtol=1e-13, atol=1e-13)


# sizes that span several 64-wide tiles with ragged tails, odd / even / tiny n3
SHAPES = [(1, 1, 1, 1), (3, 5, 2, 1), (7, 9, 4, 2), (33, 70, 65, 3), (65, 31, 129, 8), (40, 17, 23, 16),
          (20, 30, 10, 100), (130, 64, 5, 5)]


@pytest.mark.parametrize("n1,n2,n4,n3", SHAPES)
def test_tprod_fp64(api, orc, n1, n2, n4, n3):
    A, B = rand(n3, n1, n2), rand(n3, n2, n4)
    C = api.tprod(dev(A), dev(B)).cpu().numpy()
    np.testing.assert_allclose(C, orc.tprod(A, B), rtol=0, atol=1e-11 * np.sqrt(n2 * n3))


@pytest.mark.parametrize("n1,n2,n4,n3", SHAPES)
def test_tprod_fp32(api, orc, n1, n2, n4, n3):
    A, B = rand(n3, n1, n2), rand(n3, n2, n4)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    C = api.tprod(dev(A32, torch.float32), dev(B32, torch.float32)).cpu().numpy()
    ref = orc.tprod(A32.astype(np.float64), B32.astype(np.float64))
    # FP32 storage and accumulation: error ~ eps32 * sqrt(n2 n3) * |A||B|
    np.testing.assert_allclose(C, ref, rtol=0, atol=2e-6 * np.sqrt(n2 * n3) * 4)


@pytest.mark.parametrize("n1,n2,n4,n3", [(3, 4, 2, 1), (9, 17, 70, 6), (65, 40, 3, 7)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tprod_backward(api, orc, n1, n2, n4, n3, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    A, B, dC = rand(n3, n1, n2), rand(n3, n2, n4), rand(n3, n1, n4)
    if precision == "fp32":
        A, B, dC = (x.astype(np.float32).astype(np.float64) for x in (A, B, dC))
    dA, dB = api.tprod_backward(dev(A, dt), dev(B, dt), dev(dC, dt), precision)
    rA, rB = orc.tprod_backward(A, B, dC)
    tol = 1e-11 if precision == "fp64" else 2e-5
    np.testing.assert_allclose(dA.cpu().numpy(), rA, rtol=0, atol=tol * np.sqrt(n4 * n3) * 4)
    np.testing.assert_allclose(dB.cpu().numpy(), rB, rtol=0, atol=tol * np.sqrt(n1 * n3) * 4)


@pytest.mark.parametrize("n1,m,n2,n3", [(5, 2, 3, 1), (33, 7, 65, 4), (70, 20, 9, 9)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tproj_and_backward(api, orc, n1, m, n2, n3, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    Q, A, dY = rand(n3, n1, m), rand(n3, n1, n2), rand(n3, n1, n2)
    if precision == "fp32":
        Q, A, dY = (x.astype(np.float32).astype(np.float64) for x in (Q, A, dY))
    Y = api.tproj(dev(Q, dt), dev(A, dt), precision).cpu().numpy()
    Yref = orc.tprod(Q, orc.tprod(orc.ttranspose(Q), A))
    tol = 1e-11 if precision == "fp64" else 3e-5
    scale = np.sqrt(n1 * m) * n3
    np.testing.assert_allclose(Y, Yref, rtol=0, atol=tol * scale * 4)
    dQ, dA = api.tproj_backward(dev(Q, dt), dev(A, dt), dev(dY, dt), precision)
    rQ, rA = orc.tproj_backward(Q, A, dY)
    np.testing.assert_allclose(dA.cpu().numpy(), rA, rtol=0, atol=tol * scale * 4)
    np.testing.assert_allclose(dQ.cpu().numpy(), rQ, rtol=0, atol=tol * scale * 8)


def test_autograd_tprod_matches_oracle_gradient(api, orc):
    A, B = rand(6, 8, 5), rand(6, 5, 7)
    W = rand(6, 8, 7)
    At = dev(A).requires_grad_(True)
    Bt = dev(B).requires_grad_(True)
    L = (api.tprod(At, Bt) * dev(W)).sum()
    L.backward()
    rA, rB = orc.tprod_backward(A, B, W)
    np.testing.assert_allclose(At.grad.cpu().numpy(), rA, atol=1e-11)
    np.testing.assert_allclose(Bt.grad.cpu().numpy(), rB, atol=1e-11)


def test_autograd_gradcheck_fp64(api):
    A = dev(rand(5, 4, 3)).requires_grad_(True)
    B = dev(rand(5, 3, 2)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: api.tprod(a, b), (A, B), eps=1e-6, atol=1e-8)
    Q = dev(rand(4, 6, 2)).requires_grad_(True)
    X = dev(rand(4, 6, 3)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda q, x: api.tproj(q, x), (Q, X), eps=1e-6, atol=1e-8)


# tensor-core t-product: TF32 / BF16 operands, FP32 accumulation (tcgen05)
TC_SHAPES = [(128, 128, 64, 4), (200, 96, 150, 7), (33, 70, 65, 3), (256, 512, 40, 16), (64, 31, 17, 5)]


@pytest.mark.parametrize("n1,n2,n4,n3", TC_SHAPES)
@pytest.mark.parametrize("precision,tol", [("tf32", 3e-3), ("bf16", 2e-2)])
def test_tprod_tensor_core(api, orc, n1, n2, n4, n3, precision, tol):
    A, B = rand(n3, n1, n2), rand(n3, n2, n4)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    with api.profile() as pr:
        C = api.tprod(dev(A32, torch.float32), dev(B32, torch.float32), precision)
        torch.cuda.synchronize()
    assert "tprod_gemm_tc" in pr.stages  # the tcgen05 kernel ran
    C = C.cpu().numpy()
    ref = orc.tprod(A32.astype(np.float64), B32.astype(np.float64))
    # operands rounded to TF32 (11-bit) / BF16 (8-bit significand): normwise relative error
    rel = np.linalg.norm((C - ref).ravel()) / np.linalg.norm(ref.ravel())
    assert rel < tol, rel
    # and element-wise against the scale of the summands
    scale = np.sqrt(n2 * n3) * np.max(np.abs(A32)) * np.max(np.abs(B32))
    assert np.max(np.abs(C - ref)) < 10 * tol * scale


@pytest.mark.parametrize("n1,n2,n4,n3", [(128, 128, 64, 4), (200, 130, 150, 7), (256, 512, 65, 16)])
def test_tprod_split_tf32_tensor_core(api, orc, n1, n2, n4, n3):
    """The split-TF32 t-product ("tf32x3": x = hi + lo, hi*hi + hi*lo + lo*hi on
    tcgen05) against the oracle, in the form of the TF32 / BF16 test above: a
    normwise relative error of 2e-5 (one TF32 pass: 3e-3), element-wise 10x
    that against the scale of the summands.  It is not held to the FP32 SIMT
    bound: its operands carry ~22 bits and the tensor-core accumulation of the
    three partial products loses a few more (measured: 9e-6 relative at the
    worst element of the 256 x 512 x 65 x 16 case)."""
    A, B = rand(n3, n1, n2), rand(n3, n2, n4)
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    with api.profile() as pr:
        C = api.tprod(dev(A32, torch.float32), dev(B32, torch.float32), "tf32x3")
        torch.cuda.synchronize()
    assert "tprod_gemm_tc" in pr.stages
    C = C.cpu().numpy()
    ref = orc.tprod(A32.astype(np.float64), B32.astype(np.float64))
    rel = np.linalg.norm((C - ref).ravel()) / np.linalg.norm(ref.ravel())
    assert rel < 2e-5, rel
    scale = np.sqrt(n2 * n3) * np.max(np.abs(A32)) * np.max(np.abs(B32))
    assert np.max(np.abs(C - ref)) < 10 * 2e-5 * scale
