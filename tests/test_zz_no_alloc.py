"""tprod_noalloc: the t-product for callers that cannot allocate device memory
(a pool that must not grow, a plug-in whose host owns all device allocations, a
real-time loop), with its scratch in a fixed array inside the library.

Called through the C ABI and checked against the workspace-based tprod entry
point on two calls in a row, on a case that nearly fills the fixed array, and
against the FP64 CPU oracle; then for the size limit.  This file is collected
last on purpose."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2504_04989_gb300 import _lib
    return _lib.load()


def test_tprod_noalloc_matches_tprod_twice(lib):
    from paper_2504_04989_gb300 import api
    rng = np.random.default_rng(2024)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [((33, 70, 20, 16), "fp32", torch.float32, 1), ((20, 9, 31, 7), "fp64", torch.float64, 0)]
    for (n1, n2, n4, n3), prec, dt, code in cases:
        A = torch.from_numpy(rng.standard_normal((n3, n1, n2))).to("cuda", dt)
        B = torch.from_numpy(rng.standard_normal((n3, n2, n4))).to("cuda", dt)
        ref = api.tprod(A, B, prec)
        out = torch.full((n3, n1, n4), float("nan"), dtype=dt, device="cuda")
        rc = lib.tprod_noalloc(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), C.c_void_p(out.data_ptr()),
                               n1, n2, n4, n3, code, stream)
        assert rc == 0
        torch.cuda.synchronize()
        # the tolerances of the t-product parity tests
        atol = (2e-6 * 4 if prec == "fp32" else 1e-11) * np.sqrt(n2 * n3)
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=atol)


def test_tprod_noalloc_rejects_sizes_beyond_its_scratch(lib):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    A = torch.zeros(1, dtype=torch.float32, device="cuda")
    # (65 slices) x 3 x 256 x 256 complex FP32 = 102 MB > 16 MiB: rejected before any launch
    rc = lib.tprod_noalloc(C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()), C.c_void_p(A.data_ptr()),
                           256, 256, 256, 128, 1, stream)
    assert rc == -4


def _call(lib, A, B, out, n1, n2, n4, n3, code):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.tprod_noalloc(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), C.c_void_p(out.data_ptr()),
                             n1, n2, n4, n3, code, stream)


def test_tprod_noalloc_nearly_full_scratch(lib):
    """Three FP32 operands of 5 x 360 x 360 complex take 15.55 of the 16 MiB,
    leaving less room for split-K partial sums than one split needs, so the
    products run unsplit; the result still equals tprod's."""
    from paper_2504_04989_gb300 import api
    n1 = n2 = n4 = 360
    n3 = 8
    rng = np.random.default_rng(77)
    A = torch.from_numpy(rng.standard_normal((n3, n1, n2))).to("cuda", torch.float32)
    B = torch.from_numpy(rng.standard_normal((n3, n2, n4))).to("cuda", torch.float32)
    ref = api.tprod(A, B, "fp32")
    for _ in range(2):
        out = torch.full((n3, n1, n4), float("nan"), dtype=torch.float32, device="cuda")
        assert _call(lib, A, B, out, n1, n2, n4, n3, 1) == 0
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=8e-6 * np.sqrt(n2 * n3))


def test_tprod_noalloc_against_oracle(lib, orc):
    """FP64 t-product of a small ragged case against the CPU oracle's t-product
    (itself pinned to the block-circulant definition)."""
    n1, n2, n4, n3 = 13, 17, 6, 9
    rng = np.random.default_rng(78)
    An = rng.standard_normal((n3, n1, n2))
    Bn = rng.standard_normal((n3, n2, n4))
    out = torch.empty((n3, n1, n4), dtype=torch.float64, device="cuda")
    assert _call(lib, torch.from_numpy(An).cuda(), torch.from_numpy(Bn).cuda(), out, n1, n2, n4, n3, 0) == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), orc.tprod(An, Bn), rtol=0, atol=1e-11 * np.sqrt(n2 * n3))


def test_tprod_noalloc_rejects_dimensions_whose_size_wraps(lib):
    """2 slices x 2^30 x 2^30 complex FP32 = 2^64 bytes, which is 0 in 64-bit
    arithmetic: rejected before any launch rather than passing the limit."""
    A = torch.zeros(1, dtype=torch.float32, device="cuda")
    n = 1 << 30
    assert _call(lib, A, A, A, n, n, n, 2, 1) == -4
