"""tprod_noalloc: the t-product for callers that cannot allocate device memory
(a pool that must not grow, a plug-in whose host owns all device allocations, a
real-time loop), with its scratch in a fixed array inside the library.

Called through the C ABI and checked against the workspace-based tprod entry
point on two calls in a row, then for the size limit.  This file is collected
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
