"""Torch-facing API of the randomized block Krylov truncated T-SVD
(arXiv 2504.04989) on one GB300.

PyTorch supplies device memory, the current stream and autograd; every step
of the computation runs in libtsvd's CUDA kernels (see include/tsvd.h).  A
real n1 x n2 x n3 tensor is a torch tensor of shape (n3, n1, n2) (frontal
slices contiguous), float64 for precision "fp64" and float32 otherwise.
"""
import ctypes as C

import torch

from . import _lib

_DT = {"fp64": torch.float64, "fp32": torch.float32, "tf32": torch.float32, "bf16": torch.float32,
       "tf32x3": torch.float32}


def _prec(precision):
    if precision not in _lib.PRECISIONS:
        raise ValueError("precision must be one of %s" % sorted(_lib.PRECISIONS))
    return _lib.PRECISIONS[precision]


def _stream(device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need_cuda(*ts, dtype=None):
    for t in ts:
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError("libtsvd operates on CUDA tensors only (got a %s tensor)" % t.device)
        if dtype is not None and t.dtype != dtype:
            raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _flags(fp64_qr, alg1, q_trunc, deflate=False, gram_int=False):
    return ((_lib.TSVD_FLAG_FP64_QR if fp64_qr else 0) | (_lib.TSVD_FLAG_ALG1 if alg1 else 0) |
            (_lib.TSVD_FLAG_QTRUNC if q_trunc else 0) | (_lib.TSVD_FLAG_DEFLATE if deflate else 0) |
            (_lib.TSVD_FLAG_GRAM_INT if gram_int else 0))


def rbk(A, R, P=10, q=2, seed=0, precision="fp32", omega=None, return_info=False, fp64_qr=False, alg1=False,
        q_trunc=False, deflate=False, gram_int=False):
    """Randomized block Krylov truncated T-SVD (Alg. 2): A ~ U * S * V^T.

    A: (n3, n1, n2) CUDA tensor.  Returns U (n3, n1, R), S (n3, R) singular
    tubes, V (n3, n2, R) and sigma_hat (n3 // 2 + 1, R) float64 Fourier-domain
    singular values (descending per slice).  omega (n3, n2, R + P) replaces the
    Philox-drawn test tensor when given.  fp64_qr=True orthonormalises the
    Krylov blocks in FP64 on the FP32 path as well; alg1=True runs Alg. 1
    (power iteration, basis of R+P columns) instead of Alg. 2; q_trunc=True
    projects on the leading R+P basis columns only (Ex. 1's truncated Q);
    deflate=True (FP64 only) resolves singular values below ~1e-8 sigma_1 by
    deflated Rayleigh-Ritz passes in the small SVD.  gram_int=True (FP32 paths)
    takes the exact Gram of the small SVD in integer arithmetic instead of its
    digit form on the tensor cores (the same G to the bit).
    """
    lib = _lib.load()
    pr = _prec(precision)
    dt = _DT[precision]
    A = A.contiguous()
    _need_cuda(A, omega, dtype=dt)
    n3, n1, n2 = A.shape
    flags = _flags(fp64_qr, alg1, q_trunc, deflate, gram_int)
    p = _lib.TsvdParams(R=int(R), P=int(P), q=int(q), precision=pr, seed=int(seed), flags=flags)
    nbytes = C.c_size_t()
    _lib.check(lib.tsvd_rbk_workspace_size(n1, n2, n3, C.byref(p), C.byref(nbytes)), "tsvd_rbk_workspace_size")
    dev = A.device
    ws = _workspace(nbytes.value, dev)
    h = n3 // 2 + 1
    U = torch.empty((n3, n1, R), dtype=dt, device=dev)
    S = torch.empty((n3, R), dtype=dt, device=dev)
    V = torch.empty((n3, n2, R), dtype=dt, device=dev)
    sig = torch.empty((h, R), dtype=torch.float64, device=dev)
    if omega is not None:
        omega = omega.contiguous()
        if tuple(omega.shape) != (n3, n2, R + P):
            raise ValueError("omega must have shape (n3, n2, R+P)")
    info = _lib.TsvdInfo()
    with torch.cuda.device(dev):
        rc = lib.tsvd_rbk(_ptr(A), n1, n2, n3, C.byref(p), _ptr(omega), _ptr(U), _ptr(S), _ptr(V), _ptr(sig),
                          _ptr(ws), nbytes.value, _stream(dev), C.byref(info) if return_info else None)
    _lib.check(rc, "tsvd_rbk")
    if return_info:
        return U, S, V, sig, {"status": info.status, "m_eff": info.m_eff, "dead_columns": info.dead_columns}
    return U, S, V, sig


class RbkPlan:
    """Pre-allocated outputs and workspace for repeated T-SVDs of one shape
    (no allocation per call, so a loop of calls can be captured in a CUDA graph)."""

    def __init__(self, n1, n2, n3, R, P=10, q=2, seed=0, precision="fp32", device="cuda", fp64_qr=False,
                 alg1=False, q_trunc=False, deflate=False, gram_int=False):
        self.lib = _lib.load()
        self.dt = _DT[precision]
        flags = _flags(fp64_qr, alg1, q_trunc, deflate, gram_int)
        self.p = _lib.TsvdParams(R=int(R), P=int(P), q=int(q), precision=_prec(precision), seed=int(seed),
                                 flags=flags)
        self.shape = (n1, n2, n3)
        nbytes = C.c_size_t()
        _lib.check(self.lib.tsvd_rbk_workspace_size(n1, n2, n3, C.byref(self.p), C.byref(nbytes)), "workspace")
        self.nbytes = nbytes.value
        self.device = torch.device(device)
        self.ws = _workspace(self.nbytes, self.device)
        self.U = torch.empty((n3, n1, R), dtype=self.dt, device=self.device)
        self.S = torch.empty((n3, R), dtype=self.dt, device=self.device)
        self.V = torch.empty((n3, n2, R), dtype=self.dt, device=self.device)
        self.sig = torch.empty((n3 // 2 + 1, R), dtype=torch.float64, device=self.device)

    def __call__(self, A, omega=None, stream=None):
        n1, n2, n3 = self.shape
        s = C.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream)
        rc = self.lib.tsvd_rbk(_ptr(A), n1, n2, n3, C.byref(self.p), _ptr(omega), _ptr(self.U), _ptr(self.S),
                               _ptr(self.V), _ptr(self.sig), _ptr(self.ws), self.nbytes, s, None)
        _lib.check(rc, "tsvd_rbk")
        return self.U, self.S, self.V, self.sig


class RbkBatchPlan:
    """Alg. 2 on a fixed batch of independent tensors of different shapes and
    ranks (tsvd_rbk_batched: a native scheduler over `lanes` CUDA streams).
    The plan owns the input buffers, outputs and workspace, so its call can be
    captured once into a CUDA graph (graph=True) and replayed: one launch for
    the whole batch instead of ~130 per tensor.

    shapes: list of (n1, n2, n3); R: rank per tensor (int or list); P, q, seed
    as for rbk (seed + tensor index per tensor)."""

    def __init__(self, shapes, R, P=5, q=2, seed=0, precision="fp32", lanes=8, device="cuda", graph=False):
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.dt = _DT[precision]
        n = len(shapes)
        Rs = [int(R)] * n if isinstance(R, int) else [int(r) for r in R]
        self.lanes = int(lanes)
        self.A, self.U, self.S, self.V, self.sig = [], [], [], [], []
        self.descs = (_lib.TsvdRbkDesc * max(n, 1))()
        for i, ((n1, n2, n3), r) in enumerate(zip(shapes, Rs)):
            self.A.append(torch.empty((n3, n1, n2), dtype=self.dt, device=self.device))
            self.U.append(torch.empty((n3, n1, r), dtype=self.dt, device=self.device))
            self.S.append(torch.empty((n3, r), dtype=self.dt, device=self.device))
            self.V.append(torch.empty((n3, n2, r), dtype=self.dt, device=self.device))
            self.sig.append(torch.empty((n3 // 2 + 1, r), dtype=torch.float64, device=self.device))
            d = self.descs[i]
            d.A, d.n1, d.n2, d.n3 = self.A[-1].data_ptr(), n1, n2, n3
            d.params = _lib.TsvdParams(R=r, P=int(P), q=int(q), precision=_prec(precision), seed=int(seed) + i,
                                       flags=0)
            d.Omega = None
            d.U, d.S, d.V = self.U[-1].data_ptr(), self.S[-1].data_ptr(), self.V[-1].data_ptr()
            d.sigma_hat = self.sig[-1].data_ptr()
        self.count = n
        nbytes = C.c_size_t()
        _lib.check(self.lib.tsvd_rbk_batched_workspace_size(self.descs, n, self.lanes, C.byref(nbytes)),
                   "tsvd_rbk_batched_workspace_size")
        self.nbytes = nbytes.value
        self.ws = _workspace(max(self.nbytes, 256), self.device)
        self.graph = None
        if graph:
            self._launch()                      # first call creates the lane streams outside the capture
            torch.cuda.synchronize(self.device)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._launch()
            self.graph = g

    def _launch(self):
        s = C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.tsvd_rbk_batched(self.descs, self.count, self.lanes, _ptr(self.ws), self.nbytes, s),
                       "tsvd_rbk_batched")

    def __call__(self, tensors=None):
        """Copy `tensors` (if given) into the plan's inputs, run the batch;
        returns lists U, S, V, sigma_hat."""
        if tensors is not None:
            for dst, src in zip(self.A, tensors):
                dst.copy_(src, non_blocking=True)
        if self.graph is not None:
            self.graph.replay()
        else:
            self._launch()
        return self.U, self.S, self.V, self.sig


def rbk_batched(tensors, R, P=5, q=2, seed=0, precision="fp32", lanes=8):
    """Alg. 2 on a list of independent (n3, n1, n2) CUDA tensors (per-tensor
    rank R[i], seed + i); returns lists U, S, V, sigma_hat."""
    plan = RbkBatchPlan([(t.shape[1], t.shape[2], t.shape[0]) for t in tensors], R, P, q, seed, precision, lanes,
                        device=tensors[0].device)
    out = plan(tensors)
    return [list(x) for x in out]


def _tprod_raw(A, B, precision):
    lib = _lib.load()
    pr = _prec(precision)
    A, B = A.contiguous(), B.contiguous()
    _need_cuda(A, B, dtype=_DT[precision])
    n3, n1, n2 = A.shape
    n3b, n2b, n4 = B.shape
    if n3b != n3 or n2b != n2:
        raise ValueError("tprod: shapes (n3,n1,n2) and (n3,n2,n4) required")
    nbytes = C.c_size_t()
    _lib.check(lib.tprod_workspace_size(n1, n2, n4, n3, pr, C.byref(nbytes)), "tprod_workspace_size")
    ws = _workspace(nbytes.value, A.device)
    out = torch.empty((n3, n1, n4), dtype=A.dtype, device=A.device)
    with torch.cuda.device(A.device):
        _lib.check(lib.tprod(_ptr(A), _ptr(B), _ptr(out), n1, n2, n4, n3, pr, _ptr(ws), nbytes.value,
                             _stream(A.device)), "tprod")
    return out


def tprod_backward(A, B, dC, precision="fp32", need_dA=True, need_dB=True):
    """dA = dC * B^T, dB = A^T * dC (adjoint of the t-product)."""
    lib = _lib.load()
    pr = _prec(precision)
    A, B, dC = A.contiguous(), B.contiguous(), dC.contiguous()
    _need_cuda(A, B, dC, dtype=_DT[precision])
    n3, n1, n2 = A.shape
    n4 = B.shape[2]
    nbytes = C.c_size_t()
    _lib.check(lib.tprod_backward_workspace_size(n1, n2, n4, n3, pr, C.byref(nbytes)), "workspace")
    ws = _workspace(nbytes.value, A.device)
    dA = torch.empty_like(A) if need_dA else None
    dB = torch.empty_like(B) if need_dB else None
    with torch.cuda.device(A.device):
        _lib.check(lib.tprod_backward(_ptr(A), _ptr(B), _ptr(dC), _ptr(dA), _ptr(dB), n1, n2, n4, n3, pr, _ptr(ws),
                                      nbytes.value, _stream(A.device)), "tprod_backward")
    return dA, dB


def _tproj_raw(Q, A, precision):
    lib = _lib.load()
    pr = _prec(precision)
    Q, A = Q.contiguous(), A.contiguous()
    _need_cuda(Q, A, dtype=_DT[precision])
    n3, n1, m = Q.shape
    n2 = A.shape[2]
    nbytes = C.c_size_t()
    _lib.check(lib.tproj_workspace_size(n1, m, n2, n3, pr, C.byref(nbytes)), "workspace")
    ws = _workspace(nbytes.value, Q.device)
    Y = torch.empty_like(A)
    with torch.cuda.device(Q.device):
        _lib.check(lib.tproj(_ptr(Q), _ptr(A), _ptr(Y), n1, m, n2, n3, pr, _ptr(ws), nbytes.value,
                             _stream(Q.device)), "tproj")
    return Y


def tproj_backward(Q, A, dY, precision="fp32", need_dQ=True, need_dA=True):
    """dA = Q * (Q^T * dY), dQ = dY * (A^T * Q) + A * (dY^T * Q) for Y = Q * Q^T * A."""
    lib = _lib.load()
    pr = _prec(precision)
    Q, A, dY = Q.contiguous(), A.contiguous(), dY.contiguous()
    _need_cuda(Q, A, dY, dtype=_DT[precision])
    n3, n1, m = Q.shape
    n2 = A.shape[2]
    nbytes = C.c_size_t()
    _lib.check(lib.tproj_backward_workspace_size(n1, m, n2, n3, pr, C.byref(nbytes)), "workspace")
    ws = _workspace(nbytes.value, Q.device)
    dQ = torch.empty_like(Q) if need_dQ else None
    dA = torch.empty_like(A) if need_dA else None
    with torch.cuda.device(Q.device):
        _lib.check(lib.tproj_backward(_ptr(Q), _ptr(A), _ptr(dY), _ptr(dQ), _ptr(dA), n1, m, n2, n3, pr, _ptr(ws),
                                      nbytes.value, _stream(Q.device)), "tproj_backward")
    return dQ, dA


def _precision_of(t, precision):
    if precision is not None:
        return precision
    return "fp64" if t.dtype == torch.float64 else "fp32"


class TProd(torch.autograd.Function):
    """C = A * B with the hand-written adjoint as backward."""

    @staticmethod
    def forward(ctx, A, B, precision):
        ctx.save_for_backward(A, B)
        ctx.precision = precision
        return _tprod_raw(A, B, precision)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dA, dB = tprod_backward(A, B, dC, ctx.precision, ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return dA, dB, None


class TProj(torch.autograd.Function):
    """Y = Q * Q^T * A with the hand-written adjoint as backward."""

    @staticmethod
    def forward(ctx, Q, A, precision):
        ctx.save_for_backward(Q, A)
        ctx.precision = precision
        return _tproj_raw(Q, A, precision)

    @staticmethod
    def backward(ctx, dY):
        Q, A = ctx.saved_tensors
        dQ, dA = tproj_backward(Q, A, dY, ctx.precision, ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return dQ, dA, None


def tprod(A, B, precision=None):
    """t-product C = A * B (Alg. TP); differentiable."""
    return TProd.apply(A, B, _precision_of(A, precision))


def tproj(Q, A, precision=None):
    """Projection Y = Q * Q^T * A (Sec. 4: the Alg. 2 output lies in the projection Q*Q^T*A); differentiable."""
    return TProj.apply(Q, A, _precision_of(Q, precision))


def gaussian(seed, n, stream_id=0, tensor_id=0, device="cuda"):
    """Device draw of the Philox4x32-10 / Box-Muller Gaussian stream (float64)."""
    lib = _lib.load()
    out = torch.empty(int(n), dtype=torch.float64, device=device)
    _lib.check(lib.tsvd_gaussian(int(seed), stream_id, tensor_id, int(n), _ptr(out), _stream(out.device)), "gaussian")
    return out


def philox_words(key, ctr1, ctr2, ctr3, n, device="cuda"):
    """Raw Philox4x32-10 words for counters (i, ctr1, ctr2, ctr3), i < n: int64 (n, 4)."""
    lib = _lib.load()
    out = torch.empty((int(n), 4), dtype=torch.int32, device=device)
    k = (C.c_uint32 * 2)(int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF)
    _lib.check(lib.tsvd_philox_words(k, ctr1, ctr2, ctr3, int(n), _ptr(out), _stream(out.device)), "philox_words")
    return out.to(torch.int64) & 0xFFFFFFFF


class profile:
    """Context manager collecting per-stage GPU times (CUDA events recorded by
    the library around each pipeline stage).  After exit, `.stages` maps a
    stage name to (total milliseconds, executions)."""

    def __enter__(self):
        self.lib = _lib.load()
        _lib.check(self.lib.tsvd_profile_begin(), "tsvd_profile_begin")
        self.stages = {}
        return self

    def __exit__(self, *exc):
        buf = (_lib.TsvdStageTime * 64)()
        n = C.c_int()
        _lib.check(self.lib.tsvd_profile_end(buf, 64, C.byref(n)), "tsvd_profile_end")
        self.stages = {buf[i].name.decode(): (buf[i].ms, buf[i].count) for i in range(n.value)}
        return False


def launch_count():
    """Kernels launched by libtsvd so far in this process."""
    return int(_lib.load().tsvd_launch_count())


def ttranspose(A, precision=None):
    """Tensor transpose (Sec. 2): (n3, n1, n2) -> (n3, n2, n1)."""
    lib = _lib.load()
    precision = _precision_of(A, precision)
    A = A.contiguous()
    _need_cuda(A, dtype=_DT[precision])
    n3, n1, n2 = A.shape
    out = torch.empty((n3, n2, n1), dtype=A.dtype, device=A.device)
    with torch.cuda.device(A.device):
        _lib.check(lib.ttranspose(_ptr(A), _ptr(out), n1, n2, n3, _prec(precision), _stream(A.device)), "ttranspose")
    return out


def tsvd_error(X, U, S, V, precision=None):
    """||X - U * S * V^T||_F^2 (device FP64 scalar) for the layouts of rbk:
    X (n3, n1, n2), U (n3, n1, R), S (n3, R) diagonal tubes, V (n3, n2, R).
    Fused Fourier-domain evaluation (Parseval over the half spectrum)."""
    lib = _lib.load()
    precision = _precision_of(X, precision)
    pr = _prec(precision)
    X, U, S, V = (t.contiguous() for t in (X, U, S, V))
    _need_cuda(X, U, S, V, dtype=_DT[precision])
    n3, n1, n2 = X.shape
    R = U.shape[2]
    if U.shape != (n3, n1, R) or S.shape != (n3, R) or V.shape != (n3, n2, R):
        raise ValueError("tsvd_error: U (n3,n1,R), S (n3,R), V (n3,n2,R) required")
    nbytes = C.c_size_t()
    _lib.check(lib.tsvd_error_workspace_size(n1, n2, n3, R, pr, C.byref(nbytes)), "tsvd_error_workspace_size")
    ws = _workspace(nbytes.value, X.device)
    out = torch.empty((), dtype=torch.float64, device=X.device)
    with torch.cuda.device(X.device):
        _lib.check(lib.tsvd_error(_ptr(X), _ptr(U), _ptr(S), _ptr(V), n1, n2, n3, R, pr, _ptr(out), _ptr(ws),
                                  nbytes.value, _stream(X.device)), "tsvd_error")
    return out


def masked_residual(C, X, mask, out=None, loss=None, partial=None):
    """R = mask .* (C - X) and the FP64 sum of R^2 (device scalar)."""
    lib = _lib.load()
    precision = _precision_of(C, None)
    C, X = C.contiguous(), X.contiguous()
    _need_cuda(C, X, dtype=C.dtype)
    if mask.dtype != torch.uint8 or not mask.is_cuda or mask.numel() != C.numel():
        raise ValueError("mask must be a CUDA uint8 tensor with C's number of elements")
    R = torch.empty_like(C) if out is None else out
    loss = torch.empty((), dtype=torch.float64, device=C.device) if loss is None else loss
    partial = torch.empty(1024, dtype=torch.float64, device=C.device) if partial is None else partial
    with torch.cuda.device(C.device):
        _lib.check(lib.tsvd_masked_residual(_ptr(C), _ptr(X), _ptr(mask), _ptr(R), _ptr(loss), _ptr(partial),
                                            C.numel(), _prec(precision), _stream(C.device)), "masked_residual")
    return R, loss


def tqr(A, precision=None, return_info=False):
    """T-QR decomposition A = Q * R (Alg. TQR): A (n3, n1, n2) CUDA tensor;
    returns Q (n3, n1, p) and R (n3, p, n2), p = min(n1, n2), whose Fourier
    slices have diag(R_k) real and >= 0."""
    lib = _lib.load()
    precision = _precision_of(A, precision)
    pr = _prec(precision)
    A = A.contiguous()
    _need_cuda(A, dtype=_DT[precision])
    n3, n1, n2 = A.shape
    p = min(n1, n2)
    nbytes = C.c_size_t()
    _lib.check(lib.tqr_workspace_size(n1, n2, n3, pr, C.byref(nbytes)), "tqr_workspace_size")
    ws = _workspace(nbytes.value, A.device)
    Q = torch.empty((n3, n1, p), dtype=A.dtype, device=A.device)
    R = torch.empty((n3, p, n2), dtype=A.dtype, device=A.device)
    info = _lib.TsvdInfo()
    with torch.cuda.device(A.device):
        _lib.check(lib.tqr(_ptr(A), n1, n2, n3, pr, _ptr(Q), _ptr(R), _ptr(ws), nbytes.value, _stream(A.device),
                           C.byref(info) if return_info else None), "tqr")
    if return_info:
        return Q, R, {"status": info.status, "dead_columns": info.dead_columns}
    return Q, R


def tpinv(A, precision=None, return_info=False):
    """Moore-Penrose pseudoinverse (Alg. mp): A (n3, n1, n2) -> (n3, n2, n1).
    Every Fourier slice must have full rank min(n1, n2) (status
    TSVD_ERR_RANK_DEFICIENT in the info otherwise)."""
    lib = _lib.load()
    precision = _precision_of(A, precision)
    pr = _prec(precision)
    A = A.contiguous()
    _need_cuda(A, dtype=_DT[precision])
    n3, n1, n2 = A.shape
    nbytes = C.c_size_t()
    _lib.check(lib.tpinv_workspace_size(n1, n2, n3, pr, C.byref(nbytes)), "tpinv_workspace_size")
    ws = _workspace(nbytes.value, A.device)
    X = torch.empty((n3, n2, n1), dtype=A.dtype, device=A.device)
    info = _lib.TsvdInfo()
    with torch.cuda.device(A.device):
        _lib.check(lib.tpinv(_ptr(A), n1, n2, n3, pr, _ptr(X), _ptr(ws), nbytes.value, _stream(A.device),
                             C.byref(info) if return_info else None), "tpinv")
    if return_info:
        return X, {"status": info.status, "dead_columns": info.dead_columns}
    return X


_CDT = {torch.float64: torch.complex128, torch.float32: torch.complex64}


def rfft3(X, precision=None):
    """Mode-3 transform of a real (n3, rows, cols) CUDA tensor: its
    floor(n3/2)+1 non-redundant Fourier slices (h, rows, cols), complex."""
    lib = _lib.load()
    precision = _precision_of(X, precision)
    X = X.contiguous()
    _need_cuda(X, dtype=_DT[precision])
    n3 = X.shape[0]
    out = torch.empty((n3 // 2 + 1,) + tuple(X.shape[1:]), dtype=_CDT[X.dtype], device=X.device)
    plane = X[0].numel()
    with torch.cuda.device(X.device):
        _lib.check(lib.tsvd_rfft3(_ptr(X), plane, n3, _prec(precision), _ptr(out), _stream(X.device)), "tsvd_rfft3")
    return out


def irfft3(Xh, n3):
    """Inverse of rfft3: (h, rows, cols) complex -> real (n3, rows, cols)."""
    lib = _lib.load()
    Xh = Xh.contiguous()
    _need_cuda(Xh)
    rdt = torch.float64 if Xh.dtype == torch.complex128 else torch.float32
    if Xh.shape[0] != n3 // 2 + 1:
        raise ValueError("irfft3: %d slices given, n3 = %d needs %d" % (Xh.shape[0], n3, n3 // 2 + 1))
    out = torch.empty((n3,) + tuple(Xh.shape[1:]), dtype=rdt, device=Xh.device)
    plane = Xh[0].numel()
    pr = _lib.TSVD_FP64 if rdt == torch.float64 else _lib.TSVD_FP32
    with torch.cuda.device(Xh.device):
        _lib.check(lib.tsvd_irfft3(_ptr(Xh), plane, n3, pr, _ptr(out), _stream(Xh.device)), "tsvd_irfft3")
    return out


def rbk_fourier(Ahat, n3, k0, R, P=10, q=2, seed=0, precision="fp32", omega=None, return_info=False, **flags):
    """Alg. 2 on the Fourier slices k0 .. k0 + ns - 1 of an n1 x n2 x n3 tensor
    given as Ahat (ns, n1, n2) complex CUDA tensor (complex128 for "fp64",
    complex64 otherwise).  Returns Uhat (ns, n1, R), Vhat (ns, n2, R) complex
    and sigma_hat (ns, R) float64, as the slices k0.. of tsvd_rbk's factors."""
    lib = _lib.load()
    pr = _prec(precision)
    cdt = torch.complex128 if precision == "fp64" else torch.complex64
    Ahat = Ahat.contiguous()
    _need_cuda(Ahat, dtype=cdt)
    ns, n1, n2 = Ahat.shape
    p = _lib.TsvdParams(R=int(R), P=int(P), q=int(q), precision=pr, seed=int(seed), flags=_flags(**{
        "fp64_qr": flags.get("fp64_qr", False), "alg1": flags.get("alg1", False),
        "q_trunc": flags.get("q_trunc", False), "deflate": flags.get("deflate", False)}))
    nbytes = C.c_size_t()
    _lib.check(lib.tsvd_rbk_fourier_workspace_size(n1, n2, n3, k0, ns, C.byref(p), C.byref(nbytes)),
               "tsvd_rbk_fourier_workspace_size")
    dev = Ahat.device
    ws = _workspace(nbytes.value, dev)
    Uh = torch.empty((ns, n1, R), dtype=cdt, device=dev)
    Vh = torch.empty((ns, n2, R), dtype=cdt, device=dev)
    sig = torch.empty((ns, R), dtype=torch.float64, device=dev)
    if omega is not None:
        omega = omega.contiguous()
        _need_cuda(omega, dtype=_DT[precision])
    info = _lib.TsvdInfo()
    with torch.cuda.device(dev):
        _lib.check(lib.tsvd_rbk_fourier(_ptr(Ahat), n1, n2, n3, k0, ns, C.byref(p), _ptr(omega), _ptr(Uh), _ptr(Vh),
                                        _ptr(sig), _ptr(ws), nbytes.value, _stream(dev),
                                        C.byref(info) if return_info else None), "tsvd_rbk_fourier")
    if return_info:
        return Uh, Vh, sig, {"status": info.status, "m_eff": info.m_eff, "dead_columns": info.dead_columns}
    return Uh, Vh, sig


def lowrank(U, S, V, out=None, ws=None):
    """X = U * S * V^T (n3, n1, n2) from tsvd_rbk's spatial factors U (n3, n1, R),
    S (n3, R), V (n3, n2, R), fused in the Fourier domain."""
    lib = _lib.load()
    precision = _precision_of(U, None)
    U, S, V = U.contiguous(), S.contiguous(), V.contiguous()
    _need_cuda(U, S, V, dtype=U.dtype)
    n3, n1, R = U.shape
    n2 = V.shape[1]
    nbytes = C.c_size_t()
    _lib.check(lib.tsvd_lowrank_workspace_size(n1, n2, n3, R, _prec(precision), C.byref(nbytes)), "lowrank ws")
    ws = _workspace(nbytes.value, U.device) if ws is None else ws
    X = torch.empty((n3, n1, n2), dtype=U.dtype, device=U.device) if out is None else out
    with torch.cuda.device(U.device):
        _lib.check(lib.tsvd_lowrank(_ptr(U), _ptr(S), _ptr(V), n1, n2, n3, R, _prec(precision), _ptr(X), _ptr(ws),
                                    nbytes.value, _stream(U.device)), "tsvd_lowrank")
    return X


def sigma_tubes(sig_hat, n3, power=1.0, dtype=torch.float32):
    """Tubes (n3, R) of S^power from the Fourier singular values (h, R)."""
    lib = _lib.load()
    sig_hat = sig_hat.contiguous()
    _need_cuda(sig_hat, dtype=torch.float64)
    h, R = sig_hat.shape
    if h != n3 // 2 + 1:
        raise ValueError("sigma_tubes: %d slices for n3 = %d" % (h, n3))
    pr = _lib.TSVD_FP64 if dtype == torch.float64 else _lib.TSVD_FP32
    ws = _workspace(16 * h * R, sig_hat.device)
    out = torch.empty((n3, R), dtype=dtype, device=sig_hat.device)
    with torch.cuda.device(sig_hat.device):
        _lib.check(lib.tsvd_sigma_tubes(_ptr(sig_hat), R, n3, float(power), pr, _ptr(out), _ptr(ws), ws.numel(),
                                        _stream(sig_hat.device)), "tsvd_sigma_tubes")
    return out


def fill_in(Cm, M, mask, X, change2=None, partial=None):
    """In place C <- mask ? M : X; returns the device FP64 scalar sum (dC)^2."""
    lib = _lib.load()
    _need_cuda(Cm, M, X, dtype=Cm.dtype)
    if mask.dtype != torch.uint8 or not mask.is_cuda or mask.numel() != Cm.numel():
        raise ValueError("mask must be a CUDA uint8 tensor with C's number of elements")
    change2 = torch.empty((), dtype=torch.float64, device=Cm.device) if change2 is None else change2
    partial = torch.empty(1024, dtype=torch.float64, device=Cm.device) if partial is None else partial
    with torch.cuda.device(Cm.device):
        _lib.check(lib.tsvd_fill_in(_ptr(Cm), _ptr(M), _ptr(mask), _ptr(X), Cm.numel(), _prec(_precision_of(Cm, None)),
                                    _ptr(partial), _ptr(change2), _stream(Cm.device)), "tsvd_fill_in")
    return change2


def sqdiff(A, B, out=None, partial=None):
    """Device FP64 scalar sum (A - B)^2."""
    lib = _lib.load()
    _need_cuda(A, B, dtype=A.dtype)
    A, B = A.contiguous(), B.contiguous()
    out = torch.empty((), dtype=torch.float64, device=A.device) if out is None else out
    partial = torch.empty(1024, dtype=torch.float64, device=A.device) if partial is None else partial
    with torch.cuda.device(A.device):
        _lib.check(lib.tsvd_sqdiff(_ptr(A), _ptr(B), A.numel(), _prec(_precision_of(A, None)), _ptr(partial),
                                   _ptr(out), _stream(A.device)), "tsvd_sqdiff")
    return out


def psnr(X, Y, peak=255.0):
    """PSNR = 10 log10(peak^2 / MSE) dB (Sec. 5), MSE = ||X - Y||_F^2 / num(X)."""
    import math
    mse = sqdiff(X, Y).item() / X.numel()
    return float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse)
