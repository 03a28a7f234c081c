"""Low-tubal-rank tensor completion by gradient steps on the t-factors.

min_{U, W} ||P_Omega(U * W - X)||_F^2 with U (n1 x R x n3) and W = V^T
(R x n2 x n3): the t-product (Alg. TP) in the forward pass, the hand-written
adjoint (dU = dC * W^T, dW = U^T * dC) in the backward pass, the masked
residual in a fused kernel.  The factors start from the randomized block
Krylov truncated T-SVD (Alg. 2) of the zero-filled, rescaled observations
P_Omega(X) / p, split evenly as U_0 = U_R * S_R^{1/2}, W_0 = S_R^{1/2} * V_R^T
(the square roots act per Fourier slice on the singular values).  This is the
data-completion application of Ex. 3 in its gradient form.  The paper's own
fill-in iteration (Ex. 3, Ex. 4) is `FillInPlan`: every step on the GPU in
library kernels, one iteration captured in a CUDA graph and replayed.
"""
import torch

from . import api


def _sqrt_tubes(sig_hat, n3, dtype, device):
    """Spatial tubes of the f-diagonal S^{1/2}: the inverse transform of
    sqrt(sigma_hat) per Fourier slice (library kernel)."""
    return api.sigma_tubes(sig_hat.to(device), n3, 0.5, dtype)


def f_diagonal(tubes):
    n3, R = tubes.shape
    D = torch.zeros((n3, R, R), dtype=tubes.dtype, device=tubes.device)
    D.diagonal(dim1=1, dim2=2).copy_(tubes)
    return D


def spectral_init(Xobs, mask, R, P=10, q=2, seed=0, precision="fp32"):
    """U_0, W_0 from the block Krylov T-SVD of P_Omega(X) / p."""
    p = float(mask.float().mean().item())
    U, S, V, sig = api.rbk(Xobs / p, R, P, q, seed=seed, precision=precision)
    D = f_diagonal(_sqrt_tubes(sig, Xobs.shape[0], Xobs.dtype, Xobs.device))
    U0 = api.tprod(U, D, precision)
    W0 = api.tprod(D, api.ttranspose(V, precision), precision)
    return U0.contiguous(), W0.contiguous()


def masked_loss_grad(U, W, X, mask, precision="fp32"):
    """loss = ||P_Omega(U * W - X)||^2 and its gradients (dU, dW)."""
    C = api.tprod(U, W, precision)
    Rm, loss = api.masked_residual(C, X, mask)
    dU, dW = api.tprod_backward(U, W, 2.0 * Rm, precision)
    return loss, dU, dW


def complete(Xobs, mask, R, steps=100, lr=None, P=10, q=2, seed=0, precision="fp32", callback=None, c=0.3):
    """Gradient descent from the spectral initialisation; returns (U, W, losses).
    The default step size is c / (p sigma_max), sigma_max the largest
    Fourier-domain singular value of the initial factorisation."""
    U, W = spectral_init(Xobs, mask, R, P, q, seed, precision)
    p = float(mask.float().mean().item())
    if lr is None:
        _, _, _, sig = api.rbk(Xobs / p, R, P, q, seed=seed, precision=precision)
        lr = c / (p * float(sig.max().item()))
    losses = []
    for it in range(steps):
        loss, dU, dW = masked_loss_grad(U, W, Xobs, mask, precision)
        losses.append(loss)
        U = U - lr * dU
        W = W - lr * dW
        if callback is not None:
            callback(it, U, W)
    return U, W, [float(l.item()) for l in losses]


def reconstruct(U, S, V, precision="fp32"):
    """U * S * V^T from the spatial factors of api.rbk (S as singular tubes)."""
    return api.tprod(api.tprod(U, f_diagonal(S), precision), api.ttranspose(V, precision), precision)


class FillInPlan:
    """The completion iteration of Ex. 3 with every buffer allocated once:

        X^(n)   = L(C^(n))                        (Alg. 2 + U * S * V^T)
        C^(n+1) = T .* M + (1 - T) .* X^(n)       (T the mask, M the data)

    from C^(0) = T .* M (the zero-filled observations).  One iteration is the
    library's T-SVD (RbkPlan), its low-rank product (tsvd_lowrank) and the
    fill-in (tsvd_fill_in); with graph=True it is captured once in a CUDA
    graph and replayed.  `change2` holds ||C^(n+1) - C^(n)||_F^2 of the last
    iteration (a device scalar).  Alg. 1 replaces Alg. 2 with alg1=True."""

    def __init__(self, M, mask, R, P=10, q=2, seed=0, precision="fp32", graph=True, alg1=False):
        self.M = M.contiguous()
        self.mask = mask.to(torch.uint8).contiguous()
        n3, n1, n2 = self.M.shape
        dev = self.M.device
        self.plan = api.RbkPlan(n1, n2, n3, R, P, q, seed=seed, precision=precision, device=dev, alg1=alg1)
        self.X = torch.zeros_like(self.M)
        self.C = torch.zeros_like(self.M)
        self.change2 = torch.zeros((), dtype=torch.float64, device=dev)
        self.partial = torch.empty(1024, dtype=torch.float64, device=dev)
        self.lr_ws = None
        self.reset()
        self.graph = None
        if graph:
            self._iterate()                 # first run outside the capture (lazy loading, workspaces)
            torch.cuda.synchronize(dev)
            self.reset()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._iterate()
            self.graph = g
            self.reset()

    def reset(self):
        """C <- T .* M + (1 - T) .* 0."""
        self.X.zero_()
        api.fill_in(self.C, self.M, self.mask, self.X, self.change2, self.partial)

    def _iterate(self):
        U, S, V, _ = self.plan(self.C)
        if self.lr_ws is None:
            import ctypes as C
            from . import _lib
            nbytes = C.c_size_t()
            n3, n1, R = U.shape
            _lib.check(_lib.load().tsvd_lowrank_workspace_size(n1, V.shape[1], n3, R, _lib.PRECISIONS[
                "fp64" if U.dtype == torch.float64 else "fp32"], C.byref(nbytes)), "lowrank ws")
            self.lr_ws = torch.empty(nbytes.value, dtype=torch.uint8, device=U.device)
        api.lowrank(U, S, V, out=self.X, ws=self.lr_ws)
        api.fill_in(self.C, self.M, self.mask, self.X, self.change2, self.partial)

    def step(self, iters=1):
        for _ in range(iters):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._iterate()
        return self.X


def complete_fill_in(Xobs, mask, R, iters=50, P=10, q=2, seed=0, precision="fp32", callback=None, graph=True):
    """The completion iteration of Ex. 3 (FillInPlan) for `iters` iterations;
    returns the last low-rank approximation X^(n).  `callback(it, X)` sees
    every iterate (it then runs one replay at a time)."""
    plan = FillInPlan(Xobs, mask if mask.dtype == torch.uint8 else mask.to(torch.uint8), R, P, q, seed, precision,
                      graph=graph)
    if callback is None:
        return plan.step(iters)
    for it in range(iters):
        callback(it, plan.step(1))
    return plan.X
