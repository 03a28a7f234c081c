"""Low-tubal-rank tensor completion by gradient steps on the t-factors.

min_{U, W} ||P_Omega(U * W - X)||_F^2 with U (n1 x R x n3) and W = V^T
(R x n2 x n3): the t-product (Alg. TP) in the forward pass, the hand-written
adjoint (dU = dC * W^T, dW = U^T * dC) in the backward pass, the masked
residual in a fused kernel.  The factors start from the randomized block
Krylov truncated T-SVD (Alg. 2) of the zero-filled, rescaled observations
P_Omega(X) / p, split evenly as U_0 = U_R * S_R^{1/2}, W_0 = S_R^{1/2} * V_R^T
(the square roots act per Fourier slice on the singular values).  This is the
data-completion application of Ex. 3 in its gradient form; the ALS fill-in
loop of the paper is not used.
"""
import numpy as np
import torch

from . import api


def _sqrt_tubes(sig_hat, n3, dtype, device):
    """Spatial tubes of the f-diagonal S^{1/2}: inverse DFT of sqrt(sigma_hat)
    per Fourier slice (R x n3 values, assembled on the host)."""
    s = np.sqrt(np.maximum(sig_hat.detach().cpu().numpy(), 0.0))  # (h, R), real per Fourier slice
    tubes = np.fft.irfft(s.astype(np.complex128), n=n3, axis=0)    # (n3, R)
    return torch.from_numpy(tubes).to(device=device, dtype=dtype)


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


def complete_fill_in(Xobs, mask, R, iters=50, P=10, q=2, seed=0, precision="fp32", callback=None):
    """The completion iteration of Ex. 3: X^(n) = L(C^(n)) with L the
    randomized block Krylov truncated T-SVD (Alg. 2), then the fill-in
    C^(n+1) = T .* M + (1 - T) .* X^(n) (T the observation mask, M the data).
    Starts from C^(0) = the zero-filled observations."""
    Mf = mask.to(Xobs.dtype)
    C = Xobs.clone()
    X = None
    for it in range(iters):
        U, S, V, _ = api.rbk(C, R, P, q, seed=seed, precision=precision)
        X = reconstruct(U, S, V, precision)
        C = Xobs + (1 - Mf) * X
        if callback is not None:
            callback(it, X)
    return X
