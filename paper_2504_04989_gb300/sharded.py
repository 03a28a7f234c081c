"""Slice-sharded randomized block Krylov T-SVD of one tensor over several GPUs.

After the mode-3 transform every Fourier slice is an independent problem (the
remark opening Sec. 4), so one large tensor splits across ranks by slices:

  1. rank r holds the rows [r0, r1) of the real tensor (n3, n1, n2) and
     transforms them locally (tubes are complete in every row block);
  2. one all-to-all regroups row blocks into slice blocks: rank r receives
     all rows of its Fourier slices [k0, k1);
  3. every rank runs Alg. 2 on its slices (tsvd_rbk_fourier), no exchange;
  4. a second all-to-all returns U-hat to row blocks of n1 and V-hat to row
     blocks of n2, and the singular values are all-gathered;
  5. every rank inverts the transform of its rows of U and V and of the
     singular tubes.

Partitions are contiguous and balanced (sizes differ by at most one).  The
exchanges move complex data as real pairs through torch.distributed
(all_to_all_single with uneven split sizes), so NCCL carries them on GPUs and
gloo on CPU ranks; every exchanged block lands in local memory before a kernel
reads it.  The three local steps (transform, per-slice T-SVD, inverse
transform) come from a `steps` object: `CudaSteps` calls libtsvd's kernels;
tests may pass other implementations to check the partition and exchange
logic on CPU ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def partition(n: int, parts: int):
    """Contiguous balanced split of range(n) into `parts` (lo, hi) pieces."""
    base, extra = divmod(n, parts)
    out, lo = [], 0
    for p in range(parts):
        hi = lo + base + (1 if p < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def _world(group):
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def _exchange(blocks_out, recv_shapes, dtype, device, group):
    """all-to-all of complex blocks: blocks_out[s] goes to rank s; returns the
    blocks received from every rank, with the given shapes."""
    world, _ = _world(group)
    if world == 1:
        return [blocks_out[0].reshape(recv_shapes[0])]
    send = torch.cat([torch.view_as_real(b.contiguous()).reshape(-1) for b in blocks_out])
    in_sizes = [2 * b.numel() for b in blocks_out]
    out_sizes = [2 * int(torch.Size(sh).numel()) for sh in recv_shapes]
    recv = torch.empty(sum(out_sizes), dtype=send.dtype, device=device)
    dist.all_to_all_single(recv, send, output_split_sizes=out_sizes, input_split_sizes=in_sizes, group=group)
    out, off = [], 0
    for sh, n in zip(recv_shapes, out_sizes):
        out.append(torch.view_as_complex(recv[off:off + n].view(*sh, 2)))
        off += n
    return out


class CudaSteps:
    """The local steps on this rank's GPU (libtsvd kernels)."""

    def __init__(self, precision="fp32", **flags):
        from . import api
        self.api = api
        self.precision = precision
        self.flags = flags

    def rfft3(self, X):
        return self.api.rfft3(X)

    def irfft3(self, Xh, n3):
        return self.api.irfft3(Xh, n3)

    def local(self, Ahat, n3, k0, R, P, q, seed):
        return self.api.rbk_fourier(Ahat, n3, k0, R, P, q, seed=seed, precision=self.precision, **self.flags)


def rbk_sharded(A_rows, n1, n2, n3, R, P=10, q=2, seed=0, steps=None, group=None):
    """Alg. 2 on one n1 x n2 x n3 tensor spread over the ranks of `group`.

    A_rows: this rank's rows [r0, r1) of the tensor, shape (n3, r1 - r0, n2),
    with the row partition `partition(n1, world)`.  Returns this rank's rows of
    U (n3, r1 - r0, R), the singular tubes S (n3, R), this rank's rows of V
    (n3, c1 - c0, R) for the column partition `partition(n2, world)`, and the
    Fourier-domain singular values (h, R), h = n3 // 2 + 1."""
    steps = steps or CudaSteps()
    world, rank = _world(group)
    h = n3 // 2 + 1
    rows, cols, slices = partition(n1, world), partition(n2, world), partition(h, world)
    r0, r1 = rows[rank]
    c0, c1 = cols[rank]
    k0, k1 = slices[rank]
    if tuple(A_rows.shape) != (n3, r1 - r0, n2):
        raise ValueError("rank %d holds rows %d..%d: expected shape %s, got %s"
                         % (rank, r0, r1, (n3, r1 - r0, n2), tuple(A_rows.shape)))
    if k1 <= k0:
        raise ValueError("more ranks (%d) than Fourier slices (%d)" % (world, h))
    dev = A_rows.device

    # 1-2: local transform of the row block, then rows -> slices
    Ah_rows = steps.rfft3(A_rows)                                   # (h, r1 - r0, n2)
    cdt = Ah_rows.dtype
    recv = _exchange([Ah_rows[a:b] for a, b in slices],
                     [(k1 - k0, b - a, n2) for a, b in rows], cdt, dev, group)
    Ah = torch.cat(recv, dim=1) if world > 1 else recv[0]             # (k1 - k0, n1, n2)

    # 3: the per-slice method on this rank's slices
    Uh, Vh, sig = steps.local(Ah.contiguous(), n3, k0, R, P, q, seed)

    # 4: slices -> row blocks of U and V; all singular values everywhere
    Uh_rows = torch.cat(_exchange([Uh[:, a:b] for a, b in rows],
                                  [(b - a, r1 - r0, R) for a, b in slices], cdt, dev, group), dim=0)
    Vh_rows = torch.cat(_exchange([Vh[:, a:b] for a, b in cols],
                                  [(b - a, c1 - c0, R) for a, b in slices], cdt, dev, group), dim=0)
    if world > 1:
        kmax = max(b - a for a, b in slices)
        pad = torch.zeros((kmax, R), dtype=sig.dtype, device=dev)
        pad[:k1 - k0] = sig
        allsig = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(allsig, pad, group=group)
        sig_all = torch.cat([s[:b - a] for s, (a, b) in zip(allsig, slices)])
    else:
        sig_all = sig

    # 5: back to the spatial domain
    U_rows = steps.irfft3(Uh_rows, n3)
    V_rows = steps.irfft3(Vh_rows, n3)
    S = steps.irfft3(sig_all.to(cdt).reshape(h, 1, R), n3).reshape(n3, R)
    return U_rows, S, V_rows, sig_all
