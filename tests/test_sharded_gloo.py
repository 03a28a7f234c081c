"""The slice-sharded multi-rank T-SVD (paper_2504_04989_gb300/sharded.py) on
CPU ranks over gloo: the row/slice/column partitions and both all-to-all
exchanges, with the local steps done on the CPU (library FFTs of torch and the
FP64 oracle's Alg. 2 on the received Fourier slices).  The gathered result
must equal the oracle's single-process T-SVD of the whole tensor: the Fourier
singular values to 1e-12 and the reconstruction U * S * V^T to 1e-10."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

N1, N2, N3, R, P, Q, SEED = 13, 11, 8, 3, 2, 1, 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _tensor():
    from paper_2504_04989_gb300 import workloads as wl
    return wl.low_tubal_rank(N1, N2, N3, np.linspace(4.0, 0.5, 6), noise_std=1e-2, seed=SEED)


class OracleSteps:
    """CPU stand-ins for the three local steps: library FFTs along mode 3 and
    the oracle's per-slice Alg. 2 on the Fourier slices this rank received."""

    def rfft3(self, X):
        return torch.fft.rfft(X, dim=0)

    def irfft3(self, Xh, n3):
        return torch.fft.irfft(Xh, n=n3, dim=0)

    def local(self, Ahat, n3, k0, R_, P_, q_, seed):
        import oracle
        n2, b = Ahat.shape[2], R_ + P_
        om = oracle.gaussian(seed, n3 * n2 * b).reshape(n3, n2, b)
        omh = np.fft.rfft(om, axis=0)[k0:k0 + Ahat.shape[0]]
        r = oracle.rtsvd_hat(Ahat.numpy(), omh, R_, P_, q_)
        return torch.from_numpy(r["Uhat"]), torch.from_numpy(r["Vhat"]), torch.from_numpy(r["sig"])


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2504_04989_gb300 import sharded
    X = _tensor()
    r0, r1 = sharded.partition(N1, world)[rank]
    U, S, V, sig = sharded.rbk_sharded(torch.from_numpy(np.ascontiguousarray(X[:, r0:r1])), N1, N2, N3, R, P, Q,
                                       seed=SEED, steps=OracleSteps())
    np.savez(os.path.join(outdir, "rank%d.npz" % rank), U=U.numpy(), S=S.numpy(), V=V.numpy(), sig=sig.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_partition_is_contiguous_and_balanced():
    from paper_2504_04989_gb300 import sharded
    for n, parts in ((13, 2), (5, 3), (65, 8), (7, 7)):
        p = sharded.partition(n, parts)
        assert p[0][0] == 0 and p[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(p, p[1:]))
        sizes = [b - a for a, b in p]
        assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_gloo_matches_oracle(orc, world):
    from paper_2504_04989_gb300 import sharded
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_worker, args=(r, world, port, d)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert p.exitcode == 0
        parts = [np.load(os.path.join(d, "rank%d.npz" % r)) for r in range(world)]
        U = np.concatenate([pt["U"] for pt in parts], axis=1)
        V = np.concatenate([pt["V"] for pt in parts], axis=1)
        S, sig = parts[0]["S"], parts[0]["sig"]
        for pt in parts[1:]:
            np.testing.assert_array_equal(pt["sig"], sig)
    X = _tensor()
    Ur, Sr, Vr, sigr = orc.rtsvd(X, R, P, Q, seed=SEED)
    np.testing.assert_allclose(sig, sigr, rtol=1e-12)
    Xr_ref = orc.reconstruct(Ur, Sr, Vr)
    Xr = orc.reconstruct(U, S, V)
    assert np.linalg.norm(Xr - Xr_ref) <= 1e-10 * np.linalg.norm(Xr_ref)
    # every rank got its own part of the partitions
    assert U.shape == (N3, N1, R) and V.shape == (N3, N2, R)
    assert len(sharded.partition(N3 // 2 + 1, world)) == world
