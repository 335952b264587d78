"""The exchange and ordering logic of the row-sharded POD
(paper_2405_15529_gb300.sharded.pod_sharded), run as a world-size-2 gloo
process group on the CPU: each rank holds one block of rows, factors it,
all-gathers the R factors in rank order, runs the replicated top and picks
its own block B_rank.  The three device steps are replaced by CPU stand-ins
built from the oracle's routines (Householder QR of the rows, of the stacked
factors, the Jacobi SVD and the reflector product), so the test checks what
the collective part does: ranks' factors land in the right slots, every rank
gets the same S and r, and the ranks' mode rows stack to the POD of the whole
matrix (compared with the oracle's own POD of it)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

N, M, R_MAX = 3000, 12, 12
SPLIT = 1300          # rank 0: rows [0, 1300), rank 1: rows [1300, 3000)


def _matrix():
    import synth
    return synth.waves(N, M, n_waves=3, noise=1e-3, seed=61)


class CpuShardOps:
    """CPU stand-ins for the three device steps (test infrastructure)."""

    def __init__(self, energy=0.0):
        import oracle
        self.o = oracle
        self.energy = energy

    def factor(self, X, w):
        Y, mean = self.o.center_weight(X.numpy(), None, True)
        packed, tau = self.o.householder_qr(Y)
        R = np.triu(packed[:M, :])
        # column-major R_g, as the device step returns it
        return torch.from_numpy(np.asfortranarray(R)).t().contiguous().t(), (packed, tau)

    def top(self, Rstack):
        G = Rstack.shape[0]
        C = np.vstack([Rstack[g].numpy().T for g in range(G)])      # slot g holds R_g column-major
        packed, tau = self.o.householder_qr(C)
        R = np.triu(packed[:M, :])
        U_R, S, V, _ = self.o.svd(R)
        r = self.o.truncation_rank(S, self.energy, R_MAX)
        Z = np.zeros((G * M, r))
        Z[:M] = U_R[:, :r]
        Bfull = self.o.apply_q(packed, tau, Z)
        B = torch.zeros((G, R_MAX, M), dtype=torch.float64)
        for g in range(G):
            B[g, :r, :] = torch.from_numpy(Bfull[g * M:(g + 1) * M].T.copy())
        return torch.from_numpy(S), torch.from_numpy(V.T.copy()), B, torch.tensor([r]), None

    def modes(self, state, Bg, r_dev, w):
        packed, tau = state
        r = int(r_dev[0])
        Z = np.zeros((packed.shape[0], r))
        Z[:M] = Bg.numpy()[:r].T
        return torch.from_numpy(self.o.apply_q(packed, tau, Z))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2405_15529_gb300 import sharded
        X = _matrix()
        rows = slice(0, SPLIT) if rank == 0 else slice(SPLIT, N)
        U, S, VT, r = sharded.pod_sharded(torch.from_numpy(np.ascontiguousarray(X[rows])), ops=CpuShardOps())
        q.put((rank, U.numpy(), S.numpy(), r))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_exchange_gloo():
    import oracle
    from tests import parity
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, U0, S0, r0), (_, U1, S1, r1) = out
    assert r0 == r1 and np.array_equal(S0, S1)          # replicated top: identical on both ranks
    assert U0.shape[0] == SPLIT and U1.shape[0] == N - SPLIT
    ref = oracle.pod(_matrix(), remove_mean=True, r_max=R_MAX)
    parity.check_sigma(S0, ref["S"])
    parity.check_vectors(np.vstack([U0, U1]), ref["U"], ref["S"], ncols=r0)


def test_single_process_falls_back_to_one_shard():
    import oracle
    from tests import parity
    from paper_2405_15529_gb300 import sharded
    assert not dist.is_initialized()
    X = _matrix()
    U, S, VT, r = sharded.pod_sharded(torch.from_numpy(np.ascontiguousarray(X)), ops=CpuShardOps())
    ref = oracle.pod(X, remove_mean=True, r_max=R_MAX)
    parity.check_sigma(S.numpy(), ref["S"])
    parity.check_vectors(U.numpy(), ref["U"], ref["S"], ncols=r)
