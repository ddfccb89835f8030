"""The row-sharded multi-GPU design of frPCAt (Alg. 6), checked on CPU ranks
(gloo, world size 2) with the oracle's steps standing in for the kernels.

A is split into row blocks A_b (rank b holds rows r_b .. r_{b+1}-1).  The
exchange steps are exactly those the design names:
  - A Q: local, Y_b = A_b Q (Q replicated, no communication);
  - A^T Y = sum_b A_b^T Y_b: one all-reduce of an n x l block per A^T pass;
  - lu() and the power iteration's eigSVD act on the replicated n x l block
    (every rank computes the same result from the same input);
  - the final eigSVD on the row-sharded m x l block: one all-reduce of the
    l x l Gram, then each rank applies V^ diag(1./S^) to its own rows.
The sharded result must match the single-rank oracle to rounding (1e-12 on
sigma, 1e-10 on the principal-angle sines): only the order of the cross-rank
sums differs.  Even q draws the m x l Gaussian block of Alg. 6 in full and
each rank takes its rows of it, so the sketch equals the single-rank one.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _allreduce(x):
    t = torch.from_numpy(np.ascontiguousarray(x))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def _eigsvd_replicated(oracle, M):
    U, S, V = oracle.eigsvd(M)
    return U


def sharded_frpca(oracle, A, r0, r1, k, l, q, seed):
    """Alg. 6 on the row block r0..r1-1 of A, with the design's collectives."""
    m, n = A.m, A.n
    ip = A.indptr[r0:r1 + 1] - A.indptr[r0]
    ix = A.indices[A.indptr[r0]:A.indptr[r1]]
    va = A.data[A.indptr[r0]:A.indptr[r1]].astype(np.float64)
    mb = r1 - r0
    spmm = lambda X: oracle.spmm(mb, n, ip, ix, va, X)                  # A_b X   # noqa: E731
    spmm_t = lambda Y: _allreduce(oracle.spmm_t(mb, n, ip, ix, va, Y))  # sum_b A_b^T Y_b  # noqa: E731
    if q % 2 == 0:
        Om = oracle.gaussian(m, l, seed)[r0:r1]
        Q = spmm_t(Om)
        Q = _eigsvd_replicated(oracle, Q) if q == 2 else oracle.lu_ptl(Q)[0]
    else:
        Q = oracle.gaussian(n, l, seed)
    loops = (q - 1) // 2
    for i in range(1, loops + 1):
        Q = spmm_t(spmm(Q))
        Q = _eigsvd_replicated(oracle, Q) if i == loops else oracle.lu_ptl(Q)[0]
    W = spmm(Q)
    B = _allreduce(oracle.gram(W))
    w, Vh = oracle.eig_sym(B)
    S = np.sqrt(w)
    ind = np.arange(l - 1, l - 1 - k, -1)
    Ub = (W @ Vh[:, ind]) / S[ind]
    V = Q @ Vh[:, ind]
    # Sign convention of the method's output: v_j's largest-magnitude entry
    # (smallest index on ties) positive; V is replicated, so every rank agrees.
    sign = np.sign(V[np.argmax(np.abs(V), axis=0), np.arange(k)])
    return Ub * sign, S[ind], V * sign


def _worker(rank, world, port, q_out, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import oracle
    import synthetic
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = synthetic.powerlaw_csr(4000, 700, 15, 1.1, "tfidf", seed=5, dtype=np.float64)
        bounds = np.linspace(0, A.m, world + 1).astype(int)
        r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
        Ub, S, V = sharded_frpca(oracle, A, r0, r1, 8, 20, q, 3)
        q_out.put((rank, r0, r1, Ub, S, V))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("q", [3, 4, 5])
def test_row_sharded_design_matches_single_rank_oracle(q):
    sys.path.insert(0, ROOT)
    import oracle
    import synthetic
    from tests.helpers import max_principal_sine

    oracle.build()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, out, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    A = synthetic.powerlaw_csr(4000, 700, 15, 1.1, "tfidf", seed=5, dtype=np.float64)
    Uo, So, Vo = oracle.frpca(A.m, A.n, A.indptr, A.indices, A.data, 8, 20, q, 3)
    U = np.vstack([g[3] for g in got])
    assert [g[1] for g in got] == [0, got[0][2]] and got[-1][2] == A.m
    for g in got:  # S and V are replicated
        assert np.array_equal(g[4], got[0][4]) and np.array_equal(g[5], got[0][5])
    S, V = got[0][4], got[0][5]
    assert np.max(np.abs(S - So) / So) <= 1e-12
    assert max_principal_sine(U, Uo) <= 1e-10
    assert max_principal_sine(V, Vo) <= 1e-10
    # Same sign convention, so the vectors themselves agree.
    assert np.max(np.abs(V - Vo)) <= 1e-9
    assert np.max(np.abs(U - Uo)) <= 1e-9
