"""Host side of the sharded form, on CPU: the partition of mode 1 into
slabs, and the assembly of the whole blocks from the slabs' contributions by
the binding's SUM all-reduce over a real process group (2 gloo ranks).

Each rank computes its slab's contribution with the FP64 oracle (eq. 3.3 on
the slab, the A_{1,n} rows placed at the slab's rows, zeros elsewhere; the
same layout hoscf_ttvc_blocks_slab writes on the GPU) and the reduced sum
must be the oracle's blocks of the whole tensor."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W
from paper_2403_01778_gb300 import allreduce_blocks, shard_rows


@pytest.mark.parametrize("dim0,world", [(10, 3), (7, 7), (1024, 8), (5, 1), (9, 4)])
def test_partition_covers_mode_1_once_in_order(dim0, world):
    spans = [shard_rows(dim0, r, world) for r in range(world)]
    assert spans[0][0] == 0
    for (a0, an), (b0, _) in zip(spans, spans[1:]):
        assert b0 == a0 + an
    assert spans[-1][0] + spans[-1][1] == dim0
    assert max(n for _, n in spans) - min(n for _, n in spans) <= 1
    assert min(n for _, n in spans) >= 1


def test_partition_rejects_too_many_ranks():
    with pytest.raises(ValueError):
        shard_rows(3, 0, 4)
    with pytest.raises(ValueError):
        shard_rows(8, 4, 4)


def slab_contribution(T, u, row0, rows):
    """The slab's blocks in the whole tensor's packed layout (oracle)."""
    dims = list(T.shape)
    us = [u[0][row0:row0 + rows]] + u[1:]
    Hs = oracle.unpack_blocks(oracle.blocks(np.ascontiguousarray(T[row0:row0 + rows]), us),
                              [rows] + dims[1:])
    out = []
    for (m, n) in oracle.block_pairs(len(dims)):
        if m == 0:
            B = np.zeros((dims[0], dims[n]))
            B[row0:row0 + rows] = Hs[(0, n)]
        else:
            B = Hs[(m, n)]
        out.append(B.ravel())
    return np.concatenate(out)


def _rank(rank, world, port, dims, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        T = W.gaussian_tensor(dims, 5).numpy().astype(np.float64)
        u = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 6)]
        row0, rows = shard_rows(dims[0], rank, world)
        t = torch.from_numpy(slab_contribution(T, u, row0, rows))
        allreduce_blocks(t)
        if rank == 0:
            q.put(float(np.max(np.abs(t.numpy() - oracle.blocks(T, u)))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dims", [(5, 4, 6), (7, 3, 4, 5)])
def test_two_gloo_ranks_assemble_the_whole_blocks(dims):
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, dims, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) <= 1e-12
