"""Sharded form on one GPU: the tensor split into slabs of mode 1, the slab
pass scattered into the whole block layout, summed over the slabs.

Ranks are emulated on one GPU: the slab passes run one after another, or -
for whole sharded solves - as host threads, one library handle and one CUDA
stream each, whose block reduction meets on the host (every thread first
synchronises its own stream; no kernel waits for another).  The sums are
compared with the FP64 oracle's blocks of the whole tensor (eq. 3.3) and the
solves with the oracle's solve."""
import threading

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from helpers import assert_same_solution

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01778_gb300 import build
    build.build()


def P():
    import paper_2403_01778_gb300 as pkg
    return pkg


def slab_sum(T, u, world):
    """Sum over the slabs of the slab passes (the collective's result)."""
    pkg = P()
    dim0 = T.shape[0]
    parts = []
    for rank in range(world):
        row0, rows = pkg.shard_rows(dim0, rank, world)
        # a rank's own allocation (a view into T need not start 16-byte aligned)
        parts.append(pkg.hoscf_ttvc_blocks_slab(T[row0:row0 + rows].clone(), row0, dim0, u))
    tot = parts[0].clone()
    for p in parts[1:]:
        tot += p
    torch.cuda.synchronize()
    return tot, parts


@pytest.mark.parametrize("dims", [(7, 5, 6, 9), (10, 33, 40), (9, 13), (5, 4, 3, 6, 8), (12, 64, 128)])
@pytest.mark.parametrize("world", [1, 2, 3])
def test_slab_blocks_sum_to_the_whole_blocks_exactly(dims, world):
    """Integer-valued tensor and factors (every FP32 sum exact): the sum over
    the slabs equals the oracle's whole blocks bit for bit, and each slab's
    output is the oracle's blocks of that slab with the A_{1,n} rows placed
    at row0 and zeros elsewhere."""
    rng = np.random.default_rng(sum(dims) + world)
    T = rng.integers(-3, 4, size=dims).astype(np.float32)
    u = [rng.integers(-2, 3, size=n).astype(np.float64) for n in dims]
    Tg = torch.from_numpy(T).cuda()
    ug = torch.from_numpy(np.concatenate(u).astype(np.float32)).cuda()
    tot, parts = slab_sum(Tg, ug, world)
    assert np.array_equal(tot.double().cpu().numpy(), oracle.blocks(T, u))
    offs, _ = oracle.block_offsets(list(dims))
    for rank, part in enumerate(parts):
        row0, rows = P().shard_rows(dims[0], rank, world)
        us = [u[0][row0:row0 + rows]] + u[1:]
        Hs = oracle.unpack_blocks(oracle.blocks(T[row0:row0 + rows], us), [rows] + list(dims[1:]))
        got = part.double().cpu().numpy()
        for (m, n), o in zip(oracle.block_pairs(len(dims)), offs):
            B = got[o:o + dims[m] * dims[n]].reshape(dims[m], dims[n])
            if m == 0:
                want = np.zeros((dims[0], dims[n]))
                want[row0:row0 + rows] = Hs[(0, n)]
            else:
                want = Hs[(m, n)]
            assert np.array_equal(B, want), (rank, m, n)


@pytest.mark.parametrize("dims", [(40, 41, 42, 43), (300, 64, 96)])
def test_slab_blocks_gaussian_within_fp32_bound(dims):
    T = W.gaussian_tensor(dims, 3).numpy()
    u = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 4)]
    tot, _ = slab_sum(torch.from_numpy(T).cuda(),
                      torch.from_numpy(np.concatenate(u).astype(np.float32)).cuda(), 3)
    Hr = oracle.blocks(T, u)
    S = oracle.blocks(np.abs(T).astype(np.float64), [np.abs(v) for v in u])
    M = np.concatenate([np.full(dims[m] * dims[n], np.prod(dims) / (dims[m] * dims[n]))
                        for (m, n) in oracle.block_pairs(len(dims))])
    assert np.all(np.abs(tot.double().cpu().numpy() - Hr) <= 8 * EPS32 * np.sqrt(M + 3) * S + 1e-30)


def test_one_rank_sharded_solve_is_hoscf_solve():
    """world = 1: the slab is the tensor and the reduction is the identity, so
    the sharded solve is hoscf_solve bit for bit."""
    dims = (30, 40, 50)
    T, _ = W.planted_cp(dims, [2.0, 1.0], seed=31, noise_abs=0.3)
    u0 = torch.cat(W.unit_gaussian_vectors(dims, 32)).cuda()
    Tg = T.cuda()
    a = P().hoscf_solve(Tg, u0, tol=1e-6, max_iter=300)
    b = P().hoscf_solve_sharded(Tg, 0, dims[0], u0, reduce=lambda t: None, tol=1e-6, max_iter=300)
    assert a.converged and b.converged
    assert (a.iters, a.passes) == (b.iters, b.passes)
    assert a.sigma == b.sigma and torch.equal(a.u, b.u)


class HostGroup:
    """Emulated collective of `world` host threads on one GPU: each thread
    synchronises its stream, deposits its buffer, and after a barrier rank 0
    writes the sum (in rank order) into every buffer and synchronises."""

    def __init__(self, world):
        self.world = world
        self.bar = threading.Barrier(world, timeout=60)
        self.bufs = [None] * world

    def reducer(self, rank):
        def reduce(t):
            torch.cuda.current_stream().synchronize()
            self.bufs[rank] = t
            self.bar.wait()
            if rank == 0:
                tot = self.bufs[0].clone()
                for b in self.bufs[1:]:
                    tot += b
                for b in self.bufs:
                    b.copy_(tot)
                torch.cuda.current_stream().synchronize()
            self.bar.wait()
        return reduce


def sharded_solve_threads(T, u0, world, **kw):
    pkg = P()
    dim0 = T.shape[0]
    grp = HostGroup(world)
    out, errs = [None] * world, []

    def run(rank):
        h = pkg.hoscf_create_handle(0)
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                row0, rows = pkg.shard_rows(dim0, rank, world)
                Ts = T[row0:row0 + rows].clone()
                s.synchronize()
                out[rank] = pkg.hoscf_solve_sharded(Ts, row0, dim0, u0, reduce=grp.reducer(rank),
                                                    handle_=h, **kw)
                s.synchronize()
        except BaseException as exc:
            errs.append(exc)
            grp.bar.abort()
        finally:
            pkg.hoscf_destroy_handle(h)

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return out


@pytest.mark.parametrize("dims,world,variant", [((30, 40, 50), 3, "hoscf"), ((13, 9, 10, 11), 2, "hoscf"),
                                                 ((30, 40, 50), 2, "ihoscf"), ((30, 40, 50), 3, "asvd")])
def test_sharded_solve_over_emulated_ranks_matches_the_oracle(dims, world, variant):
    T, _ = W.planted_cp(dims, [4.0, 1.0], seed=41, noise_abs=0.4)
    u0 = W.unit_gaussian_vectors(dims, 42)
    fn = oracle.asvd if variant == "asvd" else oracle.hoscf
    kw = {} if variant == "asvd" else {"variant": variant}
    ref = fn(T.numpy(), [v.numpy() for v in u0], tol=1e-10, max_iter=1000, **kw)
    assert ref.converged
    res = sharded_solve_threads(T.cuda(), torch.cat(u0).cuda(), world, tol=1e-6, max_iter=1000,
                                variant=variant)
    for r in res:
        assert r.converged
        assert r.sigma == res[0].sigma and torch.equal(r.u, res[0].u)   # identical on every rank
    assert_same_solution(res[0].sigma, res[0].factors(), ref.sigma, ref.u)


def test_sharded_rejects_rows_outside_mode_1():
    pkg = P()
    T = torch.randn(4, 5, 6, device="cuda")
    u = torch.randn(10 + 5 + 6, device="cuda")
    with pytest.raises(pkg.HoscfError) as e:
        pkg.hoscf_ttvc_blocks_slab(T, 7, 10, u)
    assert e.value.status == 1
    with pytest.raises(ValueError):
        pkg.shard_rows(2, 0, 3)
