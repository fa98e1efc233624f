"""Precision form on the GPU: BF16 / FP8-e4m3 storage against the oracle's
format definitions (bit-exact codes) and the oracle's blocks of the exactly
dequantised tensor; low-precision solve with FP32 refinement against the FP64
oracle on the FP32 tensor."""
import math

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


def test_quantize_bf16_bit_exact():
    x = W.gaussian_tensor((3, 1000, 37), 1).numpy() * 50
    q, _ = P().hoscf_quantize(torch.from_numpy(x).cuda(), "bf16")
    got = q.view(torch.int16).cpu().numpy().view(np.uint16).ravel()
    assert np.array_equal(got, oracle.quantize_bf16(x).ravel())


def test_quantize_f16_bit_exact():
    """Including subnormal codes (tiny values) and overflow to infinity."""
    x = W.gaussian_tensor((3, 1000, 37), 11).numpy() * 50
    x.reshape(-1)[:1000] *= 1e-6
    x.reshape(-1)[1000:1010] = [65504, 65519, 65520, -70000, 1e5, 2 ** -24, 2 ** -25, 0.0, -0.0, 1.0]
    q, _ = P().hoscf_quantize(torch.from_numpy(x).cuda(), "f16")
    got = q.view(torch.int16).cpu().numpy().view(np.uint16).ravel()
    assert np.array_equal(got, oracle.quantize_f16(x).ravel())


@pytest.mark.parametrize("n", [128 * 7, 1000, 129, 1])
def test_quantize_e4m3_bit_exact(n):
    x = W.gaussian_tensor((n,), 2).numpy() * 3
    x[: min(n, 128)] *= 1e-3           # a group with small values (subnormal codes)
    if n > 300:
        x[128:256] = 0.0               # an all-zero group (scale 1)
    q, s = P().hoscf_quantize(torch.from_numpy(x).cuda(), "fp8")
    codes, scales = oracle.quantize_e4m3_scaled(x)
    assert np.array_equal(s.cpu().numpy().view(np.uint32), scales.view(np.uint32))
    assert np.array_equal(q.cpu().numpy().ravel(), codes)


def bound(Tq, u):
    dims = Tq.shape
    S = oracle.blocks(np.abs(Tq), [np.abs(v) for v in u])
    M = np.concatenate([np.full(dims[m] * dims[n], np.prod(dims) / (dims[m] * dims[n]))
                        for (m, n) in oracle.block_pairs(len(dims))])
    return 8 * EPS32 * np.sqrt(M + 1.0) * S + 1e-30


@pytest.mark.parametrize("dims", [(5, 64, 200), (9, 48, 128), (7, 33, 100), (9, 10, 11, 12), (5, 6, 40, 36),
                                  (4, 5, 6, 24, 20), (3, 200, 200), (30, 20), (6, 40, 256), (4, 17, 136)])
@pytest.mark.parametrize("fmt", ["fp8", "bf16", "f16"])
def test_blocks_low_precision_match_dequantised_oracle(dims, fmt):
    """Every load path of every storage format: the full-row kernel (rows of
    128 .. 256, a multiple of 8), the tiled kernel (TMA, cp.async, plain
    loads), the small-face kernel and the order-2 copy."""
    T = W.gaussian_tensor(dims, 3) * 7
    u = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 4)]
    if fmt == "fp8":
        codes, scales = oracle.quantize_e4m3_scaled(T.numpy())
        Tq = oracle.dequantize_e4m3_scaled(codes, scales).reshape(dims)
        Tg = torch.from_numpy(codes.reshape(dims)).cuda()
        sg = torch.from_numpy(scales).cuda()
    elif fmt == "f16":
        q = oracle.quantize_f16(T.numpy())
        Tq = oracle.dequantize_f16(q).reshape(dims)
        Tg = torch.from_numpy(q.view(np.int16)).cuda().view(torch.float16).reshape(dims)
        sg = None
    else:
        q = oracle.quantize_bf16(T.numpy())
        Tq = oracle.dequantize_bf16(q).reshape(dims)
        Tg = torch.from_numpy(q.view(np.int16)).cuda().view(torch.bfloat16).reshape(dims)
        sg = None
    ug = torch.from_numpy(np.concatenate(u).astype(np.float32)).cuda()
    Hg = P().hoscf_ttvc_blocks(Tg, ug, scales=sg).double().cpu().numpy()
    Hr = oracle.blocks(Tq, u)
    assert np.all(np.abs(Hg - Hr) <= bound(Tq, u))


@pytest.mark.parametrize("fmt", ["fp8", "bf16", "f16"])
def test_low_precision_solve_with_fp32_refinement(fmt):
    """Planted rank one (sigma = 100) plus noise of norm 10, like the 200^4
    precision workload at 40^4: iterate on the low-precision copy, refine on
    FP32, and match the FP64 oracle run on the FP32 tensor."""
    dims = (40, 40, 40, 40)
    T, _ = W.planted_cp(dims, [100.0], seed=5, noise_abs=10.0)
    u0 = W.unit_gaussian_vectors(dims, 6)
    ref = oracle.hoscf(T.numpy(), [v.numpy() for v in u0], tol=1e-10, max_iter=200)
    Tg = T.cuda()
    q, s = P().hoscf_quantize(Tg, fmt)
    r = P().hoscf_solve(q, torch.cat(u0).cuda(), scales=s, refine=Tg, tol=1e-6, switch_tol=1e-2)
    assert r.converged and r.passes_refine >= 1 and r.passes > r.passes_refine
    assert_same_solution(r.sigma, r.factors(), ref.sigma, ref.u)


def test_slowly_converging_solve_keeps_the_narrow_copy_until_switch_tol():
    """T = u o u o u o u + 0.3 sum over the six placements of v o v among
    u's (v orthogonal to u): the blocks at the solution keep a strong second
    singular value, so HOSCF converges slowly and steadily (the residual
    falls by ~15 % per iteration, never halving).  With switch_predict 2 the
    narrow-copy passes continue until the residual nears switch_tol - a slow
    decrease is progress, not the storage format's floor - and the FP32
    refinement then reaches the tolerance, certified by the oracle's FP64
    pass."""
    import itertools
    dims = (24, 24, 24, 24)
    rng = np.random.default_rng(25)
    u = rng.standard_normal(24)
    u /= np.linalg.norm(u)
    v = rng.standard_normal(24)
    v -= (v @ u) * u
    v /= np.linalg.norm(v)
    Tn = np.einsum("i,j,k,l->ijkl", u, u, u, u)
    for pos in itertools.combinations(range(4), 2):
        Tn = Tn + 0.3 * np.einsum("i,j,k,l->ijkl", *[v if k in pos else u for k in range(4)])
    Tn = Tn + 1e-4 * rng.standard_normal(Tn.shape)
    T = torch.from_numpy(Tn.astype(np.float32))
    u0 = torch.cat(W.unit_gaussian_vectors(dims, 26)).cuda()
    Tg = T.cuda()
    to_switch = P().hoscf_solve(Tg, u0, tol=1e-3, max_iter=3000)     # FP32 passes down to 1e-3
    q, s = P().hoscf_quantize(Tg, "f16")
    # the prediction from the slower of the last two contractions (a fast
    # first step does not end the narrow passes)
    r = P().hoscf_solve(q, u0, refine=Tg, tol=1e-6, max_iter=3000, switch_tol=1e-3, switch_predict=2)
    assert r.converged
    narrow = r.passes - r.passes_refine
    # the narrow copy carries the iteration down to switch_tol (the
    # prediction may move the switch a pass or two earlier); a rule that took
    # a residual that does not halve for the format's floor stopped after two
    assert to_switch.passes >= 10 and narrow >= to_switch.passes - 3, (narrow, to_switch.passes)
    uf = [f.double().cpu().numpy() for f in r.factors()]
    g, full = oracle.kkt_vectors(T.numpy().astype(np.float64), uf)
    rr = np.linalg.norm(np.concatenate(g) - full * np.concatenate(uf)) / abs(full)
    assert rr <= 1e-5, rr
