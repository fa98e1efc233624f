"""Full-size workloads in the launch configuration the benchmark times: the
1024^3 planted rank-5 tensor (FP32) and the 200^4 planted rank-one tensor
(FP32, BF16, FP8-e4m3 with per-128 scales), made on the device by the seeded
workload generators and passed through hoscf_ttvc_blocks as the benchmark
does.  Sampled entries of every block are compared with the oracle's
one-entry definition (eq. 3.3) evaluated on the slab of T that the entry sums
(the modes m, n fixed at i, j); for the narrow formats the oracle quantises
the FP32 slab itself (whole 128-element groups for FP8)."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01778_gb300 import build
    build.build()


def P():
    import paper_2403_01778_gb300 as pkg
    return pkg


def slab_flat_indices(dims, m, n, i, j):
    """Row-major flat indices of T[..., i (mode m), ..., j (mode n), ...], in
    the slab's own row-major order."""
    st = [int(np.prod(dims[k + 1:])) for k in range(len(dims))]
    grids = [np.arange(dims[k]) if k not in (m, n) else np.array([i if k == m else j])
             for k in range(len(dims))]
    f = np.zeros([len(g) for g in grids], dtype=np.int64)
    for k, g in enumerate(grids):
        shape = [1] * len(dims)
        shape[k] = len(g)
        f = f + (g * st[k]).reshape(shape)
    return f


def oracle_slab(T32, dims, fmt, f):
    """FP64 values of the slab at flat indices f after the oracle's own
    storage rounding of the FP32 tensor."""
    flat = T32.view(-1)
    if fmt == "fp32":
        return flat[torch.from_numpy(f.ravel()).cuda()].double().cpu().numpy().reshape(f.shape)
    if fmt == "bf16":
        x = flat[torch.from_numpy(f.ravel()).cuda()].cpu().numpy()
        return oracle.dequantize_bf16(oracle.quantize_bf16(x)).reshape(f.shape)
    # fp8: quantise every 128-element group that holds a slab element
    grp = np.unique(f.ravel() // 128)
    idx = (grp[:, None] * 128 + np.arange(128)[None, :]).ravel()
    x = flat[torch.from_numpy(idx).cuda()].cpu().numpy()
    codes, scales = oracle.quantize_e4m3_scaled(x)
    vals = oracle.dequantize_e4m3_scaled(codes, scales).reshape(len(grp), 128)
    pos = np.searchsorted(grp, f.ravel() // 128)
    return vals[pos, f.ravel() % 128].reshape(f.shape)


@pytest.mark.parametrize("name,fmt,per_block", [("cfg2a_1024cube_rank5", "fp32", 6),
                                                ("cfg3_200p4", "fp32", 3),
                                                ("cfg3_200p4", "bf16", 2),
                                                ("cfg3_200p4", "fp8", 2)])
def test_blocks_sampled_at_full_size(name, fmt, per_block):
    dims = tuple(W.CONFIGS[name]["dims"])
    d = len(dims)
    T32 = W.config_tensor(name, 0, device="cuda")
    uh = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 7)]
    ug = torch.from_numpy(np.concatenate(uh).astype(np.float32)).cuda()
    if fmt == "fp32":
        Tg, sg = T32, None
    else:
        Tg, sg = P().hoscf_quantize(T32, fmt)
    H = P().hoscf_ttvc_blocks(Tg, ug, scales=sg)
    torch.cuda.synchronize()
    offs, _ = oracle.block_offsets(list(dims))
    rng = np.random.default_rng(8)
    M = math.prod(dims)
    for (m, n), o in zip(oracle.block_pairs(d), offs):
        for _ in range(per_block):
            i, j = int(rng.integers(dims[m])), int(rng.integers(dims[n]))
            f = slab_flat_indices(dims, m, n, i, j)
            Ts = oracle_slab(T32, dims, fmt, f)
            us = list(uh)
            us[m], us[n] = uh[m][i:i + 1], uh[n][j:j + 1]
            ref = oracle.block_entry(Ts, us, m, n, 0, 0)
            sc = oracle.block_entry(np.abs(Ts), [np.abs(v) for v in us], m, n, 0, 0)
            tol = 8 * EPS32 * math.sqrt(M / (dims[m] * dims[n]) + 1) * sc + 1e-30
            got = H[o + i * dims[n] + j].item()
            assert abs(got - ref) <= tol, ((m, n), i, j, got, ref, tol)
    del T32, Tg, sg, H
    torch.cuda.empty_cache()


@pytest.mark.parametrize("name,fmt", [("cfg2a_1024cube_rank5", "fp32"), ("cfg3_200p4", "fp8")])
def test_solve_at_full_size_is_a_kkt_point_for_the_oracle(name, fmt):
    """Whole solves at full size (the 200^4 one on FP8 storage with FP32
    refinement): the oracle's FP64 pass over the FP32 tensor at the returned
    factors gives the same sigma and a KKT residual (eq. 2.4) within the
    tolerance."""
    dims = tuple(W.CONFIGS[name]["dims"])
    T32 = W.config_tensor(name, 0, device="cuda")
    u0 = torch.cat(W.unit_gaussian_vectors(dims, 9)).cuda()
    if fmt == "fp32":
        r = P().hoscf_solve(T32, u0, tol=1e-6)
    else:
        q, s = P().hoscf_quantize(T32, fmt)
        r = P().hoscf_solve(q, u0, tol=1e-6, scales=s, refine=T32)
        del q, s
    torch.cuda.synchronize()
    assert r.converged
    Th = T32.cpu().numpy()
    del T32
    torch.cuda.empty_cache()
    u = [f.double().cpu().numpy() for f in r.factors()]
    g, full = oracle.kkt_vectors(Th, u)
    rr = np.linalg.norm(np.concatenate(g) - full * np.concatenate(u)) / abs(full)
    assert abs(full - r.sigma) <= 1e-5 * abs(full), (full, r.sigma)
    assert rr <= 1e-5, rr
