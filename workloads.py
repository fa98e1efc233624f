"""Seeded synthetic inputs shaped like the paper's experiments and the bench
workloads of this project.

This module is the one place that both the CUDA path (tests, bench) and the
FP64 oracle get their inputs from.  It holds input synthesis only - random
factors, noise, the closed-form test tensors of the paper's Example 2 - and
none of the HOSCF arithmetic (no blocks, no eigen-solves, no residuals).

All generators are deterministic functions of their seed.  Tensors are
float32, row-major (last index fastest).  Generation runs on the device the
caller names; the CPU and CUDA random streams differ, so a test that compares
the two paths generates on the CPU once and copies the same bytes to the GPU.

Workload recipes (sizes and distributions follow the paper and the project's
benchmark configurations):

* ``planted_cp``: T = sum_r w_r a_r^(1) o ... o a_r^(d) + E, each a_r^(n) a
  seeded Gaussian vector normalised to unit length, E i.i.d. N(0,1) rescaled so
  that ||E||_F equals ``noise_abs`` or ``noise_rel * ||L||_F`` (L the
  noiseless part).
* ``gaussian_tensor``: i.i.d. N(0,1) entries (the paper's Example 1 and the
  pure-noise 1024^3 case).
* ``example2``: EXP (30^3), ARCSIN (20^4), TAN (10^5) of the paper's Table 2
  (1-based indices; the ARCSIN entry is read as
  sum_j arcsin((-1)^{i_j} j / i_j) when i_j >= j for every j, else 0).
* ``unit_gaussian_vectors`` / ``uniform01_vectors``: initial guesses (the
  bench's seeded unit Gaussian x0, and the paper's U[0,1] entries of Sec. 6.1).
* ``batched_dims``: the ragged batch (768 order-3 tensors with dims in [8,96],
  256 order-4 tensors with dims in [8,32], sigma ~ U[1,10], 5% noise).
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def unit_gaussian_vectors(dims, seed: int, device="cpu"):
    """One seeded N(0,1) vector per mode, each scaled to unit 2-norm (float32)."""
    g = _gen(seed, device)
    out = []
    for n in dims:
        v = torch.randn(int(n), generator=g, device=device, dtype=torch.float64)
        out.append((v / v.norm()).to(torch.float32))
    return out


def uniform01_vectors(dims, seed: int, device="cpu"):
    """Initial guess with U[0,1] entries, as in the paper's Sec. 6.1 (float32)."""
    g = _gen(seed, device)
    return [torch.rand(int(n), generator=g, device=device, dtype=torch.float32) for n in dims]


def outer(vectors):
    """v1 o v2 o ... o vd as a dense tensor (input synthesis helper)."""
    out = vectors[0]
    for v in vectors[1:]:
        out = out.unsqueeze(-1) * v
    return out


def gaussian_tensor(dims, seed: int, device="cpu"):
    g = _gen(seed, device)
    return torch.randn(*[int(n) for n in dims], generator=g, device=device,
                       dtype=torch.float32)


def coupled_pair(dims, a: float, seed: int, noise_abs: float = 0.0, device="cpu"):
    """u o ... o u plus a times every placement of v o v (two modes) among
    the u's, v a unit vector orthogonal to u (one u, v per mode), plus
    Gaussian noise of norm noise_abs - a tensor whose blocks at the best
    rank-one point keep a second singular value of about a, so that HOSCF
    converges slowly and steadily (about 15 % per iteration at a = 0.3, d = 4).
    Returns T (float32)."""
    import itertools
    dims = [int(n) for n in dims]
    d = len(dims)
    g = _gen(seed, device)
    us, vs = [], []
    for n in dims:
        u = torch.randn(n, generator=g, device=device, dtype=torch.float64)
        u /= u.norm()
        v = torch.randn(n, generator=g, device=device, dtype=torch.float64)
        v -= (v @ u) * u
        v /= v.norm()
        us.append(u.to(torch.float32))
        vs.append(v.to(torch.float32))
    T = outer(us)
    for pos in itertools.combinations(range(d), 2):
        T.add_(outer([vs[k] if k in pos else us[k] for k in range(d)]), alpha=float(a))
    if noise_abs:
        E = torch.randn(*dims, generator=g, device=device, dtype=torch.float32)
        E.mul_(float(noise_abs) / float(E.double().norm()))
        T.add_(E)
    return T


def planted_cp(dims, weights, seed: int, noise_rel=None, noise_abs=None, device="cpu"):
    """Planted CP tensor plus scaled Gaussian noise.

    Returns (T float32, factors) with factors[r][n] the unit vector of rank-one
    term r in mode n (float32)."""
    dims = [int(n) for n in dims]
    g = _gen(seed, device)
    factors = []
    L = torch.zeros(*dims, device=device, dtype=torch.float32)
    for w in weights:
        fr = []
        for n in dims:
            v = torch.randn(n, generator=g, device=device, dtype=torch.float64)
            fr.append((v / v.norm()).to(torch.float32))
        factors.append(fr)
        L.add_(outer(fr), alpha=float(w))
    if noise_abs is None and noise_rel is None:
        return L, factors
    E = torch.randn(*dims, generator=g, device=device, dtype=torch.float32)
    target = noise_abs if noise_abs is not None else noise_rel * float(
        L.double().norm())
    E.mul_(float(target) / float(E.double().norm()))
    L.add_(E)
    return L, factors


def example2(name: str, device="cpu"):
    """Closed-form tensors of the paper's Example 2 (Table 2), float32.  On a
    CUDA device the same formulas are evaluated there (FP64, then rounded)."""
    if str(device) != "cpu":
        return _example2_torch(name, device)
    name = name.upper()
    if name == "EXP":
        d, I = 3, 30
    elif name == "ARCSIN":
        d, I = 4, 20
    elif name == "TAN":
        d, I = 5, 10
    else:
        raise ValueError(name)
    idx = np.indices([I] * d, dtype=np.float64) + 1.0     # 1-based i_j
    j = np.arange(1, d + 1, dtype=np.float64).reshape([d] + [1] * d)
    if name == "EXP":
        A = np.sum(((-1.0) ** (j + 1)) * j * np.exp(-idx), axis=0)
    elif name == "ARCSIN":
        ok = np.all(idx >= j, axis=0)
        arg = np.where(idx >= j, ((-1.0) ** idx) * j / idx, 0.0)
        A = np.where(ok, np.sum(np.arcsin(arg), axis=0), 0.0)
    else:
        A = np.tan(np.sum(((-1.0) ** (j + 1)) * idx / j, axis=0))
    return torch.from_numpy(A.astype(np.float32))


def _example2_torch(name: str, device):
    """example2() with torch FP64 element-wise functions on `device`."""
    name = name.upper()
    d, I = {"EXP": (3, 30), "ARCSIN": (4, 20), "TAN": (5, 10)}[name]
    ar = torch.arange(1, I + 1, dtype=torch.float64, device=device)
    idx = torch.stack(torch.meshgrid(*([ar] * d), indexing="ij"))      # 1-based i_j
    j = torch.arange(1, d + 1, dtype=torch.float64, device=device).reshape([d] + [1] * d)
    sgn_j = torch.where(j % 2 == 1, 1.0, -1.0)                          # (-1)^(j+1)
    if name == "EXP":
        A = torch.sum(sgn_j * j * torch.exp(-idx), dim=0)
    elif name == "ARCSIN":
        ok = torch.all(idx >= j, dim=0)
        sgn_i = torch.where(idx % 2 == 0, 1.0, -1.0)                    # (-1)^(i_j)
        arg = torch.where(idx >= j, sgn_i * j / idx, torch.zeros_like(idx))
        A = torch.where(ok, torch.sum(torch.asin(arg), dim=0), torch.zeros_like(ok, dtype=torch.float64))
    else:
        A = torch.tan(torch.sum(sgn_j * idx / j, dim=0))
    return A.to(torch.float32).contiguous()


def batched_dims(seed: int, count3: int = 768, count4: int = 256,
                 lo3: int = 8, hi3: int = 96, lo4: int = 8, hi4: int = 32):
    """Ragged dims of the batched workload (inclusive uniform integer ranges)
    plus one planted weight sigma ~ U[1,10] per tensor."""
    rng = np.random.default_rng(int(seed))
    dims = [tuple(int(v) for v in rng.integers(lo3, hi3 + 1, size=3)) for _ in range(count3)]
    dims += [tuple(int(v) for v in rng.integers(lo4, hi4 + 1, size=4)) for _ in range(count4)]
    sig = rng.uniform(1.0, 10.0, size=len(dims))
    return dims, [float(s) for s in sig]


def batched_tensors(seed: int, noise_frac: float = 0.05, device="cpu", **kw):
    """The batched workload: planted rank-one sigma * u1 o ... o ud plus noise
    with ||E||_F = noise_frac * sigma, one seed per tensor."""
    dims, sig = batched_dims(seed, **kw)
    out = []
    for t, (dd, s) in enumerate(zip(dims, sig)):
        T, _ = planted_cp(dd, [s], seed=seed * 100003 + t, noise_abs=noise_frac * s,
                          device=device)
        out.append(T)
    return out, sig


# Named workloads of the project's benchmark configurations.
CONFIGS = {
    "cfg1_64cube": dict(dims=(64, 64, 64), weights=[10.0], noise_abs=1.0),
    "cfg2a_1024cube_rank5": dict(dims=(1024, 1024, 1024),
                                 weights=[2.0 ** -r for r in range(5)], noise_rel=0.05),
    "cfg2b_1024cube_gauss": dict(dims=(1024, 1024, 1024), gaussian=True),
    "cfg3_200p4": dict(dims=(200, 200, 200, 200), weights=[100.0], noise_abs=10.0),
    "cfg4a_256cube": dict(dims=(256, 256, 256), weights=[1.0], noise_abs=0.05),
    "cfg4b_order6": dict(dims=(24, 20, 24, 20, 24, 20), weights=[1.0], noise_abs=0.05),
}


def config_tensor(name: str, seed: int = 0, device="cpu"):
    """Tensor of a named workload (float32) - see CONFIGS."""
    c = CONFIGS[name]
    if c.get("gaussian"):
        return gaussian_tensor(c["dims"], seed, device)
    T, _ = planted_cp(c["dims"], c["weights"], seed, noise_rel=c.get("noise_rel"),
                      noise_abs=c.get("noise_abs"), device=device)
    return T


def table_shapes():
    """The four equal-size (16.8M element) tensors of the paper's scalability
    test (Sec. 6.2, Table 5); dims as printed (the order-7 one has 33.6M)."""
    return [(32, 32, 32, 32, 16), (16,) * 6, (16, 16, 16, 16, 8, 8, 8), (8,) * 8]


def n_elements(dims) -> int:
    return int(math.prod(int(v) for v in dims))
