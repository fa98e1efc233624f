"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: closed forms, brute force, a textbook special case (the SVD), theorem
invariants, values printed in the paper's tables, finite differences, and the
definitions of the BF16 / FP8-e4m3 formats."""
import itertools
import json
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def rand_unit(dims, seed):
    return [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, seed)]


# ------------------------------------------------------------- eq. (3.3)
@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 5), (2, 3, 2, 3, 2), (4, 3)])
def test_blocks_rank_one_closed_form(dims):
    """For T = a1 o ... o ad:  A_{m,n} = (prod_{k!=m,n} <a_k,u_k>) a_m a_n^T."""
    rng = np.random.default_rng(1)
    a = [rng.standard_normal(n) for n in dims]
    T = W.outer([torch.from_numpy(v) for v in a]).numpy()          # float64
    u = rand_unit(dims, 2)
    H = oracle.unpack_blocks(oracle.blocks(T, u), list(dims))
    d = len(dims)
    for (m, n), B in H.items():
        c = np.prod([a[k] @ u[k] for k in range(d) if k not in (m, n)])
        np.testing.assert_allclose(B, c * np.outer(a[m], a[n]), rtol=1e-12, atol=1e-14)


def test_blocks_integer_brute_force():
    """Integer tensor and integer vectors: FP64 sums are exact, so the blocks
    must equal a pure-Python brute-force sum bit for bit."""
    dims = (3, 2, 4, 3)
    rng = np.random.default_rng(3)
    T = rng.integers(-5, 6, size=dims).astype(np.float32)
    u = [rng.integers(-3, 4, size=n).astype(np.float64) for n in dims]
    H = oracle.unpack_blocks(oracle.blocks(T, u), list(dims))
    for (m, n), B in H.items():
        ref = np.zeros((dims[m], dims[n]))
        for idx in itertools.product(*[range(s) for s in dims]):
            p = float(T[idx])
            for k in range(4):
                if k not in (m, n):
                    p *= u[k][idx[k]]
            ref[idx[m], idx[n]] += p
        assert np.array_equal(B, ref)


def test_blocks_match_einsum_and_entries():
    dims = (4, 5, 3, 2)
    T = W.gaussian_tensor(dims, 5).numpy()
    u = rand_unit(dims, 6)
    Hp = oracle.blocks(T, u)
    H = oracle.unpack_blocks(Hp, list(dims))
    letters = "abcd"
    for (m, n), B in H.items():
        ops, subs = [T.astype(np.float64)], [letters]
        for k in range(4):
            if k not in (m, n):
                ops.append(u[k])
                subs.append(letters[k])
        ref = np.einsum(",".join(subs) + "->" + letters[m] + letters[n], *ops)
        np.testing.assert_allclose(B, ref, rtol=1e-12, atol=1e-13)
        for (i, j) in [(0, 0), (dims[m] - 1, dims[n] - 1), (1, 0)]:
            for fast in (True, False):
                assert abs(oracle.block_entry(T, u, m, n, i, j, fast=fast) - B[i, j]) < 1e-12


def test_kkt_vectors_match_blocks():
    """g_n from the tensor directly equals A_{n,m} u_m for every m != n."""
    dims = (5, 4, 6)
    T = W.gaussian_tensor(dims, 7).numpy()
    u = rand_unit(dims, 8)
    g, full = oracle.kkt_vectors(T, u)
    Hf = oracle.full_block_matrix(oracle.blocks(T, u), list(dims))
    off = oracle.mode_offsets(dims)
    for n in range(3):
        for m in range(3):
            if m == n:
                continue
            gnm = Hf[off[n]:off[n + 1], off[m]:off[m + 1]] @ u[m]
            np.testing.assert_allclose(gnm, g[n], rtol=1e-12, atol=1e-13)
        assert abs(full - g[n] @ u[n]) < 1e-12


def test_ttv_definition():
    dims = (3, 4, 5)
    T = W.gaussian_tensor(dims, 9).numpy()
    v = np.arange(4, dtype=np.float64)
    np.testing.assert_allclose(oracle.ttv(T, 1, v), np.einsum("abc,b->ac", T.astype(np.float64), v),
                               rtol=1e-12)


# ------------------------------------------------------------- Theorem 1
@pytest.mark.parametrize("dims", [(4, 5, 3), (3, 4, 2, 3)])
def test_spectrum_flip_theorem1_p1(dims):
    """Thm 1 (P1): negating block 1 of x negates the spectrum of J(x)."""
    T = W.gaussian_tensor(dims, 11).numpy()
    u = rand_unit(dims, 12)
    uh = [-u[0]] + u[1:]
    J = oracle.nepv_matrix(oracle.blocks(T, u), list(dims))
    Jh = oracle.nepv_matrix(oracle.blocks(T, uh), list(dims))
    w = np.sort(np.linalg.eigvalsh(J))
    wh = np.sort(np.linalg.eigvalsh(Jh))
    np.testing.assert_allclose(wh, -w[::-1], atol=1e-12)


# ------------------------------------------------------------- d = 2: SVD
def test_order2_is_top_singular_triplet():
    """d = 2: J is [[0,A],[A^T,0]] and the best rank-one approximation is the
    top singular triplet (Eckart-Young-Mirsky)."""
    A = W.gaussian_tensor((7, 5), 13).numpy()
    U, S, Vt = np.linalg.svd(A.astype(np.float64))
    res = oracle.hoscf(A, rand_unit((7, 5), 14), tol=1e-12, max_iter=10)
    assert res.converged and res.iters == 1
    assert abs(res.sigma - S[0]) < 1e-12 * S[0]
    assert abs(abs(res.u[0] @ U[:, 0]) - 1) < 1e-12
    assert abs(abs(res.u[1] @ Vt[0]) - 1) < 1e-12


# ------------------------------------------------------------- planted
@pytest.mark.parametrize("dims", [(6, 7, 8), (5, 4, 6, 3), (3, 4, 3, 2, 3)])
def test_planted_rank_one_exact_recovery(dims):
    f = [v / np.linalg.norm(v) for v in rand_unit(dims, 21)]      # unit in FP64
    T = 3.5 * W.outer([torch.from_numpy(v) for v in f]).numpy()  # exact rank one
    res = oracle.hoscf(T, rand_unit(dims, 22), tol=1e-13, max_iter=100)
    assert res.converged
    assert abs(res.sigma - 3.5) < 1e-12 * 3.5
    for n in range(len(dims)):
        assert abs(abs(res.u[n] @ f[n]) - 1) < 1e-12


def test_kkt_and_theorems_at_convergence():
    """KKT (2.4) from the tensor itself; Thm 3 (largest magnitude);
    Thm 1 (P2) equal block norms; Lemma 2 remark: sigma is the top singular
    value of every block, with singular vectors (u_m, u_n)."""
    dims = (9, 8, 7)
    T, _ = W.planted_cp(dims, [4.0], seed=31, noise_abs=1.0)
    T = T.numpy()
    res = oracle.hoscf(T, rand_unit(dims, 32), tol=1e-12, max_iter=500)
    assert res.converged
    g, full = oracle.kkt_vectors(T, res.u)
    assert abs(full - res.sigma) < 1e-10 * res.sigma
    for n in range(3):
        assert np.linalg.norm(g[n] - res.sigma * res.u[n]) < 1e-10 * res.sigma
    Hp = oracle.blocks(T, res.u)
    J = oracle.nepv_matrix(Hp, list(dims))
    w, V = np.linalg.eigh(J)
    k = np.argmax(np.abs(w))
    assert abs(w[k] - res.sigma) < 1e-10 * res.sigma
    norms = [np.linalg.norm(b) for b in oracle.split(V[:, k], dims)]
    np.testing.assert_allclose(norms, norms[0], rtol=1e-8)
    for (m, n), B in oracle.unpack_blocks(Hp, dims).items():
        U, S, Vt = np.linalg.svd(B)
        assert abs(S[0] - res.sigma) < 1e-10 * res.sigma
        assert abs(abs(U[:, 0] @ res.u[m]) - 1) < 1e-10
        assert abs(abs(Vt[0] @ res.u[n]) - 1) < 1e-10


def test_brute_force_2x2x2():
    """On 2x2x2 tensors the best of several HOSCF starts equals the maximum of
    |T(u1,u2,u3)| over a fine grid of unit vectors (cos t, sin t), refined."""
    from scipy.optimize import minimize
    th = np.linspace(0, np.pi, 181, endpoint=False)
    C = np.stack([np.cos(th), np.sin(th)], 1)
    for seed in range(3):
        T = W.gaussian_tensor((2, 2, 2), 40 + seed).numpy().astype(np.float64)
        F = np.abs(np.einsum("abc,ia,jb,kc->ijk", T, C, C, C))
        i, j, k = np.unravel_index(np.argmax(F), F.shape)

        def f(t):
            v = [np.array([np.cos(x), np.sin(x)]) for x in t]
            return -abs(np.einsum("abc,a,b,c->", T, *v))
        best = -minimize(f, [th[i], th[j], th[k]], method="Nelder-Mead",
                         options=dict(xatol=1e-12, fatol=1e-14, maxiter=4000)).fun
        sig = max(oracle.hoscf(T, rand_unit((2, 2, 2), s), tol=1e-13, max_iter=500).sigma
                  for s in range(8))
        assert abs(sig - best) < 1e-9 * best


def test_hopm_cross_check():
    dims = (8, 6, 7)
    T, _ = W.planted_cp(dims, [5.0, 1.0], seed=51, noise_abs=0.5)
    T = T.numpy()
    u0 = rand_unit(dims, 52)
    s1 = oracle.hoscf(T, u0, tol=1e-12, max_iter=500)
    s2, _ = oracle.hopm(T, u0, tol=1e-12)
    assert abs(s1.sigma - s2) < 1e-10 * s2


# ------------------------------------------------------------- Jacobi-HOPM
def test_jacobi_hopm_order2_is_power_iteration_to_top_singular_pair():
    """d = 2: the Jacobi update (u1 <- A u2, u2 <- A^T u1, both from the old
    pair, normalised) is a power iteration that converges to the top singular
    triplet (Eckart-Young-Mirsky)."""
    A = W.gaussian_tensor((30, 20), 15).numpy().astype(np.float64)
    U, S, Vt = np.linalg.svd(A)
    res = oracle.hoscf(A, rand_unit((30, 20), 16), tol=1e-11, max_iter=5000,
                       variant="jacobi_hopm")
    assert res.converged and res.iters > 1
    assert abs(res.sigma - S[0]) < 1e-10 * S[0]
    assert abs(abs(res.u[0] @ U[:, 0]) - 1) < 1e-10
    assert abs(abs(res.u[1] @ Vt[0]) - 1) < 1e-10


@pytest.mark.parametrize("dims", [(6, 7, 8), (5, 4, 6, 3)])
def test_jacobi_hopm_noiseless_rank_one_in_one_step(dims):
    """T = s a1 o ... o ad: A x_{k!=n} u^(k) = s prod_{k!=n} <a_k, u_k> a_n, so
    one Jacobi step lands on the planted factors exactly."""
    f = [v / np.linalg.norm(v) for v in rand_unit(dims, 23)]
    T = 2.5 * W.outer([torch.from_numpy(v) for v in f]).numpy()
    res = oracle.hoscf(T, rand_unit(dims, 24), tol=1e-13, max_iter=10, variant="jacobi_hopm")
    assert res.converged and res.iters == 1
    assert abs(res.sigma - 2.5) < 1e-12 * 2.5
    for n in range(len(dims)):
        assert abs(abs(res.u[n] @ f[n]) - 1) < 1e-12


def test_jacobi_hopm_reaches_the_gauss_seidel_hopm_point():
    dims = (8, 6, 7)
    T, _ = W.planted_cp(dims, [5.0, 1.0], seed=51, noise_abs=0.5)
    T = T.numpy()
    u0 = rand_unit(dims, 52)
    res = oracle.hoscf(T, u0, tol=1e-12, max_iter=2000, variant="jacobi_hopm")
    s2, u2 = oracle.hopm(T, u0, tol=1e-12)
    assert res.converged
    assert abs(res.sigma - s2) < 1e-10 * s2
    for a, b in zip(res.u, u2):
        assert abs(abs(a @ b) - 1) < 1e-9


# ------------------------------------------------------------- greedy rank-R
def test_greedy_order2_is_truncated_svd():
    """d = 2: each rank-one step takes the top singular triplet of the
    deflated matrix, so R steps give the R leading singular triplets
    (Eckart-Young-Mirsky) and ||A^(r)||_F^2 = sum_{i >= r} s_i^2."""
    A = W.gaussian_tensor((12, 9), 31).numpy().astype(np.float64)
    U, S, Vt = np.linalg.svd(A)
    g = oracle.greedy(A, 4, [rand_unit((12, 9), 40 + r) for r in range(4)], tol=1e-12)
    for r in range(4):
        assert abs(g.sigmas[r] - S[r]) < 1e-10 * S[0]
        assert abs(abs(g.factors[r][0] @ U[:, r]) - 1) < 1e-8
        assert abs(abs(g.factors[r][1] @ Vt[r]) - 1) < 1e-8
    nrm = np.linalg.norm(A)
    for r in range(5):
        assert abs(g.res[r] - np.sqrt(np.sum(S[r:] ** 2)) / nrm) < 1e-10


def test_greedy_orthogonal_cp_exact_recovery():
    """A sum of rank-one terms with mutually orthogonal factors in every mode
    and distinct weights: greedy recovers the terms in decreasing order and
    the residual vanishes after the last one."""
    dims, w = (6, 7, 5), [5.0, 3.0, 1.5]
    Q = [np.linalg.qr(np.random.default_rng(60 + n).standard_normal((m, 3)))[0] for n, m in enumerate(dims)]
    T = sum(wr * np.einsum("i,j,k->ijk", Q[0][:, r], Q[1][:, r], Q[2][:, r]) for r, wr in enumerate(w))
    g = oracle.greedy(T, 3, [rand_unit(dims, 70 + r) for r in range(3)], tol=1e-13)
    for r in range(3):
        assert abs(g.sigmas[r] - w[r]) < 1e-11 * w[0]
        for n in range(3):
            assert abs(abs(g.factors[r][n] @ Q[n][:, r]) - 1) < 1e-10
    assert g.res[3] < 1e-12


def test_greedy_residual_norm_identity():
    """At a KKT point <A, B> = sigma^2 = ||B||^2, so the deflation removes
    exactly sigma^2 of squared norm: ||A^(r+1)||^2 = ||A^(r)||^2 - sigma_r^2."""
    dims = (7, 6, 5, 4)
    T, _ = W.planted_cp(dims, [3.0, 2.0, 1.0], seed=81, noise_abs=0.3)
    T = T.numpy().astype(np.float64)
    g = oracle.greedy(T, 3, [rand_unit(dims, 90 + r) for r in range(3)], tol=1e-12)
    n0 = np.linalg.norm(T)
    for r in range(3):
        lhs = (g.res[r + 1] * n0) ** 2
        rhs = (g.res[r] * n0) ** 2 - g.sigmas[r] ** 2
        assert abs(lhs - rhs) < 1e-9 * n0 ** 2


def test_example2_device_generator_matches_the_pinned_formulas():
    """The on-device Example 2 generator (torch FP64) evaluates the same
    closed forms as the numpy one the Table 2 / 3 pins use (run here on the
    CPU through the same torch code)."""
    for name in ("EXP", "ARCSIN", "TAN"):
        a = W.example2(name).numpy()
        b = W._example2_torch(name, "cpu").numpy()
        assert a.shape == b.shape
        np.testing.assert_allclose(b, a, rtol=1e-6, atol=1e-6)


# ------------------------------------------------------------- Tables 1-3
@pytest.mark.parametrize("name", ["EXP", "ARCSIN"])
def test_example2_table2_rho_and_table3_iterations(name):
    ref = GOLD["table2_rho"][name]
    it_ref = GOLD["table3_iterations"][name]
    T = W.example2(name).numpy()
    nrm = np.linalg.norm(T.astype(np.float64))
    rho, its, its_i = [], [], []
    for s in range(6):
        u0 = [v.numpy() for v in W.uniform01_vectors(T.shape, s)]
        r = oracle.hoscf(T, u0, tol=1e-4, max_iter=500)
        ri = oracle.hoscf(T, u0, tol=1e-4, max_iter=500, variant="ihoscf")
        rho.append(r.sigma / nrm)
        its.append(r.iters)
        its_i.append(ri.iters)
        assert abs(ri.sigma - r.sigma) < 1e-4 * r.sigma
    assert abs(np.mean(rho) - ref["rho"]) <= ref["pm"] + 0.005     # two printed digits
    m, sd = it_ref["hoscf"]
    assert abs(np.mean(its) - m) <= 2 * sd
    assert np.mean(its_i) < np.mean(its)                            # iHOSCF needs fewer


def test_example1_table1_mean_lambda():
    """Loose statistical check of Table 1 (HOSCF column): Gaussian 10x10x10."""
    m, sd = GOLD["table1_lambda"]["3"]
    lam = []
    for s in range(12):
        T = W.gaussian_tensor((10, 10, 10), 600 + s).numpy()
        u0 = [v.numpy() for v in W.uniform01_vectors((10, 10, 10), 700 + s)]
        lam.append(oracle.hoscf(T, u0, tol=1e-4, max_iter=500).sigma)
    assert abs(np.mean(lam) - m) < 2 * sd


# ------------------------------------------------------------- final fix / gauge
def test_final_fix_and_gauge_keep_the_rank_one_term():
    dims = (4, 3, 5)
    u = rand_unit(dims, 61)
    s, uf = oracle.gauge(*oracle.final_fix(-2.0, u))
    assert s == 2.0
    for n in range(1, 3):
        assert uf[n][np.argmax(np.abs(uf[n]))] > 0
    a = -2.0 * W.outer([torch.from_numpy(v) for v in u]).numpy()
    b = s * W.outer([torch.from_numpy(v) for v in uf]).numpy()
    np.testing.assert_allclose(a, b, atol=1e-15)


# ------------------------------------------------------------- adjoint
@pytest.mark.parametrize("dims", [(5, 6, 7), (3, 4, 3, 4)])
def test_adjoint_matches_central_differences(dims):
    T, _ = W.planted_cp(dims, [3.0], seed=71, noise_abs=0.3)
    T = T.numpy().astype(np.float64)
    res = oracle.hoscf(T, rand_unit(dims, 72), tol=1e-14, max_iter=500)
    rng = np.random.default_rng(73)
    w = [rng.standard_normal(n) for n in dims]
    c = 0.7
    G, a, _ = oracle.adjoint(T, res.u, res.sigma, c, w)
    for n in range(len(dims)):
        assert abs(a[n] @ res.u[n]) < 1e-10
    D = rng.standard_normal(T.shape)

    def L(Tp):
        r = oracle.hoscf(Tp, res.u, tol=1e-14, max_iter=500)
        return c * r.sigma + sum(wn @ un for wn, un in zip(w, r.u))
    h = 1e-5
    fd = (L(T + h * D) - L(T - h * D)) / (2 * h)
    an = float(np.sum(G * D))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


# ------------------------------------------------------------- formats
def test_bf16_rounding_definition():
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 1 + 2 ** -8 + 2 ** -20,
                     3.0e38, 1e-40, 0.0, -0.0], dtype=np.float32)
    q = oracle.quantize_bf16(vals)
    assert [hex(v) for v in q[:5]] == ["0x3f80", "0x3f80", "0x3f82", "0xbf80", "0x3f81"]
    assert q[5] == 0x7F80 or q[5] == 0x7F62
    assert oracle.dequantize_bf16(q[7:9]).tolist() == [0.0, 0.0]
    x = W.gaussian_tensor((4096,), 81).numpy() * 37
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.quantize_bf16(x), ref)


def test_f16_rounding_definition():
    """IEEE binary16 round-to-nearest-even worked by hand (ties at 1 + 2^-11
    and 1 + 3 * 2^-11, the largest finite 65504, the overflow threshold
    65520, the smallest subnormal 2^-24 and the tie below it), then against
    numpy's and torch's own FP32 -> FP16 conversions on Gaussian values over
    many magnitudes."""
    vals = np.array([1.0, 1 + 2 ** -11, 1 + 3 * 2 ** -11, -(1 + 2 ** -11), 65504.0, 65519.0, 65520.0,
                     2.0 ** -24, 2.0 ** -25, 1.5 * 2.0 ** -25, 0.0, -0.0], dtype=np.float32)
    q = oracle.quantize_f16(vals)
    assert [hex(v) for v in q] == ["0x3c00", "0x3c00", "0x3c02", "0xbc00", "0x7bff", "0x7bff", "0x7c00",
                                   "0x1", "0x0", "0x1", "0x0", "0x8000"]
    assert oracle.dequantize_f16(q[7:8])[0] == 2.0 ** -24 and np.isinf(oracle.dequantize_f16(q[6:7])[0])
    rng = np.random.default_rng(82)
    x = (rng.standard_normal(8192) * 10.0 ** rng.integers(-8, 5, 8192)).astype(np.float32)
    assert np.array_equal(oracle.quantize_f16(x), x.astype(np.float16).view(np.uint16))
    ref = torch.from_numpy(x).to(torch.float16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.quantize_f16(x), ref)


def test_e4m3_definition():
    tab = oracle.e4m3_table()
    assert tab[0x7E] == 448.0 and tab[0x38] == 1.0 and tab[0x08] == 2.0 ** -6
    assert tab[0x01] == 2.0 ** -9 and np.isnan(tab[0x7F]) and tab[0xB8] == -1.0
    y = np.array([1.0625, 1.1875, 500.0, -1000.0, 2.0 ** -10, 3 * 2.0 ** -10, 0.0, 17.0])
    codes = oracle._e4m3_round(y)
    # 1.0625 ties between 1.0 (0x38) and 1.125 (0x39) -> even 0x38; 1.1875 -> 0x3A
    assert codes.tolist() == [0x38, 0x3A, 0x7E, 0xFE, 0x00, 0x02, 0x00, 0x58]
    x = W.gaussian_tensor((8192,), 82).numpy() * 3
    codes = oracle._e4m3_round(x.astype(np.float64))
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(codes, ref)


def test_e4m3_scaled_roundtrip_error_bound():
    x = W.gaussian_tensor((1000,), 83).numpy()
    codes, scales = oracle.quantize_e4m3_scaled(x)
    assert scales.shape == (8,)
    xq = oracle.dequantize_e4m3_scaled(codes, scales)
    amax = np.repeat(scales * 448.0, 128)[:1000]
    # e4m3 keeps 3 mantissa bits: relative error <= 2^-4 for normals, and the
    # subnormal spacing 2^-9 * scale bounds the rest
    err = np.abs(xq - x)
    assert np.all(err <= np.maximum(np.abs(x) * 2.0 ** -4, 2.0 ** -10 * amax / 448.0 * 1.0001))


# ------------------------------------------------------------- RQI step (Sec. 4.4)
def _rqi_spectral(Q, lam, x):
    """One Rayleigh-quotient step written in the eigenbasis of J = Q diag(lam) Q^T:
    rho = sum_j lam_j c_j^2 / sum_j c_j^2 and y ~ sum_j c_j / (lam_j - rho) q_j,
    c = Q^T x; unit length, <y, x> >= 0."""
    c = Q.T @ x
    rho = float(np.sum(lam * c * c) / np.sum(c * c))
    y = Q @ (c / (lam - rho))
    y /= np.linalg.norm(y)
    return (y if y @ x >= 0 else -y), rho


def test_rqi_step_matches_the_spectral_form():
    """oracle.rqi_step on one block (d = 1: x~ = u, plain RQI) against the step
    written in a known eigenbasis."""
    rng = np.random.default_rng(5)
    n = 7
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.array([4.0, 2.5, 1.0, -0.5, -1.5, -3.0, 0.25])
    J = (Q * lam) @ Q.T
    u = rng.standard_normal(n)
    u /= np.linalg.norm(u)
    y_ref, rho_ref = _rqi_spectral(Q, lam, u)
    assert np.min(np.abs(lam - rho_ref)) > 0.05       # a well-posed shift
    (y,), rho = oracle.rqi_step(J, [u], [n])
    assert abs(rho - rho_ref) <= 1e-13
    assert np.max(np.abs(y - y_ref)) <= 1e-11


def test_rqi_step_order2_block_form():
    """d = 2, A = diag(s1, s2): J = [[0, A], [A, 0]] has eigenpairs +-s_i,
    (e_i, +-e_i)/sqrt(2); the step from x~ = [u1; u2]/sqrt(2) is the spectral
    form, then each block is normalised (Alg. 1 lines 6-9)."""
    s1, s2 = 3.0, 1.0
    A = np.diag([s1, s2])
    Hp = A.ravel()
    J = oracle.nepv_matrix(Hp, [2, 2])
    a, b = 0.3, -0.8
    u1, u2 = np.array([np.cos(a), np.sin(a)]), np.array([np.cos(b), np.sin(b)])
    r2 = 1 / np.sqrt(2)
    Q = np.array([[r2, 0, r2, 0], [0, r2, 0, r2], [r2, 0, -r2, 0], [0, r2, 0, -r2]])
    lam = np.array([s1, s2, -s1, -s2])
    xt = np.concatenate([u1, u2]) * r2
    y_ref, rho_ref = _rqi_spectral(Q, lam, xt)
    assert abs(rho_ref - (s1 * u1[0] * u2[0] + s2 * u1[1] * u2[1])) <= 1e-14
    (v1, v2), rho = oracle.rqi_step(J, [u1, u2], [2, 2])
    assert abs(rho - rho_ref) <= 1e-14
    assert np.max(np.abs(v1 - y_ref[:2] / np.linalg.norm(y_ref[:2]))) <= 1e-12
    assert np.max(np.abs(v2 - y_ref[2:] / np.linalg.norm(y_ref[2:]))) <= 1e-12


def test_rqi_step_converges_cubically():
    """Near an eigenvector at angle eps, one RQI step leaves an angle O(eps^3)
    (symmetric J): a tenfold smaller eps gives a ~1000-fold smaller angle."""
    rng = np.random.default_rng(6)
    n = 9
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(-2.0, 5.0, n)
    J = (Q * lam) @ Q.T
    w = rng.standard_normal(n)
    w -= (w @ Q[:, -1]) * Q[:, -1]
    w /= np.linalg.norm(w)
    ang = []
    q = Q[:, -1]
    for eps in (3e-2, 3e-3):
        u = q + eps * w
        u /= np.linalg.norm(u)
        (y,), _ = oracle.rqi_step(J, [u], [n])
        ang.append(np.linalg.norm(y - (y @ q) * q))   # sine of the angle to q
    assert ang[0] <= 3e-4 and 3e-4 <= ang[1] / ang[0] <= 3e-3


def test_ihoscf_rejects_an_rqi_step_that_lowers_sigma(monkeypatch):
    """Acceptance rule of iHOSCF (Sec. 4.4 reading): a y with a smaller
    |sigma| that its pass does not certify is rejected, so the loop keeps the
    eigen-step iterates x_k - exactly plain HOSCF's sequence - with one extra
    pass per iteration and no acceptances."""
    dims = (6, 5, 4)
    T, _ = W.planted_cp(dims, [3.0], seed=41, noise_abs=0.3)
    T = T.numpy().astype(np.float64)
    u0 = rand_unit(dims, 42)
    bad = rand_unit(dims, 43)
    monkeypatch.setattr(oracle, "rqi_step", lambda J, u, d: ([v.copy() for v in bad], 0.0))
    assert abs(oracle.kkt_vectors(T, bad)[1]) < 0.5 * 3.0     # bad lowers sigma
    ref = oracle.hoscf(T, u0, tol=1e-10, max_iter=100, variant="hoscf")
    r = oracle.hoscf(T, u0, tol=1e-10, max_iter=100, variant="ihoscf")
    assert r.rqi_accepts == 0
    assert r.iters == ref.iters and abs(r.sigma - ref.sigma) <= 1e-14 * abs(ref.sigma)
    for a, b in zip(r.u, ref.u):
        assert np.max(np.abs(a - b)) <= 1e-12
    # per iteration: the pass of x_k, then the rejected pass of y (the last
    # iteration's x_k certifies and takes no RQI step)
    assert r.passes == 1 + 2 * r.iters - 1


def test_ihoscf_accepts_an_rqi_step_its_pass_certifies(monkeypatch):
    """Acceptance rule, other branch: a y whose pass certifies convergence is
    kept at once.  The step is made to return the maximiser found beforehand
    by plain HOSCF to 1e-13, from a start where plain HOSCF needs several
    iterations to reach 1e-8."""
    dims = (6, 5, 4)
    T, _ = W.planted_cp(dims, [3.0], seed=41, noise_abs=0.3)
    T = T.numpy().astype(np.float64)
    u0 = rand_unit(dims, 42)
    best = oracle.hoscf(T, u0, tol=1e-13, max_iter=500, variant="hoscf")
    plain = oracle.hoscf(T, u0, tol=1e-8, max_iter=500, variant="hoscf")
    assert best.converged and plain.iters >= 3
    monkeypatch.setattr(oracle, "rqi_step", lambda J, u, d: ([v.copy() for v in best.u], 0.0))
    r = oracle.hoscf(T, u0, tol=1e-8, max_iter=500, variant="ihoscf")
    assert r.converged and r.rqi_accepts == 1 and r.iters == 1
    assert abs(r.sigma - best.sigma) <= 1e-12 * abs(best.sigma)
    # the |sigma| branch: an uncertified y with a larger |sigma| than x_1 is
    # kept too (passes: x_0, x_1, then y)
    rng = np.random.default_rng(46)
    near = [v + 1e-3 * rng.standard_normal(v.size) for v in best.u]
    near = [v / np.linalg.norm(v) for v in near]
    monkeypatch.setattr(oracle, "rqi_step", lambda J, u, d: ([v.copy() for v in near], 0.0))
    r = oracle.hoscf(T, u0, tol=1e-8, max_iter=500, variant="ihoscf")
    (s1, r1), (sy, ry) = r.history[1], r.history[2]
    assert ry > 1e-8 and abs(sy) >= abs(s1) and r1 > 1e-8
    assert r.rqi_accepts >= 1 and r.converged


# ------------------------------------------------------------- planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """A dropped 1/(d-1), a transposed block and a wrong gauge sign each break
    one of the pins above."""
    dims = (6, 5, 4)
    T, _ = W.planted_cp(dims, [2.0], seed=91)
    T = T.numpy().astype(np.float64)
    u0 = rand_unit(dims, 92)
    good = oracle.nepv_matrix
    monkeypatch.setattr(oracle, "nepv_matrix", lambda Hp, d: good(Hp, d) * (len(d) - 1))
    r = oracle.hoscf(T, u0, tol=1e-12, max_iter=50)
    lam = oracle.largest_magnitude_eigpair(oracle.nepv_matrix(oracle.blocks(T, r.u), dims))[0]
    assert abs(lam - r.sigma) > 0.5            # Thm 3 check would fail
    monkeypatch.setattr(oracle, "nepv_matrix", good)

    A = W.gaussian_tensor((5, 5), 93).numpy().astype(np.float64)
    U, S, Vt = np.linalg.svd(A)
    gfull = oracle.full_block_matrix
    monkeypatch.setattr(oracle, "full_block_matrix",
                        lambda Hp, d: gfull(Hp.reshape(5, 5).T.ravel(), d))
    r = oracle.hoscf(A, rand_unit((5, 5), 94), tol=1e-12, max_iter=5)
    assert abs(abs(r.u[0] @ U[:, 0]) - 1) > 1e-3   # SVD pin would fail
    monkeypatch.setattr(oracle, "full_block_matrix", gfull)

    s, uf = oracle.final_fix(-1.0, rand_unit(dims, 95))
    assert s > 0 and abs(uf[0][0]) > 0


# ------------------------------------------------------------- eq. (4.1)
@pytest.mark.parametrize("t", [0.0, 0.3, 1.1, np.pi / 2, 2.5])
def test_residual_4_1_order2_closed_form(t):
    """Eq. (4.1) worked by hand for d = 2, A = diag(3, 1), u = e1,
    v = (cos t, sin t): x = [u; v]/sqrt(2), J = [[0, A], [A^T, 0]],
    rho = x^T J x = 3 cos t, ||J x - rho x|| = sqrt(5) |sin t| and
    ||J||_F = 2 sqrt(5), so the residual is
    sqrt(5) |sin t| / (2 sqrt(5) + 3 |cos t|)."""
    Hp = np.array([3.0, 0.0, 0.0, 1.0])
    u = [np.array([1.0, 0.0]), np.array([np.cos(t), np.sin(t)])]
    want = np.sqrt(5.0) * abs(np.sin(t)) / (2.0 * np.sqrt(5.0) + 3.0 * abs(np.cos(t)))
    assert abs(oracle.residual_4_1(Hp, [2, 2], u) - want) <= 1e-15


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 3, 5, 2), (3, 2, 4, 2, 3)])
def test_residual_4_1_against_the_kkt_vectors(dims):
    """For the balanced x = [u]/sqrt(d), (J x)_n = g_n / sqrt(d) with
    g_n = A x_{k!=n} u^(k) and rho = A(u^(1), ..., u^(d)) (eq. 3.2-3.3), so
    eq. (4.1) equals ||g - rho u|| / (sqrt(d) (||J||_F + |rho|)) with
    ||J||_F^2 = 2 sum_{m<n} ||A_{m,n}||_F^2 / (d-1)^2.  g and rho come from
    the direct contraction of the tensor (not from the blocks)."""
    d = len(dims)
    T = W.gaussian_tensor(dims, 71).numpy().astype(np.float64)
    u = rand_unit(dims, 72)
    g, rho = oracle.kkt_vectors(T, u)
    Hp = oracle.blocks(T, u)
    jf = np.sqrt(2.0 * sum(float(np.sum(B * B)) for B in oracle.unpack_blocks(Hp, list(dims)).values())) / (d - 1)
    num = np.linalg.norm(np.concatenate(g) - rho * np.concatenate(u)) / np.sqrt(d)
    want = num / (jf + abs(rho))
    got = oracle.residual_4_1(Hp, list(dims), u)
    assert abs(got - want) <= 1e-12 * want
    # invariant under scaling of the tensor and under sign flips of factor pairs
    assert abs(oracle.residual_4_1(oracle.blocks(7.0 * T, u), list(dims), u) - got) <= 1e-12 * got
    uf = [-u[0]] + [-u[1]] + u[2:]
    assert abs(oracle.residual_4_1(oracle.blocks(T, uf), list(dims), uf) - got) <= 1e-12 * got


def test_residual_4_1_vanishes_at_a_singular_pair():
    """At the factors of an exact rank-one tensor x is an eigenvector of
    J(x) (Thm 2), so eq. (4.1) is zero to rounding."""
    dims = (6, 5, 4, 3)
    f = [v / np.linalg.norm(v) for v in rand_unit(dims, 73)]
    T = 2.5 * W.outer([torch.from_numpy(v) for v in f]).numpy()
    assert oracle.residual_4_1(oracle.blocks(T, f), list(dims), f) <= 1e-15
    r = oracle.hoscf(T, rand_unit(dims, 74), tol=1e-13, max_iter=50)
    assert r.resid_4_1 <= 1e-14


# ------------------------------------------------------------- Alg. 1 line 5, ARPACK branch
@pytest.mark.parametrize("lo,hi", [(-5.0, 4.0), (-4.0, 5.0), (-3.0, 3.0)])
def test_largest_magnitude_arpack_branch_matches_eigh(lo, hi):
    """The branch for large matrices (ARPACK on both spectrum ends) against a
    matrix of known spectrum Q diag(w) Q^T: the largest-|w| end is chosen
    and the eigenvector is the matching column of Q, sign-aligned with
    x_prev.  On a tie (w = -3 and 3) the computed ends differ only by
    rounding and either may win (both give the same rank-one term after
    Alg. 1 lines 12-15); the vector must belong to the end chosen."""
    n = 300
    rng = np.random.default_rng(75)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    w = np.concatenate([[lo, hi], rng.uniform(-0.9 * min(-lo, hi), 0.9 * min(-lo, hi), n - 2)])
    J = (Q * w) @ Q.T
    J = 0.5 * (J + J.T)
    x_prev = rng.standard_normal(n)
    lam, x = oracle.largest_magnitude_eigpair(J, x_prev, dense_max=0)
    k = 1 if hi > -lo else 0 if hi < -lo else (1 if lam > 0 else 0)
    assert abs(lam - w[k]) <= 1e-10 * abs(w[k])
    q = Q[:, k] if Q[:, k] @ x_prev >= 0 else -Q[:, k]
    assert np.linalg.norm(x - q) <= 1e-8
    if hi != -lo:
        lam_d, x_d = oracle.largest_magnitude_eigpair(J, x_prev)
        assert abs(lam - lam_d) <= 1e-10 * abs(lam_d) and np.linalg.norm(x - x_d) <= 1e-8


# ------------------------------------------------------------- ASVD (Sec. 1)
def test_asvd_order2_is_one_svd():
    """d = 2: the intermediate matrix is A itself, so one sub-step gives the
    top singular triplet and the next pass certifies it."""
    A = W.gaussian_tensor((9, 6), 81).numpy()
    U, S, Vt = np.linalg.svd(A.astype(np.float64))
    r = oracle.asvd(A, rand_unit((9, 6), 82), tol=1e-12, max_iter=10)
    assert r.converged and r.iters == 1 and r.passes == 2
    assert abs(r.sigma - S[0]) <= 1e-12 * S[0]
    assert abs(abs(r.u[0] @ U[:, 0]) - 1) <= 1e-12 and abs(abs(r.u[1] @ Vt[0]) - 1) <= 1e-12


def test_asvd_noiseless_rank_one_in_two_sub_steps():
    """T = s a1 o a2 o a3: the first block A x_1 u1 = s <a1,u1> a2 a3^T gives
    (a2, a3) exactly; the second, A x_2 a2 = s a1 a3^T, gives a1: the third
    pass certifies the exact solution."""
    dims = (7, 5, 6)
    f = [v / np.linalg.norm(v) for v in rand_unit(dims, 83)]
    T = 2.0 * W.outer([torch.from_numpy(v) for v in f]).numpy()
    r = oracle.asvd(T, rand_unit(dims, 84), tol=1e-13, max_iter=20)
    assert r.converged and r.iters == 2 and r.passes == 3
    assert abs(r.sigma - 2.0) <= 1e-13 * 2.0
    for n in range(3):
        assert abs(abs(r.u[n] @ f[n]) - 1) <= 1e-13


@pytest.mark.parametrize("seed", [85, 86, 87])
def test_asvd_is_monotone_and_reaches_the_hopm_point(seed):
    """Each sub-step maximises |A(u1, u2, u3)| over the two free factors, so
    |sigma| never decreases along the iterates (a wrong pair, block or
    transpose breaks this); on a planted case ASVD, HOPM and HOSCF reach the
    same maximum."""
    dims = (8, 9, 7)
    T, _ = W.planted_cp(dims, [4.0, 1.5], seed=seed, noise_abs=0.8)
    T = T.numpy().astype(np.float64)
    u0 = rand_unit(dims, seed + 10)
    r = oracle.asvd(T, u0, tol=1e-12, max_iter=500)
    assert r.converged
    s = [abs(h[0]) for h in r.history]
    assert all(b >= a - 1e-12 * b for a, b in zip(s, s[1:]))
    s_hopm, _ = oracle.hopm(T, u0, tol=1e-12)
    s_hoscf = oracle.hoscf(T, u0, tol=1e-12, max_iter=500).sigma
    assert abs(r.sigma - s_hopm) <= 1e-10 * s_hopm
    assert abs(r.sigma - s_hoscf) <= 1e-10 * s_hoscf


def test_asvd_brute_force_2x2x2():
    """On 2x2x2 tensors the best of several ASVD starts equals the maximum of
    |T(u1,u2,u3)| over unit vectors (grid + local refinement)."""
    from scipy.optimize import minimize
    th = np.linspace(0, np.pi, 181, endpoint=False)
    C = np.stack([np.cos(th), np.sin(th)], 1)
    for seed in range(3):
        T = W.gaussian_tensor((2, 2, 2), 60 + seed).numpy().astype(np.float64)
        F = np.abs(np.einsum("abc,ia,jb,kc->ijk", T, C, C, C))
        i, j, k = np.unravel_index(np.argmax(F), F.shape)

        def f(t):
            v = [np.array([np.cos(x), np.sin(x)]) for x in t]
            return -abs(np.einsum("abc,a,b,c->", T, *v))
        best = -minimize(f, [th[i], th[j], th[k]], method="Nelder-Mead",
                         options=dict(xatol=1e-12, fatol=1e-14, maxiter=4000)).fun
        sig = max(oracle.asvd(T, rand_unit((2, 2, 2), s), tol=1e-13, max_iter=500).sigma
                  for s in range(8))
        assert abs(sig - best) < 1e-9 * best


def test_asvd_rejects_other_orders():
    with pytest.raises(ValueError):
        oracle.asvd(np.ones((2, 2, 2, 2)), rand_unit((2, 2, 2, 2), 1))
