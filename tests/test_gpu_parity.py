"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Floating-point tolerances follow from FP32 accumulation:
an entry that sums M terms is compared with an error bound of
c * eps32 * sqrt(M) * S, where S is the same entry computed from |T| and |u|."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from helpers import assert_same_solution, check_gauge

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01778_gb300 import build
    build.build()


def P():
    import paper_2403_01778_gb300 as pkg
    return pkg


def to_gpu(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def blocks_gpu(T, u_list, dtype=torch.float32):
    Tg = to_gpu(T).to(dtype)
    ug = to_gpu(np.concatenate(u_list).astype(np.float32))
    H = P().hoscf_ttvc_blocks(Tg, ug)
    torch.cuda.synchronize()
    return H.double().cpu().numpy()


def bound(T, u_list, c=8.0):
    """Per-entry error bound for FP32 block sums (see module docstring)."""
    dims = T.shape
    S = oracle.blocks(np.abs(T).astype(np.float64), [np.abs(v) for v in u_list])
    Ms = []
    for (m, n) in oracle.block_pairs(len(dims)):
        Ms.append(np.full(dims[m] * dims[n], np.prod(dims) / (dims[m] * dims[n])))
    M = np.concatenate(Ms)
    return c * EPS32 * np.sqrt(M + 1.0) * S + 1e-30


SHAPES = [
    (7, 5),                  # d = 2: the block is the matrix
    (64, 64, 64),            # aligned, one face tile
    (37, 50, 129),           # ragged, unaligned rows (plain loads)
    (3, 130, 260),           # several face tiles in both directions
    (200, 70, 68),           # more CTAs than outer indices per tile
    (9, 10, 11, 12),         # d = 4
    (5, 4, 3, 6, 8),         # d = 5
    (3, 2, 4, 3, 2, 5),      # d = 6
    (1, 1, 5),               # unit dims
    (5, 6, 40, 36),          # d = 4, tiled path (face 1440) with outer folds
    (7, 9, 11, 13, 5),       # small-face path, d = 5
    (2, 3, 2, 3, 2, 3, 2, 3),  # d = 8
    (4, 5, 3, 7, 2, 9, 2),   # d = 7, ragged
    (33, 1, 17, 32),         # a unit mode among outer ones
    (3, 200, 200),           # 13 rows per warp (tiles of 104 rows)
    (4, 96, 36),             # vector loads without TMA (36 floats = 144 B rows)
]


@pytest.mark.parametrize("dims", SHAPES)
def test_blocks_integer_exact(dims):
    """Integer-valued tensor and factors: every FP32 partial sum is exact, so
    the blocks must match the oracle bit for bit (index/layout check)."""
    rng = np.random.default_rng(sum(dims))
    T = rng.integers(-3, 4, size=dims).astype(np.float32)
    u = [rng.integers(-2, 3, size=n).astype(np.float64) for n in dims]
    Hg = blocks_gpu(T, u)
    Hr = oracle.blocks(T, u)
    assert np.array_equal(Hg, Hr)


@pytest.mark.parametrize("dims", SHAPES + [(96, 96, 96), (40, 41, 42, 43)])
def test_blocks_gaussian_within_fp32_bound(dims):
    T = W.gaussian_tensor(dims, 3).numpy()
    u = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 4)]
    Hg = blocks_gpu(T, u)
    Hr = oracle.blocks(T, u)
    assert np.all(np.abs(Hg - Hr) <= bound(T, u))


def test_blocks_bf16_match_dequantised_oracle():
    dims = (33, 64, 128)
    T = W.gaussian_tensor(dims, 5).numpy()
    q = oracle.quantize_bf16(T)
    Tq = oracle.dequantize_bf16(q).reshape(dims)           # exact bf16 values, FP64
    u = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 6)]
    Tg = torch.from_numpy(q.view(np.int16)).cuda().view(torch.bfloat16).reshape(dims)
    ug = to_gpu(np.concatenate(u).astype(np.float32))
    Hg = P().hoscf_ttvc_blocks(Tg, ug).double().cpu().numpy()
    Hr = oracle.blocks(Tq, u)
    assert np.all(np.abs(Hg - Hr) <= bound(Tq, u))


@pytest.mark.parametrize("dims,nsample", [((24, 20, 24, 20, 24, 20), 40), ((8,) * 8, 40),
                                           ((32, 32, 32, 32, 16), 24)])
def test_blocks_full_size_sampled_entries(dims, nsample):
    """Paper-scale small-face shapes: sampled entries of every block against the
    oracle's one-entry definition (eq. 3.3)."""
    T = W.planted_cp(dims, [1.0], seed=61, noise_abs=0.05)[0]
    u = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 62)]
    Hg = P().hoscf_ttvc_blocks(T.cuda(), to_gpu(np.concatenate(u).astype(np.float32)))
    Hg = Hg.double().cpu().numpy()
    Tn = T.numpy()
    Ta = np.abs(Tn)
    ua = [np.abs(v) for v in u]
    rng = np.random.default_rng(63)
    offs, _ = oracle.block_offsets(list(dims))
    M = np.prod(dims)
    for (m, n), o in zip(oracle.block_pairs(len(dims)), offs):
        for _ in range(max(1, nsample // len(offs))):
            i, j = int(rng.integers(dims[m])), int(rng.integers(dims[n]))
            ref = oracle.block_entry(Tn, u, m, n, i, j)
            sc = oracle.block_entry(Ta, ua, m, n, i, j)
            tol = 8 * EPS32 * math.sqrt(M / (dims[m] * dims[n]) + 1) * sc + 1e-30
            assert abs(Hg[o + i * dims[n] + j] - ref) <= tol, ((m, n), i, j)


def test_eig_step_matches_dense_eigh():
    dims = (20, 30, 25)
    T, _ = W.planted_cp(dims, [3.0], seed=7, noise_abs=1.0)
    T = T.numpy()
    u = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 8)]
    Hr = oracle.blocks(T, u)
    J = oracle.nepv_matrix(Hr, list(dims))
    x_prev = np.concatenate(u) / math.sqrt(3)
    lam, x = oracle.largest_magnitude_eigpair(J, x_prev)
    Hg = to_gpu(Hr.astype(np.float32))
    xg, ug, lg = P().hoscf_eig_step(dims, Hg, to_gpu(x_prev), eig_adapt=0.0)
    torch.cuda.synchronize()
    assert abs(lg.item() - lam) <= 1e-5 * abs(lam)
    # both sides align the eigenvector with x_prev, so x is compared with its sign
    assert abs(float(xg.cpu().numpy() @ x) - 1) <= 1e-6
    assert float(xg.cpu().numpy() @ x_prev) >= 0
    for n, un in enumerate(oracle.normalise_blocks(x, list(dims))):
        o = int(sum(dims[:n]))
        assert abs(float(ug.double().cpu().numpy()[o:o + dims[n]] @ un) - 1) <= 1e-5


@pytest.mark.parametrize("dims", [(512, 512, 1024), (200, 200, 200, 200)])
def test_eig_step_many_ctas_matches_dense_eigh(dims):
    """Eigen step (Alg. 1 line 5) with J spread over many CTAs: cached row
    blocks, grid barriers, cross-CTA sums, and on the first shape (rows of
    1024+ floats) the 16-byte mat-vec loads.  Blocks sigma u_m u_n^T plus
    noise, a random start, against LAPACK's dense eigh of the same J."""
    rng = np.random.default_rng(91)
    d = len(dims)
    u = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 92)]
    Hr = np.concatenate([(5.0 * np.outer(u[m], u[n]) +
                          0.01 * rng.standard_normal((dims[m], dims[n]))).ravel()
                         for m, n in oracle.block_pairs(d)]).astype(np.float32)
    J = oracle.nepv_matrix(Hr.astype(np.float64), list(dims))
    x_prev = np.concatenate([v.numpy().astype(np.float64)
                             for v in W.unit_gaussian_vectors(dims, 93)]) / math.sqrt(d)
    lam, x = oracle.largest_magnitude_eigpair(J, x_prev)
    xg, ug, lg = P().hoscf_eig_step(dims, to_gpu(Hr), to_gpu(x_prev), eig_adapt=0.0)
    torch.cuda.synchronize()
    assert abs(lg.item() - lam) <= 1e-5 * abs(lam)
    assert abs(float(xg.cpu().numpy() @ x) - 1) <= 1e-5
    assert float(xg.cpu().numpy() @ x_prev) >= 0


def test_rqi_step_matches_oracle_near_a_maximum():
    """iHOSCF's RQI step (Sec. 4.4) from a point near the maximum: the shift
    rho and the normalised blocks of y = (J - rho I)^-1 x~ against the
    oracle's dense solve on the same FP32 blocks and factors."""
    dims = (20, 30, 25)
    T, _ = W.planted_cp(dims, [3.0], seed=17, noise_abs=0.5)
    T = T.numpy().astype(np.float64)
    u0 = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 18)]
    near = oracle.hoscf(T, u0, tol=1e-2, max_iter=50)
    uk = [v.astype(np.float32).astype(np.float64) for v in near.u]
    Hr = oracle.blocks(T, uk).astype(np.float32)
    J = oracle.nepv_matrix(Hr.astype(np.float64), list(dims))
    v_ref, rho_ref = oracle.rqi_step(J, uk, list(dims))
    xg, ug, rg = P().hoscf_rqi_step(dims, to_gpu(Hr), to_gpu(np.concatenate(uk).astype(np.float32)))
    torch.cuda.synchronize()
    assert abs(rg.item() - rho_ref) <= 1e-6 * abs(rho_ref)
    ugn = ug.double().cpu().numpy()
    o = 0
    for n, vr in zip(dims, v_ref):
        assert float(ugn[o:o + n] @ vr) >= 1 - 1e-5
        o += n


def test_rqi_step_many_ctas_matches_oracle():
    """The RQI step with J spread over many CTAs (512x512x1024 blocks
    sigma a_m a_n^T plus noise, a start near the top eigenvector)."""
    dims = (512, 512, 1024)
    rng = np.random.default_rng(95)
    d = len(dims)
    a = [v.numpy().astype(np.float64) for v in W.unit_gaussian_vectors(dims, 96)]
    Hr = np.concatenate([(5.0 * np.outer(a[m], a[n]) +
                          0.01 * rng.standard_normal((dims[m], dims[n]))).ravel()
                         for m, n in oracle.block_pairs(d)]).astype(np.float32)
    J = oracle.nepv_matrix(Hr.astype(np.float64), list(dims))
    uk = []
    for v in a:
        w = v + 0.05 * rng.standard_normal(v.shape) / np.sqrt(v.size)
        uk.append((w / np.linalg.norm(w)).astype(np.float32).astype(np.float64))
    v_ref, rho_ref = oracle.rqi_step(J, uk, list(dims))
    xg, ug, rg = P().hoscf_rqi_step(dims, to_gpu(Hr), to_gpu(np.concatenate(uk).astype(np.float32)))
    torch.cuda.synchronize()
    assert abs(rg.item() - rho_ref) <= 1e-6 * abs(rho_ref)
    ugn = ug.double().cpu().numpy()
    o = 0
    for n, vr in zip(dims, v_ref):
        assert float(ugn[o:o + n] @ vr) >= 1 - 1e-5
        o += n


def compare_solution(res, ref, tol=1e-5):
    """sigma and the factors with their signs (final fix + gauge on both sides)."""
    assert_same_solution(res.sigma, res.factors(), ref.sigma, ref.u, tol)


def test_solve_order2_is_svd():
    A = W.gaussian_tensor((40, 30), 11).numpy()
    U, S, Vt = np.linalg.svd(A.astype(np.float64))
    u0 = torch.cat(W.unit_gaussian_vectors((40, 30), 12)).cuda()
    r = P().hoscf_solve(to_gpu(A), u0, tol=1e-6, max_iter=20)
    assert r.converged
    # the top singular pair with the gauge applied: u2's largest-|.| entry positive
    a, b = U[:, 0].copy(), Vt[0].copy()
    if b[int(np.argmax(np.abs(b)))] < 0:
        a, b = -a, -b
    assert_same_solution(r.sigma, r.factors(), S[0], [a, b])


def test_solve_64cube_matches_oracle():
    """T = 10 u1 o u2 o u3 + E, ||E||_F = 1, 64^3; tol 1e-8 (FP32 stops at its floor
    or 200 iterations); compared on sigma and factors."""
    T = W.config_tensor("cfg1_64cube", seed=0)
    u0 = W.unit_gaussian_vectors(T.shape, 1)
    ref = oracle.hoscf(T.numpy(), [v.numpy() for v in u0], tol=1e-8, max_iter=200)
    assert ref.converged
    r = P().hoscf_solve(T.cuda(), torch.cat(u0).cuda(), tol=1e-8, max_iter=200)
    compare_solution(r, ref)
    assert r.resid < 1e-5


@pytest.mark.parametrize("dims,seed", [((9, 10, 11, 12), 21), ((5, 6, 7, 5, 6), 22),
                                        ((3, 4, 3, 4, 3, 4), 23), ((130, 70, 260), 24)])
def test_solve_planted_matches_oracle(dims, seed):
    T, _ = W.planted_cp(dims, [5.0], seed=seed, noise_abs=0.5)
    u0 = W.unit_gaussian_vectors(dims, seed + 100)
    ref = oracle.hoscf(T.numpy(), [v.numpy() for v in u0], tol=1e-10, max_iter=300)
    r = P().hoscf_solve(T.cuda(), torch.cat(u0).cuda(), tol=1e-6, max_iter=300)
    assert r.converged
    compare_solution(r, ref)


@pytest.mark.parametrize("variant", ["ihoscf", "ihoscf_prev"])
@pytest.mark.parametrize("name", ["EXP", "ARCSIN"])
def test_ihoscf_matches_oracle_on_example2(name, variant):
    """Both iHOSCF readings reach the oracle's (and plain HOSCF's) solution on
    the paper's Example 2 tensors; the default reading needs fewer eigen steps
    than HOSCF (Table 3's direction)."""
    T = W.example2(name)
    u0 = W.uniform01_vectors(T.shape, 3)
    ref = oracle.hoscf(T.numpy(), [v.numpy() for v in u0], tol=1e-8, max_iter=500,
                       variant=variant)
    r = P().hoscf_solve(T.cuda(), torch.cat(u0).cuda(), tol=1e-6, max_iter=500, variant=variant)
    h = P().hoscf_solve(T.cuda(), torch.cat(u0).cuda(), tol=1e-6, max_iter=500)
    assert r.converged and h.converged
    compare_solution(r, ref)
    if variant == "ihoscf":
        assert r.iters < h.iters
        assert r.passes <= 2 * r.iters + 1


@pytest.mark.parametrize("dims,seed", [((20, 30, 25), 41), ((8, 9, 10, 11), 42), ((30, 20), 43)])
def test_jacobi_hopm_matches_oracle(dims, seed):
    """The paper's Jacobi-HOPM comparison method (every factor at once from
    the same blocks) reaches the oracle's Jacobi-HOPM point; HOSCF needs no
    more iterations (Table 1's direction)."""
    T, _ = W.planted_cp(dims, [4.0, 1.0], seed=seed, noise_abs=0.3)
    u0 = W.unit_gaussian_vectors(dims, seed + 1)
    ref = oracle.hoscf(T.numpy(), [v.numpy() for v in u0], tol=1e-9, max_iter=5000,
                       variant="jacobi_hopm")
    assert ref.converged
    r = P().hoscf_solve(T.cuda(), torch.cat(u0).cuda(), tol=1e-6, max_iter=5000,
                        variant="jacobi_hopm")
    assert r.converged
    compare_solution(r, ref)
    h = P().hoscf_solve(T.cuda(), torch.cat(u0).cuda(), tol=1e-6, max_iter=5000)
    assert h.iters <= r.iters


def test_solve_reports_kkt_consistent_with_oracle():
    """The residual and sigma the GPU certifies at its returned point agree
    with the oracle's direct KKT vectors at that same point."""
    dims = (30, 40, 50)
    T, _ = W.planted_cp(dims, [2.0, 1.0], seed=31, noise_abs=0.3)
    u0 = torch.cat(W.unit_gaussian_vectors(dims, 32)).cuda()
    r = P().hoscf_solve(T.cuda(), u0, tol=1e-6, max_iter=300)
    uf = [v.double().cpu().numpy() for v in r.factors()]
    g, full = oracle.kkt_vectors(T.numpy(), uf)
    assert abs(full - r.sigma) <= 1e-5 * abs(r.sigma)
    rr = np.linalg.norm(np.concatenate(g) - full * np.concatenate(uf)) / abs(full)
    assert rr <= 1e-5


def test_invalid_arguments_are_rejected():
    pkg = P()
    T = torch.zeros(4, 5, 6, device="cuda")
    with pytest.raises(pkg.HoscfError) as e:
        pkg.hoscf_solve(T + 1, torch.zeros(15, device="cuda"))
    assert e.value.status == 1


def test_misaligned_tensor_is_rejected():
    """The descriptor's data must be 16-byte aligned (every load path - TMA,
    bulk copies, vector loads - assumes it): a 4-byte offset is EINVAL, and the
    handle stays usable."""
    pkg = P()
    dims = (6, 5, 24, 20)
    buf = torch.zeros(int(np.prod(dims)) + 1, device="cuda")
    T = buf[1:].view(dims)
    assert T.data_ptr() % 16 != 0
    u = torch.cat(W.unit_gaussian_vectors(dims, 1)).cuda()
    with pytest.raises(pkg.HoscfError) as e:
        pkg.hoscf_ttvc_blocks(T, u)
    assert e.value.status == 1
    H = pkg.hoscf_ttvc_blocks(torch.zeros(dims, device="cuda"), u)
    assert float(H.abs().max()) == 0.0


@pytest.mark.parametrize("max_iter", [0, 1, 3, 300])
def test_reported_residuals_match_the_oracle_at_the_returned_point(max_iter):
    """hoscf_info's KKT residual, eq. (4.1) residual and raw sigma against the
    oracle's values (blocks by eq. 3.3 in FP64) at the factors the library
    returns, both at unconverged points (max_iter 0, 1, 3) and at the
    converged one.  Both residuals are invariant under the sign flips of the
    final fix and the gauge.  Tolerance: relative 1e-4 plus an absolute 2e-6
    for the FP32 blocks' rounding in J x - rho x."""
    dims = (30, 40, 50)
    T, _ = W.planted_cp(dims, [2.0, 1.0], seed=31, noise_abs=0.3)
    u0 = torch.cat(W.unit_gaussian_vectors(dims, 33)).cuda()
    r = P().hoscf_solve(T.cuda(), u0, tol=1e-6, max_iter=max_iter)
    assert r.converged == (max_iter == 300)
    uf = [v.double().cpu().numpy() for v in r.factors()]
    Hr = oracle.blocks(T.numpy(), uf)
    r41 = oracle.residual_4_1(Hr, list(dims), uf)
    _, sig, rk = oracle.kkt_from_blocks(Hr, list(dims), uf)
    assert abs(r.resid_4_1 - r41) <= 1e-4 * r41 + 2e-6, (r.resid_4_1, r41)
    assert abs(r.resid - rk) <= 1e-4 * rk + 2e-6, (r.resid, rk)
    assert abs(abs(r.sigma_raw) - abs(sig)) <= 1e-5 * abs(sig)
    assert abs(r.sigma - abs(sig)) <= 1e-5 * abs(sig)
    if max_iter == 0:
        assert r.iters == 0 and r.passes == 1


@pytest.mark.parametrize("dims,seed", [((20, 30, 25), 51), ((40, 7, 33), 52), ((130, 70, 260), 53),
                                        ((30, 20), 54)])
def test_asvd_matches_oracle(dims, seed):
    """The ASVD comparison method (Sec. 1): two factors at a time from the
    largest singular pair of the block of the free modes, Gauss-Seidel over
    the fixed mode.  The solve reaches the oracle's ASVD point (sigma and the
    signed factors), and the first sub-steps agree iterate by iterate: after
    each one sigma = a^T A_mn b = s_1 > 0 on both sides."""
    T, _ = W.planted_cp(dims, [4.0, 1.0], seed=seed, noise_abs=0.3)
    u0 = W.unit_gaussian_vectors(dims, seed + 1)
    ref = oracle.asvd(T.numpy(), [v.numpy() for v in u0], tol=1e-10, max_iter=2000)
    assert ref.converged
    u0g = torch.cat(u0).cuda()
    r = P().hoscf_solve(T.cuda(), u0g, tol=1e-6, max_iter=2000, variant="asvd")
    assert r.converged and r.passes == r.iters + 1
    compare_solution(r, ref)
    for k in range(1, min(4, ref.iters) + 1):
        rk = P().hoscf_solve(T.cuda(), u0g, tol=0.0, max_iter=k, variant="asvd", eig_adapt=0.0)
        sr = ref.history[k][0]
        assert sr > 0 and abs(rk.sigma_raw - sr) <= 1e-5 * sr, (k, rk.sigma_raw, sr)


def test_asvd_rejects_order_4():
    pkg = P()
    T = torch.randn(4, 5, 6, 3, device="cuda")
    with pytest.raises(pkg.HoscfError) as e:
        pkg.hoscf_solve(T, torch.cat(W.unit_gaussian_vectors(T.shape, 1)).cuda(), variant="asvd")
    assert e.value.status == 7
