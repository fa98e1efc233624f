"""Greedy rank-R approximation (Sec. 1, Example 3) on the GPU: implicit
deflation (the blocks of A minus the earlier terms' contributions) against the
oracle, which forms every deflated tensor A^(r+1) = A^(r) - B^(r) explicitly."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from helpers import assert_same_solution

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01778_gb300 import build
    build.build()


def P():
    import paper_2403_01778_gb300 as pkg
    return pkg


def guesses(dims, R, seed):
    return [[v.numpy() for v in W.unit_gaussian_vectors(dims, seed + r)] for r in range(R)]


def run_gpu(T, R, u0, **kw):
    u = torch.from_numpy(np.stack([np.concatenate(g) for g in u0]).astype(np.float32)).cuda()
    return P().hoscf_solve_greedy(torch.as_tensor(np.ascontiguousarray(T)).cuda(), R, u, **kw)


def compare(g, ref, R, tol=1e-5):
    for r in range(R):
        assert_same_solution(g.sigmas[r], g.factors(r), ref.sigmas[r], ref.factors[r], tol,
                             sigma_atol=tol * abs(ref.sigmas[0]))
    # res_r^2 = 1 - sum_{s<r} sigma_s^2 / ||A||^2: each sigma_s within tol
    # (relative) moves it by at most 2 tol sigma_s^2 / ||A||^2 (the square
    # root itself amplifies that near zero)
    for r in range(R + 1):
        assert abs(g.res[r] ** 2 - ref.res[r] ** 2) <= 2 * tol


def test_greedy_order2_is_truncated_svd():
    A = W.gaussian_tensor((40, 30), 5).numpy()
    U, S, Vt = np.linalg.svd(A.astype(np.float64))
    g = run_gpu(A, 3, guesses((40, 30), 3, 10), tol=1e-6, max_iter=100)
    assert g.converged
    for r in range(3):
        assert abs(g.sigmas[r] - S[r]) <= 1e-5 * S[0]
        a, b = U[:, r].copy(), Vt[r].copy()
        if b[int(np.argmax(np.abs(b)))] < 0:      # the gauge: u2's largest entry positive
            a, b = -a, -b
        assert_same_solution(g.sigmas[r], g.factors(r), S[r], [a, b], sigma_atol=1e-5 * S[0])
    for r in range(4):
        assert abs(g.res[r] - np.sqrt(np.sum(S[r:] ** 2)) / np.linalg.norm(A)) <= 1e-5


def test_greedy_orthogonal_cp_matches_oracle():
    dims, w = (40, 30, 20), [5.0, 3.0, 1.5]
    Q = [np.linalg.qr(np.random.default_rng(7 + n).standard_normal((m, 3)))[0] for n, m in enumerate(dims)]
    T = sum(wr * np.einsum("i,j,k->ijk", Q[0][:, r], Q[1][:, r], Q[2][:, r]) for r, wr in enumerate(w))
    T = T.astype(np.float32)
    u0 = guesses(dims, 3, 20)
    ref = oracle.greedy(T, 3, u0, tol=1e-10)
    g = run_gpu(T, 3, u0, tol=1e-6, max_iter=300)
    assert g.converged
    compare(g, ref, 3)
    assert g.res[3] < 1e-3


def test_greedy_planted_order4_with_noise_matches_oracle():
    dims = (12, 14, 10, 16)
    T, _ = W.planted_cp(dims, [3.0, 2.0, 1.0], seed=33, noise_abs=0.3)
    T = T.numpy()
    u0 = guesses(dims, 3, 40)
    ref = oracle.greedy(T, 3, u0, tol=1e-10, max_iter=2000)
    g = run_gpu(T, 3, u0, tol=1e-6, max_iter=2000)
    assert g.converged
    compare(g, ref, 3)


def test_greedy_rejects_bad_rank():
    pkg = P()
    T = torch.randn(4, 5, 6, device="cuda")
    with pytest.raises(ValueError):
        pkg.hoscf_solve_greedy(T, 2, torch.randn(3, 15, device="cuda"))
    with pytest.raises(pkg.HoscfError) as e:
        pkg.hoscf_solve_greedy(T, 33, torch.randn(33, 15, device="cuda"))
    assert e.value.status == 1
