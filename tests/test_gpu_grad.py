"""Differentiation form on the GPU: dL/dT for L = c*sigma + sum_n <w_n, u_n>
against the FP64 oracle adjoint (rel <= 1e-5) and against central finite
differences of the GPU solve (h = 1e-3, rel <= 1e-3)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_01778_gb300 import build
    build.build()


def P():
    import paper_2403_01778_gb300 as pkg
    return pkg


def solve(T, u0, tol=1e-6):
    r = P().hoscf_solve(T, u0, tol=tol, max_iter=500)
    assert r.converged
    return r


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims", [(20, 24, 28), (6, 7, 5, 8), (3, 4, 3, 4, 3, 4), (30, 40)])
def test_backward_matches_oracle_adjoint(dims):
    T, _ = W.planted_cp(dims, [1.0], seed=11, noise_abs=0.05)
    u0 = torch.cat(W.unit_gaussian_vectors(dims, 12)).cuda()
    Tg = T.cuda()
    r = solve(Tg, u0)
    rng = np.random.default_rng(13)
    w = rng.standard_normal(sum(dims)).astype(np.float32)
    c = 0.7
    gT = P().hoscf_backward(Tg, r.u, r.sigma, c, torch.from_numpy(w).cuda())
    u64 = [v.double().cpu().numpy() for v in r.factors()]
    ref, a, _ = oracle.adjoint(T.numpy().astype(np.float64), u64, r.sigma, c,
                               oracle.split(w.astype(np.float64), list(dims)))
    assert rel(gT.double().cpu().numpy(), ref) <= 1e-5
    gs = P().hoscf_backward(Tg, r.u, r.sigma, 1.0, None)       # d sigma / dT alone
    ref_s, _, _ = oracle.adjoint(T.numpy().astype(np.float64), u64, r.sigma, 1.0, None)
    assert rel(gs.double().cpu().numpy(), ref_s) <= 1e-6


@pytest.mark.parametrize("dims", [(256, 256, 256), (24, 20, 24, 20, 24, 20)])
def test_backward_full_size_against_oracle_and_fd(dims):
    """The differentiation workloads at full size: planted rank one plus 5%
    noise; loss sigma + <w, u> with seeded Gaussian w."""
    T, _ = W.planted_cp(dims, [1.0], seed=21, noise_abs=0.05)
    Tg = T.cuda()
    u0 = torch.cat(W.unit_gaussian_vectors(dims, 22)).cuda()
    r = solve(Tg, u0)
    w = torch.from_numpy(np.random.default_rng(23).standard_normal(sum(dims)).astype(np.float32))
    gT = P().hoscf_backward(Tg, r.u, r.sigma, 1.0, w.cuda())
    u64 = [v.double().cpu().numpy() for v in r.factors()]
    ref, _, _ = oracle.adjoint(T.numpy().astype(np.float64), u64, r.sigma, 1.0,
                               oracle.split(w.numpy().astype(np.float64), list(dims)))
    assert rel(gT.double().cpu().numpy(), ref) <= 1e-5
    # central differences (h = 1e-3) along two unit directions: the gradient
    # itself (error relative to the derivative) and a seeded Gaussian
    # direction (error relative to |grad L|, the largest directional
    # derivative; its own derivative is ~|grad L| / sqrt(N) and below the
    # FP32 noise of the solve)
    h = 1e-3

    def L(Tp):
        # run to the FP32 floor (the certificate may stop short of 2e-7)
        rr = P().hoscf_solve(Tp, r.u, tol=2e-7, max_iter=60)
        assert rr.resid < 1e-6
        return rr.sigma + float((w.cuda() * rr.u).sum())
    gnorm = float(gT.norm())
    for k, D in enumerate([gT / gT.norm(), W.gaussian_tensor(dims, 24).cuda()]):
        D = D / D.norm()
        fd = (L(Tg + h * D) - L(Tg - h * D)) / (2 * h)
        an = float((gT * D).sum())
        scale = abs(an) if k == 0 else gnorm
        assert abs(fd - an) <= 1e-3 * scale, (k, fd, an)


def test_autograd_function():
    dims = (16, 18, 20)
    T, _ = W.planted_cp(dims, [2.0], seed=31, noise_abs=0.1)
    Tg = T.cuda().requires_grad_(True)
    u0 = torch.cat(W.unit_gaussian_vectors(dims, 32)).cuda()
    w = torch.from_numpy(np.random.default_rng(33).standard_normal(sum(dims)).astype(np.float32)).cuda()
    sigma, u = P().hoscf(Tg, u0, tol=1e-6)
    loss = 0.5 * sigma + (w * u).sum()
    loss.backward()
    u64 = [v.astype(np.float64) for v in np.split(u.detach().cpu().numpy(), np.cumsum(dims)[:-1])]
    ref, _, _ = oracle.adjoint(T.numpy().astype(np.float64), u64, float(sigma.detach()), 0.5,
                               oracle.split(w.cpu().numpy().astype(np.float64), list(dims)))
    assert rel(Tg.grad.double().cpu().numpy(), ref) <= 1e-5


def test_adjoint_directions_are_tangent():
    """a_n must be orthogonal to u_n: grad_T contracted with u on all modes but n,
    then with u_n, equals c exactly when only the factor term is zeroed."""
    dims = (12, 10, 14)
    T, _ = W.planted_cp(dims, [1.5], seed=41, noise_abs=0.1)
    Tg = T.cuda()
    r = solve(Tg, torch.cat(W.unit_gaussian_vectors(dims, 42)).cuda())
    w = torch.randn(sum(dims), generator=torch.Generator().manual_seed(43)).cuda()
    gT = P().hoscf_backward(Tg, r.u, r.sigma, 0.0, w).double().cpu().numpy()
    # <gT, u1 o u2 o u3> = c - sum_n <a_n, u_n> = 0 when c = 0 and a_n ⟂ u_n
    f = [v.double().cpu().numpy() for v in r.factors()]
    val = np.einsum("abc,a,b,c->", gT, *f)
    assert abs(val) <= 1e-5 * np.linalg.norm(gT)
