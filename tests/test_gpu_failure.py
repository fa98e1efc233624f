"""Failure detection on the GPU without a fault, and the kernel-timing aid.

Every spin-wait in the library's kernels is bounded.  A wait whose condition
nothing can satisfy (an mbarrier phase no copy completes; the grid barrier
with an arrival missing) must give up after its bound, record the timeout in
the device status word and return, so that the host call reports
HOSCF_TIMEOUT and the context stays usable: the next calls on it give
correct results.  No kernel is made to fault, trap or hang."""
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


@pytest.mark.parametrize("kind", [0, 1])
def test_wait_that_runs_out_reports_timeout_and_context_survives(kind):
    pkg = P()
    assert pkg.hoscf_selftest_timeout(kind, 2_000_000) == 6      # HOSCF_TIMEOUT
    torch.cuda.synchronize()
    # same context: exact blocks on an integer-valued tensor, then a solve
    dims = (40, 50, 136)
    rng = np.random.default_rng(7)
    Ti = rng.integers(-3, 4, size=dims).astype(np.float32)
    ui = [rng.integers(-2, 3, size=n).astype(np.float64) for n in dims]
    H = pkg.hoscf_ttvc_blocks(torch.from_numpy(Ti).cuda(),
                              torch.from_numpy(np.concatenate(ui).astype(np.float32)).cuda())
    assert np.array_equal(H.double().cpu().numpy(), oracle.blocks(Ti, ui))
    T, _ = W.planted_cp((60, 70, 80), [4.0], seed=11, noise_abs=0.5)
    u0 = torch.cat(W.unit_gaussian_vectors((60, 70, 80), 12)).cuda()
    r = pkg.hoscf_solve(T.cuda(), u0, tol=1e-6, max_iter=300)   # its grid barriers work again
    assert r.converged


def test_selftest_rejects_bad_arguments():
    pkg = P()
    assert pkg.hoscf_selftest_timeout(3, 1000) == 1
    assert pkg.hoscf_selftest_timeout(0, 0) == 1


def test_asynchronous_timeout_is_reported_by_device_status():
    """A bounded wait that gives up inside an asynchronous call (kind 2: the
    pass's mbarrier wait, launched on the caller's stream) is not known when
    the call returns; hoscf_device_status reports it once and clears it, and
    the handle then gives exact blocks and a working eigen step again."""
    pkg = P()
    assert pkg.hoscf_device_status() == 0
    assert pkg.hoscf_selftest_timeout(2, 2_000_000) == 0       # launched, not read back
    assert pkg.hoscf_device_status() == 6                      # HOSCF_TIMEOUT
    assert pkg.hoscf_device_status() == 0                      # cleared
    dims = (40, 50, 136)
    rng = np.random.default_rng(9)
    Ti = rng.integers(-3, 4, size=dims).astype(np.float32)
    ui = [rng.integers(-2, 3, size=n).astype(np.float64) for n in dims]
    H = pkg.hoscf_ttvc_blocks(torch.from_numpy(Ti).cuda(),
                              torch.from_numpy(np.concatenate(ui).astype(np.float32)).cuda())
    assert np.array_equal(H.double().cpu().numpy(), oracle.blocks(Ti, ui))
    x0 = torch.from_numpy(np.concatenate(ui) / np.linalg.norm(np.concatenate(ui))).cuda()
    pkg.hoscf_eig_step(dims, H, x0)
    assert pkg.hoscf_device_status() == 0


def test_kernel_timing_aid_counts_each_pass():
    pkg = P()
    dims = (128, 128, 256)
    T = W.gaussian_tensor(dims, 8).cuda()
    u = torch.cat(W.unit_gaussian_vectors(dims, 9)).cuda()
    H = pkg.hoscf_ttvc_blocks(T, u)
    pkg.hoscf_profile_enable(0, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        pkg.hoscf_ttvc_blocks(T, u, H)
    e1.record()
    pkg.hoscf_profile_enable(0, False)
    pkg.hoscf_ttvc_blocks(T, u, H)          # not recorded
    n, ms = pkg.hoscf_profile_read(0)
    torch.cuda.synchronize()
    assert n == 3
    assert 0.0 < ms <= e0.elapsed_time(e1)
    pkg.hoscf_profile_enable(0, True)       # re-enabling clears the records
    pkg.hoscf_profile_enable(0, False)
    assert pkg.hoscf_profile_read(0)[0] == 0


def test_timing_aid_records_the_backward_write_and_adjoint_solve():
    """Kinds 1 and 2 of the timing aid: one gradient-write record per
    hoscf_backward call, one adjoint-solve record per call that solves
    (grad_u given), each a positive duration within the call's wall time."""
    pkg = P()
    dims = (20, 24, 28)
    T, _ = W.planted_cp(dims, [1.0], seed=11, noise_abs=0.05)
    Tg = T.cuda()
    r = pkg.hoscf_solve(Tg, torch.cat(W.unit_gaussian_vectors(dims, 12)).cuda(), tol=1e-6)
    w = torch.randn(sum(dims), generator=torch.Generator().manual_seed(3)).cuda()
    pkg.hoscf_profile_enable(0, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    pkg.hoscf_backward(Tg, r.u, r.sigma, 1.0, w)
    pkg.hoscf_backward(Tg, r.u, r.sigma, 1.0, None)      # d sigma / dT only: no solve
    e1.record()
    pkg.hoscf_profile_enable(0, False)
    torch.cuda.synchronize()
    nw, wms = pkg.hoscf_profile_read(0, pkg.PROFILE_GRAD_WRITE)
    na, ams = pkg.hoscf_profile_read(0, pkg.PROFILE_ADJOINT)
    assert (nw, na) == (2, 1)
    assert 0.0 < wms and 0.0 < ams and wms + ams <= e0.elapsed_time(e1)
    assert pkg.hoscf_profile_read(0, pkg.PROFILE_PASS_KERNEL)[0] == 0


def test_timing_aid_records_every_eigen_step():
    """Kind 3: one record per eigen-step launch - a hoscf_eig_step call, and
    the certificate + eigen step that follows every pass of a solve - their
    total a positive duration within the calls' wall time; kind 0 counts
    hoscf_ttvc_blocks calls only, so it stays empty here."""
    pkg = P()
    dims = (40, 30, 50)
    T, _ = W.planted_cp(dims, [1.0], seed=13, noise_abs=0.05)
    Tg = T.cuda()
    u = torch.cat(W.unit_gaussian_vectors(dims, 14)).cuda()
    H = pkg.hoscf_ttvc_blocks(Tg, u)
    pkg.hoscf_profile_enable(0, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    pkg.hoscf_eig_step(dims, H, u.double())
    r = pkg.hoscf_solve(Tg, u, tol=1e-6)
    e1.record()
    pkg.hoscf_profile_enable(0, False)
    torch.cuda.synchronize()
    ne, ems = pkg.hoscf_profile_read(0, pkg.PROFILE_EIG_STEP)
    npass, _ = pkg.hoscf_profile_read(0, pkg.PROFILE_PASS_KERNEL)
    assert r.converged
    assert npass == 0
    assert ne == 1 + r.passes     # the certificate rides on an eigen-step launch at every pass
    assert 0.0 < ems <= e0.elapsed_time(e1)
