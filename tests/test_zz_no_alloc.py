"""The allocation-free TTVc entry point (hoscf_ttvc_blocks_static), called
through the C ABI, must give the same blocks as hoscf_ttvc_blocks.

It serves callers that cannot call cudaMalloc (their host application owns
the device memory, or they must not allocate after start-up): its scratch is
the library's fixed device array, shared by all calls.  Two calls in a row
check that what one call leaves in that array does not leak into the next.
This file is collected last so a failure here stops a -x run only after every
other test has run."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    from paper_2403_01778_gb300 import _lib, build
    build.build()
    return _lib


def call_static(lib, T, u, H, status=None):
    dims = (ctypes.c_int64 * T.dim())(*T.shape)
    dtype = lib.HOSCF_BF16 if T.dtype == torch.bfloat16 else lib.HOSCF_F32
    desc = lib.TensorDesc(T.dim(), dims, dtype, ctypes.c_void_p(T.data_ptr()), None)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sp = ctypes.c_void_p(status.data_ptr() if status is not None else 0)
    return lib.load().hoscf_ttvc_blocks_static(ctypes.byref(desc), ctypes.c_void_p(u.data_ptr()),
                                               ctypes.c_void_p(H.data_ptr()), sp, stream)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("dims", [(64, 96, 128), (9, 10, 11, 12), (37, 50, 129)])
def test_static_entry_matches_workspace_entry(lib, dims, dtype):
    """Tiled and small-face kernels, FP32 and BF16 instantiations; the pass's
    device status comes back as 0 in the caller's status word."""
    import paper_2403_01778_gb300 as P
    T = W.gaussian_tensor(dims, 7).cuda().to(dtype)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        u = torch.cat(W.unit_gaussian_vectors(dims, 8 + call)).cuda()
        expect = P.hoscf_ttvc_blocks(T, u)
        H = torch.full_like(expect, float("nan"))
        status.fill_(-1)
        assert call_static(lib, T, u, H, status) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        a, b = H.double().cpu().numpy(), expect.double().cpu().numpy()
        scale = np.abs(b).max()
        np.testing.assert_allclose(a, b, rtol=0, atol=64 * EPS32 * scale)


def test_static_entry_rejects_oversized_problem(lib):
    T = torch.empty(1024, 1024, 1024, device="cuda")   # needs ~106 MiB of scratch
    u = torch.ones(sum(T.shape), device="cuda")
    H = torch.empty(3 * 1024 * 1024, device="cuda")
    assert call_static(lib, T, u, H) == 1   # HOSCF_EINVAL
