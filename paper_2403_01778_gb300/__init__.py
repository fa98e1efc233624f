"""GB300 (sm_103a) HOSCF / iHOSCF: best rank-one approximation of dense
tensors (arXiv 2403.01778) behind a C ABI (include/hoscf.h).

The compute path is libhoscf.so (hand-written CUDA); this package only
marshals torch tensors into it.  There is no CPU fallback: importing the
functions works everywhere, calling them needs the built library and a GPU.
"""
from .api import (HoscfError, SolveResult, handle, hoscf_backward, hoscf_device_status,  # noqa: F401
                  hoscf_eig_step, hoscf_opts_default, hoscf_profile_enable, hoscf_profile_read, hoscf_quantize,
                  hoscf_rqi_step, hoscf_selftest_timeout, hoscf_solve, hoscf_solve_batched,
                  hoscf_solve_greedy,
                  hoscf_ttvc_blocks, hoscf_ttvc_blocks_static, hoscf_workspace_size, n_blocks,
                  n_tot, hoscf_create_handle, hoscf_destroy_handle, shard_rows, allreduce_blocks,
                  hoscf_ttvc_blocks_slab, hoscf_solve_sharded, PROFILE_PASS_KERNEL,
                  PROFILE_GRAD_WRITE, PROFILE_ADJOINT, PROFILE_EIG_STEP)
from .autograd import HOSCFFunction, hoscf  # noqa: F401
