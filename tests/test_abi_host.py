"""Host-side checks of the C ABI and of the bench's multi-rank logic (no GPU).

* the library builds for sm_103a, loads, and exports every function that
  include/hoscf.h declares (parsed from the header, not from the binding);
* the entry points that need no device behave as documented: defaults,
  rejection of NULL / invalid arguments, host-only workspace sizing;
* a status code from the library becomes a typed Python exception (the
  failure is made on the host, by a fake of the failing call);
* the bench's max-over-ranks timing and whole-job throughput over a gloo
  process group of world size 2, and the reference arm's rank gating."""
import argparse
import ctypes
import multiprocessing as mp
import os
import re
import socket

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hoscf.h")

EINVAL = 1


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    pat = r"^\s*(?:hoscf_status|const\s+char\s*\*)\s*(hoscf_\w+)\s*\("
    return sorted(set(re.findall(pat, txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_01778_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_and_binding_list_the_same_functions():
    from paper_2403_01778_gb300 import _lib
    declared = header_functions()
    assert len(declared) >= 14
    assert set(declared) == set(_lib.EXPORTS)


def test_library_exports_every_declared_function(lib):
    from paper_2403_01778_gb300 import build
    handle = ctypes.CDLL(build.LIB)
    missing = [n for n in header_functions() if not hasattr(handle, n)]
    assert not missing, missing


def test_opts_default_values(lib):
    from paper_2403_01778_gb300 import _lib
    o = _lib.Opts()
    assert lib.hoscf_opts_default(ctypes.byref(o)) == 0
    assert (o.tol, o.max_iter, o.variant) == (1e-6, 200, 0)
    assert (o.eig_tol, o.eig_max_steps, o.eig_adapt) == (1e-10, 64, 1e-3)
    assert not o.refine and o.switch_tol == 1e-3 and o.timeout_ns == 2_000_000_000
    assert o.switch_predict == 1


def test_null_and_invalid_arguments_are_rejected_on_the_host(lib):
    from paper_2403_01778_gb300 import _lib
    assert lib.hoscf_opts_default(None) == EINVAL
    assert lib.hoscf_destroy(None) == EINVAL
    assert lib.hoscf_last_error(None) == b"null handle"
    assert lib.hoscf_ttvc_blocks(None, None, None, None, None) == EINVAL
    assert lib.hoscf_solve(None, None, None, None, None, None, None, None) == EINVAL
    arr3 = (ctypes.c_int64 * 3)(4, 5, 6)
    assert lib.hoscf_eig_step(None, 3, arr3, None, None, None, None, None, None, None) == EINVAL
    assert lib.hoscf_rqi_step(None, 3, arr3, None, None, None, None, None, None, None) == EINVAL
    assert lib.hoscf_backward(None, None, None, 0.0, 0.0, None, None, None) == EINVAL
    assert lib.hoscf_profile_enable(None, 1) == EINVAL
    n, ms = ctypes.c_int(), ctypes.c_double()
    assert lib.hoscf_profile_read(None, 0, ctypes.byref(n), ctypes.byref(ms)) == EINVAL
    assert lib.hoscf_ttvc_blocks_static(None, None, None, None, None) == EINVAL
    assert lib.hoscf_device_status(None, None) == EINVAL
    assert lib.hoscf_selftest_timeout(None, 0, 1000, None) == EINVAL
    # a descriptor of order 9 is rejected before any device call
    dims = (ctypes.c_int64 * 9)(*([2] * 9))
    desc = _lib.TensorDesc(9, dims, 0, ctypes.c_void_p(16), None)
    buf = ctypes.c_void_p(16)
    assert lib.hoscf_ttvc_blocks_static(ctypes.byref(desc), buf, buf, None, None) == EINVAL
    size = ctypes.c_size_t()
    for order, dd in [(3, (4, 0, 5)), (1, (4,)), (9, (2,) * 9)]:
        arr = (ctypes.c_int64 * len(dd))(*dd)
        assert lib.hoscf_workspace_size(order, arr, 0, ctypes.byref(size)) == EINVAL


def test_workspace_size_is_host_only_and_grows_with_the_problem(lib):
    sizes = []
    for dd in [(16, 16, 16), (64, 64, 64), (256, 256, 256), (24, 20, 24, 20, 24, 20)]:
        arr = (ctypes.c_int64 * len(dd))(*dd)
        b = ctypes.c_size_t()
        assert lib.hoscf_workspace_size(len(dd), arr, 0, ctypes.byref(b)) == 0
        sizes.append(b.value)
    assert sizes[0] > 0 and sizes[0] < sizes[1] < sizes[2]
    # the FP8 form sizes for its FP32 refinement copy as well
    arr = (ctypes.c_int64 * 4)(200, 200, 200, 200)
    b8, b32 = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.hoscf_workspace_size(4, arr, 2, ctypes.byref(b8)) == 0
    assert lib.hoscf_workspace_size(4, arr, 0, ctypes.byref(b32)) == 0
    assert b8.value >= b32.value


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_create_without_a_device_fails_cleanly(lib):
    h = ctypes.c_void_p(123)
    assert lib.hoscf_create(ctypes.byref(h), 0) != 0
    assert not h.value


def test_status_codes_become_typed_errors(monkeypatch):
    from paper_2403_01778_gb300 import _lib, api

    class FakeLib:
        def hoscf_last_error(self, h):
            return b"a device-side wait exceeded its time limit"

    monkeypatch.setattr(_lib, "load", lambda: FakeLib())
    with pytest.raises(api.HoscfError) as e:
        api._check(_lib.HOSCF_TIMEOUT, None)
    assert e.value.status == _lib.HOSCF_TIMEOUT
    assert str(e.value).startswith("TIMEOUT:") and "time limit" in str(e.value)
    with pytest.raises(api.HoscfError) as e:
        api._check(_lib.HOSCF_NONFINITE, None)
    assert e.value.status == _lib.HOSCF_NONFINITE
    assert api._check(_lib.HOSCF_NOT_CONVERGED, None,
                      allow=(0, _lib.HOSCF_NOT_CONVERGED)) == _lib.HOSCF_NOT_CONVERGED


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2403_01778_gb300 import _lib
    monkeypatch.setattr(_lib, "_LIB", None)
    monkeypatch.setattr(_lib, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, ms, bench.whole_job_gbs(2e9, 4, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_takes_the_slowest_rank_and_whole_job_bytes_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [15.0, 15.0]
    assert all(abs(g[2] - 2e9 * 4 * 2 / 0.015 / 1e9) < 1e-9 for g in got)


def test_reference_arm_runs_on_rank_zero_only():
    import bench
    args = argparse.Namespace(workload="cfg1_64cube", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert bench.max_over_ranks(7.5) == 7.5


def test_binding_rejects_bad_tensors_before_any_device_call():
    """The Python binding checks dtypes, sizes and placement on the host and
    raises ValueError before it touches the library or a device."""
    import paper_2403_01778_gb300 as P
    dims = (4, 5, 6)
    H = torch.zeros(P.n_blocks(dims))
    with pytest.raises(ValueError):
        P.hoscf_eig_step(dims, H, torch.zeros(15, dtype=torch.float32))     # x_prev must be FP64
    with pytest.raises(ValueError):
        P.hoscf_eig_step(dims, H, torch.zeros(14, dtype=torch.float64))     # wrong length
    with pytest.raises(ValueError):
        P.hoscf_rqi_step(dims, H, torch.zeros(15, dtype=torch.float64))     # u must be FP32
    with pytest.raises(ValueError):
        P.hoscf_rqi_step(dims, H, torch.zeros(16, dtype=torch.float32))     # wrong length
    with pytest.raises(ValueError):
        P.hoscf_quantize(torch.zeros(8), "bf16")                            # host tensor
    with pytest.raises(ValueError):
        P.hoscf_ttvc_blocks(torch.zeros(dims), torch.zeros(15))             # host tensor


def test_reference_arm_times_the_oracle_step_on_the_host(capsys):
    """--impl reference: the FP64 oracle's HOSCF iteration (blocks by
    definition + dense eigen step) on the host cores, over the whole tensor
    when the steps fit their budget; one JSON line with the contract's keys."""
    import json
    import bench
    args = argparse.Namespace(workload="cfg1_64cube", steps=2, warmup=1, gpus=1)
    assert bench.run_reference(args, rank=0, world=1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "GB/s"
    assert line["config"]["sample_slices"] == 64                 # the whole 64^3 tensor
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["steps"] == 2 and line["warmup"] == 1


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor: shape, dtype, contiguity and an address."""

    def __init__(self, shape, ptr):
        self.shape = torch.Size(shape)
        self.dtype = torch.float32
        self.is_cuda = True
        self._ptr = ptr

    def is_contiguous(self):
        return True

    def dim(self):
        return len(self.shape)

    def data_ptr(self):
        return self._ptr


def test_batch_descriptors_are_filled_as_the_c_struct_expects():
    """The batched call fills its descriptor array field by field with numpy:
    every field lands where the C struct has it (order, dims pointer into a
    kept buffer, dtype, data, no scales), and orders other than 3 and 4 are
    rejected on the host."""
    from paper_2403_01778_gb300 import _lib, api
    ts = [_FakeDeviceTensor((3, 4, 5), 4096), _FakeDeviceTensor((6, 7, 8, 9), 8192),
          _FakeDeviceTensor((9, 1, 2), 65536)]
    arr, keep = api._batch_descs(ts)
    for d, t in zip(arr, ts):
        assert d.order == len(t.shape)
        assert [d.dims[k] for k in range(d.order)] == list(t.shape)
        assert d.dtype == _lib.HOSCF_F32 and d.data == t.data_ptr() and not d.scales
    with pytest.raises(ValueError):
        api._batch_descs([_FakeDeviceTensor((2, 3), 16)])
    with pytest.raises(ValueError):
        api._batch_descs([_FakeDeviceTensor((2, 3, 4, 5, 6), 16)])


def test_batched_binding_rejects_bad_input_on_the_host():
    """hoscf_solve_batched checks counts, placement and start-vector lengths
    before it touches the library or a device."""
    import paper_2403_01778_gb300 as P
    with pytest.raises(ValueError):
        P.hoscf_solve_batched([], [])                                   # empty batch
    with pytest.raises(ValueError):
        P.hoscf_solve_batched([torch.zeros(3, 4, 5)], [])               # one start per tensor
    with pytest.raises(ValueError):
        P.hoscf_solve_batched([torch.zeros(3, 4, 5)], [torch.zeros(12)])   # host tensor
