"""Python binding of the HOSCF C ABI: same names, argument marshalling only.

Tensors are torch CUDA tensors (PyTorch supplies device memory and the
current stream); every computation runs in libhoscf.so.  A tensor may be
float32, bfloat16, float16, or FP8-e4m3 (torch.float8_e4m3fn or uint8 codes,
with a float32 ``scales`` tensor of one scale per 128 consecutive elements).
"""
from __future__ import annotations

import ctypes
import math
import threading
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import Info, Opts, TensorDesc


class HoscfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_handles = {}
_hlock = threading.Lock()


def handle(device=None) -> ctypes.c_void_p:
    """Per-device library handle, created on first use."""
    if device is None:
        device = torch.cuda.current_device()
    device = int(torch.device("cuda", device).index if not isinstance(device, int) else device)
    with _hlock:
        h = _handles.get(device)
        if h is None:
            lib = _lib.load()
            h = ctypes.c_void_p()
            st = lib.hoscf_create(ctypes.byref(h), device)
            if st != 0:
                raise HoscfError(st, f"hoscf_create(device={device}) failed")
            _handles[device] = h
        return h


def _check(st: int, h, allow=(0,)):
    if st not in allow:
        msg = _lib.load().hoscf_last_error(h)
        raise HoscfError(st, msg.decode() if msg else "")
    return st


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(T: torch.Tensor):
    if T.dtype == torch.float32:
        return _lib.HOSCF_F32
    if T.dtype == torch.bfloat16:
        return _lib.HOSCF_BF16
    if T.dtype == torch.float16:
        return _lib.HOSCF_F16
    if T.dtype in (torch.uint8, getattr(torch, "float8_e4m3fn", None)):
        return _lib.HOSCF_F8E4M3
    raise TypeError(f"unsupported tensor dtype {T.dtype}")


class _Desc:
    """Keeps the dims array alive alongside the descriptor."""

    def __init__(self, T: torch.Tensor, scales=None, dims=None):
        if not T.is_cuda:
            raise ValueError("tensor must be on a CUDA device")
        if not T.is_contiguous():
            raise ValueError("tensor must be contiguous (row-major)")
        shape = tuple(int(v) for v in (dims if dims is not None else T.shape))
        self.dims = (ctypes.c_int64 * len(shape))(*shape)
        self.shape = shape
        self.T = T
        self.scales = scales
        self.desc = TensorDesc(len(shape), self.dims, _dtype_code(T), ctypes.c_void_p(T.data_ptr()),
                               ctypes.c_void_p(scales.data_ptr() if scales is not None else 0))


def n_tot(dims):
    return int(sum(dims))


def n_blocks(dims):
    return int(sum(dims[m] * dims[n] for m in range(len(dims)) for n in range(m + 1, len(dims))))


def hoscf_opts_default() -> Opts:
    o = Opts()
    _lib.load().hoscf_opts_default(ctypes.byref(o))
    return o


def hoscf_workspace_size(dims, dtype=_lib.HOSCF_F32) -> int:
    arr = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    out = ctypes.c_size_t()
    st = _lib.load().hoscf_workspace_size(len(dims), arr, int(dtype), ctypes.byref(out))
    if st != 0:
        raise HoscfError(st, "hoscf_workspace_size failed")
    return int(out.value)


def hoscf_ttvc_blocks(T: torch.Tensor, u: torch.Tensor, H: torch.Tensor | None = None,
                      scales=None, stream=None) -> torch.Tensor:
    """All coupling blocks (eq. 3.3), packed (m<n lexicographic, each row-major)."""
    d = _Desc(T, scales)
    u = u.contiguous()
    if u.dtype != torch.float32 or u.numel() != n_tot(d.shape):
        raise ValueError("u must be float32 with sum(dims) entries")
    if H is None:
        H = torch.empty(n_blocks(d.shape), device=T.device, dtype=torch.float32)
    h = handle(T.device.index)
    _check(_lib.load().hoscf_ttvc_blocks(h, ctypes.byref(d.desc), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(H.data_ptr()), _stream_ptr(stream)), h)
    return H


PROFILE_PASS_KERNEL, PROFILE_GRAD_WRITE, PROFILE_ADJOINT, PROFILE_EIG_STEP = 0, 1, 2, 3


def hoscf_profile_enable(device: int = 0, enable: bool = True) -> None:
    """Start (clearing earlier records) or stop timing, on this device's
    handle, the pass's streaming kernel of every hoscf_ttvc_blocks call and
    the gradient write and adjoint solve of every hoscf_backward call."""
    h = handle(device)
    _check(_lib.load().hoscf_profile_enable(h, 1 if enable else 0), h)


def hoscf_profile_read(device: int = 0, which: int = PROFILE_PASS_KERNEL) -> tuple[int, float]:
    """(number of timed calls, total milliseconds) of one recorded kind."""
    h = handle(device)
    n, ms = ctypes.c_int(0), ctypes.c_double(0.0)
    _check(_lib.load().hoscf_profile_read(h, int(which), ctypes.byref(n), ctypes.byref(ms)), h)
    return n.value, ms.value


def hoscf_selftest_timeout(kind: int, timeout_ns: int = 1_000_000, device: int = 0,
                           stream=None) -> int:
    """Run a bounded device wait that can never be satisfied (kind 0: an
    mbarrier phase, 1: the grid barrier with an arrival missing, 2: kind 0
    launched asynchronously, reported later by hoscf_device_status) and
    return the library's status for it (HOSCF_TIMEOUT = 6 when the failure
    path works; OK for a launched kind 2)."""
    h = handle(device)
    return int(_lib.load().hoscf_selftest_timeout(h, int(kind), int(timeout_ns),
                                                  _stream_ptr(stream)))


def hoscf_device_status(device: int = 0, stream=None) -> int:
    """Failures the asynchronous calls recorded on the device: synchronises
    the stream, returns the status (0 = OK, 6 = TIMEOUT, 5 = NONFINITE) and
    clears it."""
    h = handle(device)
    return int(_lib.load().hoscf_device_status(h, _stream_ptr(stream)))


def hoscf_ttvc_blocks_static(T: torch.Tensor, u: torch.Tensor, H: torch.Tensor | None = None,
                             status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """hoscf_ttvc_blocks without allocation inside the library: scratch comes
    from the library's fixed 64 MiB device array (calls must not overlap).
    The output tensor is allocated here by torch unless H is given; `status`
    (a 1-element int32 CUDA tensor, optional) receives the pass's device
    status (0 = H valid)."""
    d = _Desc(T)
    u = u.contiguous()
    if u.dtype != torch.float32 or u.numel() != n_tot(d.shape):
        raise ValueError("u must be float32 with sum(dims) entries")
    if H is None:
        H = torch.empty(n_blocks(d.shape), device=T.device, dtype=torch.float32)
    if status is not None and (status.dtype != torch.int32 or not status.is_cuda):
        raise ValueError("status must be an int32 CUDA tensor")
    st = _lib.load().hoscf_ttvc_blocks_static(ctypes.byref(d.desc), ctypes.c_void_p(u.data_ptr()),
                                              ctypes.c_void_p(H.data_ptr()),
                                              ctypes.c_void_p(status.data_ptr() if status is not None else 0),
                                              _stream_ptr(stream))
    if st != 0:
        raise HoscfError(st, "hoscf_ttvc_blocks_static failed")
    return H


def _opts(tol=None, max_iter=None, variant=None, eig_tol=None, eig_max_steps=None,
          refine_desc=None, switch_tol=None, timeout_ns=None, eig_adapt=None,
          switch_predict=None) -> Opts:
    o = hoscf_opts_default()
    if switch_predict is not None:
        o.switch_predict = int(switch_predict)
    if eig_adapt is not None:
        o.eig_adapt = float(eig_adapt)
    if tol is not None:
        o.tol = float(tol)
    if max_iter is not None:
        o.max_iter = int(max_iter)
    if variant is not None:
        o.variant = _lib.VARIANTS[variant] if isinstance(variant, str) else int(variant)
    if eig_tol is not None:
        o.eig_tol = float(eig_tol)
    if eig_max_steps is not None:
        o.eig_max_steps = int(eig_max_steps)
    if refine_desc is not None:
        o.refine = ctypes.pointer(refine_desc)
    if switch_tol is not None:
        o.switch_tol = float(switch_tol)
    if timeout_ns is not None:
        o.timeout_ns = int(timeout_ns)
    return o


def hoscf_eig_step(dims, H: torch.Tensor, x_prev: torch.Tensor, eig_tol=None, eig_max_steps=None,
                   eig_adapt=None, stream=None):
    """Largest-magnitude eigenpair of J (Alg. 1 line 5) and the normalised
    factors (lines 6-9).  Returns (x float64, u float32, lambda float64 tensor)."""
    dims = [int(v) for v in dims]
    n = n_tot(dims)
    x_prev = x_prev.contiguous()
    if x_prev.dtype != torch.float64 or x_prev.numel() != n:
        raise ValueError("x_prev must be float64 with sum(dims) entries")
    x = torch.empty(n, device=H.device, dtype=torch.float64)
    u = torch.empty(n, device=H.device, dtype=torch.float32)
    lam = torch.empty(1, device=H.device, dtype=torch.float64)
    arr = (ctypes.c_int64 * len(dims))(*dims)
    o = _opts(eig_tol=eig_tol, eig_max_steps=eig_max_steps, eig_adapt=eig_adapt)
    h = handle(H.device.index)
    _check(_lib.load().hoscf_eig_step(h, len(dims), arr, ctypes.c_void_p(H.data_ptr()),
                                      ctypes.c_void_p(x_prev.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                      ctypes.c_void_p(lam.data_ptr()), ctypes.byref(o),
                                      _stream_ptr(stream)), h)
    return x, u, lam


def hoscf_rqi_step(dims, H: torch.Tensor, u: torch.Tensor, eig_tol=None, eig_max_steps=None,
                   stream=None):
    """One Rayleigh-quotient step of iHOSCF (Sec. 4.4) from the factors u:
    y = (J - rho I)^-1 x~ with x~ = [u] / sqrt(d), rho its Rayleigh quotient,
    then the block normalisation (Alg. 1 lines 6-9).  Returns (x float64 unit
    y, u float32 normalised blocks, rho float64 tensor)."""
    dims = [int(v) for v in dims]
    n = n_tot(dims)
    u = u.contiguous()
    if u.dtype != torch.float32 or u.numel() != n:
        raise ValueError("u must be float32 with sum(dims) entries")
    x = torch.empty(n, device=H.device, dtype=torch.float64)
    uo = torch.empty(n, device=H.device, dtype=torch.float32)
    rho = torch.empty(1, device=H.device, dtype=torch.float64)
    arr = (ctypes.c_int64 * len(dims))(*dims)
    o = _opts(eig_tol=eig_tol, eig_max_steps=eig_max_steps)
    h = handle(H.device.index)
    _check(_lib.load().hoscf_rqi_step(h, len(dims), arr, ctypes.c_void_p(H.data_ptr()),
                                      ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(uo.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
                                      ctypes.byref(o), _stream_ptr(stream)), h)
    return x, uo, rho


@dataclass
class SolveResult:
    sigma: float
    u: torch.Tensor          # concatenated factors, float32
    dims: tuple
    iters: int
    passes: int
    passes_refine: int
    rqi_accepts: int
    resid: float
    resid_4_1: float
    sigma_raw: float
    converged: bool

    def factors(self):
        out, o = [], 0
        for n in self.dims:
            out.append(self.u[o:o + n])
            o += n
        return out


def hoscf_solve(T: torch.Tensor, u0: torch.Tensor, tol=1e-6, max_iter=200, variant="hoscf",
                eig_tol=None, eig_max_steps=None, scales=None, refine: torch.Tensor | None = None,
                switch_tol=None, timeout_ns=None, u_out: torch.Tensor | None = None,
                eig_adapt=None, refine_scales=None, stream=None, switch_predict=None) -> SolveResult:
    """HOSCF / iHOSCF (Algorithm 1, Sec. 4.4).  Synchronous."""
    d = _Desc(T, scales)
    u0 = u0.contiguous()
    n = n_tot(d.shape)
    if u0.dtype != torch.float32 or u0.numel() != n:
        raise ValueError("u0 must be float32 with sum(dims) entries")
    rd = _Desc(refine) if refine is not None else None
    o = _opts(tol, max_iter, variant, eig_tol, eig_max_steps,
              rd.desc if rd is not None else None, switch_tol, timeout_ns, eig_adapt, switch_predict)
    if u_out is None:
        u_out = torch.empty(n, device=T.device, dtype=torch.float32)
    sigma = ctypes.c_double()
    info = Info()
    h = handle(T.device.index)
    st = _lib.load().hoscf_solve(h, ctypes.byref(d.desc), ctypes.c_void_p(u0.data_ptr()),
                                 ctypes.byref(o), ctypes.c_void_p(u_out.data_ptr()),
                                 ctypes.byref(sigma), ctypes.byref(info), _stream_ptr(stream))
    _check(st, h, allow=(0, _lib.HOSCF_NOT_CONVERGED))
    return SolveResult(sigma.value, u_out, d.shape, info.iters, info.passes, info.passes_refine,
                       info.rqi_accepts, info.resid, info.resid_4_1, info.sigma_raw, st == 0)


@dataclass
class GreedyResult:
    sigmas: list             # sigma_r of each rank-one term
    u: torch.Tensor          # R x n_tot factors, float32
    dims: tuple
    infos: list              # per-term (iters, passes, resid, converged)
    res: list                # ||A^(r)||_F / ||A||_F, r = 1 .. R+1
    converged: bool

    def factors(self, r):
        out, o = [], 0
        for n in self.dims:
            out.append(self.u[r, o:o + n])
            o += n
        return out


def hoscf_solve_greedy(T: torch.Tensor, R: int, u0: torch.Tensor, tol=1e-6, max_iter=200,
                       variant="hoscf", scales=None, refine: torch.Tensor | None = None,
                       switch_tol=None, eig_tol=None, eig_max_steps=None, eig_adapt=None,
                       timeout_ns=None, stream=None) -> GreedyResult:
    """Greedy rank-R approximation (Sec. 1, Example 3) with implicit deflation.
    u0: R x n_tot float32 initial guesses.  Synchronous."""
    d = _Desc(T, scales)
    n = n_tot(d.shape)
    u0 = u0.contiguous()
    if u0.dtype != torch.float32 or u0.shape != (R, n):
        raise ValueError("u0 must be float32 of shape (R, sum(dims))")
    rd = _Desc(refine) if refine is not None else None
    o = _opts(tol, max_iter, variant, eig_tol, eig_max_steps,
              rd.desc if rd is not None else None, switch_tol, timeout_ns, eig_adapt)
    u_out = torch.empty(R, n, device=T.device, dtype=torch.float32)
    sig = (ctypes.c_double * R)()
    infos = (Info * R)()
    res = (ctypes.c_double * (R + 1))()
    h = handle(T.device.index)
    st = _lib.load().hoscf_solve_greedy(h, ctypes.byref(d.desc), int(R),
                                        ctypes.c_void_p(u0.data_ptr()), ctypes.byref(o),
                                        ctypes.c_void_p(u_out.data_ptr()), sig, infos, res,
                                        _stream_ptr(stream))
    _check(st, h, allow=(0, _lib.HOSCF_NOT_CONVERGED))
    return GreedyResult([sig[i] for i in range(R)], u_out, d.shape,
                        [(infos[i].iters, infos[i].passes, infos[i].resid) for i in range(R)],
                        [res[i] for i in range(R + 1)], st == 0)


def hoscf_quantize(x: torch.Tensor, dtype: str, stream=None):
    """FP32 -> ("bf16": bfloat16 tensor), ("f16": float16 tensor) or ("fp8":
    uint8 e4m3 codes, float32 scales)."""
    x = x.contiguous()
    if x.dtype != torch.float32 or not x.is_cuda:
        raise ValueError("x must be a float32 CUDA tensor")
    n = x.numel()
    h = handle(x.device.index)
    if dtype == "bf16":
        q = torch.empty(x.shape, device=x.device, dtype=torch.bfloat16)
        _check(_lib.load().hoscf_quantize(h, ctypes.c_void_p(x.data_ptr()), n, _lib.HOSCF_BF16,
                                          ctypes.c_void_p(q.data_ptr()), None, _stream_ptr(stream)), h)
        return q, None
    if dtype == "f16":
        q = torch.empty(x.shape, device=x.device, dtype=torch.float16)
        _check(_lib.load().hoscf_quantize(h, ctypes.c_void_p(x.data_ptr()), n, _lib.HOSCF_F16,
                                          ctypes.c_void_p(q.data_ptr()), None, _stream_ptr(stream)), h)
        return q, None
    if dtype == "fp8":
        q = torch.empty(x.shape, device=x.device, dtype=torch.uint8)
        s = torch.empty((n + 127) // 128, device=x.device, dtype=torch.float32)
        _check(_lib.load().hoscf_quantize(h, ctypes.c_void_p(x.data_ptr()), n, _lib.HOSCF_F8E4M3,
                                          ctypes.c_void_p(q.data_ptr()),
                                          ctypes.c_void_p(s.data_ptr()), _stream_ptr(stream)), h)
        return q, s
    raise ValueError(dtype)


def hoscf_backward(T: torch.Tensor, u: torch.Tensor, sigma: float, grad_sigma: float,
                   grad_u: torch.Tensor | None = None, grad_T: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """dL/dT for L = grad_sigma*sigma + <grad_u, u> at a converged solution."""
    d = _Desc(T)
    u = u.contiguous()
    if grad_T is None:
        grad_T = torch.empty(d.shape, device=T.device, dtype=torch.float32)
    gu = grad_u.contiguous() if grad_u is not None else None
    h = handle(T.device.index)
    _check(_lib.load().hoscf_backward(h, ctypes.byref(d.desc), ctypes.c_void_p(u.data_ptr()),
                                      float(sigma), float(grad_sigma),
                                      ctypes.c_void_p(gu.data_ptr() if gu is not None else 0),
                                      ctypes.c_void_p(grad_T.data_ptr()), _stream_ptr(stream)), h)
    return grad_T


def _batch_descs(tensors):
    """The descriptor array of a batch, filled field by field with numpy (a
    Python object per tensor costs more than the whole launch at a thousand
    tensors).  Returns (array, dims buffer to keep alive)."""
    import numpy as np
    cnt = len(tensors)
    for T in tensors:
        if not (T.is_cuda and T.is_contiguous() and T.dtype == torch.float32):
            raise ValueError("batched tensors must be contiguous FP32 CUDA tensors")
    shapes = [tuple(T.shape) for T in tensors]
    if any(len(sh) not in (3, 4) for sh in shapes):
        raise ValueError("batched tensors have order 3 or 4")
    dims = np.array([sh + (0,) * (4 - len(sh)) for sh in shapes], dtype=np.int64).reshape(cnt, 4)
    orders = np.array([len(sh) for sh in shapes], dtype=np.int32)
    arr = (TensorDesc * cnt)()
    rec = np.ndarray((cnt,), dtype=np.dtype({
        "names": ["order", "dims", "dtype", "data", "scales"],
        "formats": [np.int32, np.uint64, np.int32, np.uint64, np.uint64],
        "offsets": [TensorDesc.order.offset, TensorDesc.dims.offset, TensorDesc.dtype.offset,
                    TensorDesc.data.offset, TensorDesc.scales.offset],
        "itemsize": ctypes.sizeof(TensorDesc)}), buffer=arr)
    rec["order"] = orders
    rec["dims"] = dims.ctypes.data + dims.strides[0] * np.arange(cnt, dtype=np.uint64)
    rec["dtype"] = _lib.HOSCF_F32
    rec["data"] = np.fromiter((T.data_ptr() for T in tensors), dtype=np.uint64, count=cnt)
    rec["scales"] = 0
    return arr, dims


def hoscf_solve_batched(tensors, u0s, tol=1e-6, max_iter=200, eig_tol=None, timeout_ns=None,
                        batch_threads=None, batch_faces=None, stream=None):
    """Many small independent F32 tensors (orders 3-4) in one persistent,
    graph-captured launch.  Returns (sigmas, factor tensors, infos, status);
    the factor tensors are views of one buffer."""
    import numpy as np
    cnt = len(tensors)
    if cnt == 0 or len(u0s) != cnt:
        raise ValueError("need one start vector per tensor, at least one tensor")
    arr, dims_keep = _batch_descs(tensors)
    u0c = [u.contiguous() for u in u0s]
    ns = [u.numel() for u in u0c]
    if ns != [sum(T.shape) for T in tensors]:
        raise ValueError("each start vector holds sum(dims) entries")
    flat = torch.empty(sum(ns), dtype=torch.float32, device=tensors[0].device)
    uo = list(flat.split(ns))
    offs = np.zeros(cnt, dtype=np.uint64)
    np.cumsum(np.asarray(ns[:-1], dtype=np.uint64) * 4, out=offs[1:])
    pin = (ctypes.c_void_p * cnt)()
    np.ndarray((cnt,), dtype=np.uint64, buffer=pin)[:] = [u.data_ptr() for u in u0c]
    pout = (ctypes.c_void_p * cnt)()
    np.ndarray((cnt,), dtype=np.uint64, buffer=pout)[:] = flat.data_ptr() + offs
    sig = (ctypes.c_double * cnt)()
    infos = (Info * cnt)()
    o = _opts(tol, max_iter, None, eig_tol, None, None, None, timeout_ns)
    if batch_threads is not None:
        o.batch_threads = int(batch_threads)
    if batch_faces is not None:
        o.batch_faces = int(batch_faces)
    dev = tensors[0].device.index
    h = handle(dev)
    st = _lib.load().hoscf_solve_batched(h, cnt, arr, pin, ctypes.byref(o), pout, sig, infos,
                                         _stream_ptr(stream))
    del dims_keep
    _check(st, h, allow=(0, _lib.HOSCF_NOT_CONVERGED))
    return list(sig), uo, list(infos), st


# ------------------------------------------------------------------ sharded form
def hoscf_create_handle(device: int = 0) -> ctypes.c_void_p:
    """A library handle of one's own (a handle serves one host thread and one
    stream at a time; the functions above share one handle per device).
    Release it with hoscf_destroy_handle."""
    h = ctypes.c_void_p()
    st = _lib.load().hoscf_create(ctypes.byref(h), int(device))
    if st != 0:
        raise HoscfError(st, f"hoscf_create(device={device}) failed")
    return h


def hoscf_destroy_handle(h: ctypes.c_void_p) -> None:
    _lib.load().hoscf_destroy(h)


def shard_rows(dim0: int, rank: int, world: int) -> tuple[int, int]:
    """(row0, rows): the contiguous slab of mode 1 that `rank` of `world`
    holds; the first dim0 % world ranks hold one row more.  Every rank holds
    at least one row."""
    dim0, rank, world = int(dim0), int(rank), int(world)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if dim0 < world:
        raise ValueError(f"mode 1 has {dim0} rows for {world} ranks (at least one row each)")
    base, more = divmod(dim0, world)
    return rank * base + min(rank, more), base + (1 if rank < more else 0)


def allreduce_blocks(t: torch.Tensor, group=None) -> None:
    """The sharded form's collective: SUM of the whole blocks over the ranks
    of `group`, in place (torch.distributed; NCCL for CUDA tensors)."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


class _DeviceView:
    """__cuda_array_interface__ of `count` float32 at a library device
    pointer, so torch can name the buffer without copying it."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f4",
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None, "stream": None}


def hoscf_ttvc_blocks_slab(T: torch.Tensor, row0: int, dim0: int, u: torch.Tensor,
                           H: torch.Tensor | None = None, scales=None, handle_=None,
                           stream=None) -> torch.Tensor:
    """This slab's contribution to the whole tensor's blocks (T = rows
    [row0, row0 + T.shape[0]) of mode 1 of a tensor with dim0 rows)."""
    d = _Desc(T, scales)
    full = (int(dim0),) + d.shape[1:]
    u = u.contiguous()
    if u.dtype != torch.float32 or u.numel() != n_tot(full):
        raise ValueError("u must be float32 with the whole tensor's sum(dims) entries")
    if H is None:
        H = torch.empty(n_blocks(full), device=T.device, dtype=torch.float32)
    h = handle_ if handle_ is not None else handle(T.device.index)
    _check(_lib.load().hoscf_ttvc_blocks_slab(h, ctypes.byref(d.desc), int(row0), int(dim0),
                                              ctypes.c_void_p(u.data_ptr()),
                                              ctypes.c_void_p(H.data_ptr()), _stream_ptr(stream)), h)
    return H


def hoscf_solve_sharded(T: torch.Tensor, row0: int, dim0: int, u0: torch.Tensor, reduce=None,
                        group=None, tol=1e-6, max_iter=200, variant="hoscf", eig_tol=None,
                        eig_max_steps=None, eig_adapt=None, scales=None,
                        refine: torch.Tensor | None = None, switch_tol=None, timeout_ns=None,
                        handle_=None, stream=None) -> SolveResult:
    """HOSCF on a tensor sharded by slabs of mode 1: T is this rank's slab
    (rows [row0, row0 + T.shape[0]) of dim0), u0 the whole initial guess.
    `reduce(t)` sums the whole blocks t over the ranks in place; by default
    allreduce_blocks over `group`.  Every rank gets the same result."""
    d = _Desc(T, scales)
    full = (int(dim0),) + d.shape[1:]
    n = n_tot(full)
    u0 = u0.contiguous()
    if u0.dtype != torch.float32 or u0.numel() != n:
        raise ValueError("u0 must be float32 with the whole tensor's sum(dims) entries")
    rd = _Desc(refine) if refine is not None else None
    o = _opts(tol, max_iter, variant, eig_tol, eig_max_steps,
              rd.desc if rd is not None else None, switch_tol, timeout_ns, eig_adapt)
    fn = reduce if reduce is not None else (lambda t: allreduce_blocks(t, group))
    dev = T.device
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    errors = []

    def _cb(hptr, count, stream_ptr, user):
        try:
            with torch.cuda.stream(s):
                fn(torch.as_tensor(_DeviceView(hptr, count), device=dev))
            return 0
        except BaseException as exc:   # reported after the call returns
            errors.append(exc)
            return 1

    cb = _lib.REDUCE_FN(_cb)
    sh = _lib.Shard(int(row0), int(dim0), cb, None)
    u_out = torch.empty(n, device=dev, dtype=torch.float32)
    sigma = ctypes.c_double()
    info = Info()
    h = handle_ if handle_ is not None else handle(dev.index)
    st = _lib.load().hoscf_solve_sharded(h, ctypes.byref(d.desc), ctypes.byref(sh),
                                         ctypes.c_void_p(u0.data_ptr()), ctypes.byref(o),
                                         ctypes.c_void_p(u_out.data_ptr()), ctypes.byref(sigma),
                                         ctypes.byref(info), ctypes.c_void_p(s.cuda_stream))
    if errors:
        raise errors[0]
    _check(st, h, allow=(0, _lib.HOSCF_NOT_CONVERGED))
    return SolveResult(sigma.value, u_out, full, info.iters, info.passes, info.passes_refine,
                       info.rqi_accepts, info.resid, info.resid_4_1, info.sigma_raw, st == 0)
