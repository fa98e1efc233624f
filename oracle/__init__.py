"""FP64 CPU oracle for HOSCF / iHOSCF (best rank-one approximation, arXiv 2403.01778).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import, call or link anything
under ``oracle/``.  The product path (``paper_2403_01778_gb300``) never does,
and this module imports nothing from it: the two share no code.

Everything here is a plain, slow, obviously correct restatement of the paper
in FP64.  The heavy loops (eq. (3.3) blocks, eq. (2.4) KKT vectors) live in
``hoscf_ref.c``; the driver loop, the dense eigen-solve and the linear solves
use numpy/scipy routines as single steps.

What each function follows
--------------------------
``blocks``                eq. (3.3): A_{m,n}(x) = A x_{k!=m,n} u^(k), all m<n.
``nepv_matrix``           eq. (3.2): J(x) = (1/(d-1)) [[0, A_12, ...], ...].
``largest_magnitude_eigpair``  Alg. 1 line 5 (largest *magnitude*, Sec. 4.1).
``kkt_from_blocks``       eq. (2.4) with g_n = (1/(d-1)) sum_{m!=n} A_{n,m} u^(m),
                          i.e. g = sqrt(d) J(x) x for the balanced x = [u]/sqrt(d).
``hoscf``                 Algorithm 1 (lines 1-15) with the readings below.
``rqi_step``              Sec. 4.4 (iHOSCF), reading below.  The step is pinned
                          (the spectral form in a known eigenbasis, the order-2
                          block case, cubic convergence); the acceptance rule of
                          the iHOSCF loop (keep y when its pass certifies or
                          |sigma(y)| >= |sigma(x_k)|) by steps made to return a
                          certified point, an uncertified point of larger
                          |sigma|, and a point of smaller |sigma| (then the loop
                          must reproduce plain HOSCF's iterates).
``hopm``                  the HOPM (ALS) baseline named in Sec. 1 / Sec. 6.1,
                          used as an independent cross-check only.
``asvd``                  the ASVD comparison method of Sec. 1 (d = 2, 3): two
                          factors at a time from the largest singular pair of
                          the coupling block of the two free modes, Gauss-Seidel
                          over the fixed mode.
``greedy``                the greedy rank-one update of Sec. 1 / Example 3:
                          B^(r) = best rank-one approximation of A^(r),
                          A^(r+1) = A^(r) - B^(r), A^(1) = A; the deflated tensor
                          is formed explicitly (the definition).
``adjoint``               not in the paper: the implicit-function adjoint of the
                          KKT system (2.4), checked against finite differences.
``quantize_*``            not in the paper: BF16 and IEEE FP16 (round to nearest even) and
                          FP8-e4m3 (per-128-element FP32 scales, saturating,
                          round to nearest even) storage, from the formats'
                          definitions.

Readings of the paper (where it is silent, ambiguous or garbled)
----------------------------------------------------------------
* Stopping rule: eq. (4.1) evaluated literally at (J_{k-1}, x_k) is ~0 at every
  step (x_k is an eigenvector of J_{k-1}).  The oracle certifies the point
  where the blocks were built: r = ||g - sigma u||_2 / |sigma| with
  sigma = mean_n <u_n, g_n>, and returns that iterate.  Eq. (4.1) at the new
  point is reported too (``residual_4_1``).
* Largest-magnitude ties (d = 2 has a symmetric spectrum): the positive
  eigenvalue wins.
* Eigenvector sign: chosen so that <x_k, x_{k-1}> >= 0 (x_{k-1} balanced).
* Gauge: after Alg. 1 lines 12-15, pairs (u^(1), u^(n)) are flipped so that the
  largest-|.| entry of u^(n) (lowest index on ties) is positive for n >= 2;
  sigma stays >= 0.
* iHOSCF: taken literally (rho_k and the RQI from x_k with J_{k-1}) the step is
  singular, because x_k is an eigenvector of J_{k-1}.  The default reading
  ("ihoscf") builds J(x_k) at the new point (one more pass) and runs the RQI
  rho = x~^T J x~, y = (J - rho I)^{-1} x~ from the block-balanced
  x~ = [u_k^(n)]/sqrt(d), normalised and sign-aligned with x~; y is kept when
  its own pass certifies convergence or |sigma(y)| >= |sigma(x_k)| ("only if
  lambda increases"), else x_k is kept.  The other reading ("ihoscf_prev")
  uses J_{k-1}; one RQI step from x~_k then lands back on x_k (to third
  order), so it tracks plain HOSCF iteration for iteration.
* Initial guess: each block of x0 is normalised; a zero block is an error.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hoscf_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhoscf_ref.so")
_lib = None

_I64P = ctypes.POINTER(ctypes.c_int64)
_F64P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile hoscf_ref.c with gcc (plain C99 + OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                        _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i = ctypes.c_void_p, ctypes.c_int
        lib.ref_blocks.argtypes = [vp, i, i, _I64P, _F64P, _F64P, i]
        lib.ref_block_entry.argtypes = [vp, i, i, _I64P, _F64P, i, i,
                                        ctypes.c_int64, ctypes.c_int64, _F64P]
        lib.ref_block_entry_fast.argtypes = lib.ref_block_entry.argtypes
        lib.ref_kkt_vectors.argtypes = [vp, i, i, _I64P, _F64P, _F64P, _F64P, i]
        lib.ref_ttv.argtypes = [vp, i, i, _I64P, i, _F64P, _F64P]
        lib.ref_grad_tensor.argtypes = [i, _I64P, _F64P, _F64P, ctypes.c_double, _F64P]
        for f in (lib.ref_blocks, lib.ref_block_entry, lib.ref_block_entry_fast,
                  lib.ref_kkt_vectors, lib.ref_ttv, lib.ref_grad_tensor):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


# ---------------------------------------------------------------- helpers
def _tensor_arg(T):
    T = np.ascontiguousarray(T)
    if T.dtype == np.float32:
        return T, 0
    if T.dtype == np.float64:
        return T, 1
    raise TypeError(f"oracle tensors are float32 or float64, got {T.dtype}")


def _dims_arg(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int64))


def _p(a, typ):
    return a.ctypes.data_as(typ)


def block_pairs(d: int):
    """(m, n) pairs with m < n in the packed (lexicographic) order."""
    return [(m, n) for m in range(d) for n in range(m + 1, d)]


def block_offsets(dims):
    offs, p = [], 0
    for m, n in block_pairs(len(dims)):
        offs.append(p)
        p += dims[m] * dims[n]
    return offs, p


def mode_offsets(dims):
    return np.concatenate([[0], np.cumsum(dims)]).astype(np.int64)


def concat(u_list):
    return np.concatenate([np.asarray(v, dtype=np.float64).ravel() for v in u_list])


def split(x, dims):
    off = mode_offsets(dims)
    return [np.array(x[off[k]:off[k + 1]], dtype=np.float64) for k in range(len(dims))]


# ----------------------------------------------------------- eq. (3.3)
def blocks(T, u_list, nthreads: int = 0) -> np.ndarray:
    """All coupling blocks A_{m,n} (m<n), packed, FP64 (eq. 3.3)."""
    T, dt = _tensor_arg(T)
    dims = _dims_arg(T.shape)
    u = np.ascontiguousarray(concat(u_list))
    _, P = block_offsets(list(T.shape))
    H = np.empty(P, dtype=np.float64)
    rc = _load().ref_blocks(T.ctypes.data, dt, T.ndim, _p(dims, _I64P), _p(u, _F64P),
                            _p(H, _F64P), int(nthreads))
    if rc:
        raise ValueError(f"ref_blocks failed ({rc})")
    return H


def unpack_blocks(Hp, dims):
    offs, _ = block_offsets(dims)
    return {(m, n): Hp[o:o + dims[m] * dims[n]].reshape(dims[m], dims[n])
            for (m, n), o in zip(block_pairs(len(dims)), offs)}


def block_entry(T, u_list, m, n, i, j, fast: bool = True) -> float:
    """One entry A_{m,n}[i, j] by its definition (eq. 3.3)."""
    T, dt = _tensor_arg(T)
    dims = _dims_arg(T.shape)
    u = np.ascontiguousarray(concat(u_list))
    out = ctypes.c_double()
    fn = _load().ref_block_entry_fast if fast else _load().ref_block_entry
    rc = fn(T.ctypes.data, dt, T.ndim, _p(dims, _I64P), _p(u, _F64P), int(m), int(n),
            int(i), int(j), ctypes.byref(out))
    if rc:
        raise ValueError("ref_block_entry failed")
    return out.value


def kkt_vectors(T, u_list, nthreads: int = 0):
    """g_n = A x_{k!=n} u^(k) for all n and the full contraction (eq. 2.4)."""
    T, dt = _tensor_arg(T)
    dims = _dims_arg(T.shape)
    u = np.ascontiguousarray(concat(u_list))
    g = np.empty_like(u)
    full = ctypes.c_double()
    rc = _load().ref_kkt_vectors(T.ctypes.data, dt, T.ndim, _p(dims, _I64P), _p(u, _F64P),
                                 _p(g, _F64P), ctypes.byref(full), int(nthreads))
    if rc:
        raise ValueError("ref_kkt_vectors failed")
    return split(g, list(T.shape)), full.value


def ttv(T, n, v):
    """A x_n v (Sec. 2), FP64, shape = T.shape without mode n."""
    T, dt = _tensor_arg(T)
    dims = _dims_arg(T.shape)
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    shape = [s for k, s in enumerate(T.shape) if k != n]
    out = np.empty(int(np.prod(shape)), dtype=np.float64)
    rc = _load().ref_ttv(T.ctypes.data, dt, T.ndim, _p(dims, _I64P), int(n), _p(v, _F64P),
                         _p(out, _F64P))
    if rc:
        raise ValueError("ref_ttv failed")
    return out.reshape(shape)


# ----------------------------------------------------------- eq. (3.2)
def full_block_matrix(Hp, dims) -> np.ndarray:
    """The symmetric block matrix with A_{m,n} off the diagonal, zero diagonal
    blocks; J(x) of eq. (3.2) is this divided by (d - 1)."""
    d = len(dims)
    off = mode_offsets(dims)
    n_tot = int(off[-1])
    M = np.zeros((n_tot, n_tot))
    for (m, n), B in unpack_blocks(Hp, dims).items():
        M[off[m]:off[m + 1], off[n]:off[n + 1]] = B
        M[off[n]:off[n + 1], off[m]:off[m + 1]] = B.T
    return M


def nepv_matrix(Hp, dims) -> np.ndarray:
    return full_block_matrix(Hp, dims) / (len(dims) - 1)


def largest_magnitude_eigpair(J, x_prev=None, dense_max: int = 4096):
    """Largest-magnitude eigenpair of a symmetric matrix (Alg. 1 line 5).

    Ties between +l and -l go to the positive one.  The eigenvector is unit
    length with <x, x_prev> >= 0 when x_prev is given.  Matrices of order up
    to `dense_max` use LAPACK's dense eigh; larger ones ARPACK (both ends of
    the spectrum)."""
    n = J.shape[0]
    if n <= dense_max:
        w, V = np.linalg.eigh(J)
        lo, hi = 0, n - 1
        k = hi if w[hi] >= -w[lo] else lo
        lam, x = float(w[k]), V[:, k].copy()
    else:  # large n: ARPACK on the dense matrix, both spectrum ends
        from scipy.sparse.linalg import eigsh
        v0 = None if x_prev is None else np.asarray(x_prev, dtype=np.float64)
        wa, Va = eigsh(J, k=1, which="LA", v0=v0, tol=1e-14)
        ws, Vs = eigsh(J, k=1, which="SA", v0=v0, tol=1e-14)
        if wa[0] >= -ws[0]:
            lam, x = float(wa[0]), Va[:, 0].copy()
        else:
            lam, x = float(ws[0]), Vs[:, 0].copy()
    x /= np.linalg.norm(x)
    if x_prev is not None and float(np.dot(x, x_prev)) < 0:
        x = -x
    return lam, x


# ----------------------------------------------------------- eq. (2.4)
def kkt_from_blocks(Hp, dims, u_list):
    """g_n = (1/(d-1)) sum_{m != n} A_{n,m} u^(m); sigma = mean_n <u_n, g_n>;
    r = ||g - sigma u||_2 / |sigma| (stacked 2-norm)."""
    d = len(dims)
    M = full_block_matrix(Hp, dims)
    u = concat(u_list)
    g = M @ u / (d - 1)
    gs, us = split(g, dims), split(u, dims)
    sig_n = np.array([float(np.dot(a, b)) for a, b in zip(us, gs)])
    sigma = float(sig_n.mean())
    r = float(np.linalg.norm(g - sigma * u) / abs(sigma)) if sigma != 0 else float("inf")
    return gs, sigma, r


def residual_4_1(Hp, dims, u_list):
    """Eq. (4.1) evaluated at the point where J was built: x = [u]/sqrt(d),
    rho = x^T J x, ||J x - rho x|| / (||J||_F + |rho|)."""
    J = nepv_matrix(Hp, dims)
    x = concat(u_list) / np.sqrt(len(dims))
    Jx = J @ x
    rho = float(x @ Jx)
    return float(np.linalg.norm(Jx - rho * x) / (np.linalg.norm(J) + abs(rho)))


def normalise_blocks(x, dims):
    """u^(n) = x_{index_n} / ||x_{index_n}|| (eq. 3.4 / Alg. 1 lines 6-9);
    a zero block stays zero, as eq. (3.4) prescribes."""
    out = []
    for v in split(x, dims):
        nv = np.linalg.norm(v)
        out.append(v / nv if nv != 0 else np.zeros_like(v))
    return out


def final_fix(sigma, u_list):
    """Alg. 1 lines 12-15: if lambda < 0, negate it and u^(1)."""
    u = [v.copy() for v in u_list]
    if sigma < 0:
        sigma = -sigma
        u[0] = -u[0]
    return sigma, u


def gauge(sigma, u_list):
    """Sign gauge (reading): for n >= 2 make the largest-|.| entry of u^(n)
    positive (lowest index on ties), flipping u^(1) along with it."""
    u = [v.copy() for v in u_list]
    for n in range(1, len(u)):
        k = int(np.argmax(np.abs(u[n])))
        if u[n][k] < 0:
            u[n] = -u[n]
            u[0] = -u[0]
    return sigma, u


# ----------------------------------------------------------- Algorithm 1
@dataclass
class Result:
    sigma: float
    u: list
    iters: int            # eigen steps taken (Alg. 1 loop trips)
    passes: int           # block constructions (line 4), incl. the certifying one
    resid: float          # KKT residual at the returned point
    converged: bool
    history: list = field(default_factory=list)   # (sigma, r) per pass
    rqi_accepts: int = 0
    resid_4_1: float = float("nan")


def _unit_blocks(u0_list):
    u = []
    for v in u0_list:
        v = np.asarray(v, dtype=np.float64).ravel()
        nv = np.linalg.norm(v)
        if not np.isfinite(nv) or nv == 0:
            raise ValueError("initial guess has a zero or non-finite block")
        u.append(v / nv)
    return u


def rqi_step(J, u_list, dims):
    """One Rayleigh-quotient iteration (Sec. 4.4) on the balanced x~ = [u]/sqrt(d)."""
    d = len(dims)
    xt = concat(u_list) / np.sqrt(d)
    rho = float(xt @ (J @ xt)) / float(xt @ xt)
    y = np.linalg.solve(J - rho * np.eye(J.shape[0]), xt)
    y /= np.linalg.norm(y)
    if float(y @ xt) < 0:
        y = -y
    return normalise_blocks(y, dims), rho


def hoscf(T, u0_list, tol: float = 1e-8, max_iter: int = 200, variant: str = "hoscf",
          nthreads: int = 0, keep_history: bool = True) -> Result:
    """HOSCF (Algorithm 1) and iHOSCF (Sec. 4.4) in FP64 with the readings above.

    variant = "hoscf": Algorithm 1.
    variant = "ihoscf": after line 5, build J at the new point x_k (one more
        pass) and run one RQI step with it from the balanced x~_k; the RQI
        iterate y is kept if its pass certifies convergence or
        |sigma(y)| >= |sigma(x_k)|, else x_k (whose blocks are already built)
        is kept.
    variant = "ihoscf_prev": the RQI step uses J_{k-1} (the matrix line 5 just
        used); y is kept if certified or |sigma(y)| >= |sigma(x_{k-1})|, else
        x_k is restored with one extra pass.  (One RQI step from x~_k with
        J_{k-1} returns x_k up to third-order terms, so this variant tracks
        plain HOSCF.)
    variant = "jacobi_hopm": the Jacobi form of HOPM the paper compares with
        (Sec. 1, Sec. 6.1): every factor at once from the previous iterate,
        u^(n) <- A x_{k!=n} u^(k) / ||.|| = g_n / ||g_n||, g_n read off the
        blocks; same certificate and stopping rule as HOSCF."""
    dims = list(T.shape)
    d = len(dims)
    if d < 2:
        raise ValueError("order must be >= 2")
    if variant not in ("hoscf", "ihoscf", "ihoscf_prev", "jacobi_hopm"):
        raise ValueError(variant)
    u = _unit_blocks(u0_list)
    hist = []
    iters = passes = accepts = 0

    def build(uu):
        nonlocal passes
        Hq = blocks(T, uu, nthreads)                      # line 4
        passes += 1
        _, sg, rr = kkt_from_blocks(Hq, dims, uu)
        if keep_history:
            hist.append((sg, rr))
        return Hq, sg, rr

    Hp, sigma, r = build(u)
    while not (r <= tol or iters >= max_iter):
        if variant == "jacobi_hopm":
            g, _, _ = kkt_from_blocks(Hp, dims, u)
            nrm = [np.linalg.norm(gn) for gn in g]
            if min(nrm) == 0.0:
                raise ZeroDivisionError("a factor's update A x_{k!=n} u^(k) is zero")
            u = [gn / nn for gn, nn in zip(g, nrm)]
            iters += 1
            Hp, sigma, r = build(u)
            continue
        J = nepv_matrix(Hp, dims)
        _, x = largest_magnitude_eigpair(J, concat(u) / np.sqrt(d))   # line 5
        u_k = normalise_blocks(x, dims)                   # lines 6-9
        iters += 1
        if variant == "hoscf":
            u = u_k
            Hp, sigma, r = build(u)
        elif variant == "ihoscf_prev":
            u_y, _ = rqi_step(J, u_k, dims)
            Hy, sy, ry = build(u_y)
            if ry <= tol or abs(sy) >= abs(sigma):
                u, Hp, sigma, r = u_y, Hy, sy, ry
                accepts += 1
            else:
                u = u_k
                Hp, sigma, r = build(u)
        else:
            Hk, sk, rk = build(u_k)
            if rk <= tol:
                u, Hp, sigma, r = u_k, Hk, sk, rk
                break
            u_y, _ = rqi_step(nepv_matrix(Hk, dims), u_k, dims)
            Hy, sy, ry = build(u_y)
            if ry <= tol or abs(sy) >= abs(sk):
                u, Hp, sigma, r = u_y, Hy, sy, ry
                accepts += 1
            else:
                u, Hp, sigma, r = u_k, Hk, sk, rk
    r41 = residual_4_1(Hp, dims, u)
    sigma_f, u_f = gauge(*final_fix(sigma, u))            # lines 12-15 + gauge
    return Result(sigma_f, u_f, iters, passes, r, r <= tol, hist, accepts, r41)


def asvd(T, u0_list, tol: float = 1e-8, max_iter: int = 500, nthreads: int = 0,
         keep_history: bool = True) -> Result:
    """ASVD, the alternating-SVD comparison method of Sec. 1, for d = 3 (and
    the degenerate d = 2, where it is one SVD).

    A Gauss-Seidel sweep over the fixed mode f = 1, 2, 3, 1, ...: with u^(f)
    fixed, the other two factors (m, n) become the largest singular pair of
    the intermediate matrix A x_f u^(f), which is the coupling block A_{m,n}
    of eq. (3.3).  Reading for the sign: (a, b) with a^T A_{m,n} b = +s_1, the
    pair negated together when <a, u^(m)> + <b, u^(n)> < 0.  One sub-step is
    one eigen step (iters); the blocks at every new point are one pass, and
    the certificate and stopping rule are HOSCF's (KKT residual at the point
    the blocks were built for)."""
    dims = list(T.shape)
    d = len(dims)
    if d not in (2, 3):
        raise ValueError("ASVD is defined here for orders 2 and 3")
    u = _unit_blocks(u0_list)
    hist = []
    iters = passes = 0

    def build(uu):
        nonlocal passes
        Hq = blocks(T, uu, nthreads)
        passes += 1
        _, sg, rr = kkt_from_blocks(Hq, dims, uu)
        if keep_history:
            hist.append((sg, rr))
        return Hq, sg, rr

    Hp, sigma, r = build(u)
    while not (r <= tol or iters >= max_iter):
        if d == 2:
            m, n = 0, 1
        else:
            f = iters % 3
            m, n = [k for k in range(3) if k != f]
        B = unpack_blocks(Hp, dims)[(m, n)]
        U, S, Vt = np.linalg.svd(B)
        a, b = U[:, 0].copy(), Vt[0].copy()
        if float(a @ u[m]) + float(b @ u[n]) < 0:
            a, b = -a, -b
        u = list(u)
        u[m], u[n] = a, b
        iters += 1
        Hp, sigma, r = build(u)
    r41 = residual_4_1(Hp, dims, u)
    sigma_f, u_f = gauge(*final_fix(sigma, u))
    return Result(sigma_f, u_f, iters, passes, r, r <= tol, hist, 0, r41)


def hopm(T, u0_list, tol: float = 1e-10, max_iter: int = 2000):
    """HOPM / ALS (Gauss-Seidel): u^(n) <- A x_{k!=n} u^(k), normalised, one mode
    at a time.  Cross-check baseline only."""
    dims = list(T.shape)
    u = _unit_blocks(u0_list)
    sigma = 0.0
    for it in range(max_iter):
        for n in range(len(dims)):
            g, _ = kkt_vectors(T, u)
            gn = g[n]
            u[n] = gn / np.linalg.norm(gn)
        g, sigma = kkt_vectors(T, u)
        r = np.linalg.norm(concat(g) - sigma * concat(u)) / abs(sigma)
        if r <= tol:
            break
    return gauge(*final_fix(sigma, u))


# ----------------------------------------------------------- greedy rank-R
class GreedyResult:
    def __init__(self, sigmas, factors, results, res):
        self.sigmas = sigmas      # sigma_r of each rank-one term B^(r)
        self.factors = factors    # [r][n] unit factor vectors
        self.results = results    # per-term Result of the rank-one solve
        self.res = res            # ||A^(r)||_F / ||A||_F for r = 1 .. R+1


def greedy(T, R: int, u0_lists, tol: float = 1e-8, max_iter: int = 500,
           variant: str = "hoscf") -> GreedyResult:
    """Greedy rank-one update (Sec. 1, Example 3): for r = 1..R, B^(r) =
    sigma_r u_1^(r) o ... o u_d^(r) is the best rank-one approximation of A^(r)
    (by ``hoscf`` from u0_lists[r-1]), and A^(r+1) = A^(r) - B^(r) is formed
    explicitly.  res[r-1] = ||A^(r)||_F / ||A^(1)||_F."""
    A = np.array(T, dtype=np.float64)
    n0 = float(np.linalg.norm(A))
    sig, fac, runs, res = [], [], [], [float(np.linalg.norm(A)) / n0]
    for r in range(R):
        out = hoscf(A, u0_lists[r], tol=tol, max_iter=max_iter, variant=variant)
        B = out.sigma
        for v in out.u:
            B = np.multiply.outer(B, v)
        A = A - B
        sig.append(out.sigma)
        fac.append(out.u)
        runs.append(out)
        res.append(float(np.linalg.norm(A)) / n0)
    return GreedyResult(sig, fac, runs, res)


# ----------------------------------------------------------- adjoint
def adjoint(T, u_list, sigma, c=1.0, w_list=None):
    """Gradient of L = c*sigma + sum_n <w_n, u_n> w.r.t. the tensor at a
    converged rank-one solution.

    Linearising the KKT system g_n(T, u) = mu_n u_n, ||u_n|| = 1 gives
      (H - sigma I) du - U dmu = -b,  U^T du = 0,  b_n = dT x_{k!=n} u_k,
    with H the full symmetric block matrix (blocks A_{n,m}) and U = blockdiag(u_n).
    The adjoint solves M [a; nu] = [w; 0], M = [[H - sigma I, -U], [-U^T, 0]],
    and dL/dT = c * u1 o ... o ud - sum_n u1 o ... o a_n o ... o ud."""
    dims = list(T.shape)
    d = len(dims)
    n_tot = sum(dims)
    off = mode_offsets(dims)
    Hp = blocks(T, u_list)
    Hf = full_block_matrix(Hp, dims)
    if w_list is None:
        a = np.zeros(n_tot)
        nu = np.zeros(d)
    else:
        U = np.zeros((n_tot, d))
        for k in range(d):
            U[off[k]:off[k + 1], k] = u_list[k]
        M = np.zeros((n_tot + d, n_tot + d))
        M[:n_tot, :n_tot] = Hf - sigma * np.eye(n_tot)
        M[:n_tot, n_tot:] = -U
        M[n_tot:, :n_tot] = -U.T
        rhs = np.concatenate([concat(w_list), np.zeros(d)])
        sol = np.linalg.solve(M, rhs)
        a, nu = sol[:n_tot], sol[n_tot:]
    dims_a = _dims_arg(dims)
    u = np.ascontiguousarray(concat(u_list))
    a = np.ascontiguousarray(a)
    out = np.empty(int(np.prod(dims)), dtype=np.float64)
    rc = _load().ref_grad_tensor(d, _p(dims_a, _I64P), _p(u, _F64P), _p(a, _F64P),
                                 float(c), _p(out, _F64P))
    if rc:
        raise ValueError("ref_grad_tensor failed")
    return out.reshape(dims), split(a, dims), nu


# ----------------------------------------------------------- storage formats
def quantize_bf16(x) -> np.ndarray:
    """FP32 -> BF16 bit patterns (uint16), round to nearest, ties to even.

    Candidates are the truncation toward zero and the next pattern away from
    zero; the nearer one in exact (FP64) arithmetic wins, ties go to the
    pattern whose last kept bit is 0.  The pattern after the largest finite
    one is infinity, whose distance is measured from 2^128 (the value the
    exponent range would give it).  Inputs must be finite."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if not np.all(np.isfinite(x)):
        raise ValueError("quantize_bf16 expects finite inputs")
    bits = x.view(np.uint32).astype(np.uint64)
    lo = bits & 0xFFFF0000
    hi = lo + 0x10000
    xv = np.abs(x.astype(np.float64))
    lov = np.abs((lo.astype(np.uint32)).view(np.float32).astype(np.float64))
    hi_is_inf = (hi & 0x7FFFFFFF) == 0x7F800000
    with np.errstate(over="ignore", invalid="ignore"):
        hiv = np.abs((hi.astype(np.uint32)).view(np.float32).astype(np.float64))
    hiv = np.where(hi_is_inf, 2.0 ** 128, hiv)
    dlo = xv - lov
    dhi = hiv - xv
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (((lo >> 16) & 1) == 1))
    return (np.where(pick_hi, hi, lo) >> 16).astype(np.uint16)


def dequantize_bf16(q) -> np.ndarray:
    q = np.asarray(q, dtype=np.uint16).astype(np.uint32) << 16
    return q.view(np.float32).astype(np.float64)


def f16_table() -> np.ndarray:
    """Value of each of the 65536 IEEE binary16 patterns: 1 sign bit, 5
    exponent bits (bias 15), 10 mantissa bits; exponent 0 = subnormal
    (m / 1024) 2^-14, exponent 31 = infinity (m = 0) or NaN."""
    code = np.arange(65536, dtype=np.int64)
    s = np.where(code & 0x8000, -1.0, 1.0)
    e = (code >> 10) & 0x1F
    m = (code & 0x3FF).astype(np.float64)
    val = np.where(e == 0, (m / 1024.0) * 2.0 ** -14, (1.0 + m / 1024.0) * 2.0 ** (e - 15.0))
    val = np.where(e == 31, np.where(m == 0, np.inf, np.nan), val)
    return s * val


def quantize_f16(x) -> np.ndarray:
    """FP32 -> IEEE binary16 bit patterns (uint16), round to nearest, ties to
    even: the nearer of the two patterns around |x| in exact (FP64)
    arithmetic, the even one (mantissa's last bit 0) on a tie.  Past the
    largest finite value 65504 the next pattern is infinity, whose distance
    is measured from 2^16 (the value the exponent range would give it), so
    |x| >= 65520 rounds to infinity.  Inputs must be finite."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    if not np.all(np.isfinite(x)):
        raise ValueError("quantize_f16 expects finite inputs")
    pos = f16_table()[:0x7C01].copy()       # codes 0x0000 .. 0x7C00 (+inf), increasing
    pos[0x7C00] = 2.0 ** 16
    a = np.abs(x)
    k = np.clip(np.searchsorted(pos, a, side="left"), 1, 0x7C00)   # pos[k-1] < a <= pos[k]
    lo, hi = pos[k - 1], pos[k]
    dlo, dhi = a - lo, hi - a
    take_hi = (hi == a) | (dhi < dlo) | ((dhi == dlo) & ((k & 1) == 0))
    code = np.where(a == 0, 0, np.where(take_hi, k, k - 1))
    return (code | np.where(np.signbit(x), 0x8000, 0)).astype(np.uint16)


def dequantize_f16(q) -> np.ndarray:
    return f16_table()[np.asarray(q, dtype=np.uint16).astype(np.int64)]


def e4m3_table() -> np.ndarray:
    """Value of each of the 256 FP8-e4m3 (fn variant) codes: 1 sign bit, 4
    exponent bits (bias 7), 3 mantissa bits, no infinities, S.1111.111 = NaN."""
    vals = np.empty(256)
    for code in range(256):
        s = -1.0 if code & 0x80 else 1.0
        e = (code >> 3) & 0xF
        m = code & 0x7
        if e == 0xF and m == 0x7:
            vals[code] = np.nan
        elif e == 0:
            vals[code] = s * (m / 8.0) * 2.0 ** (1 - 7)
        else:
            vals[code] = s * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return vals


def _e4m3_round(y64):
    """Nearest e4m3 code of each value (ties to the even mantissa), saturating
    at +-448; the sign bit is the sign bit of the input (so -0 -> 0x80)."""
    y64 = np.asarray(y64, dtype=np.float64)
    if not np.all(np.isfinite(y64)):
        raise ValueError("e4m3 rounding expects finite inputs")
    pos_vals = e4m3_table()[:0x7F]            # codes 0x00..0x7E, increasing
    a = np.minimum(np.abs(y64), 448.0)
    k = np.searchsorted(pos_vals, a, side="left")   # pos_vals[k-1] < a <= pos_vals[k]
    km1 = np.maximum(k - 1, 0)
    below, above = pos_vals[km1], pos_vals[k]
    db, da = a - below, above - a
    take_above = (above == a) | (da < db) | ((da == db) & ((k & 1) == 0))
    code = np.where(take_above, k, km1)
    sign = np.where(np.signbit(y64), 0x80, 0)
    return (code | sign).astype(np.uint8)


def quantize_e4m3_scaled(x, group: int = 128):
    """FP32 tensor -> (e4m3 codes, FP32 scales), one scale per `group`
    consecutive elements of the flat (row-major) order.

    scale = fp32(amax / 448) (1 if the group is all zero); y = fp32(x / scale);
    code = nearest e4m3 of y with saturation.  Both divisions are single
    correctly rounded FP32 operations, so the codes are reproducible exactly."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).ravel()
    N = x.size
    G = (N + group - 1) // group
    pad = np.zeros(G * group, dtype=np.float32)
    pad[:N] = x
    amax = np.abs(pad.reshape(G, group)).max(axis=1).astype(np.float32)
    scale = (amax / np.float32(448.0)).astype(np.float32)
    scale = np.where(amax == 0, np.float32(1.0), scale).astype(np.float32)
    y = (pad.reshape(G, group) / scale[:, None]).astype(np.float32).ravel()[:N]
    return _e4m3_round(y.astype(np.float64)), scale


def dequantize_e4m3_scaled(codes, scales, group: int = 128) -> np.ndarray:
    """Exact FP64 value of code * scale for each element."""
    codes = np.asarray(codes, dtype=np.uint8).ravel()
    tab = e4m3_table()
    s = np.repeat(np.asarray(scales, dtype=np.float64), group)[:codes.size]
    return tab[codes] * s
