"""Comparison helpers shared by the GPU tests.

Solutions are compared WITH their signs.  Both sides apply Algorithm 1's
final fix (lines 12-15: sigma >= 0, carried by u^(1)) and the sign gauge (for
n >= 2 the largest-|.| entry of u^(n), lowest index on ties, is positive, the
flip carried by u^(1)), so the factors are fixed exactly, not up to sign.

The one place where the data may not fix a sign is a mode whose two largest
|entries| are closer together than the entry-wise difference of the two
solutions: there FP32 and FP64 may legitimately pick different entries as
"largest".  For such a mode the sign is compared up to a flip; the product of
all the signs (the sign of the rank-one term sigma u1 o ... o ud itself) is
still checked, so a final fix that flips the wrong factor pair fails."""
import numpy as np


def as_np(v):
    if hasattr(v, "detach"):
        return v.detach().double().cpu().numpy()
    return np.asarray(v, dtype=np.float64)


def check_gauge(u_list, sigma):
    """The returned point satisfies the final fix and the gauge on its own."""
    assert sigma >= 0.0, sigma
    for n, u in enumerate(u_list):
        if n == 0:
            continue
        u = as_np(u)
        k = int(np.argmax(np.abs(u)))        # first maximum = lowest index on ties
        assert u[k] >= 0.0, (n, k, u[k])


def assert_same_solution(sigma, u_list, sigma_ref, u_ref, tol=1e-5, sigma_atol=None):
    """sigma within tol (relative; or within sigma_atol when given); every
    factor within |1 - <u, u_ref>| <= tol with the sign the gauge fixes; the
    rank-one term's sign equal."""
    check_gauge(u_list, sigma)
    s_tol = tol * abs(sigma_ref) if sigma_atol is None else sigma_atol
    assert abs(sigma - sigma_ref) <= s_tol, (sigma, sigma_ref)
    signs = []
    for n, (u, r) in enumerate(zip(u_list, u_ref)):
        u, r = as_np(u), as_np(r)
        c = float(u @ r)
        assert abs(1.0 - abs(c)) <= tol, (n, c)
        s = 1.0 if c >= 0 else -1.0
        signs.append(s)
        if n >= 1:
            a = np.sort(np.abs(r))[::-1]
            err = float(np.max(np.abs(u - s * r)))
            if a.size == 1 or a[0] - a[1] > 2.0 * err:
                assert s > 0, f"mode {n}: the gauge fixes this factor's sign and it differs"
    assert np.prod(signs) > 0, f"the rank-one term has the opposite sign ({signs})"


def split(u, dims):
    out, o = [], 0
    for n in dims:
        out.append(u[o:o + n])
        o += n
    return out
