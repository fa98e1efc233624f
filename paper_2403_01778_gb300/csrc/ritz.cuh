// Small symmetric tridiagonal problems of the Lanczos kernels (k <= 128):
// extreme eigenvalues by warp multisection, eigenvectors by inverse
// iteration, and the shifted solves of the RQI / adjoint modes.
#pragma once

#include "common.cuh"

namespace hoscf {

constexpr int kMaxLanczos = 128;

// --- small symmetric tridiagonal Ritz problem (k <= kMaxLanczos), one warp.
// Sturm count of eigenvalues < x (FP32, fast reciprocal: only signs matter).
static __device__ __forceinline__ int sturm_count(const float* al, const float* be2, int k, float x,
                                           float pivmin) {
    int c = 0;
    float q = al[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
    for (int i = 1; i < k; ++i) {
        q = (al[i] - x) - __fdividef(be2[i - 1], q);
        if (fabsf(q) < pivmin) q = -pivmin;
        c += q < 0.f;
    }
    return c;
}

// Both extreme eigenvalues by multisection with the pivot-form Sturm count,
// one full warp: lanes 0-15 bracket the largest, lanes 16-31 the smallest,
// 16 points each per round, one whole-warp ballot per round, until both
// brackets are small.  Returns the midpoint of the lane's final bracket.
static __device__ float extreme_eig(const float* al, const float* be2, int k, float lo, float hi,
                                    float pivmin) {
    const int lane = threadIdx.x & 31;
    const bool upper = lane >= 16;
    for (int round = 0; round < 7; ++round) {
        const float w = (hi - lo) * (1.f / 17.f);
        const float x = lo + w * (float)((lane & 15) + 1);
        const int c = sturm_count(al, be2, k, x, pivmin);
        // largest: first point with all k eigenvalues below it; smallest:
        // first point with one below it
        const bool hit = upper ? (c >= 1) : (c == k);
        const unsigned bal = __ballot_sync(HOSCF_FULLMASK, hit);
        const unsigned mine = upper ? (bal >> 16) : (bal & 0xffffu);
        const int first = mine ? __ffs(mine) - 1 : 16;
        const float nlo = lo + w * (float)first;
        const float nhi = (first == 16) ? hi : lo + w * (float)(first + 1);
        lo = nlo;
        hi = nhi;
        if (__all_sync(HOSCF_FULLMASK, hi - lo <= 4.f * 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi)))) break;
    }
    return 0.5f * (lo + hi);
}

// Sturm count without divisions for k <= KM, on T scaled by a power of two so
// that every entry is at most 1 in magnitude (x in the same units): the
// leading principal minors p_i of T - x I, p_i = (a_i - x) p_{i-1} -
// b_{i-1}^2 p_{i-2} (p_0 = 1), change sign once per eigenvalue below x, a
// zero minor taking the sign opposite to its predecessor's (the limit of the
// pivot form's replacement of a zero pivot by a small negative one).
// |p_i| <= (1 + sqrt 2)^i, so nothing overflows for KM <= 32; a pair of
// minors below 2^-32 is rescaled by 2^32 at once (the recurrence is
// homogeneous in the pair; branch-free), which keeps clustered spectra,
// whose minors can shrink by many orders of magnitude per step, clear of
// underflow.
template <int KM>
static __device__ __forceinline__ int sturm_count_poly(const float (&a)[KM], const float (&b2)[KM],
                                                       int k, float x) {
    float pp = 1.f, pc = a[0] - x;
    bool nc = pc <= 0.f;   // p_0 > 0
    int c = nc ? 1 : 0;
#pragma unroll
    for (int i = 1; i < KM; ++i) {
        if (i < k) {
            const float pn = fmaf(a[i] - x, pc, -b2[i - 1] * pp);
            pp = pc;
            pc = pn;
            const bool nn = pn < 0.f || (pn == 0.f && !nc);
            c += nn != nc ? 1 : 0;
            nc = nn;
            const float f = fmaxf(fabsf(pp), fabsf(pc)) < 0x1p-32f ? 0x1p32f : 1.f;
            pp *= f;
            pc *= f;
        }
    }
    return c;
}

// Both extreme eigenvalues for k <= KM with sturm_count_poly, one full warp:
// lanes 0-15 bracket the largest, lanes 16-31 the smallest, 16 points each
// per round, one whole-warp ballot per round; the entries are scaled by
// scale = 2^-e (exact) so that the Gershgorin bound is below 1, the
// multisection runs on [-1, 1] until both brackets are small and the result
// (the lane's end) is scaled back.
template <int KM>
static __device__ float extreme_eig_poly(const float* al, const float* be2, int k, float scale) {
    const int lane = threadIdx.x & 31;
    const bool upper = lane >= 16;
    float a[KM], b2[KM];
    const float s2 = scale * scale;
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        a[i] = i < k ? al[i] * scale : 0.f;
        b2[i] = i < k - 1 ? be2[i] * s2 : 0.f;
    }
    float lo = -1.f, hi = 1.f;
    for (int round = 0; round < 8; ++round) {
        const float w = (hi - lo) * (1.f / 17.f);
        const float x = lo + w * (float)((lane & 15) + 1);
        const int c = sturm_count_poly<KM>(a, b2, k, x);
        // largest: first point with every eigenvalue below it; smallest:
        // first point with one below it
        const bool hit = upper ? (c >= 1) : (c == k);
        const unsigned bal = __ballot_sync(HOSCF_FULLMASK, hit);
        const unsigned mine = upper ? (bal >> 16) : (bal & 0xffffu);
        const int first = mine ? __ffs(mine) - 1 : 16;
        const float nlo = lo + w * (float)first;
        const float nhi = (first == 16) ? hi : lo + w * (float)(first + 1);
        lo = nlo;
        hi = nhi;
        if (__all_sync(HOSCF_FULLMASK, hi - lo <= 4.f * 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi)))) break;
    }
    return 0.5f * (lo + hi) / scale;
}

// Eigenvector of the tridiagonal T for eigenvalue approx theta: two steps of
// inverse iteration with partial-pivot LU (FP32).  s has k entries, unit norm.
static __device__ void tridiag_inverse_iteration(const float* al, const float* be, int k, float theta,
                                          float bound, float* s, float* wa, float* wb, float* wc,
                                          float* wd, int* piv) {
    // LU of (T - theta I): rows i with sub-diagonal be[i-1], super be[i].
    // Zero pivots are replaced by eps32 * ||T|| (standard inverse iteration).
    const float eps = fmaxf(1.2e-7f * bound, 1e-30f);
    for (int i = 0; i < k; ++i) s[i] = 1.f;
    for (int i = 0; i < k; ++i) {
        wa[i] = al[i] - theta;
        wb[i] = (i < k - 1) ? be[i] : 0.f;
        wc[i] = 0.f;
    }
    for (int i = 0; i < k - 1; ++i) {
        const float sub = be[i];   // element (i+1, i)
        if (fabsf(wa[i]) >= fabsf(sub)) {
            piv[i] = 0;
            const float l = (wa[i] != 0.f) ? __fdividef(sub, wa[i]) : 0.f;
            wd[i] = l;
            wa[i + 1] -= l * wb[i];
        } else {
            piv[i] = 1;
            const float l = __fdividef(wa[i], sub);
            wd[i] = l;
            const float a_ip1 = wa[i + 1];
            wa[i] = sub;
            const float t = wb[i];
            wb[i] = a_ip1;
            wa[i + 1] = t - l * a_ip1;
            if (i < k - 2) {
                wc[i] = wb[i + 1];
                wb[i + 1] = -l * wb[i + 1];
            }
        }
    }
    for (int i = 0; i < k; ++i)
        if (fabsf(wa[i]) <= eps) wa[i] = (wa[i] < 0.f) ? -eps : eps;
    for (int it = 0; it < 2; ++it) {
        for (int i = 0; i < k - 1; ++i) {
            if (piv[i]) {
                const float t = s[i];
                s[i] = s[i + 1];
                s[i + 1] = t - wd[i] * s[i];
            } else {
                s[i + 1] -= wd[i] * s[i];
            }
        }
        float mx = 0.f;
        for (int i = k - 1; i >= 0; --i) {
            float v = s[i];
            if (i + 1 < k) v -= wb[i] * s[i + 1];
            if (i + 2 < k) v -= wc[i] * s[i + 2];
            s[i] = __fdividef(v, wa[i]);
            if (fabsf(s[i]) > 1e30f) {   // rescale to stay finite
                for (int t = i; t < k; ++t) s[t] *= 1e-30f;
            }
        }
        for (int i = 0; i < k; ++i) mx = fmaxf(mx, fabsf(s[i]));
        if (!(mx > 0.f) || !isfinite(mx)) {
            for (int i = 0; i < k; ++i) s[i] = (i == 0) ? 1.f : 0.f;
            mx = 1.f;
        }
        const float inv = 1.f / mx;
        for (int i = 0; i < k; ++i) s[i] *= inv;
    }
}

// The same for k <= KM with every array in registers (one thread, loops
// unrolled over KM); the result is written to s[0..k).
template <int KM>
static __device__ void tridiag_inverse_iteration_reg(const float* al, const float* be, int k,
                                                     float theta, float bound, float* s_out) {
    const float eps = fmaxf(1.2e-7f * bound, 1e-30f);
    float wa[KM], wb[KM], wc[KM], wd[KM], s[KM];
    unsigned piv = 0u;
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        wa[i] = i < k ? al[i] - theta : 1.f;
        wb[i] = i < k - 1 ? be[i] : 0.f;
        wc[i] = 0.f;
        wd[i] = 0.f;
        s[i] = 1.f;
    }
#pragma unroll
    for (int i = 0; i < KM - 1; ++i) {
        if (i < k - 1) {
            const float sub = be[i];   // element (i+1, i)
            if (fabsf(wa[i]) >= fabsf(sub)) {
                const float l = (wa[i] != 0.f) ? __fdividef(sub, wa[i]) : 0.f;
                wd[i] = l;
                wa[i + 1] -= l * wb[i];
            } else {
                piv |= 1u << i;
                const float l = __fdividef(wa[i], sub);
                wd[i] = l;
                const float a_ip1 = wa[i + 1];
                wa[i] = sub;
                const float t = wb[i];
                wb[i] = a_ip1;
                wa[i + 1] = t - l * a_ip1;
                if (i + 1 < KM - 1 && i < k - 2) {
                    wc[i] = wb[i + 1];
                    wb[i + 1] = -l * wb[i + 1];
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < KM; ++i)
        if (i < k && fabsf(wa[i]) <= eps) wa[i] = (wa[i] < 0.f) ? -eps : eps;
    for (int it = 0; it < 2; ++it) {
#pragma unroll
        for (int i = 0; i < KM - 1; ++i) {
            if (i < k - 1) {
                if (piv & (1u << i)) {
                    const float t = s[i];
                    s[i] = s[i + 1];
                    s[i + 1] = t - wd[i] * s[i];
                } else {
                    s[i + 1] -= wd[i] * s[i];
                }
            }
        }
#pragma unroll
        for (int i = KM - 1; i >= 0; --i) {
            if (i < k) {
                float v = s[i];
                if (i + 1 < KM && i + 1 < k) v -= wb[i] * s[i + 1];
                if (i + 2 < KM && i + 2 < k) v -= wc[i] * s[i + 2];
                s[i] = __fdividef(v, wa[i]);
                if (fabsf(s[i]) > 1e30f) {   // rescale to stay finite
#pragma unroll
                    for (int t = 0; t < KM; ++t)
                        if (t >= i && t < k) s[t] *= 1e-30f;
                }
            }
        }
        float mx = 0.f;
#pragma unroll
        for (int i = 0; i < KM; ++i)
            if (i < k) mx = fmaxf(mx, fabsf(s[i]));
        if (!(mx > 0.f) || !isfinite(mx)) {
#pragma unroll
            for (int i = 0; i < KM; ++i) s[i] = (i == 0) ? 1.f : 0.f;
            mx = 1.f;
        }
        const float inv = 1.f / mx;
#pragma unroll
        for (int i = 0; i < KM; ++i) s[i] *= inv;
    }
#pragma unroll
    for (int i = 0; i < KM; ++i)
        if (i < k) s_out[i] = s[i];
}

// Solution z of (T - shift I) z = e_1 for the k x k tridiagonal T (FP32,
// partial-pivot LU as above); returns |z_k| / ||z|| and writes z / ||z|| to
// s_out (FP64).  One thread.
static __device__ double tridiag_shifted_solve(const double* alpha, const double* beta, int k,
                                        double shift, double* s_out, float* wa, float* wb,
                                        float* wc, float* wd, float* z, int* piv,
                                        double* znorm) {
    float bound = 0.f;
    for (int i = 0; i < k; ++i) {
        wa[i] = (float)(alpha[i] - shift);
        wb[i] = (i < k - 1) ? (float)beta[i] : 0.f;
        wc[i] = 0.f;
        z[i] = (i == 0) ? 1.f : 0.f;
        bound = fmaxf(bound, fabsf(wa[i]) + fabsf(wb[i]) + (i > 0 ? (float)fabs(beta[i - 1]) : 0.f));
    }
    const float eps = fmaxf(1.2e-7f * bound, 1e-30f);
    for (int i = 0; i < k - 1; ++i) {
        const float sub = (float)beta[i];
        if (fabsf(wa[i]) >= fabsf(sub)) {
            piv[i] = 0;
            const float l = (wa[i] != 0.f) ? sub / wa[i] : 0.f;
            wd[i] = l;
            wa[i + 1] -= l * wb[i];
        } else {
            piv[i] = 1;
            const float l = wa[i] / sub;
            wd[i] = l;
            const float a_ip1 = wa[i + 1];
            wa[i] = sub;
            const float t = wb[i];
            wb[i] = a_ip1;
            wa[i + 1] = t - l * a_ip1;
            if (i < k - 2) {
                wc[i] = wb[i + 1];
                wb[i + 1] = -l * wb[i + 1];
            }
        }
    }
    for (int i = 0; i < k - 1; ++i) {
        if (piv[i]) {
            const float t = z[i];
            z[i] = z[i + 1];
            z[i + 1] = t - wd[i] * z[i];
        } else {
            z[i + 1] -= wd[i] * z[i];
        }
    }
    for (int i = k - 1; i >= 0; --i) {
        float v = z[i];
        if (i + 1 < k) v -= wb[i] * z[i + 1];
        if (i + 2 < k) v -= wc[i] * z[i + 2];
        const float dd = fabsf(wa[i]) > eps ? wa[i] : (wa[i] < 0.f ? -eps : eps);
        z[i] = v / dd;
        if (fabsf(z[i]) > 1e30f)
            for (int t = i; t < k; ++t) z[t] *= 1e-30f;
    }
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += (double)z[i] * (double)z[i];
    nrm = sqrt(nrm);
    if (!(nrm > 0.0) || !isfinite(nrm)) {
        for (int i = 0; i < k; ++i) s_out[i] = (i == 0) ? 1.0 : 0.0;
        *znorm = NAN;
        return 1.0;
    }
    *znorm = nrm;
    for (int i = 0; i < k; ++i) s_out[i] = (double)z[i] / nrm;
    return fabs((double)z[k - 1]) / nrm;
}

struct RitzOut {
    double theta;
    double resid;   // |beta_k * s_k| / ||s||
};

// |s_k| of the unit eigenvector of the k x k tridiagonal T for its extreme
// eigenvalue near th, without the vector: with p_j the leading principal
// minors of T - th I, s_k^2 = -p_{k-1}(th) / p_k'(th), from the pivots
// q_j = p_j / p_{j-1} and the ratios r_j = p_j' / p_j of one pass,
//   q_j = (a_j - th) - b_{j-1}^2 / q_{j-1},
//   p_j' / p_{j-1} = -1 + (a_j - th) r_{j-1} - b_{j-1}^2 r_{j-2} / q_{j-1},
//   r_j = (p_j' / p_{j-1}) / q_j.
// At an extreme eigenvalue every pivot q_j (j < k) has one sign and stays
// away from zero (the eigenvalues of T_j lie strictly inside by interlacing),
// so the pass is stable; in FP32 it is accurate while |s_k| >= ~3e-3 and
// flattens out near sqrt(eps32) below that (measured on Lanczos
// tridiagonals), so only values well above that floor are used.  One thread.
static __device__ float ritz_last_component(const float* al, const float* be2, int k, float th) {
    float rq = __fdividef(1.f, al[0] - th);   // 1 / q_1
    float r1 = -rq, r2 = 0.f;                 // r_1, r_0
    float num = -1.f;                         // p_1' / p_0
    for (int j = 1; j < k; ++j) {
        const float aj = al[j] - th;
        const float bq = be2[j - 1] * rq;     // b_{j-1}^2 / q_{j-1}
        num = -1.f + aj * r1 - bq * r2;
        if (j + 1 < k) {
            const float rqn = __fdividef(1.f, aj - bq);
            r2 = r1;
            r1 = num * rqn;
            rq = rqn;
        }
    }
    return sqrtf(1.f / fabsf(num));
}

// Largest-magnitude Ritz pair of T_k (alpha, beta in FP64, k >= 1), FP32
// part: the extreme eigenvalue (multisection on both ends, ties to the
// positive end) and its eigenvector by inverse iteration, left (unit max
// norm) in scratch[3k'..] (k' = kMaxLanczos); resid = |beta_k s_k| / ||s||.
// The trailing component of a converged Ritz vector is far below what an
// FP32 eigenvalue resolves through the pivots of T - theta I, so it is read
// off the inverse-iteration vector.  Enough to decide convergence; the FP64
// refined pair comes from ritz_refine_fp64 on the same scratch.  Called by
// one full warp.
// When the eigenvector is not needed (need_vec false) and the estimate of
// ritz_last_component at both ends of the eigenvalue's FP32 bracket agrees
// (within a factor 2) on |s_k| >= 1e-2 and a residual above 4 * tol_rel *
// |theta| - a pair that is clearly not converged - the inverse iteration is
// skipped and that estimate returned (the caller only learns "not
// converged").
// The same with the FP32 tridiagonal already in scratch (al = scratch[0..k),
// be = scratch[k'..], be2 = scratch[2k'..], k' = kMaxLanczos; be[k-1] and
// be2[k-1] are not read): callers that build T one step at a time keep those
// arrays current instead of converting alpha and beta at every check.
// poly selects the division-free multisection for k <= 32 (its register
// arrays suit kernels with registers to spare; the pivot form otherwise).
static __device__ RitzOut ritz_extreme_core(int k, double beta_k, float* scratch,
                                            double tol_rel = 0.0, bool need_vec = true,
                                            bool poly = true) {
    const int lane = threadIdx.x & 31;
    float* al = scratch;
    float* be = al + kMaxLanczos;
    float* be2 = be + kMaxLanczos;
    float* sv = be2 + kMaxLanczos;
    float* wa = sv + kMaxLanczos;
    float* wb = wa + kMaxLanczos;
    float* wc = wb + kMaxLanczos;
    float* wd = wc + kMaxLanczos;
    int* piv = reinterpret_cast<int*>(wd + kMaxLanczos);
    float bound = 0.f;
    for (int i = lane; i < k; i += 32) {
        const float r = fabsf(al[i]) + (i < k - 1 ? fabsf(be[i]) : 0.f) + (i > 0 ? fabsf(be[i - 1]) : 0.f);
        bound = fmaxf(bound, r);
    }
    for (int o = 16; o > 0; o >>= 1) bound = fmaxf(bound, __shfl_xor_sync(HOSCF_FULLMASK, bound, o));
    bound = bound * 1.0001f + 1e-30f;
    const float pivmin = fmaxf(bound * 1e-30f, 1e-35f);
    // lanes 0-15: largest eigenvalue, lanes 16-31: smallest
    float ext;
    if (k == 1) {
        ext = al[0];
    } else if (poly && k <= 32) {
        // power-of-two scale putting the Gershgorin bound below 1
        int e;
        frexpf(bound, &e);
        const float scale = ldexpf(1.f, -e);
        if (k <= 8)
            ext = extreme_eig_poly<8>(al, be2, k, scale);
        else if (k <= 16)
            ext = extreme_eig_poly<16>(al, be2, k, scale);
        else
            ext = extreme_eig_poly<32>(al, be2, k, scale);
    } else {
        ext = extreme_eig(al, be2, k, -bound, bound, pivmin);
    }
    const float tmax = __shfl_sync(HOSCF_FULLMASK, ext, 0);
    const float tmin = __shfl_sync(HOSCF_FULLMASK, ext, 16);
    // ties between +l and -l go to the positive end
    const float theta32 = (tmax >= -tmin) ? tmax : tmin;
    // the cheap estimate at both ends of the bracket, on lanes 0 and 1
    float est = -1.f;
    if (!need_vec && k >= 2 && lane < 2) {
        const float h = 4.8e-7f * fabsf(theta32) + 1e-30f;
        est = ritz_last_component(al, be2, k, lane == 0 ? theta32 - h : theta32 + h);
    }
    const float e0 = __shfl_sync(HOSCF_FULLMASK, est, 0);
    const float e1 = __shfl_sync(HOSCF_FULLMASK, est, 1);
    float s_est = -1.f;
    if (!need_vec && k >= 2) {
        const float lim = __fdividef((float)(4.0 * tol_rel) * fabsf(theta32), (float)fabs(beta_k));
        if (isfinite(e0) && isfinite(e1) && fminf(e0, e1) >= 1e-2f && fminf(e0, e1) > lim &&
            fmaxf(e0, e1) <= 2.f * fminf(e0, e1))
            s_est = fminf(e0, e1);
    }
    if (s_est >= 0.f) {
        RitzOut ro;
        ro.theta = theta32;
        ro.resid = fabs(beta_k) * (double)s_est;
        return ro;
    }
    if (lane == 0) {
        if (k == 1)
            sv[0] = 1.f;
        else if (poly && k <= 8)
            tridiag_inverse_iteration_reg<8>(al, be, k, theta32, bound, sv);
        else if (poly && k <= 16)
            tridiag_inverse_iteration_reg<16>(al, be, k, theta32, bound, sv);
        else
            tridiag_inverse_iteration(al, be, k, theta32, bound, sv, wa, wb, wc, wd, piv);
    }
    __syncwarp();
    float ss = 0.f;
    for (int i = lane; i < k; i += 32) ss = fmaf(sv[i], sv[i], ss);
    ss = warp_sum(ss);
    RitzOut ro;
    ro.theta = theta32;
    ro.resid = fabs(beta_k) * (double)(fabsf(sv[k - 1]) * rsqrtf(ss));
    return ro;
}

static __device__ RitzOut ritz_extreme_fp32(const double* alpha, const double* beta, int k,
                                            double beta_k, float* scratch, double tol_rel = 0.0,
                                            bool need_vec = true) {
    const int lane = threadIdx.x & 31;
    float* al = scratch;
    float* be = al + kMaxLanczos;
    float* be2 = be + kMaxLanczos;
    for (int i = lane; i < k; i += 32) {
        al[i] = (float)alpha[i];
        be[i] = (i < k - 1) ? (float)beta[i] : 0.f;
        be2[i] = be[i] * be[i];
    }
    __syncwarp();
    return ritz_extreme_core(k, beta_k, scratch, tol_rel, need_vec, false);
}

// FP64 refinement of the pair ritz_extreme_fp32 left in scratch: Rayleigh
// quotient theta = s^T T s / s^T s, residual |beta_k s_k| / ||s||, and the
// unit vector s (FP64) in s_out.  Called by one full warp.
static __device__ RitzOut ritz_refine_fp64(const double* alpha, const double* beta, int k,
                                           double beta_k, double* s_out, const float* scratch) {
    const int lane = threadIdx.x & 31;
    const float* sv = scratch + 3 * kMaxLanczos;
    double num = 0.0, den = 0.0;
    for (int i = lane; i < k; i += 32) {
        const double si = sv[i];
        double ts = alpha[i] * si;
        if (i > 0) ts += beta[i - 1] * (double)sv[i - 1];
        if (i < k - 1) ts += beta[i] * (double)sv[i + 1];
        num += si * ts;
        den += si * si;
    }
    num = warp_sum_d(num);
    den = warp_sum_d(den);
    const double inv = rsqrt_nr(den);
    for (int i = lane; i < k; i += 32) s_out[i] = (double)sv[i] * inv;
    RitzOut ro;
    ro.theta = num * (inv * inv);
    ro.resid = fabs(beta_k * (double)sv[k - 1]) * inv;
    return ro;
}

// Both parts: the refined largest-magnitude Ritz pair.
static __device__ RitzOut ritz_largest_magnitude(const double* alpha, const double* beta, int k,
                                                 double beta_k, double* s_out, float* scratch) {
    ritz_extreme_fp32(alpha, beta, k, beta_k, scratch);
    return ritz_refine_fp64(alpha, beta, k, beta_k, s_out, scratch);
}

}  // namespace hoscf
