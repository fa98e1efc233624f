// Eigen step of HOSCF: the largest-magnitude eigenpair of J(x) (Algorithm 1
// line 5), the block normalisation of lines 6-9, the KKT certificate of the
// point the blocks were built at (eq. 2.4 / eq. 4.1), and the final sign fix
// of lines 12-15.
//
// J is never formed densely.  `Jr` holds the rows of the full symmetric block
// matrix with its zero diagonal blocks dropped (row q of mode m is the
// concatenation of A_{m,n} rows for n > m and A_{n,m}^T rows for n < m), so a
// mat-vec is a set of independent contiguous row dot products.
//
// Lanczos runs as one cooperative kernel over G CTAs: rows are split across
// CTAs, every step does one mat-vec and one full (classical Gram-Schmidt)
// reorthogonalisation against the whole FP64 basis, with two grid barriers.
// Scalars (dot products, the tridiagonal matrix, Ritz values) are reduced in
// a fixed order and recomputed identically by every CTA, so all CTAs take the
// same decisions without another barrier.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hoscf {

constexpr int kEigThreads = 256;
constexpr int kEigWarps = kEigThreads / 32;
constexpr int kMaxLanczos = 128;

struct EigArgs {
    const float* Jr;        // 2P floats
    int d;
    int n;
    int64_t moff[kMaxOrder + 1];
    int64_t jroff[kMaxOrder + 1];   // Jr offset of the first row of each mode
    float scale;            // 1 / (d - 1)
    const double* x0;       // start vector (n), or NULL: start = u0 / sqrt(d)
    const float* u0;
    double* V;              // (mmax + 1) x n
    double* Y;              // n
    double* part;           // 2 x G x pstride (two alternating reduction buffers)
    int pstride;
    double* scal;           // outputs (see EigScal)
    double* x_out;          // n or NULL
    float* u_out;           // n or NULL
    double* lambda_out;     // 1 or NULL
    int mmax;
    double eig_tol;
    int check;              // 1: certify the start point first, stop if r <= kkt_tol
    double kkt_tol;
    unsigned* bar;
    int* err;
    uint64_t timeout_ns;
};

__device__ __forceinline__ int mode_of(const EigArgs& a, int q) {
    int m = 0;
    while (m < a.d - 1 && q >= a.moff[m + 1]) ++m;
    return m;
}

// y[q] = (1/(d-1)) * Jr_row(q) . v  for the rows of this CTA, one warp per
// row; FP32 products summed in FP32 over runs of 32 terms per lane, FP64
// beyond.  Also accumulates the squared row norms (for ||J||_F) when asked.
__device__ void matvec_rows(const EigArgs& a, const float* __restrict__ vf, int r0, int r1,
                            double* sq) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double sqacc = 0.0;
    for (int q = r0 + warp; q < r1; q += kEigWarps) {
        const int m = mode_of(a, q);
        const int64_t Im = a.moff[m + 1] - a.moff[m];
        const int64_t len = a.n - Im;
        const float* row = a.Jr + a.jroff[m] + (int64_t)(q - a.moff[m]) * len;
        const int64_t lo = a.moff[m];
        double acc = 0.0;
        double sacc = 0.0;
        for (int64_t j0 = 0; j0 < len; j0 += 1024) {
            float f = 0.f, s2 = 0.f;
            const int64_t j1 = min(len, j0 + 1024);
            for (int64_t j = j0 + lane; j < j1; j += 32) {
                const float h = __ldg(row + j);
                const int64_t col = j < lo ? j : j + Im;
                f = fmaf(h, vf[col], f);
                s2 = fmaf(h, h, s2);
            }
            acc += (double)f;
            sacc += (double)s2;
        }
        acc = warp_sum_d(acc);
        if (sq) sacc = warp_sum_d(sacc);
        if (lane == 0) {
            a.Y[q] = acc * (double)a.scale;
            sqacc += sacc;
        }
    }
    if (sq && lane == 0) atomicAdd(sq, sqacc);   // shared-memory scratch, per CTA
}

// --- small symmetric tridiagonal Ritz problem (k <= kMaxLanczos), one warp.
// Sturm count of eigenvalues < x (FP32, fast reciprocal: only signs matter).
__device__ __forceinline__ int sturm_count(const float* al, const float* be2, int k, float x,
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

// Largest (want_max) or smallest eigenvalue by 16-way multisection on one
// half-warp.  Returns the midpoint of the final bracket.
__device__ float extreme_eig(const float* al, const float* be2, int k, float lo, float hi,
                             bool want_max, int sublane, unsigned halfmask, float pivmin) {
    for (int round = 0; round < 7; ++round) {
        const float x = lo + (hi - lo) * (float)(sublane + 1) / 17.f;
        const int c = sturm_count(al, be2, k, x, pivmin);
        // want_max: first shift with all k eigenvalues below it
        const bool hit = want_max ? (c == k) : (c >= 1);
        const unsigned bal = __ballot_sync(halfmask, hit);
        const unsigned mine = (halfmask == 0xffffu) ? bal : (bal >> 16);
        const int first = mine ? __ffs(mine) - 1 : 16;   // first hit shift index
        const float w = (hi - lo) / 17.f;
        const float nlo = lo + w * (float)first;
        const float nhi = (first == 16) ? hi : lo + w * (float)(first + 1);
        lo = nlo;
        hi = nhi;
        if (hi - lo <= 4.f * 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
    }
    return 0.5f * (lo + hi);
}

// Eigenvector of the tridiagonal T for eigenvalue approx theta: two steps of
// inverse iteration with partial-pivot LU (FP32).  s has k entries, unit norm.
__device__ void tridiag_inverse_iteration(const float* al, const float* be, int k, float theta,
                                          float bound, float* s, float* wa, float* wb, float* wc,
                                          float* wd, int* piv) {
    // LU of (T - theta I): rows i with sub-diagonal be[i-1], super be[i].
    // Zero pivots are replaced by eps32 * ||T|| (standard inverse iteration).
    const float eps = fmaxf(1.2e-7f * bound, 1e-30f);
    for (int i = 0; i < k; ++i) s[i] = 1.f;
    // factorisation (LAPACK gttrf-style): diag wa, super wb, super2 wc, multipliers wd
    for (int i = 0; i < k; ++i) {
        wa[i] = al[i] - theta;
        wb[i] = (i < k - 1) ? be[i] : 0.f;
        wc[i] = 0.f;
    }
    for (int i = 0; i < k - 1; ++i) {
        const float sub = be[i];   // element (i+1, i)
        if (fabsf(wa[i]) >= fabsf(sub)) {
            piv[i] = 0;
            const float l = (wa[i] != 0.f) ? sub / wa[i] : 0.f;
            wd[i] = l;
            wa[i + 1] -= l * wb[i];
        } else {
            piv[i] = 1;
            const float l = wa[i] / sub;
            wd[i] = l;
            // swap rows i and i+1
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
    for (int it = 0; it < 2; ++it) {
        // forward: apply row interchanges and multipliers
        for (int i = 0; i < k - 1; ++i) {
            if (piv[i]) {
                const float t = s[i];
                s[i] = s[i + 1];
                s[i + 1] = t - wd[i] * s[i];
            } else {
                s[i + 1] -= wd[i] * s[i];
            }
        }
        // backward
        for (int i = k - 1; i >= 0; --i) {
            float v = s[i];
            if (i + 1 < k) v -= wb[i] * s[i + 1];
            if (i + 2 < k) v -= wc[i] * s[i + 2];
            const float dd = fabsf(wa[i]) > eps ? wa[i] : (wa[i] < 0 ? -eps : eps);
            s[i] = v / dd;
            if (fabsf(s[i]) > 1e30f) {   // rescale to stay finite
                for (int t = i; t < k; ++t) s[t] *= 1e-30f;
            }
        }
        float mx = 0.f;
        for (int i = 0; i < k; ++i) mx = fmaxf(mx, fabsf(s[i]));
        if (!(mx > 0.f) || !isfinite(mx)) {
            for (int i = 0; i < k; ++i) s[i] = (i == 0) ? 1.f : 0.f;
            mx = 1.f;
        }
        float nrm = 0.f;
        for (int i = 0; i < k; ++i) {
            s[i] /= mx;
            nrm = fmaf(s[i], s[i], nrm);
        }
        nrm = rsqrtf(nrm);
        for (int i = 0; i < k; ++i) s[i] *= nrm;
    }
}

struct RitzOut {
    double theta;
    double resid;   // |beta_k * s_k|
};

// Largest-magnitude Ritz pair of T_k (alpha, beta in FP64, k >= 1); writes s
// (FP64) to shared memory.  Called by warp 0; result broadcast by the caller.
__device__ RitzOut ritz_largest_magnitude(const double* alpha, const double* beta, int k,
                                          double beta_k, double* s_out, float* scratch) {
    const int lane = threadIdx.x & 31;
    float* al = scratch;                 // k
    float* be = al + kMaxLanczos;        // k
    float* be2 = be + kMaxLanczos;       // k
    float* sv = be2 + kMaxLanczos;       // k
    float* wa = sv + kMaxLanczos;
    float* wb = wa + kMaxLanczos;
    float* wc = wb + kMaxLanczos;
    float* wd = wc + kMaxLanczos;
    int* piv = reinterpret_cast<int*>(wd + kMaxLanczos);
    float bound = 0.f;
    for (int i = lane; i < k; i += 32) {
        al[i] = (float)alpha[i];
        be[i] = (i < k - 1) ? (float)beta[i] : 0.f;
        be2[i] = be[i] * be[i];
    }
    __syncwarp();
    for (int i = lane; i < k; i += 32) {
        const float r = fabsf(al[i]) + fabsf(be[i]) + (i > 0 ? fabsf(be[i - 1]) : 0.f);
        bound = fmaxf(bound, r);
    }
    for (int o = 16; o > 0; o >>= 1) bound = fmaxf(bound, __shfl_xor_sync(HOSCF_FULLMASK, bound, o));
    bound = bound * 1.0001f + 1e-30f;
    const float pivmin = fmaxf(bound * 1e-30f, 1e-35f);
    // half-warp 0: largest eigenvalue, half-warp 1: smallest
    const bool upper = lane >= 16;
    const unsigned hm = upper ? 0xffff0000u : 0x0000ffffu;
    float ext;
    if (k == 1) {
        ext = al[0];
    } else {
        ext = extreme_eig(al, be2, k, -bound, bound, !upper, lane & 15, hm, pivmin);
    }
    const float tmax = __shfl_sync(HOSCF_FULLMASK, ext, 0);
    const float tmin = __shfl_sync(HOSCF_FULLMASK, ext, 16);
    // ties between +l and -l go to the positive end
    const float theta32 = (tmax >= -tmin) ? tmax : tmin;
    RitzOut ro;
    if (lane == 0) {
        if (k == 1) {
            sv[0] = 1.f;
        } else {
            tridiag_inverse_iteration(al, be, k, theta32, bound, sv, wa, wb, wc, wd, piv);
        }
        // refine theta with the FP64 Rayleigh quotient of s
        double num = 0.0, den = 0.0;
        for (int i = 0; i < k; ++i) {
            const double si = sv[i];
            double ts = alpha[i] * si;
            if (i > 0) ts += beta[i - 1] * (double)sv[i - 1];
            if (i < k - 1) ts += beta[i] * (double)sv[i + 1];
            num += si * ts;
            den += si * si;
            s_out[i] = si;
        }
        ro.theta = num / den;
        ro.resid = fabs(beta_k * (double)sv[k - 1]) / sqrt(den);
    }
    ro.theta = __shfl_sync(HOSCF_FULLMASK, ro.theta, 0);
    ro.resid = __shfl_sync(HOSCF_FULLMASK, ro.resid, 0);
    return ro;
}

// Sum over CTAs of partial vectors: out[i] = sum_c part[c * stride + i],
// i < cnt, fixed order (lane stride then butterfly), one warp per index.
// Callers alternate between two partial buffers so that a CTA writing the
// next reduction's partials never overwrites ones another CTA is still
// reading (consecutive reductions are separated by one grid barrier only).
__device__ void sum_partials(const double* part, int stride, int G, int cnt, double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < cnt; i += kEigWarps) {
        double s = 0.0;
        for (int c = lane; c < G; c += 32) s += ((volatile const double*)part)[(size_t)c * stride + i];
        s = warp_sum_d(s);
        if (lane == 0) out[i] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kEigThreads, 1) lanczos_kernel(EigArgs a) {
    const int G = gridDim.x;
    const int c = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n;
    const int R = (n + G - 1) / G;
    const int r0 = min(n, c * R), r1 = min(n, r0 + R);

    extern __shared__ __align__(16) uint8_t sm_raw[];
    float* vf = reinterpret_cast<float*>(sm_raw);                       // n floats
    double* hsum = reinterpret_cast<double*>(vf + ((n + 3) & ~3));       // kMaxLanczos + 8
    double* alpha = hsum + kMaxLanczos + 8;                              // kMaxLanczos
    double* beta = alpha + kMaxLanczos;                                  // kMaxLanczos
    double* sv = beta + kMaxLanczos;                                     // kMaxLanczos
    double* misc = sv + kMaxLanczos;                                     // 16
    float* rscratch = reinterpret_cast<float*>(misc + 16);               // 9 * kMaxLanczos

    double* V = a.V;
    const int ps = a.pstride;
    int phase = 0;
    auto pbuf = [&]() { return a.part + (size_t)(phase & 1) * G * ps; };
    const double sqrt_d = sqrt((double)a.d);

    // ---- start vector V[0] (unnormalised) for my rows
    for (int q = r0 + tid; q < r1; q += kEigThreads) {
        double v;
        if (a.x0) {
            v = a.x0[q];
        } else {
            v = (double)a.u0[q] / sqrt_d;
        }
        V[q] = v;
    }
    if (tid == 0) misc[0] = 0.0;
    if (!grid_barrier(a.bar, G, a.err, a.timeout_ns)) return;

    int k = 0;             // basis size
    double beta_last = 0.0;
    RitzOut ro;
    ro.theta = 0.0;
    ro.resid = 0.0;
    bool done = false;
    int j = 0;
    for (j = 0; j < a.mmax && !done; ++j) {
        // stage V[j] into shared memory as FP32
        for (int q = tid; q < n; q += kEigThreads) vf[q] = (float)((volatile double*)V)[(size_t)j * n + q];
        __syncthreads();
        matvec_rows(a, vf, r0, r1, j == 0 ? &misc[0] : nullptr);
        __syncthreads();
        // partial dots over my rows: h_i = V[i].y (i <= j), yy, and (j==0) xx, ||J||^2
        const int cnt = j + 2 + (j == 0 ? 2 : 0);
        for (int i = warp; i < cnt; i += kEigWarps) {
            double s = 0.0;
            if (i <= j) {
                for (int q = r0 + lane; q < r1; q += 32) s += V[(size_t)i * n + q] * a.Y[q];
            } else if (i == j + 1) {
                for (int q = r0 + lane; q < r1; q += 32) s += a.Y[q] * a.Y[q];
            } else if (i == j + 2) {
                for (int q = r0 + lane; q < r1; q += 32) s += V[q] * V[q];
            }
            s = warp_sum_d(s);
            if (lane == 0) pbuf()[(size_t)c * ps + i] = (i == j + 3) ? misc[0] : s;
        }
        if (!grid_barrier(a.bar, G, a.err, a.timeout_ns)) return;
        sum_partials(pbuf(), ps, G, cnt, hsum);
        ++phase;
        if (j == 0) {
            // normalise the start vector (delayed): v0 = x0/|x0|, y = J v0
            const double xx = hsum[2];
            if (!(xx > 0.0) || !isfinite(xx)) {
                if (tid == 0) atomicCAS(a.err, 0, (int)DEV_NONFINITE);
                return;
            }
            const double inv = 1.0 / sqrt(xx);
            for (int q = r0 + tid; q < r1; q += kEigThreads) {
                V[q] *= inv;
                a.Y[q] *= inv;
            }
            if (tid == 0) {
                hsum[0] *= inv * inv;
                hsum[1] *= inv * inv;
                misc[1] = sqrt(hsum[3]) * (double)a.scale;   // ||J||_F
            }
            __syncthreads();
            // exact ||y - alpha0 v0||^2 over my rows (one more reduction)
            const double al0 = hsum[0];
            double s = 0.0;
            for (int q = r0 + tid; q < r1; q += kEigThreads) {
                const double w = a.Y[q] - al0 * V[q];
                a.Y[q] = w;
                s += w * w;
            }
            s = warp_sum_d(s);
            __shared__ double red[kEigWarps];
            if (lane == 0) red[warp] = s;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w8 = 0; w8 < kEigWarps; ++w8) t += red[w8];
                pbuf()[(size_t)c * ps + 0] = t;
            }
            if (!grid_barrier(a.bar, G, a.err, a.timeout_ns)) return;
            sum_partials(pbuf(), ps, G, 1, misc + 2);
            ++phase;
            const double b0 = sqrt(fmax(misc[2], 0.0));
            const double rho = al0;
            if (c == 0 && tid == 0) {
                a.scal[SC_SIGMA] = rho;
                a.scal[SC_KKT] = (rho != 0.0) ? sqrt_d * b0 / fabs(rho) : INFINITY;
                a.scal[SC_R41] = b0 / (misc[1] + fabs(rho));
                a.scal[SC_JFRO] = misc[1];
                a.scal[SC_CONVERGED] = 0.0;
            }
            if (!isfinite(rho) || !isfinite(b0)) {
                if (tid == 0) atomicCAS(a.err, 0, (int)DEV_NONFINITE);
                return;
            }
            if (a.check && rho != 0.0 && sqrt_d * b0 / fabs(rho) <= a.kkt_tol) {
                // the start point is certified: no eigen step
                if (c == 0 && tid == 0) {
                    a.scal[SC_CONVERGED] = 1.0;
                    a.scal[SC_LAMBDA] = rho;
                    a.scal[SC_STEPS] = 0.0;
                    a.scal[SC_RITZRES] = b0;
                }
                return;
            }
            alpha[0] = rho;
            // w = y - alpha0 v0 -> V[1] after normalisation
            beta_last = b0;
            if (tid == 0) beta[0] = b0;
            k = 1;
        } else {
            // full classical Gram-Schmidt against V[0..j]
            double ssq = 0.0;
            for (int i = 0; i <= j; ++i) ssq += hsum[i] * hsum[i];
            const double yy = hsum[j + 1];
            double b2 = yy - ssq;
            if (tid == 0) alpha[j] = hsum[j];
            __syncthreads();
            for (int q = r0 + tid; q < r1; q += kEigThreads) {
                double w = a.Y[q];
                for (int i = 0; i <= j; ++i) w -= hsum[i] * V[(size_t)i * n + q];
                a.Y[q] = w;
            }
            if (b2 < 0.25 * yy) {
                // heavy cancellation: second Gram-Schmidt pass with exact norm
                __syncthreads();
                for (int i = warp; i < j + 2; i += kEigWarps) {
                    double s = 0.0;
                    if (i <= j) {
                        for (int q = r0 + lane; q < r1; q += 32) s += V[(size_t)i * n + q] * a.Y[q];
                    } else {
                        for (int q = r0 + lane; q < r1; q += 32) s += a.Y[q] * a.Y[q];
                    }
                    s = warp_sum_d(s);
                    if (lane == 0) pbuf()[(size_t)c * ps + i] = s;
                }
                if (!grid_barrier(a.bar, G, a.err, a.timeout_ns)) return;
                sum_partials(pbuf(), ps, G, j + 2, hsum);
                ++phase;
                double ssq2 = 0.0;
                for (int i = 0; i <= j; ++i) ssq2 += hsum[i] * hsum[i];
                b2 = hsum[j + 1] - ssq2;
                if (tid == 0) alpha[j] += hsum[j];
                __syncthreads();
                for (int q = r0 + tid; q < r1; q += kEigThreads) {
                    double w = a.Y[q];
                    for (int i = 0; i <= j; ++i) w -= hsum[i] * V[(size_t)i * n + q];
                    a.Y[q] = w;
                }
            }
            beta_last = sqrt(fmax(b2, 0.0));
            if (tid == 0) beta[j] = beta_last;
            k = j + 1;
        }
        __syncthreads();
        // convergence test on the Ritz pair (every 4 steps, and at the limits)
        const bool last = (k == a.mmax) || (k == n) || beta_last <= 1e-300;
        if (k >= 2 && ((k % 4) == 0 || last)) {
            __shared__ RitzOut s_ro;
            if (warp == 0) {
                RitzOut t = ritz_largest_magnitude(alpha, beta, k, beta_last, sv, rscratch);
                if (lane == 0) s_ro = t;
            }
            __syncthreads();
            ro = s_ro;
            if (ro.resid <= a.eig_tol * fabs(ro.theta) || last) done = true;
        } else if (last) {
            if (tid == 0) sv[0] = 1.0;
            ro.theta = alpha[0];
            ro.resid = beta_last;
            done = true;
        }
        __syncthreads();
        if (!done) {
            const double inv = 1.0 / beta_last;
            for (int q = r0 + tid; q < r1; q += kEigThreads) V[(size_t)(j + 1) * n + q] = a.Y[q] * inv;
            if (!grid_barrier(a.bar, G, a.err, a.timeout_ns)) return;
        }
    }
    // ---- Ritz vector x = V[0..k-1] s for my rows; block norms and sign
    const int d = a.d;
    for (int q = r0 + tid; q < r1; q += kEigThreads) {
        double x = 0.0;
        for (int i = 0; i < k; ++i) x += sv[i] * V[(size_t)i * n + q];
        a.Y[q] = x;
    }
    __syncthreads();
    // partials: [0..d-1] block norms^2, [d] x . v0
    for (int i = warp; i < d + 1; i += kEigWarps) {
        double s = 0.0;
        if (i < d) {
            const int lo = max(r0, (int)a.moff[i]), hi = min(r1, (int)a.moff[i + 1]);
            for (int q = lo + lane; q < hi; q += 32) s += a.Y[q] * a.Y[q];
        } else {
            for (int q = r0 + lane; q < r1; q += 32) s += a.Y[q] * V[q];
        }
        s = warp_sum_d(s);
        if (lane == 0) pbuf()[(size_t)c * ps + i] = s;
    }
    if (!grid_barrier(a.bar, G, a.err, a.timeout_ns)) return;
    sum_partials(pbuf(), ps, G, d + 1, hsum);
    double tot = 0.0;
    for (int m = 0; m < d; ++m) tot += hsum[m];
    const double sgn = (hsum[d] < 0.0) ? -1.0 : 1.0;
    const double invx = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    for (int q = r0 + tid; q < r1; q += kEigThreads) {
        const double x = a.Y[q] * sgn;
        if (a.x_out) a.x_out[q] = x * invx;
        if (a.u_out) {
            const int m = mode_of(a, q);
            const double nb = hsum[m];
            a.u_out[q] = nb > 0.0 ? (float)(x / sqrt(nb)) : 0.f;
        }
    }
    if (c == 0 && tid == 0) {
        a.scal[SC_LAMBDA] = ro.theta;
        a.scal[SC_STEPS] = (double)k;
        a.scal[SC_RITZRES] = ro.resid;
        if (a.lambda_out) *a.lambda_out = ro.theta;
    }
}

// ---------------------------------------------------------------- Jr build
// Jr rows from the packed blocks: block (m,n) goes to rows of mode m as is
// and to rows of mode n transposed (32x32 smem tiles, coalesced both ways).
struct JrBuildArgs {
    int d, nblk;
    int64_t n;
    int64_t dims[kMaxOrder];
    int64_t moff[kMaxOrder + 1];
    int64_t jroff[kMaxOrder + 1];
    int64_t boff[kMaxBlocks + 1];
    int bm[kMaxBlocks], bn[kMaxBlocks];
    int64_t tstart[kMaxBlocks + 1];   // tile prefix
};

__global__ void build_jr_kernel(const float* __restrict__ H, float* __restrict__ Jr, JrBuildArgs a) {
    __shared__ float tile[32][33];
    const int64_t tix = blockIdx.x;
    int b = 0;
    while (tix >= a.tstart[b + 1]) ++b;
    const int m = a.bm[b], nn = a.bn[b];
    const int64_t Im = a.dims[m], In = a.dims[nn];
    const int64_t tj_count = (In + 31) / 32;
    const int64_t loc = tix - a.tstart[b];
    const int64_t ti = loc / tj_count, tj = loc % tj_count;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    const float* blk = H + a.boff[b];
    const int64_t lenm = a.n - Im, lenn = a.n - In;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = ti * 32 + r, jj = tj * 32 + tx;
        float v = 0.f;
        if (i < Im && jj < In) {
            v = blk[i * In + jj];
            // row (moff[m] + i), column (moff[nn] + jj) of J; drop the m block
            Jr[a.jroff[m] + i * lenm + (a.moff[nn] - Im) + jj] = v;
        }
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t jj = tj * 32 + r, i = ti * 32 + tx;
        if (i < Im && jj < In) {
            // row (moff[nn] + jj), column (moff[m] + i), m < nn so no shift
            Jr[a.jroff[nn] + jj * lenn + a.moff[m] + i] = tile[tx][r];
        }
    }
}

// ---------------------------------------------------------------- small kernels
// Per-mode norms of u (FP64) into out[0..d-1]; one CTA.
__global__ void mode_norms_kernel(const float* __restrict__ u, int d, ModeInfoArr mi, double* out) {
    __shared__ double red[32];
    for (int m = 0; m < d; ++m) {
        double s = 0.0;
        for (int64_t q = mi.off[m] + threadIdx.x; q < mi.off[m + 1]; q += blockDim.x) {
            const double v = u[q];
            s += v * v;
        }
        s = warp_sum_d(s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            out[m] = t;
        }
        __syncthreads();
    }
}

__global__ void scale_modes_kernel(const float* __restrict__ u, int d, ModeInfoArr mi,
                                   const double* __restrict__ nrm2, float* __restrict__ out) {
    const int64_t n = mi.off[d];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        int m = 0;
        while (m < d - 1 && q >= mi.off[m + 1]) ++m;
        out[q] = (float)((double)u[q] / sqrt(nrm2[m]));
    }
}

// Alg. 1 lines 12-15 (sign of sigma) plus the sign gauge: for n >= 1 the
// largest-|.| entry of u^(n) (lowest index on ties) is made positive, the
// flip carried by u^(0).  One CTA; sigma in/out in FP64.
__global__ void final_fix_kernel(float* __restrict__ u, int d, ModeInfoArr mi, double* sigma) {
    __shared__ float bv[32];
    __shared__ int bi[32];
    __shared__ int flips;
    if (threadIdx.x == 0) flips = (*sigma < 0.0) ? 1 : 0;
    __syncthreads();
    for (int m = 1; m < d; ++m) {
        float best = -1.f;
        int bidx = 0x7fffffff;
        for (int64_t q = mi.off[m] + threadIdx.x; q < mi.off[m + 1]; q += blockDim.x) {
            const float v = fabsf(u[q]);
            if (v > best || (v == best && (int)q < bidx)) {
                best = v;
                bidx = (int)q;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(HOSCF_FULLMASK, best, o);
            const int oi = __shfl_xor_sync(HOSCF_FULLMASK, bidx, o);
            if (ov > best || (ov == best && oi < bidx)) {
                best = ov;
                bidx = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            bv[threadIdx.x >> 5] = best;
            bi[threadIdx.x >> 5] = bidx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = bv[0];
            int ix = bi[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (bv[w] > b || (bv[w] == b && bi[w] < ix)) {
                    b = bv[w];
                    ix = bi[w];
                }
            bi[0] = ix;
        }
        __syncthreads();
        const bool neg = u[bi[0]] < 0.f;
        __syncthreads();
        if (neg) {
            for (int64_t q = mi.off[m] + threadIdx.x; q < mi.off[m + 1]; q += blockDim.x) u[q] = -u[q];
            if (threadIdx.x == 0) flips ^= 1;
        }
        __syncthreads();
    }
    if (flips)
        for (int64_t q = mi.off[0] + threadIdx.x; q < mi.off[1]; q += blockDim.x) u[q] = -u[q];
    if (threadIdx.x == 0) *sigma = fabs(*sigma);
}

// ---------------------------------------------------------------- host
static size_t lanczos_smem(int64_t n) {
    return sizeof(float) * (size_t)((n + 3) & ~3) +
           sizeof(double) * (size_t)(kMaxLanczos + 8 + 3 * kMaxLanczos + 16) +
           sizeof(float) * 9 * kMaxLanczos + 64;
}

int lanczos_blocks_per_sm(int64_t n_tot) {
    int nb = 0;
    const size_t sm = lanczos_smem(n_tot);
    cudaFuncSetAttribute(lanczos_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lanczos_kernel, kEigThreads, sm) !=
        cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}

bool make_eig_plan(const Shape& s, int nsm, int blocks_per_sm, int mmax, EigPlan& e) {
    e = EigPlan();
    if (mmax < 2) mmax = 2;
    if (mmax > kMaxLanczos) mmax = kMaxLanczos;
    e.mmax = mmax;
    if (lanczos_smem(s.n_tot) > 200 * 1024) return false;
    const int64_t want = (s.n_tot + 15) / 16;   // ~16 rows per CTA
    int64_t G = std::min<int64_t>(want, (int64_t)nsm * std::max(1, blocks_per_sm));
    e.G = (int)std::max<int64_t>(1, G);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    e.off_jr = take(sizeof(float) * 2 * (size_t)s.P);
    e.off_V = take(sizeof(double) * (size_t)(mmax + 1) * s.n_tot);
    e.off_Y = take(sizeof(double) * (size_t)s.n_tot);
    e.off_part = take(sizeof(double) * 2 * (size_t)e.G * (mmax + 8));
    e.bytes = off;
    return true;
}

static void jr_offsets(const Shape& s, int64_t* jroff) {
    jroff[0] = 0;
    for (int m = 0; m < s.d; ++m) jroff[m + 1] = jroff[m] + s.dims[m] * (s.n_tot - s.dims[m]);
}

cudaError_t launch_build_jr(const Shape& s, const float* H, float* Jr, cudaStream_t st) {
    JrBuildArgs a;
    memset(&a, 0, sizeof(a));
    a.d = s.d;
    a.n = s.n_tot;
    for (int k = 0; k < s.d; ++k) a.dims[k] = s.dims[k];
    for (int k = 0; k <= s.d; ++k) a.moff[k] = s.moff[k];
    jr_offsets(s, a.jroff);
    int b = 0;
    for (int m = 0; m < s.d; ++m)
        for (int n = m + 1; n < s.d; ++n) {
            a.bm[b] = m;
            a.bn[b] = n;
            a.boff[b] = s.boff[b];
            a.tstart[b + 1] = a.tstart[b] + ((s.dims[m] + 31) / 32) * ((s.dims[n] + 31) / 32);
            ++b;
        }
    a.nblk = b;
    const int64_t tiles = a.tstart[b];
    build_jr_kernel<<<(unsigned)tiles, 256, 0, st>>>(H, Jr, a);
    return cudaGetLastError();
}

cudaError_t launch_lanczos(const Shape& s, const LanczosLaunch& l, cudaStream_t st) {
    EigArgs a;
    memset(&a, 0, sizeof(a));
    a.Jr = l.Jr;
    a.d = s.d;
    a.n = (int)s.n_tot;
    for (int k = 0; k <= s.d; ++k) a.moff[k] = s.moff[k];
    jr_offsets(s, a.jroff);
    a.scale = 1.0f / (float)(s.d - 1);
    a.x0 = l.x0;
    a.u0 = l.u0;
    a.V = l.V;
    a.Y = l.Y;
    a.part = l.part;
    a.pstride = l.mmax + 8;
    a.scal = l.scal;
    a.x_out = l.x_out;
    a.u_out = l.u_out;
    a.lambda_out = l.lambda_out;
    a.mmax = l.mmax;
    a.eig_tol = l.eig_tol;
    a.check = l.check;
    a.kkt_tol = l.kkt_tol;
    a.bar = l.bar;
    a.err = l.err;
    a.timeout_ns = l.timeout_ns;
    const size_t sm = lanczos_smem(s.n_tot);
    cudaError_t e = cudaFuncSetAttribute(lanczos_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)lanczos_kernel, dim3(l.G), dim3(kEigThreads),
                                       args, sm, st);
}

static ModeInfoArr mode_info(const Shape& s) {
    ModeInfoArr mi;
    memset(&mi, 0, sizeof(mi));
    for (int k = 0; k <= s.d; ++k) mi.off[k] = s.moff[k];
    return mi;
}

cudaError_t launch_mode_norms(const Shape& s, const float* u, double* out, cudaStream_t st) {
    mode_norms_kernel<<<1, 256, 0, st>>>(u, s.d, mode_info(s), out);
    return cudaGetLastError();
}

cudaError_t launch_scale_modes(const Shape& s, const float* u, const double* nrm2, float* out,
                               cudaStream_t st) {
    const int64_t n = s.n_tot;
    scale_modes_kernel<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, st>>>(
        u, s.d, mode_info(s), nrm2, out);
    return cudaGetLastError();
}

cudaError_t launch_final_fix(const Shape& s, float* u, double* sigma, cudaStream_t st) {
    final_fix_kernel<<<1, 256, 0, st>>>(u, s.d, mode_info(s), sigma);
    return cudaGetLastError();
}

}  // namespace hoscf
