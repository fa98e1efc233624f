// Differentiation form (no paper counterpart): gradient of
//   L = c * sigma + sum_n <w_n, u_n>
// with respect to the tensor at a converged rank-one solution.
//
// Envelope theorem: d sigma / dT = u1 o ... o ud.  Linearising the KKT system
// (eq. 2.4) with per-mode multipliers gives, for the factors,
//   (H - sigma I) du - U dmu = -b,  U^T du = 0,  b_n = dT x_{k!=n} u_k,
// H the full symmetric block matrix (blocks A_{n,m}, eq. 3.3), U = blockdiag(u_n).
// Its adjoint: on the factors' tangent space P = I - U U^T solve
//   P (H - sigma I) P a = P w,
// (negative definite at a nondegenerate maximum), then
//   dL/dT = c u1 o ... o ud - sum_n u1 o .. o a_n o .. o ud.
// The solve runs in the Lanczos kernel (operator mode: full blocks, shift
// -sigma, blockwise projection; a Galerkin tridiagonal solve).  The write is
// one HBM pass over dT:  with w_o = prod_{outer} u_k[o_k] and
// alpha_o = sum_{n outer} a_n[o_n] prod_{k != n} u_k[o_k],
//   dT[o,a,b] = (c w_o - alpha_o) uA[a] uB[b] - w_o (aA[a] uB[b] + uA[a] aB[b]).
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hoscf {

// b = P w in FP64 (one CTA; per-mode dots then subtraction).
__global__ void tangent_project_kernel(const float* __restrict__ u, const float* __restrict__ w,
                                       int d, ModeInfoArr mi, double* __restrict__ b,
                                       double* __restrict__ bnorm2) {
    __shared__ double red[32];
    __shared__ double mu;
    double tot = 0.0;
    for (int m = 0; m < d; ++m) {
        double s = 0.0;
        for (int64_t q = mi.off[m] + threadIdx.x; q < mi.off[m + 1]; q += blockDim.x)
            s += (double)u[q] * (double)w[q];
        s = warp_sum_d(s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
            mu = t;
        }
        __syncthreads();
        double ss = 0.0;
        for (int64_t q = mi.off[m] + threadIdx.x; q < mi.off[m + 1]; q += blockDim.x) {
            const double v = (double)w[q] - mu * (double)u[q];
            b[q] = v;
            ss += v * v;
        }
        ss = warp_sum_d(ss);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) *bnorm2 = tot;
}

struct GradArgs {
    int d, D;
    int dims[kMaxOrder];
    int64_t st[kMaxOrder];
    int64_t moff[kMaxOrder + 1];
    int64_t O, A, B, F;
    int64_t OT;   // outer indices per block row
    double c;
};

// Per outer index: coef1 = c w_o - alpha_o, coef2 = w_o.
__global__ void grad_coef_kernel(const float* __restrict__ u, const double* __restrict__ a, GradArgs g,
                                 float* __restrict__ coef1, float* __restrict__ coef2) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < g.O;
         o += (int64_t)gridDim.x * blockDim.x) {
        double uv[kMaxOrder], av[kMaxOrder];
        double w = 1.0;
        for (int k = 0; k < g.D; ++k) {
            const int dk = (int)((o / g.st[k]) % g.dims[k]);
            uv[k] = u[g.moff[k] + dk];
            av[k] = a ? a[g.moff[k] + dk] : 0.0;
            w *= uv[k];
        }
        double al = 0.0;
        for (int n = 0; n < g.D; ++n) {
            double p = av[n];
            for (int k = 0; k < g.D; ++k)
                if (k != n) p *= uv[k];
            al += p;
        }
        coef1[o] = (float)(g.c * w - al);
        coef2[o] = (float)w;
    }
}

// dT[o, f] for a tile of 16 outer indices per block row; f over threads.
__global__ void grad_write_kernel(const float* __restrict__ u, const double* __restrict__ a,
                                  const float* __restrict__ coef1, const float* __restrict__ coef2,
                                  GradArgs g, float* __restrict__ out) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= g.F) return;
    const int64_t ia = f / g.B, ib = f - (f / g.B) * g.B;
    const float uA = u[g.moff[g.d - 2] + ia], uB = u[g.moff[g.d - 1] + ib];
    const float aA = a ? (float)a[g.moff[g.d - 2] + ia] : 0.f;
    const float aB = a ? (float)a[g.moff[g.d - 1] + ib] : 0.f;
    const float p1 = uA * uB, p2 = fmaf(aA, uB, uA * aB);
    const int64_t o0 = (int64_t)blockIdx.y * g.OT;
    const int64_t o1 = min(g.O, o0 + g.OT);
    for (int64_t o = o0; o < o1; ++o)
        __stcs(out + o * g.F + f, fmaf(coef1[o], p1, -coef2[o] * p2));
}

cudaError_t launch_tangent_project(const Shape& s, const float* u, const float* w, double* b,
                                   double* bnorm2, cudaStream_t st) {
    ModeInfoArr mi;
    memset(&mi, 0, sizeof(mi));
    for (int k = 0; k <= s.d; ++k) mi.off[k] = s.moff[k];
    tangent_project_kernel<<<1, 256, 0, st>>>(u, w, s.d, mi, b, bnorm2);
    return cudaGetLastError();
}

cudaError_t launch_grad_write(const Shape& s, const float* u, const double* a, double c,
                              float* coef, float* out, cudaStream_t st, const KernelEvents* kev) {
    GradArgs g;
    memset(&g, 0, sizeof(g));
    g.d = s.d;
    g.D = s.D;
    for (int k = 0; k < s.D; ++k) {
        g.dims[k] = (int)s.dims[k];
        g.st[k] = s.ost[k];
    }
    for (int k = 0; k <= s.d; ++k) g.moff[k] = s.moff[k];
    g.O = s.O;
    g.A = s.A;
    g.B = s.B;
    g.F = s.A * s.B;
    g.c = c;
    float* coef1 = coef;
    float* coef2 = coef + s.O;
    const int64_t cb = std::min<int64_t>(4096, (s.O + 255) / 256);
    if (kev) cudaEventRecord(kev->begin, st);
    grad_coef_kernel<<<(unsigned)std::max<int64_t>(cb, 1), 256, 0, st>>>(u, a, g, coef1, coef2);
    g.OT = std::max<int64_t>(16, (s.O + 65534) / 65535);
    dim3 grid((unsigned)((g.F + 255) / 256), (unsigned)((s.O + g.OT - 1) / g.OT));
    grad_write_kernel<<<grid, 256, 0, st>>>(u, a, coef1, coef2, g, out);
    if (kev) cudaEventRecord(kev->end, st);
    return cudaGetLastError();
}

}  // namespace hoscf
