// Greedy rank-R approximation by repeated best rank-one approximation
// (Sec. 1 and Example 3: B^(r) = best rank-one approximation of A^(r),
// A^(r+1) = A^(r) - B^(r)) without rewriting the tensor.  The coupling
// blocks of the deflated tensor A - sum_{s<r} sigma_s u_1^(s) o ... o u_d^(s)
// at a point u follow from those of A (eq. 3.3) by a rank-(r-1) correction:
//   H_{m,n} - sum_s sigma_s (prod_{k != m,n} <u_k^(s), u_k>) u_m^(s) u_n^(s)^T,
// so every pass still reads only A.  Also the squared Frobenius norm of a
// tensor in any storage format (residual norms of the greedy terms).
#include <algorithm>
#include <cstring>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hoscf {

struct DeflArgs {
    int d, R;
    int64_t n;
    int64_t moff[kMaxOrder + 1];
    int64_t dims[kMaxOrder];
    int npairs;
    int pm[kMaxBlocks], pn[kMaxBlocks];
    int64_t boff[kMaxBlocks + 1];
};

// c[s d + k] = <u_k^(s), u_k>, one warp per (s, k), FP64 sums.
__global__ void defl_dots_kernel(const float* __restrict__ uprev, const float* __restrict__ u,
                                 DeflArgs a, double* __restrict__ c) {
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= a.R * a.d) return;
    const int s = w / a.d, k = w - (w / a.d) * a.d;
    const int64_t lo = a.moff[k], hi = a.moff[k + 1];
    double acc = 0.0;
    for (int64_t i = lo + lane; i < hi; i += 32)
        acc += (double)uprev[(int64_t)s * a.n + i] * (double)u[i];
    acc = warp_sum_d(acc);
    if (lane == 0) c[w] = acc;
}

// H[e] -= sum_s sigma_s prod_{k != m,n} c[s d + k] u_m^(s)[i] u_n^(s)[j]
__global__ void defl_blocks_kernel(float* __restrict__ H, const float* __restrict__ uprev,
                                   const double* __restrict__ sigma,
                                   const double* __restrict__ c, DeflArgs a) {
    const int64_t P = a.boff[a.npairs];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P;
         e += (int64_t)gridDim.x * blockDim.x) {
        int b = 0;
        while (e >= a.boff[b + 1]) ++b;
        const int m = a.pm[b], nn = a.pn[b];
        const int64_t loc = e - a.boff[b];
        const int64_t i = loc / a.dims[nn], j = loc - (loc / a.dims[nn]) * a.dims[nn];
        double corr = 0.0;
        for (int s = 0; s < a.R; ++s) {
            double w = sigma[s];
            for (int k = 0; k < a.d; ++k)
                if (k != m && k != nn) w *= c[s * a.d + k];
            const float* us = uprev + (int64_t)s * a.n;
            corr += w * (double)us[a.moff[m] + i] * (double)us[a.moff[nn] + j];
        }
        H[e] = (float)((double)H[e] - corr);
    }
}

cudaError_t launch_deflate(const Shape& s, float* H, const float* u, const float* uprev,
                           const double* sigma, int R, double* dots, cudaStream_t st) {
    if (R <= 0 || s.d < 2) return cudaSuccess;
    DeflArgs a;
    memset(&a, 0, sizeof(a));
    a.d = s.d;
    a.R = R;
    a.n = s.n_tot;
    for (int k = 0; k <= s.d; ++k) a.moff[k] = s.moff[k];
    for (int k = 0; k < s.d; ++k) a.dims[k] = s.dims[k];
    int np = 0;
    for (int m = 0; m < s.d; ++m)
        for (int n = m + 1; n < s.d; ++n) {
            a.pm[np] = m;
            a.pn[np] = n;
            a.boff[np] = s.boff[block_index(s.d, m, n)];
            ++np;
        }
    a.npairs = np;
    a.boff[np] = s.P;
    const int warps = R * s.d;
    defl_dots_kernel<<<(warps * 32 + 255) / 256, 256, 0, st>>>(uprev, u, a, dots);
    const int64_t blocks = std::min<int64_t>((s.P + 255) / 256, 4096);
    defl_blocks_kernel<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(H, uprev, sigma,
                                                                             dots, a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- ||A||_F^2
template <typename E>
__device__ __forceinline__ float elem_value(const E* p, const float* scales, int64_t i);
template <>
__device__ __forceinline__ float elem_value<float>(const float* p, const float*, int64_t i) {
    return p[i];
}
template <>
__device__ __forceinline__ float elem_value<bf16_t>(const bf16_t* p, const float*, int64_t i) {
    const uint16_t b = reinterpret_cast<const uint16_t*>(p)[i];
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
}
template <>
__device__ __forceinline__ float elem_value<f16_t>(const f16_t* p, const float*, int64_t i) {
    return __half2float(__ushort_as_half(reinterpret_cast<const unsigned short*>(p)[i]));
}
template <>
__device__ __forceinline__ float elem_value<fp8_t>(const fp8_t* p, const float* scales, int64_t i) {
    const uint8_t c = reinterpret_cast<const uint8_t*>(p)[i];
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3);
    return __half2float(*reinterpret_cast<const __half*>(&h)) * scales[i >> 7];
}

// per-CTA partial sums of squares (FP64), then one CTA adds them in order
template <typename E>
__global__ void sumsq_kernel(const E* __restrict__ x, const float* __restrict__ scales, int64_t n,
                             double* __restrict__ part) {
    __shared__ double red[8];
    // FP32 sums of up to 256 squares, flushed to FP64 (GB300's FP64 rate is
    // 1/64 of FP32, so no FP64 work per element)
    double acc = 0.0;
    float acc32 = 0.f;
    int cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float v = elem_value<E>(x, scales, i);
        acc32 = fmaf(v, v, acc32);
        if (++cnt == 256) {
            acc += (double)acc32;
            acc32 = 0.f;
            cnt = 0;
        }
    }
    acc += (double)acc32;
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < np; ++i) t += part[i];
        *out = t;
    }
}

cudaError_t launch_sumsq(int dtype, const void* data, const float* scales, int64_t n,
                         double* part, int nparts, double* out, cudaStream_t st) {
    if (dtype == HOSCF_F32)
        sumsq_kernel<float><<<nparts, 256, 0, st>>>((const float*)data, scales, n, part);
    else if (dtype == HOSCF_BF16)
        sumsq_kernel<bf16_t><<<nparts, 256, 0, st>>>((const bf16_t*)data, scales, n, part);
    else if (dtype == HOSCF_F16)
        sumsq_kernel<f16_t><<<nparts, 256, 0, st>>>((const f16_t*)data, scales, n, part);
    else
        sumsq_kernel<fp8_t><<<nparts, 256, 0, st>>>((const fp8_t*)data, scales, n, part);
    sum_parts_kernel<<<1, 32, 0, st>>>(part, nparts, out);
    return cudaGetLastError();
}

}  // namespace hoscf
