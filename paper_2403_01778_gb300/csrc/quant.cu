// Precision-form storage (no paper counterpart): FP32 -> BF16 or IEEE FP16
// (round to nearest even; FP16 overflows to infinity beyond 65504 as IEEE
// rounding prescribes) and FP32 -> FP8-e4m3 with one FP32 scale per 128 consecutive
// elements of the flat (row-major) order:
//   scale = fp32(amax / 448)  (1 for an all-zero group)
//   code  = e4m3(fp32(x / scale)), round to nearest even, saturating at 448.
// Both divisions are single correctly rounded FP32 operations and the
// conversions are the hardware's round-to-nearest-even instructions, so the
// codes are reproducible bit for bit.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"

namespace hoscf {

__global__ void quant_bf16_kernel(const float* __restrict__ x, int64_t n, uint16_t* __restrict__ q) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const __nv_bfloat16 b = __float2bfloat16_rn(x[i]);
        q[i] = *reinterpret_cast<const uint16_t*>(&b);
    }
}

__global__ void quant_f16_kernel(const float* __restrict__ x, int64_t n, uint16_t* __restrict__ q) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        q[i] = __half_as_ushort(__float2half_rn(x[i]));
}

// One warp per 128-element group; lane l handles elements 4l..4l+3.
__global__ void quant_e4m3_kernel(const float* __restrict__ x, int64_t n, uint8_t* __restrict__ q,
                                  float* __restrict__ scales) {
    const int lane = threadIdx.x & 31;
    const int64_t ng = (n + 127) / 128;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < ng;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t base = g * 128 + 4 * lane;
        float v[4];
        float amax = 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            v[c] = (base + c < n) ? x[base + c] : 0.f;
            amax = fmaxf(amax, fabsf(v[c]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(HOSCF_FULLMASK, amax, o));
        const float scale = amax == 0.f ? 1.f : __fdiv_rn(amax, 448.f);
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
            const float2 pair = make_float2(__fdiv_rn(v[c], scale), __fdiv_rn(v[c + 1], scale));
            const __nv_fp8x2_storage_t p2 = __nv_cvt_float2_to_fp8x2(pair, __NV_SATFINITE, __NV_E4M3);
            if (base + c < n) q[base + c] = (uint8_t)(p2 & 0xff);
            if (base + c + 1 < n) q[base + c + 1] = (uint8_t)(p2 >> 8);
        }
        if (lane == 0) scales[g] = scale;
    }
}

cudaError_t launch_quantize(const float* x, int64_t n, int dtype, void* q, float* scales,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (dtype == HOSCF_BF16) {
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 65535);
        quant_bf16_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, static_cast<uint16_t*>(q));
    } else if (dtype == HOSCF_F16) {
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 65535);
        quant_f16_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, static_cast<uint16_t*>(q));
    } else {
        const int64_t groups = (n + 127) / 128;
        const int64_t blocks = std::min<int64_t>((groups * 32 + 255) / 256, 65535);
        quant_e4m3_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, static_cast<uint8_t*>(q), scales);
    }
    return cudaGetLastError();
}

}  // namespace hoscf
