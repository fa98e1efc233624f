// Shared device helpers and host-side plan structures of the HOSCF library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hoscf.h"

#define HOSCF_WARP 32
#define HOSCF_FULLMASK 0xffffffffu

namespace hoscf {

// ------------------------------------------------------------------ status
struct Err {
    hoscf_status code = HOSCF_OK;
    char msg[512] = {0};
};

// Device-side error codes written to a status word by kernels.
enum DevErr : int {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,      // a bounded wait gave up
    DEV_NONFINITE = 2,    // NaN / Inf met
    DEV_BADARG = 3
};

// ------------------------------------------------------------------ launch helpers
// Opt a kernel into the device's largest dynamic shared memory per CTA; each
// launch still passes its own size (which is what occupancy and the
// cooperative-launch check use).  Setting the attribute to a per-launch size
// instead would race between host threads launching the same kernel with
// different sizes (one thread lowering it between another's set and launch).
// (The opt-in limit counts the kernel's static shared memory as well.)
template <typename Kernel>
inline cudaError_t allow_max_dynamic_smem(Kernel kern) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
    return e;
}

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Asynchronous global->shared copy of N = 4, 8 or 16 bytes; `valid` false
// zero-fills the destination without reading the source.
template <int N>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
    if (N == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)),
                     "l"(src), "r"(valid ? 16 : 0)
                     : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_addr(dst)),
                     "l"(src), "n"(N), "r"(valid ? N : 0)
                     : "memory");
    }
}

// Wait until every cp.async this thread issued has landed (they always
// complete: sources are valid addresses).
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Close the group of this thread's cp.async issued since the last commit;
// wait until at most N of its committed groups are still in flight.
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The barrier receives one arrival (counted in its init count) once every
// cp.async this thread issued before has landed.
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// The same test with a suspend-time hint: a thread whose phase is not
// complete sleeps until it completes or about `hint_ns` pass, instead of
// returning at once (waiting warps then do not take issue slots).
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity,
                                                   uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Wait for an mbarrier phase with a wall-clock bound.  Returns false (and
// leaves the caller to record the timeout) when the bound passes.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    const uint32_t hint = (uint32_t)(limit_ns < 100000ull ? limit_ns : 100000ull);
    while (true) {
        if (mbar_try_wait_hint(bar, parity, hint)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// Packed FP32 (two lanes per instruction, IEEE fma / mul per lane, so the
// results equal the scalar ones bit for bit).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const uint64_t*>(&a)), "l"(*reinterpret_cast<const uint64_t*>(&b)),
          "l"(*reinterpret_cast<const uint64_t*>(&c)));
    return *reinterpret_cast<const float2*>(&d);
}

// Contiguous bulk copy global -> shared (cp.async.bulk): both addresses and
// the size multiples of 16 bytes; completion counted on `bar` as
// transaction bytes.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 3-D tiled TMA load: box at coordinates (c0 innermost, c1, c2) into smem,
// completion signalled on `bar` as transaction bytes.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

// Hint: fetch the 128-byte line holding p into L2 (no register result, no
// wait; a line past the end of an allocation is never touched by callers).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(HOSCF_FULLMASK, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(HOSCF_FULLMASK, v, o);
    return v;
}

// 1/sqrt(x) and 1/x in FP64 from the FP32 hardware approximation and two
// Newton steps (each squares the relative error: ~1e-7, ~1e-14, then below
// FP64 rounding) - far fewer FP64 instructions than the correctly rounded
// routines, whose results they match to a few ulps; arguments outside FP32's
// normal range take those routines.
__device__ __forceinline__ double rsqrt_nr(double x) {
    if (!(x >= 1.2e-38 && x <= 3.0e38)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf((float)x);
    const double hx = 0.5 * x;
    y = y * fma(-hx * y, y, 1.5);
    y = y * fma(-hx * y, y, 1.5);
    return y;
}

__device__ __forceinline__ double rcp_nr(double x) {
    const double ax = fabs(x);
    if (!(ax >= 1.2e-38 && ax <= 3.0e38)) return 1.0 / x;
    double y = (double)__fdividef(1.f, (float)x);
    y = y * fma(-x, y, 2.0);
    y = y * fma(-x, y, 2.0);
    return y;
}

// Double-float accumulation (hi + lo, ~46 significant bits) with FP32
// instructions, for sums that need more than FP32 on parts where FP64 issues
// slowly: (hi, lo) += a by Knuth's two-sum, += x y with the product's exact
// error from an FMA.
__device__ __forceinline__ void df_add(float& hi, float& lo, float a) {
    const float s = hi + a;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (a - bb);
    hi = s;
}

__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float x, float y) {
    const float p = x * y;
    df_add(hi, lo, p);
    lo += fmaf(x, y, -p);
}

// ------------------------------------------------------------------ grid barrier
// Software barrier across the co-resident CTAs of a cooperative launch.
// `*count` is zero when the launch starts (the launcher's preceding kernel
// on the same stream clears it) and only grows: every CTA adds one per
// barrier with a fire-and-forget release reduction (it publishes the CTA's
// earlier writes), then polls with acquire loads until the count reaches
// epoch x nblocks, `epoch` being the number of barriers this CTA has passed
// (uniform over the CTA).  One round trip per barrier, no release flag, no
// full fences.  Every wait is bounded by `limit_ns`; on timeout *err is set
// and false is returned (the caller then leaves the kernel).
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned nblocks, unsigned& epoch,
                                             int* err, uint64_t limit_ns) {
    __syncthreads();
    __shared__ int s_ok;
    ++epoch;
    if (threadIdx.x == 0) {
        // release: the CTA's writes (ordered before this thread by the CTA
        // barrier above) become visible before the arrival; no reply awaited
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
        const unsigned target = epoch * nblocks;
        auto seen = [count]() {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            return v;
        };
        int ok = 1;
        if ((int)(seen() - target) < 0) {
            const uint64_t t0 = global_timer_ns();
            unsigned spins = 0;
            while ((int)(seen() - target) < 0) {
                __nanosleep(20);
                if ((++spins & 255u) == 0) {
                    if (*(volatile int*)err) { ok = 0; break; }
                    if (global_timer_ns() - t0 > limit_ns) {
                        atomicCAS(err, 0, (int)DEV_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        s_ok = ok;   // the acquire load that saw the target orders the reads after the barrier
    }
    __syncthreads();
    return s_ok != 0;
}

// The same barrier in two halves, so that a CTA can work between its arrival
// and its wait: grid_arrive publishes the CTA's earlier writes and counts it
// in (after a CTA barrier); grid_wait polls (bounded) until every CTA of
// this epoch has arrived.  Each grid_arrive must be followed by exactly one
// grid_wait, or by the CTA leaving the kernel.
__device__ __forceinline__ void grid_arrive(unsigned* count, unsigned& epoch) {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0)
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
}

__device__ __forceinline__ bool grid_wait(unsigned* count, unsigned nblocks, unsigned epoch, int* err,
                                          uint64_t limit_ns) {
    __shared__ int s_okw;
    if (threadIdx.x == 0) {
        const unsigned target = epoch * nblocks;
        auto seen = [count]() {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            return v;
        };
        int ok = 1;
        if ((int)(seen() - target) < 0) {
            const uint64_t t0 = global_timer_ns();
            unsigned spins = 0;
            while ((int)(seen() - target) < 0) {
                __nanosleep(20);
                if ((++spins & 255u) == 0) {
                    if (*(volatile int*)err) { ok = 0; break; }
                    if (global_timer_ns() - t0 > limit_ns) {
                        atomicCAS(err, 0, (int)DEV_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        s_okw = ok;
    }
    __syncthreads();
    return s_okw != 0;
}

// grid_wait for a group of warps of the CTA: thread `leader` polls, then the
// group's nthreads threads meet at named barrier `bar_id` (not 0, which
// __syncthreads uses).  Same bound and error handling as grid_wait.
__device__ __forceinline__ bool grid_wait_group(unsigned* count, unsigned nblocks, unsigned epoch,
                                                int* err, uint64_t limit_ns, int leader,
                                                int bar_id, int nthreads, int* ok_out) {
    if ((int)threadIdx.x == leader) {
        const unsigned target = epoch * nblocks;
        auto seen = [count]() {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            return v;
        };
        int ok = 1;
        if ((int)(seen() - target) < 0) {
            const uint64_t t0 = global_timer_ns();
            unsigned spins = 0;
            while ((int)(seen() - target) < 0) {
                __nanosleep(20);
                if ((++spins & 255u) == 0) {
                    if (*(volatile int*)err) { ok = 0; break; }
                    if (global_timer_ns() - t0 > limit_ns) {
                        atomicCAS(err, 0, (int)DEV_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        *ok_out = ok;
    }
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthreads) : "memory");
    return *ok_out != 0;
}

// ------------------------------------------------------------------ element loads
template <typename E>
struct ElemTraits;

template <>
struct ElemTraits<float> {
    static constexpr int size = 4;
    __device__ static __forceinline__ float to_f(float v) { return v; }
};

struct bf16_t { uint16_t bits; };
struct f16_t { uint16_t bits; };
struct fp8_t { uint8_t bits; };

template <>
struct ElemTraits<bf16_t> {
    static constexpr int size = 2;
    __device__ static __forceinline__ float to_f(bf16_t v) {
        return __uint_as_float(static_cast<uint32_t>(v.bits) << 16);
    }
};

}  // namespace hoscf
