// Streaming pass for the narrow storage formats (BF16, FP16, FP8-e4m3 with
// one FP32 scale per 128 consecutive elements) when the face row is 128 .. 256
// elements long and a multiple of 8 (e.g. the 200^4 precision workload).
// Same factorisation and outputs as the tiled kernel in ttvc.cu (eq. 3.3):
//     face[a][b] += w_o T[o][a][b],  y1[o][a] = sum_b T u_B[b],  y2[o][b] = sum_a T u_A[a],
// but built for formats whose bytes carry less work per instruction:
//  * a tile spans the whole row: lane l owns columns 8l .. 8l+7 (one 8-byte
//    FP8 / 16-byte BF16 shared-memory load), warp w rows [w ROWS, (w+1) ROWS)
//    of an 8 ROWS-row band, so the per-item costs (row-sum transpose, column
//    exchange, waits, copy issue) are paid once per 8 ROWS x B elements;
//  * a warp's rows of one outer index are contiguous in memory: one 1-D bulk
//    copy (cp.async.bulk, rounded out to 16-byte granules, so no row-pitch
//    alignment rule) per warp and item, issued by lane 0 into the warp's ring;
//  * FP8: an 8-element chunk starts at a multiple of 8 of the flat index, so
//    it never straddles a 128-element scale group; the group scale s is
//    folded into the per-row multipliers (w_o s, u_A[a] s) and applied once
//    to the row partial, instead of one multiply per element.  The scales a
//    band spans arrive by a second bulk copy on the same mbarrier.
// Partials (per-CTA face tiles of FA x 256, per-tile y2, y1) go to the same
// workspace layout as the tiled kernel and are summed by the same reduce.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hoscf {

namespace {

// Eight consecutive elements (one aligned shared-memory load) -> float.
__device__ __forceinline__ void unpack8(const bf16_t* p, float2 (&x)[4]) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = make_float2(__uint_as_float(w[j] << 16), __uint_as_float(w[j] & 0xffff0000u));
}

__device__ __forceinline__ void unpack8(const f16_t* p, float2 (&x)[4]) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = __half22float2(*reinterpret_cast<const __half2*>(&w[j]));
}

__device__ __forceinline__ void unpack8(const fp8_t* p, float2 (&x)[4]) {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    const uint32_t w[2] = {q.x, q.y};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[j] & 0xffffu), __NV_E4M3);
        const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[j] >> 16), __NV_E4M3);
        x[2 * j] = __half22float2(*reinterpret_cast<const __half2*>(&lo));
        x[2 * j + 1] = __half22float2(*reinterpret_cast<const __half2*>(&hi));
    }
}

}  // namespace

// RMAX rows per warp at most; a tile of FA = a.FA rows is split as evenly as
// possible over the 8 warps (warp w: rows [w base + min(w, extra), +base +
// (w < extra)), base = FA / 8, extra = FA % 8), so e.g. A = 200 is covered
// by 2 tiles of 100 or 4 of 50 rows with no idle warp.  OCC CTAs per SM.
template <typename E, int RMAX, int OCC>
__global__ void __launch_bounds__(256, OCC) ttvc_narrow_kernel(const NarrowArgs a) {
    constexpr int FB = 256;
    constexpr bool F8 = std::is_same<E, fp8_t>::value;
    constexpr int ES = (int)sizeof(E);
    const int S = a.nstage;
    const int G = a.group;
    const int FA = a.FA;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const NarrowSmem L = narrow_smem(S, G, RMAX, a.B, ES, F8);
    float* s_y2 = reinterpret_cast<float*>(smem + L.y2);          // [2][G][8][FB]
    int64_t* s_off = reinterpret_cast<int64_t*>(smem + L.off);    // [2][G]
    int* s_cnt = reinterpret_cast<int*>(smem + L.cnt);            // [2][G]

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    float* s_rs = reinterpret_cast<float*>(smem + L.ysc) + (size_t)warp * RMAX * kRowSumStride;
    float* s_ua = reinterpret_cast<float*>(smem + L.ua) + warp * 16;
    const int64_t c = blockIdx.x;
    int64_t i0, i1;
    if (a.P > 0) {
        const int64_t t = c / a.P, o0 = (c - t * a.P) * a.W;
        i0 = t * a.O + o0;
        i1 = t * a.O + min(o0 + a.W, a.O);
    } else {
        i0 = c * a.W;
        i1 = min(i0 + a.W, a.items);
    }
    if (i0 >= i1) return;
    const int nloc = (int)(i1 - i0);
    const int64_t AB = a.A * a.B;
    const int B = (int)a.B;
    const bool colok = 8 * lane < B;                                // lane holds columns
    const int wbase = FA >> 3, wextra = FA & 7;
    const int wrow0 = warp * wbase + min(warp, wextra);             // warp's first row in a tile
    const int wrows = wbase + (warp < wextra ? 1 : 0);              // its rows (<= RMAX)

    uint8_t* ring = smem + (size_t)warp * S * L.slot;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars) + warp * S;
    // zero the warp's ring once (its pad and every byte a copy does not
    // write then hold finite values), then the barriers
    for (uint32_t q = 16u * lane; q < (uint32_t)(S * L.slot); q += 512u)
        *reinterpret_cast<uint4*>(ring + q) = make_uint4(0u, 0u, 0u, 0u);
    if (lane == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&full[q], 1u);
        fence_mbar_init();
    }
    __syncwarp();
    // a lane past the row end reads 8 zero elements (slot byte 0 .. 15 is
    // never written by a copy: every copy starts at the slot's data + 16)
    const uint32_t lane_off = colok ? 16u + 8u * lane * ES : 0u;
    const uint32_t row_step = colok ? (uint32_t)(B * ES) : 0u;

    // ---- issue side (lane 0)
    int64_t ii_o = 0, ii_t = i0 / a.O;
    ii_o = i0 - ii_t * a.O;
    auto issue = [&](int slot) {
        const int64_t ar0 = ii_t * FA + wrow0;
        const int nrows = (int)max((int64_t)0, min((int64_t)wrows, a.A - ar0));
        uint8_t* dst = ring + (size_t)slot * L.slot;
        if (nrows == 0) {
            mbar_arrive(&full[slot]);   // nothing to copy for this warp (ragged last band)
            return;
        }
        const int64_t f0 = ii_o * AB + ar0 * a.B;                   // flat index of the band
        const uintptr_t gb = reinterpret_cast<uintptr_t>(a.T) + (uintptr_t)(f0 * ES);
        const uintptr_t gal = gb & ~(uintptr_t)15;
        // the copy is rounded out to whole 16-byte granules; the bytes past the
        // band (at most 15, inside the granule of its last element) are unused
        const uint32_t bytes = (uint32_t)((gb - gal) + (uintptr_t)nrows * a.B * ES + 15) & ~15u;
        uint32_t sbytes = 0;
        uintptr_t sal = 0;
        if (F8) {
            const int64_t g0 = f0 >> 7, g1 = (f0 + (int64_t)nrows * a.B - 1) >> 7;
            const uintptr_t sb = reinterpret_cast<uintptr_t>(a.scales + g0);
            sal = sb & ~(uintptr_t)15;
            sbytes = (uint32_t)((sb - sal) + (uintptr_t)(g1 - g0 + 1) * 4 + 15) & ~15u;
        }
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[slot], bytes + sbytes);
        bulk_load(dst + 16, reinterpret_cast<const void*>(gal), bytes, &full[slot]);
        if (F8) bulk_load(dst + L.data, reinterpret_cast<const void*>(sal), sbytes, &full[slot]);
    };
    auto ii_next = [&]() {
        if (++ii_o == a.O) {
            ii_o = 0;
            ++ii_t;
        }
    };

    // ---- consume side
    float2 acc[RMAX][4];
    float2 uB2[4];
    const int64_t t_first = i0 / a.O;
    int64_t cc_o = i0 - t_first * a.O, cc_t = t_first - 1;
    int64_t y2off = 0, f0 = 0;
    int nrows = 0;
    const float* wp = a.w + cc_o;
    float* y1p = nullptr;

    auto flush = [&](int64_t t) {
        const int seg = (int)(t - t_first);
        float* dst = a.hp + ((size_t)(c * 2 + seg) * FA) * FB;
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            if (r < wrows) {
                float4* q = reinterpret_cast<float4*>(dst + (size_t)(wrow0 + r) * FB + 8 * lane);
                q[0] = make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y);
                q[1] = make_float4(acc[r][2].x, acc[r][2].y, acc[r][3].x, acc[r][3].y);
            }
        }
    };
    auto new_tile = [&](int64_t t) {
        const int64_t ar0 = t * FA + wrow0;
        nrows = (int)max((int64_t)0, min((int64_t)wrows, a.A - ar0));
        y1p = a.y1p + cc_o * a.A + ar0;
        y2off = (t * a.O + cc_o) * a.B;
        f0 = cc_o * AB + ar0 * a.B;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = 8 * lane + 2 * j;
            uB2[j] = colok ? make_float2(a.uB[b], a.uB[b + 1]) : make_float2(0.f, 0.f);
        }
        __syncwarp();
        if (lane < RMAX) s_ua[lane] = lane < nrows ? a.uA[ar0 + lane] : 0.f;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[r][j] = make_float2(0.f, 0.f);
    };

    int si = 0, nis = 0;
    if (lane == 0)
        for (; nis < S - 1 && nis < nloc; ++nis) {
            issue(si);
            ii_next();
            si = si + 1 == S ? 0 : si + 1;
        }
    nis = __shfl_sync(HOSCF_FULLMASK, nis, 0);
    si = __shfl_sync(HOSCF_FULLMASK, si, 0);

    bool ok = true;
    int kfail = nloc;
    int cs = 0;
    uint32_t cph = 0;
    int gbuf = 0, gj = 0;
    for (int k = 0; k < nloc; ++k) {
        if (ok && nis < nloc) {
            if (lane == 0) {
                issue(si);
                ii_next();
            }
            si = si + 1 == S ? 0 : si + 1;
            ++nis;
        }
        if (k == 0 || cc_o == 0) {
            if (k > 0) flush(cc_t);
            ++cc_t;
            new_tile(cc_t);
        }
        const float wo = __ldg(wp);
        float2 y2[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                        make_float2(0.f, 0.f)};
        float y1[RMAX];
        if (ok) {
            const bool got = mbar_wait_bounded(&full[cs], cph, a.timeout_ns);
            if (!__all_sync(HOSCF_FULLMASK, got)) {
                if (lane == 0) atomicCAS(a.err, 0, (int)DEV_TIMEOUT);
                ok = false;
                kfail = k;
            }
        }
        // the band's first element sits `head` bytes into the slot's data
        // (the copy starts at the granule below it); rows past the band and
        // lanes past the row end contribute only to outputs nobody reads or
        // read the zero pad (no branch per row)
        const uint8_t* slot = ring + (size_t)cs * L.slot;
        const uint32_t head = (uint32_t)((uintptr_t)(f0 * ES) & 15u);
        const uint8_t* base = slot + (colok ? head : 0u) + lane_off;
        const float* scl = reinterpret_cast<const float*>(slot + L.data);
        uint32_t gl = 0;        // FP8: flat offset of the lane's chunk past the band's group start
        int32_t gsh = 0;        // and the copied run's first group offset in the slot
        if (F8) {
            gl = (uint32_t)(f0 & 127) + 8u * lane;
            gsh = (int32_t)(((reinterpret_cast<uintptr_t>(a.scales + (f0 >> 7))) & 15u) >> 2);
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            float2 x[4];
            unpack8(reinterpret_cast<const E*>(base + r * row_step), x);
            float m1 = wo, m2 = s_ua[r], sc = 1.f;
            if (F8) {
                sc = scl[(int32_t)((gl + (uint32_t)(r * B)) >> 7) + gsh];
                m1 *= sc;
                m2 *= sc;
            }
            const float2 m12 = make_float2(m1, m1), m22 = make_float2(m2, m2);
            float2 p = make_float2(x[0].x * uB2[0].x, x[0].y * uB2[0].y);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[r][j] = ffma2(m12, x[j], acc[r][j]);
                y2[j] = ffma2(m22, x[j], y2[j]);
                if (j > 0) p = ffma2(x[j], uB2[j], p);
            }
            y1[r] = F8 ? (p.x + p.y) * sc : p.x + p.y;
        }
        __syncwarp();   // every lane is done with slot cs (refilled at the next issue)
        if (++cs == S) {
            cs = 0;
            cph ^= 1u;
        }
        // row sums -> y1: transpose through shared memory (row r, lane l at
        // r*36 + l), then lanes 2r, 2r+1 add 16 partials each
#pragma unroll
        for (int r = 0; r < RMAX; ++r) s_rs[r * kRowSumStride + lane] = y1[r];
        __syncwarp();
        {
            const int row = lane >> 1;
            float ys = 0.f;
            if (row < RMAX) {
                const float4* src = reinterpret_cast<const float4*>(s_rs + row * kRowSumStride + 16 * (lane & 1));
                const float4 q0 = src[0], q1 = src[1], q2 = src[2], q3 = src[3];
                ys = ((q0.x + q0.y) + (q0.z + q0.w)) + ((q1.x + q1.y) + (q1.z + q1.w)) +
                     (((q2.x + q2.y) + (q2.z + q2.w)) + ((q3.x + q3.y) + (q3.z + q3.w)));
            }
            ys += __shfl_xor_sync(HOSCF_FULLMASK, ys, 1);
            if ((lane & 1) == 0 && row < nrows) y1p[row] = ys;
        }
        __syncwarp();
        // column partials -> exchange ring; summed over the 8 warps every G items
        float* sy = s_y2 + ((size_t)(gbuf * G + gj) * 8 + warp) * FB + 8 * lane;
        reinterpret_cast<float4*>(sy)[0] = make_float4(y2[0].x, y2[0].y, y2[1].x, y2[1].y);
        reinterpret_cast<float4*>(sy)[1] = make_float4(y2[2].x, y2[2].y, y2[3].x, y2[3].y);
        if (tid == 0) {
            s_off[gbuf * G + gj] = y2off;
            s_cnt[gbuf * G + gj] = B;
        }
        if (gj == G - 1 || k == nloc - 1) {
            asm volatile("bar.sync 1, 256;" ::: "memory");
            const float* gb = s_y2 + (size_t)gbuf * G * 8 * FB;
            const int n = (gj + 1) * FB;
            for (int e = tid; e < n; e += 256) {
                const int jj = e >> 8, b = e & (FB - 1);
                if (b < s_cnt[gbuf * G + jj]) {
                    float sum = 0.f;
#pragma unroll
                    for (int w8 = 0; w8 < 8; ++w8) sum += gb[((size_t)jj * 8 + w8) * FB + b];
                    a.y2p[s_off[gbuf * G + jj] + b] = sum;
                }
            }
            gbuf ^= 1;
            gj = 0;
        } else {
            ++gj;
        }
        ++wp;
        y1p += a.A;
        y2off += a.B;
        f0 += AB;
        if (++cc_o == a.O) {
            cc_o = 0;
            wp = a.w;
        }
    }
    flush(cc_t);
    if (!ok) {
        // a wait gave up (the code is in the device status word): every copy
        // already issued must still land before the CTA's shared memory is
        // released, so wait for each with a bound of at least 1 s
        const uint64_t drain_ns = a.timeout_ns > 1000000000ull ? a.timeout_ns : 1000000000ull;
        for (int k = kfail; k < nis; ++k) mbar_wait_bounded(&full[k % S], (uint32_t)((k / S) & 1), drain_ns);
    }
}

template <typename E, int RMAX, int OCC>
static cudaError_t launch_narrow_k(const PassPlan& p, const NarrowArgs& a, cudaStream_t st,
                                   const KernelEvents* kev) {
    auto kern = ttvc_narrow_kernel<E, RMAX, OCC>;
    cudaError_t e = allow_max_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
    if (kev) cudaEventRecord(kev->begin, st);
    kern<<<p.grid, 256, p.smem, st>>>(a);
    if (kev) cudaEventRecord(kev->end, st);
    return cudaGetLastError();
}

template <typename E>
static cudaError_t launch_narrow_rows(const PassPlan& p, const NarrowArgs& a, cudaStream_t st,
                                      const KernelEvents* kev) {
    if (p.rows == kNarrowRowsOcc2) return launch_narrow_k<E, kNarrowRowsOcc2, 2>(p, a, st, kev);
    if (p.rows == 16) return launch_narrow_k<E, 16, 1>(p, a, st, kev);
    return launch_narrow_k<E, 13, 1>(p, a, st, kev);
}

cudaError_t launch_narrow(const PassPlan& p, int dtype, const NarrowArgs& a, cudaStream_t st,
                          const KernelEvents* kev) {
    if (dtype == HOSCF_BF16) return launch_narrow_rows<bf16_t>(p, a, st, kev);
    if (dtype == HOSCF_F16) return launch_narrow_rows<f16_t>(p, a, st, kev);
    return launch_narrow_rows<fp8_t>(p, a, st, kev);
}

}  // namespace hoscf
