// All-pairs TTVc pass: every coupling block A_{m,n} = A x_{k!=m,n} u^(k)
// (paper eq. 3.3, Algorithm 1 line 4) from ONE read of the tensor.
//
// Factorisation used (derived from eq. 3.3).  View the row-major tensor as
// T[o][a][b], o over the D = d-2 leading modes, (a, b) the two fastest modes
// ("face").  With w_o = prod_{k<D} u_k[o_k]:
//     H_{D,D+1}[a][b]  = sum_o w_o T[o][a][b]                  (face block)
//     y1[o][a]         = sum_b T[o][a][b] u_{D+1}[b]
//     y2[o][b]         = sum_a T[o][a][b] u_D[a]
// Every other block is a contraction of y1 / y2 over outer modes only:
//     H_{m,D}[i][a]    = sum_{o: o_m=i} prod_{k!=m} u_k[o_k] y1[o][a]
//     H_{m,D+1}[i][b]  = same with y2
//     H_{m,n}[i][j]    = sum_{o: o_m=i,o_n=j} prod_{k!=m,n} u_k[o_k] r[o],
//                        r[o] = sum_a y1[o][a] u_D[a]      (m < n < D)
// so the streaming pass does three FMAs per element and everything after it
// touches tensors smaller by a factor A or B.
//
// Streaming kernel: face tiles of FA x 128, stream-K split of the
// (tile, o) items over a persistent grid.  Each CTA keeps its tile's face
// accumulator in registers, reduces row sums with warp shuffles and column
// sums through a small shared-memory exchange, and writes per-CTA partials;
// the reduce kernels then sum them in a fixed order (no global atomics).
// Tensor slabs arrive by TMA (cp.async.bulk.tensor) into a shared-memory
// ring when the row pitch is 16-byte aligned, else by plain loads.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hoscf {

// ---------------------------------------------------------------- shape/plan
bool make_shape(int d, const int64_t* dims, Shape& s) {
    if (d < 2 || d > kMaxOrder || !dims) return false;
    s = Shape();
    s.d = d;
    s.N = 1;
    for (int k = 0; k < d; ++k) {
        if (dims[k] < 1 || dims[k] > (int64_t(1) << 31)) return false;
        s.dims[k] = dims[k];
        s.moff[k + 1] = s.moff[k] + dims[k];
        if (s.N > (int64_t(1) << 40) / dims[k]) return false;
        s.N *= dims[k];
    }
    s.n_tot = s.moff[d];
    int b = 0;
    for (int m = 0; m < d; ++m)
        for (int n = m + 1; n < d; ++n) {
            s.boff[b + 1] = s.boff[b] + dims[m] * dims[n];
            ++b;
        }
    s.P = s.boff[b];
    s.D = d >= 2 ? d - 2 : 0;
    s.A = dims[d - 2];
    s.B = dims[d - 1];
    s.O = 1;
    for (int k = s.D - 1; k >= 0; --k) {
        s.ost[k] = s.O;
        s.O *= dims[k];
    }
    return true;
}

static int elem_size(int dtype) { return dtype == HOSCF_F32 ? 4 : (dtype == HOSCF_BF16 ? 2 : 1); }

bool make_pass_plan(const Shape& s, int dtype, int nsm, bool tma_ok, PassPlan& p) {
    p = PassPlan();
    if (s.d == 2) {
        p.copy_only = true;
        return true;
    }
    const int es = elem_size(dtype);
    if (make_small_plan(s, nsm, p.sp)) {
        p.small = true;
        size_t off = 0;
        p.sp.off_patch = off;
        off = align_up(off + sizeof(float) * (size_t)p.sp.G * p.sp.patch_floats, 256);
        p.sp.off_cover = off;
        off = align_up(off + sizeof(int) * (size_t)p.sp.G * std::max(1, s.D) * 2, 256);
        p.bytes = off;
        return true;
    }
    // rows per warp: the candidate whose tiles waste the fewest rows of A
    {
        const int cand[3] = {8, 13, 16};
        int best = 8;
        double bw = 1e30;
        for (int r : cand) {
            const int64_t fa = 8 * r, ta = (s.A + fa - 1) / fa;
            const double waste = (double)(ta * fa) / (double)s.A + (r == 8 ? 0.0 : 1e-3 * r);
            if (waste < bw - 1e-9) {
                bw = waste;
                best = r;
            }
        }
        p.rows = best;
    }
    p.FA = 8 * p.rows;
    p.FB = 128;
    p.TA = (s.A + p.FA - 1) / p.FA;
    p.TB = (s.B + p.FB - 1) / p.FB;
    p.TT = p.TA * p.TB;
    p.items = p.TT * s.O;
    // TMA needs 16-byte row and slab pitches and coordinates below 2^31.
    p.tma = tma_ok && (s.B * es) % 16 == 0 && s.O < (int64_t(1) << 31);
    p.vec = (s.B % 4) == 0;
    int64_t grid = std::max<int64_t>(nsm, p.TT);
    if (!p.tma) grid = std::max<int64_t>(grid, 4 * (int64_t)nsm);
    grid = std::min<int64_t>(grid, p.items);
    p.W = (p.items + grid - 1) / grid;
    // W <= O keeps every CTA within two consecutive tiles.
    if (p.W > s.O) {
        p.W = s.O;
    }
    p.grid = (int)((p.items + p.W - 1) / p.W);
    const size_t stage = (size_t)p.FA * p.FB * es;
    if (p.tma) {
        p.nstage = (int)std::min<size_t>(16, std::max<size_t>(2, (192 * 1024) / stage));
        p.smem = 1024 + p.nstage * stage + 2 * p.nstage * 8 + 2 * 8 * p.FB * sizeof(float) + 64;
    } else {
        p.nstage = 0;
        p.smem = 2 * 8 * p.FB * sizeof(float);
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    p.off_w = take(sizeof(float) * (size_t)s.O);
    p.off_hp = take(sizeof(float) * (size_t)p.grid * 2 * p.FA * p.FB);
    p.off_y1p = take(sizeof(float) * (size_t)p.TB * s.O * s.A);
    p.off_y2p = take(sizeof(float) * (size_t)p.TA * s.O * s.B);
    if (s.d >= 4) {
        p.off_y1 = take(sizeof(float) * (size_t)s.O * s.A);
        p.off_y2 = take(sizeof(float) * (size_t)s.O * s.B);
        p.off_r = take(sizeof(float) * (size_t)s.O);
    }
    p.bytes = off;
    return true;
}

// ---------------------------------------------------------------- kernels
struct OuterInfo {
    int D;
    int dims[kMaxOrder];
    int st[kMaxOrder];       // outer strides (o = sum digit_k * st[k])
    int uoff[kMaxOrder];     // factor offsets of the outer modes
};

__device__ __forceinline__ int outer_digit(const OuterInfo& oi, int64_t o, int k) {
    return (int)((o / oi.st[k]) % oi.dims[k]);
}

// w[o] = prod_{k<D} u_k[o_k]
__global__ void outer_weights_kernel(const float* __restrict__ u, OuterInfo oi, int64_t O,
                                     float* __restrict__ w) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < O;
         o += (int64_t)gridDim.x * blockDim.x) {
        float p = 1.f;
        for (int k = 0; k < oi.D; ++k) p *= u[oi.uoff[k] + outer_digit(oi, o, k)];
        w[o] = p;
    }
}

struct TiledArgs {
    const void* T;
    int64_t O, A, B;
    int64_t TB, items, W;
    const float* w;      // O outer weights
    const float* uA;     // factor of mode d-2 (length A)
    const float* uB;     // factor of mode d-1 (length B)
    float* hp;           // grid x 2 x FA x FB face partials
    float* y1p;          // TB x O x A
    float* y2p;          // TA x O x B
    int* err;
    uint64_t timeout_ns;
    const float* scales;   // FP8 only: one per 128 flat elements
};

// Reduce-scatter of NV per-lane row partials over the 32 lanes; returns the
// full sum of row `row` (lanes sharing a row hold the same value).
template <int NV>
__device__ __forceinline__ float rs_reduce(float (&y)[NV], int lane, int& row) {
    row = 0;
    int mask = 16;
#pragma unroll
    for (int h = NV / 2; h >= 1; h >>= 1) {
        const bool up = (lane & mask) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const float send = up ? y[k] : y[k + h];
            const float keep = up ? y[k + h] : y[k];
            y[k] = keep + __shfl_xor_sync(HOSCF_FULLMASK, send, mask);
        }
        row += up ? h : 0;
        mask >>= 1;
    }
#pragma unroll
    for (int m = 16 / NV; m >= 1; m >>= 1) y[0] += __shfl_xor_sync(HOSCF_FULLMASK, y[0], m);
    return y[0];
}

// Four consecutive elements -> float (no scaling).
__device__ __forceinline__ void unpack4(float4 q, float (&v)[4]) {
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void unpack4(uint2 q, float (&v)[4]) {   // 4 x bf16
    v[0] = __uint_as_float(q.x << 16);
    v[1] = __uint_as_float(q.x & 0xffff0000u);
    v[2] = __uint_as_float(q.y << 16);
    v[3] = __uint_as_float(q.y & 0xffff0000u);
}
__device__ __forceinline__ void unpack4(uint32_t q, float (&v)[4]) {   // 4 x fp8 e4m3
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q & 0xffffu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(q >> 16), __NV_E4M3);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&lo));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&hi));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename E> struct Pack4;
template <> struct Pack4<float> { using T = float4; };
template <> struct Pack4<bf16_t> { using T = uint2; };
template <> struct Pack4<fp8_t> { using T = uint32_t; };

template <typename E>
__device__ __forceinline__ void load4_smem(const E* row, int col, float (&v)[4]) {
    unpack4(*reinterpret_cast<const typename Pack4<E>::T*>(row + col), v);
}

template <typename E>
__device__ __forceinline__ void load4_global_vec(const E* p, float (&v)[4]) {
    unpack4(__ldcs(reinterpret_cast<const typename Pack4<E>::T*>(p)), v);
}

template <typename E>
__device__ __forceinline__ float load1_global(const E* p);
template <>
__device__ __forceinline__ float load1_global<float>(const float* p) { return __ldcs(p); }
template <>
__device__ __forceinline__ float load1_global<bf16_t>(const bf16_t* p) {
    const uint16_t b = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(static_cast<uint32_t>(b) << 16);
}
template <>
__device__ __forceinline__ float load1_global<fp8_t>(const fp8_t* p) {
    const uint8_t c = __ldcs(reinterpret_cast<const unsigned char*>(p));
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3);
    return __half2float(*reinterpret_cast<const __half*>(&h));
}

// FP8 storage: multiply each of the lane's four values by the scale of its
// 128-element group (flat row-major index f0 .. f0+3 spans at most two groups).
__device__ __forceinline__ void apply_scales(const float* __restrict__ scales, int64_t f0,
                                             float (&v)[4]) {
    const int64_t g0 = f0 >> 7;
    const float s0 = __ldg(scales + g0);
    const float s1 = ((f0 + 3) >> 7) != g0 ? __ldg(scales + g0 + 1) : s0;
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] *= (((f0 + c) >> 7) == g0) ? s0 : s1;
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

// How the consumer warps get their tile rows.
enum LoadMode : int { LOAD_TMA = 0, LOAD_VEC = 1, LOAD_SCALAR = 2 };

// The streaming kernel.  Threads 0..255 are 8 consumer warps; with TMA a
// ninth warp issues the bulk tensor copies.  Consumer warp w owns rows
// [w*ROWS, (w+1)*ROWS) of the FA x 128 tile, lane l owns columns 4l..4l+3.
// Without TMA the consumers load their own rows (16-byte vector loads when
// rows are aligned, else element by element).
template <typename E, int MODE, int ROWS>
__global__ void __launch_bounds__(MODE == LOAD_TMA ? 288 : 256, 1)
    ttvc_tiled_kernel(const __grid_constant__ CUtensorMap tmap, const TiledArgs a, int nstage) {
    constexpr bool TMA = MODE == LOAD_TMA;
    constexpr int FA = 8 * ROWS;
    constexpr int FB = 128;
    constexpr int STAGE = FA * FB;   // elements
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~uintptr_t(1023));
    E* stages = reinterpret_cast<E*>(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (TMA ? (size_t)nstage * STAGE * sizeof(E) : 0));
    uint64_t* empty = full + (TMA ? nstage : 0);
    float* s_y2 = reinterpret_cast<float*>(empty + (TMA ? nstage : 0));   // [2][8][FB]

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t c = blockIdx.x;
    const int64_t i0 = c * a.W;
    const int64_t i1 = min(i0 + a.W, a.items);
    if (i0 >= i1) return;
    const int64_t nloc = i1 - i0;

    if (TMA) {
        if (tid == 0) {
            for (int s = 0; s < nstage; ++s) {
                mbar_init(&full[s], 1);
                mbar_init(&empty[s], 8);
            }
            fence_mbar_init();
        }
        __syncthreads();
        if (warp == 8) {
            if (lane == 0) {
                prefetch_tmap(&tmap);
                for (int64_t k = 0; k < nloc; ++k) {
                    const int64_t item = i0 + k;
                    const int64_t t = item / a.O;
                    const int64_t o = item - t * a.O;
                    const int s = (int)(k % nstage);
                    if (k >= nstage) {
                        const uint32_t par = (uint32_t)(((k / nstage) - 1) & 1);
                        if (!mbar_wait_bounded(&empty[s], par, a.timeout_ns)) {
                            atomicCAS(a.err, 0, (int)DEV_TIMEOUT);
                            break;
                        }
                    }
                    mbar_arrive_expect_tx(&full[s], STAGE * sizeof(E));
                    tma_load_3d(stages + (size_t)s * STAGE, &tmap, (int)((t % a.TB) * FB),
                                (int)((t / a.TB) * FA), (int)o, &full[s]);
                }
            }
            return;
        }
    }

    float2 acc[ROWS][2];
    float2 uB2[2];
    float uAr[ROWS];
    int64_t cur_t = -1;
    int64_t ta = 0, tb = 0;
    const int64_t t_first = i0 / a.O;

    auto flush = [&](int64_t t) {
        const int seg = (int)(t - t_first);
        float* dst = a.hp + ((size_t)(c * 2 + seg) * FA) * FB;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            float4 q = make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y);
            *reinterpret_cast<float4*>(dst + (size_t)(warp * ROWS + r) * FB + 4 * lane) = q;
        }
    };

    bool ok = true;
    for (int64_t k = 0; k < nloc; ++k) {
        const int64_t item = i0 + k;
        const int64_t t = item / a.O;
        const int64_t o = item - t * a.O;
        if (t != cur_t) {
            if (cur_t >= 0) flush(cur_t);
            cur_t = t;
            ta = t / a.TB;
            tb = t - ta * a.TB;
            float ub[4];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int64_t b = tb * FB + 4 * lane + cc;
                ub[cc] = b < a.B ? a.uB[b] : 0.f;
            }
            uB2[0] = make_float2(ub[0], ub[1]);
            uB2[1] = make_float2(ub[2], ub[3]);
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const int64_t ar = ta * FA + warp * ROWS + r;
                uAr[r] = ar < a.A ? a.uA[ar] : 0.f;
                acc[r][0] = make_float2(0.f, 0.f);
                acc[r][1] = make_float2(0.f, 0.f);
            }
        }
        const float wo = __ldg(a.w + o);
        const float2 wo2 = make_float2(wo, wo);
        constexpr int RP = ROWS <= 8 ? 8 : (ROWS <= 16 ? 16 : 32);
        float y1[RP];
#pragma unroll
        for (int r = ROWS; r < RP; ++r) y1[r] = 0.f;
        float2 y2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        const int s = TMA ? (int)(k % nstage) : 0;
        if (TMA) {
            const uint32_t par = (uint32_t)((k / nstage) & 1);
            if (ok && !mbar_wait_bounded(&full[s], par, a.timeout_ns)) {
                atomicCAS(a.err, 0, (int)DEV_TIMEOUT);
                ok = false;
            }
        }
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            float v[4];
            const int64_t ar = ta * FA + warp * ROWS + r;
            const int64_t b0 = tb * FB + 4 * lane;
            if (TMA) {
                load4_smem<E>(stages + (size_t)s * STAGE + (size_t)(warp * ROWS + r) * FB,
                              4 * lane, v);
            } else if (MODE == LOAD_VEC) {
                const E* rowp = reinterpret_cast<const E*>(a.T) + ((size_t)o * a.A + ar) * a.B;
                if (ar < a.A && b0 < a.B) {
                    load4_global_vec<E>(rowp + b0, v);   // B % 4 == 0: all four in range
                } else {
                    v[0] = v[1] = v[2] = v[3] = 0.f;
                }
            } else {
                const E* rowp = reinterpret_cast<const E*>(a.T) + ((size_t)o * a.A + ar) * a.B;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int64_t b = b0 + cc;
                    v[cc] = (ar < a.A && b < a.B) ? load1_global<E>(rowp + b) : 0.f;
                }
            }
            if (std::is_same<E, fp8_t>::value && ar < a.A && b0 < a.B)
                apply_scales(a.scales, ((int64_t)o * a.A + ar) * a.B + b0, v);
            const float2 v0 = make_float2(v[0], v[1]), v1 = make_float2(v[2], v[3]);
            acc[r][0] = ffma2(wo2, v0, acc[r][0]);
            acc[r][1] = ffma2(wo2, v1, acc[r][1]);
            const float2 ua2 = make_float2(uAr[r], uAr[r]);
            y2[0] = ffma2(v0, ua2, y2[0]);
            y2[1] = ffma2(v1, ua2, y2[1]);
            const float2 dd = ffma2(v1, uB2[1], make_float2(v0.x * uB2[0].x, v0.y * uB2[0].y));
            y1[r] = dd.x + dd.y;
        }
        if (TMA) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        // row sums -> y1 partial of this b-tile
        int row;
        const float ys = rs_reduce<RP>(y1, lane, row);
        if ((lane & ((32 / RP) - 1)) == 0 && row < ROWS) {
            const int64_t ar = ta * FA + warp * ROWS + row;
            if (ar < a.A) a.y1p[((size_t)tb * a.O + o) * a.A + ar] = ys;
        }
        // column sums over the 8 warps -> y2 partial of this a-tile
        float* sy = s_y2 + (size_t)(k & 1) * 8 * FB;
        *reinterpret_cast<float4*>(sy + warp * FB + 4 * lane) = make_float4(y2[0].x, y2[0].y, y2[1].x, y2[1].y);
        asm volatile("bar.sync 1, 256;" ::: "memory");
        if (tid < FB) {
            float sum = 0.f;
#pragma unroll
            for (int w8 = 0; w8 < 8; ++w8) sum += sy[w8 * FB + tid];
            const int64_t b = tb * FB + tid;
            if (b < a.B) a.y2p[((size_t)ta * a.O + o) * a.B + b] = sum;
        }
    }
    if (cur_t >= 0) flush(cur_t);
    if (TMA && !ok) {
        // a wait gave up: let copies already issued land before the CTA exits
        for (int64_t k = (nloc > nstage ? nloc - nstage : 0); k < nloc; ++k)
            mbar_wait_bounded(&full[k % nstage], (uint32_t)((k / nstage) & 1), a.timeout_ns);
    }
}

// H_{D,D+1}[a][b] = sum of the face partials of every CTA that touched the
// tile, in CTA order.
__global__ void reduce_face_kernel(const float* __restrict__ hp, float* __restrict__ out,
                                   int64_t A, int64_t B, int FA, int FB, int64_t TB, int64_t O,
                                   int64_t W) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < A * B;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t aa = idx / B, bb = idx - (idx / B) * B;
        const int64_t ta = aa / FA, tb = bb / FB;
        const int64_t t = ta * TB + tb;
        const int64_t c_lo = (t * O) / W, c_hi = ((t + 1) * O - 1) / W;
        float s = 0.f;
        for (int64_t c = c_lo; c <= c_hi; ++c) {
            const int64_t seg = t - (c * W) / O;
            s += hp[((size_t)(c * 2 + seg) * FA + (aa - ta * FA)) * FB + (bb - tb * FB)];
        }
        out[idx] = s;
    }
}

// out[i] = sum_{p < np} part[p * stride + i]
__global__ void reduce_parts_kernel(const float* __restrict__ part, float* __restrict__ out,
                                    int64_t n, int64_t np, int64_t stride) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int64_t p = 0; p < np; ++p) s += part[p * stride + i];
        out[i] = s;
    }
}

// Cross blocks H_{m,face}[i][col] = sum_{o: o_m = i} prod_{k!=m} u_k[o_k] y[o][col]
// for every outer mode m; one CTA row per (m, i), columns over threads.
struct ModeOffs {
    int64_t off[kMaxOrder];
};

__global__ void fold_cross_kernel(const float* __restrict__ y, int64_t C, const float* __restrict__ u,
                                  OuterInfo oi, int64_t O, float* __restrict__ H,
                                  const ModeOffs row_block_off) {
    // blockIdx.x enumerates (m, i) rows: rows of mode m start at sum_{k<m} I_k
    int m = 0;
    int64_t row = blockIdx.x;
    while (m < oi.D - 1 && row >= oi.dims[m]) {
        row -= oi.dims[m];
        ++m;
    }
    const int i = (int)row;
    const int64_t Im = oi.dims[m];
    const int64_t stm = oi.st[m];
    const int64_t pre = O / (Im * stm);
    const int64_t col = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
    if (col >= C) return;
    float acc = 0.f;
    for (int64_t p = 0; p < pre; ++p) {
        for (int64_t s = 0; s < stm; ++s) {
            const int64_t o = (p * Im + i) * stm + s;
            float pi = 1.f;
            for (int k = 0; k < oi.D; ++k)
                if (k != m) pi *= __ldg(u + oi.uoff[k] + outer_digit(oi, o, k));
            acc = fmaf(pi, __ldg(y + o * C + col), acc);
        }
    }
    H[row_block_off.off[m] + (int64_t)i * C + col] = acc;
}

// r[o] = sum_a y1[o][a] uA[a]   (one warp per o)
__global__ void fold_r_kernel(const float* __restrict__ y1, const float* __restrict__ uA, int64_t O,
                              int64_t A, float* __restrict__ r) {
    const int lane = threadIdx.x & 31;
    for (int64_t o = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; o < O;
         o += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
        for (int64_t aa = lane; aa < A; aa += 32) s = fmaf(y1[o * A + aa], uA[aa], s);
        s = warp_sum(s);
        if (lane == 0) r[o] = s;
    }
}

// Outer pairs H_{m,n}[i][j] = sum_{o: o_m=i, o_n=j} prod_{k!=m,n} u_k[o_k] r[o].
struct PairInfo {
    int npairs;
    int pm[kMaxBlocks], pn[kMaxBlocks];
    int64_t start[kMaxBlocks + 1];   // prefix of I_m*I_n over the pairs
    int64_t hoff[kMaxBlocks];        // packed block offsets
};

__global__ void fold_pairs_kernel(const float* __restrict__ r, const float* __restrict__ u,
                                  OuterInfo oi, PairInfo pi_, int64_t O, float* __restrict__ H) {
    const int64_t total = pi_.start[pi_.npairs];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int p = 0;
        while (e >= pi_.start[p + 1]) ++p;
        const int m = pi_.pm[p], n = pi_.pn[p];
        const int64_t loc = e - pi_.start[p];
        const int i = (int)(loc / oi.dims[n]), j = (int)(loc % oi.dims[n]);
        const int64_t M = O / ((int64_t)oi.dims[m] * oi.dims[n]);
        float acc = 0.f;
        for (int64_t q = 0; q < M; ++q) {
            // digits of the other outer modes from q (row-major over them)
            int64_t rem = q, o = (int64_t)i * oi.st[m] + (int64_t)j * oi.st[n];
            float pw = 1.f;
            for (int k = oi.D - 1; k >= 0; --k) {
                if (k == m || k == n) continue;
                const int dk = (int)(rem % oi.dims[k]);
                rem /= oi.dims[k];
                o += (int64_t)dk * oi.st[k];
                pw *= __ldg(u + oi.uoff[k] + dk);
            }
            acc = fmaf(pw, r[o], acc);
        }
        H[pi_.hoff[p] + loc] = acc;
    }
}

// d == 2: the only block is the matrix itself.
__global__ void copy_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void bf16_to_f32_kernel(const uint16_t* __restrict__ src, float* __restrict__ dst,
                                   int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __uint_as_float(static_cast<uint32_t>(src[i]) << 16);
}

// ---------------------------------------------------------------- host
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

static OuterInfo make_outer(const Shape& s) {
    OuterInfo oi;
    memset(&oi, 0, sizeof(oi));
    oi.D = s.D;
    for (int k = 0; k < s.D; ++k) {
        oi.dims[k] = (int)s.dims[k];
        oi.st[k] = (int)s.ost[k];
        oi.uoff[k] = (int)s.moff[k];
    }
    return oi;
}

static int grid_for(int64_t n, int threads, int cap) {
    int64_t g = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

template <typename E, int MODE, int ROWS>
static cudaError_t launch_tiled_k(const PassPlan& p, const CUtensorMap& map, const TiledArgs& a,
                                  cudaStream_t st) {
    auto kern = ttvc_tiled_kernel<E, MODE, ROWS>;
    const size_t smem = MODE == LOAD_TMA ? p.smem : (size_t)2 * 8 * 128 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<p.grid, MODE == LOAD_TMA ? 288 : 256, smem, st>>>(map, a, p.nstage);
    return cudaGetLastError();
}

template <typename E, int MODE>
static cudaError_t launch_tiled_rows(const PassPlan& p, const CUtensorMap& map, const TiledArgs& a,
                                     cudaStream_t st) {
    if (MODE == LOAD_SCALAR || p.rows == 8) return launch_tiled_k<E, MODE, 8>(p, map, a, st);
    if (p.rows == 13) return launch_tiled_k<E, MODE, 13>(p, map, a, st);
    return launch_tiled_k<E, MODE, 16>(p, map, a, st);
}

template <typename E>
static cudaError_t launch_tiled(const PassPlan& p, int mode, const CUtensorMap& map,
                                const TiledArgs& a, cudaStream_t st) {
    if (mode == LOAD_TMA) return launch_tiled_rows<E, LOAD_TMA>(p, map, a, st);
    if (mode == LOAD_VEC) return launch_tiled_rows<E, LOAD_VEC>(p, map, a, st);
    return launch_tiled_rows<E, LOAD_SCALAR>(p, map, a, st);
}

__global__ void fp8_to_f32_kernel(const uint8_t* __restrict__ src, const float* __restrict__ scales,
                                  float* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)src[i], __NV_E4M3);
        dst[i] = __half2float(*reinterpret_cast<const __half*>(&h)) * scales[i >> 7];
    }
}

// Runs the whole pass: blocks H (P floats, packed) from T and u.
hoscf_status run_ttvc(const Shape& s, const PassPlan& p, int dtype, const void* data,
                      const float* scales, const float* u, float* H, char* ws, int* dev_err,
                      uint64_t timeout_ns, cudaStream_t st, Err& err) {
    (void)scales;
    cudaError_t ce;
#define HOSCF_CK(x)                                                                  \
    do {                                                                             \
        ce = (x);                                                                    \
        if (ce != cudaSuccess) {                                                     \
            err.code = HOSCF_ECUDA;                                                  \
            snprintf(err.msg, sizeof(err.msg), "%s: %s", #x, cudaGetErrorString(ce)); \
            return err.code;                                                         \
        }                                                                            \
    } while (0)
    if (p.copy_only) {
        if (dtype == HOSCF_F32) {
            copy_kernel<<<grid_for(s.N, 256, 4096), 256, 0, st>>>((const float*)data, H, s.N);
        } else if (dtype == HOSCF_BF16) {
            bf16_to_f32_kernel<<<grid_for(s.N, 256, 4096), 256, 0, st>>>((const uint16_t*)data, H,
                                                                         s.N);
        } else {
            fp8_to_f32_kernel<<<grid_for(s.N, 256, 4096), 256, 0, st>>>((const uint8_t*)data,
                                                                        scales, H, s.N);
        }
        HOSCF_CK(cudaGetLastError());
        return HOSCF_OK;
    }
    if (p.small) {
        HOSCF_CK(run_small(s, p.sp, dtype, data, scales, u, H, ws, st));
        return HOSCF_OK;
    }
    const OuterInfo oi = make_outer(s);
    float* w = reinterpret_cast<float*>(ws + p.off_w);
    const float* wptr;
    if (s.D == 1) {
        wptr = u;   // w[o] = u_0[o]
    } else {
        outer_weights_kernel<<<grid_for(s.O, 256, 4096), 256, 0, st>>>(u, oi, s.O, w);
        HOSCF_CK(cudaGetLastError());
        wptr = w;
    }
    TiledArgs a;
    a.T = data;
    a.O = s.O;
    a.A = s.A;
    a.B = s.B;
    a.TB = p.TB;
    a.items = p.items;
    a.W = p.W;
    a.w = wptr;
    a.uA = u + s.moff[s.d - 2];
    a.uB = u + s.moff[s.d - 1];
    a.hp = reinterpret_cast<float*>(ws + p.off_hp);
    a.y1p = reinterpret_cast<float*>(ws + p.off_y1p);
    a.y2p = reinterpret_cast<float*>(ws + p.off_y2p);
    a.err = dev_err;
    a.timeout_ns = timeout_ns;
    a.scales = scales;

    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    bool use_tma = p.tma;
    if (use_tma) {
        EncodeTiledFn enc = get_encode_fn();
        const int es = elem_size(dtype);
        cuuint64_t gdim[3] = {(cuuint64_t)s.B, (cuuint64_t)s.A, (cuuint64_t)s.O};
        cuuint64_t gstr[2] = {(cuuint64_t)(s.B * es), (cuuint64_t)(s.A * s.B * es)};
        cuuint32_t box[3] = {(cuuint32_t)p.FB, (cuuint32_t)p.FA, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        CUtensorMapDataType dt = dtype == HOSCF_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : dtype == HOSCF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_UINT8;
        if (!enc || (reinterpret_cast<uintptr_t>(data) & 15) != 0 ||
            enc(&map, dt, 3, const_cast<void*>(data), gdim, gstr, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            use_tma = false;
    }
    const int mode = use_tma ? LOAD_TMA
                     : (p.vec && (reinterpret_cast<uintptr_t>(data) & 15) == 0) ? LOAD_VEC
                                                                                : LOAD_SCALAR;
    if (dtype == HOSCF_F32) {
        HOSCF_CK(launch_tiled<float>(p, mode, map, a, st));
    } else if (dtype == HOSCF_BF16) {
        HOSCF_CK(launch_tiled<bf16_t>(p, mode, map, a, st));
    } else {
        HOSCF_CK(launch_tiled<fp8_t>(p, mode, map, a, st));
    }
    // face block (d-2, d-1)
    float* Hface = H + s.boff[block_index(s.d, s.d - 2, s.d - 1)];
    reduce_face_kernel<<<grid_for(s.A * s.B, 256, 8192), 256, 0, st>>>(
        a.hp, Hface, s.A, s.B, p.FA, p.FB, p.TB, s.O, p.W);
    HOSCF_CK(cudaGetLastError());
    if (s.d == 3) {
        // y1 = H_{0,1} (I_0 x A), y2 = H_{0,2} (I_0 x B)
        reduce_parts_kernel<<<grid_for(s.O * s.A, 256, 8192), 256, 0, st>>>(
            a.y1p, H + s.boff[block_index(3, 0, 1)], s.O * s.A, p.TB, s.O * s.A);
        reduce_parts_kernel<<<grid_for(s.O * s.B, 256, 8192), 256, 0, st>>>(
            a.y2p, H + s.boff[block_index(3, 0, 2)], s.O * s.B, p.TA, s.O * s.B);
        HOSCF_CK(cudaGetLastError());
        return HOSCF_OK;
    }
    float* y1 = reinterpret_cast<float*>(ws + p.off_y1);
    float* y2 = reinterpret_cast<float*>(ws + p.off_y2);
    float* r = reinterpret_cast<float*>(ws + p.off_r);
    reduce_parts_kernel<<<grid_for(s.O * s.A, 256, 8192), 256, 0, st>>>(a.y1p, y1, s.O * s.A, p.TB,
                                                                       s.O * s.A);
    reduce_parts_kernel<<<grid_for(s.O * s.B, 256, 8192), 256, 0, st>>>(a.y2p, y2, s.O * s.B, p.TA,
                                                                       s.O * s.B);
    HOSCF_CK(cudaGetLastError());
    // cross blocks (m, d-2) from y1 and (m, d-1) from y2
    int64_t rows = 0;
    for (int k = 0; k < s.D; ++k) rows += s.dims[k];
    ModeOffs off1, off2;
    for (int m = 0; m < s.D; ++m) {
        off1.off[m] = s.boff[block_index(s.d, m, s.d - 2)];
        off2.off[m] = s.boff[block_index(s.d, m, s.d - 1)];
    }
    {
        dim3 g1((unsigned)rows, (unsigned)((s.A + 255) / 256));
        fold_cross_kernel<<<g1, 256, 0, st>>>(y1, s.A, u, oi, s.O, H, off1);
        dim3 g2((unsigned)rows, (unsigned)((s.B + 255) / 256));
        fold_cross_kernel<<<g2, 256, 0, st>>>(y2, s.B, u, oi, s.O, H, off2);
        HOSCF_CK(cudaGetLastError());
    }
    if (s.D >= 2) {
        fold_r_kernel<<<grid_for(s.O * 32, 256, 8192), 256, 0, st>>>(y1, a.uA, s.O, s.A, r);
        PairInfo pi_;
        memset(&pi_, 0, sizeof(pi_));
        int np = 0;
        for (int m = 0; m < s.D; ++m)
            for (int n = m + 1; n < s.D; ++n) {
                pi_.pm[np] = m;
                pi_.pn[np] = n;
                pi_.hoff[np] = s.boff[block_index(s.d, m, n)];
                pi_.start[np + 1] = pi_.start[np] + s.dims[m] * s.dims[n];
                ++np;
            }
        pi_.npairs = np;
        fold_pairs_kernel<<<grid_for(pi_.start[np], 128, 8192), 128, 0, st>>>(r, u, oi, pi_, s.O, H);
        HOSCF_CK(cudaGetLastError());
    }
    return HOSCF_OK;
#undef HOSCF_CK
}

}  // namespace hoscf
