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

static int elem_size(int dtype) {
    return dtype == HOSCF_F32 ? 4 : (dtype == HOSCF_BF16 || dtype == HOSCF_F16) ? 2 : 1;
}

bool make_pass_plan(const Shape& s, int dtype, int nsm, bool tma_ok, PassPlan& p) {
    p = PassPlan();
    p.nsm = nsm;
    if (s.d == 2) {
        p.copy_only = true;
        return true;
    }
    const int es = elem_size(dtype);
    if (make_small_plan(s, dtype, nsm, p.sp)) {
        p.small = true;
        size_t off = 0;
        p.sp.off_patch = off;
        off = align_up(off + sizeof(float) * (size_t)p.sp.G * p.sp.patch_floats, 256);
        p.sp.off_cover = off;
        off = align_up(off + sizeof(int) * (size_t)p.sp.G * std::max(1, s.D) * 2, 256);
        p.bytes = off;
        return true;
    }
    // Narrow formats with rows of 128 .. 256 elements, a multiple of 8: the
    // full-row kernel (narrow.cu), 8 columns per lane, HOSCF_NARROW_OCC CTAs
    // per SM (2: at most kNarrowRowsOcc2 rows per warp; 1: 13 or 16).
    p.narrow = es < 4 && s.B % 8 == 0 && s.B >= 128 && s.B <= 256;
    // CTAs per SM (see TiledOcc): 2 for the narrow formats in the tiled
    // kernel, which then get half the shared memory and at most 13 rows per warp.
    const int occ = es == 4 ? 1 : (p.narrow ? HOSCF_NARROW_OCC : 2);
    if (p.narrow) {
        // rows per warp at most, then the fewest tiles and their rows split
        // evenly over the 8 warps (no idle warp for e.g. A = 200)
        int rmax = kNarrowRowsOcc2;
        if (occ == 1) rmax = (s.A + 103) / 104 <= (s.A + 127) / 128 ? 13 : 16;
        const int64_t ta = (s.A + 8 * rmax - 1) / (8 * rmax);
        p.rows = rmax;
        p.FA = (int)((s.A + ta - 1) / ta);
    } else
    // rows per warp: the candidate whose tiles waste the fewest rows of A,
    // the taller tile on ties (fewer column partials, per-item work spread
    // over more rows)
    {
        const int cand[3] = {8, 13, 16};
        int best = 8;
        double bw = 1e30;
        for (int r : cand) {
            if (occ == 2 && r > 13) continue;
            const int64_t fa = 8 * r, ta = (s.A + fa - 1) / fa;
            const double waste = (double)(ta * fa) / (double)s.A - 1e-4 * r;
            if (waste < bw - 1e-9) {
                bw = waste;
                best = r;
            }
        }
        p.rows = best;
        p.FA = 8 * p.rows;
    }
    p.FB = p.narrow ? 256 : 128;
    p.TA = (s.A + p.FA - 1) / p.FA;
    p.TB = (s.B + p.FB - 1) / p.FB;
    p.TT = p.TA * p.TB;
    p.items = p.TT * s.O;
    // TMA needs 16-byte row and slab pitches and coordinates below 2^31.
    p.tma = tma_ok && (s.B * es) % 16 == 0 && s.O < (int64_t(1) << 31);
    p.vec = (s.B % 4) == 0;
    // Work split.  Stream-K: CTA c takes items [c W, (c+1) W) of the
    // tile-major item list, W <= O, so it meets at most two tiles.  Per tile:
    // CTA c takes chunk c % P of tile c / P's outer indices, so the CTAs of
    // the column tiles of one row band walk the same outer indices at the
    // same time and share the DRAM lines where a row crosses from one
    // column tile to the next.  Per tile is used when it finishes no later
    // (in items per CTA times waves of resident CTAs) than stream-K.
    const int64_t R = (int64_t)occ * nsm;
    int64_t grid = std::max<int64_t>(R, p.TT);
    grid = std::min<int64_t>(grid, p.items);
    p.W = (p.items + grid - 1) / grid;
    if (p.W > s.O) {
        p.W = s.O;
    }
    p.grid = (int)((p.items + p.W - 1) / p.W);
    p.P = 0;
    {
        const int64_t sk_span = p.W * ((p.grid + R - 1) / R);
        int64_t best_span = -1, best_P = 0, best_W = 0;
        const int64_t pmax = std::min<int64_t>(s.O, 2 * R / p.TT + 1);
        for (int64_t P = 1; P <= pmax; ++P) {
            const int64_t W = (s.O + P - 1) / P;
            const int64_t Pn = (s.O + W - 1) / W;   // no empty chunk
            const int64_t span = W * ((p.TT * Pn + R - 1) / R);
            if (best_span < 0 || span < best_span) {
                best_span = span;
                best_P = Pn;
                best_W = W;
            }
        }
        if (best_span >= 0 && best_span * 100 <= sk_span * 102 && p.TT * best_P < (int64_t(1) << 31)) {
            p.P = best_P;
            p.W = best_W;
            p.grid = (int)(p.TT * best_P);
        }
    }
    // Ring depth S (>= 3) and exchange group G: a group of up to 4 items
    // first, then a deeper ring (up to 8), then a larger group.
    {
        const size_t cap = occ == 1 ? 227 * 1024 - 1024 : 112 * 1024;
        const bool fp8 = dtype == HOSCF_F8E4M3;
        int S = 0, G = 0, best = -1;
        for (int g = 8; g >= 1; g /= 2) {
            int sg = 16;
            while (sg >= 3 && tiled_smem(sg, g, p.rows, es, fp8).total > cap) --sg;
            if (sg < 3) continue;
            const int score = std::min(g, 4) * 100 + std::min(sg, 8) * 10 + g;
            if (score > best) {
                best = score;
                S = sg;
                G = g;
            }
        }
        if (G < 1) return false;
        p.group = G;
        if (p.narrow) {
            // ring depth first (up to 8 items in flight per warp), then the group
            const size_t ncap = occ == 1 ? 227 * 1024 - 1024 : 113 * 1024 - 1024;
            int Sn = 0, Gn = 0, bestn = -1;
            for (int g = 8; g >= 1; g /= 2) {
                int sg = 16;
                while (sg >= 3 && narrow_smem(sg, g, p.rows, s.B, es, fp8).total > ncap) --sg;
                if (sg < 3) continue;
                const int score = std::min(sg, 8) * 100 + std::min(g, 4) * 10 + g;
                if (score > bestn) {
                    bestn = score;
                    Sn = sg;
                    Gn = g;
                }
            }
            if (Gn < 1) {
                p.narrow = false;   // cannot happen for B <= 256; keep the tiled kernel
            } else {
                p.group = Gn;
                p.nstage = Sn;
                p.slot_bytes = (int)narrow_slot_bytes(p.rows, s.B, es, fp8);
                p.smem = 1024 + narrow_smem(Sn, Gn, p.rows, s.B, es, fp8).total;
                p.tma = false;
            }
        }
        if (p.narrow) {
        } else if (p.tma || p.vec) {
            p.nstage = S;
            p.smem = 1024 + tiled_smem(S, G, p.rows, es, fp8).total;
        } else {
            p.nstage = 0;
            p.smem = 1024 + tiled_smem(0, G, p.rows, es, fp8).total;
        }
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
        p.off_wx = take(sizeof(float) * (size_t)s.D * s.O);
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
    int nstage;            // ring slots per warp
    int group;             // items per column-sum exchange
    int64_t P;             // outer-index chunks per tile (0: stream-K split)
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

__device__ __forceinline__ void unpack4_f16(uint2 q, float (&v)[4]) {   // 4 x IEEE half
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename E> struct Pack4;
template <> struct Pack4<float> { using T = float4; };
template <> struct Pack4<bf16_t> { using T = uint2; };
template <> struct Pack4<f16_t> { using T = uint2; };
template <> struct Pack4<fp8_t> { using T = uint32_t; };

// Four consecutive elements of type E (packed as Pack4<E>::T) -> float.
template <typename E>
__device__ __forceinline__ void unpack4e(typename Pack4<E>::T q, float (&v)[4]) { unpack4(q, v); }
template <>
__device__ __forceinline__ void unpack4e<f16_t>(uint2 q, float (&v)[4]) { unpack4_f16(q, v); }

template <typename E>
__device__ __forceinline__ void load4_smem(const E* row, int col, float (&v)[4]) {
    unpack4e<E>(*reinterpret_cast<const typename Pack4<E>::T*>(row + col), v);
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
__device__ __forceinline__ float load1_global<f16_t>(const f16_t* p) {
    const unsigned short b = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __half2float(__ushort_as_half(b));
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

// How each warp gets its tile rows.
enum LoadMode : int { LOAD_TMA = 0, LOAD_ASYNC = 1, LOAD_SCALAR = 2 };

// CTAs per SM of the streaming kernel: one for FP32 (HBM-bound with 8 warps),
// two for the narrow formats, whose per-element instruction count needs
// more warps in flight to keep up with HBM.
template <typename E>
struct TiledOcc {
    static constexpr int value = sizeof(E) == 4 ? 1 : 2;
};

// The streaming kernel: 8 warps, warp w owns rows [w*ROWS, (w+1)*ROWS) of
// the FA x 128 face tile and lane l its columns 4l..4l+3.  Every warp runs
// its own ring of S slots (its rows of one item each): a TMA box of ROWS x
// 128 issued by lane 0, or per-lane cp.async of the lane's four elements;
// FP8 group scales ride along as per-lane cp.async.  One mbarrier per slot
// tracks both, so warps proceed independently; they meet only every G items
// to sum their column partials (double-buffered, one barrier per group).
// LOAD_SCALAR (rows not a multiple of 4 elements) reads global memory
// directly, element by element.  Items of a CTA are consecutive outer
// indices of at most two tiles, so per-item offsets advance by constant
// strides and are recomputed only when the tile changes.
template <typename E, int MODE, int ROWS>
__global__ void __launch_bounds__(256, TiledOcc<E>::value)
    ttvc_tiled_kernel(const __grid_constant__ CUtensorMap tmap, const TiledArgs a) {
    constexpr int FA = 8 * ROWS;
    constexpr int FB = 128;
    constexpr int SLOT = ROWS * FB;   // elements of one warp slot
    constexpr bool F8 = std::is_same<E, fp8_t>::value;
    constexpr bool RING = MODE != LOAD_SCALAR;
    constexpr bool CPA = MODE == LOAD_ASYNC || (F8 && RING);   // lanes issue cp.async
    using P4 = typename Pack4<E>::T;
    const int S = RING ? a.nstage : 0;
    const int G = a.group;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment by an offset into the shared array itself, so the
    // compiler keeps shared-space (32-bit) addressing for everything below
    uint8_t* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const TiledSmem L = tiled_smem(S, G, ROWS, (int)sizeof(E), F8);
    float* s_y2 = reinterpret_cast<float*>(smem + L.y2);          // [2][G][8][FB]
    // row-sum transpose: the warp's just-consumed ring slot when its rows are
    // wide enough (FP32, BF16), else a dedicated per-warp region
    constexpr bool RS_IN_SLOT = RING && !F8 && 128 * sizeof(E) >= kRowSumStride * 4;
    float* s_rs_own = reinterpret_cast<float*>(smem + L.ysc) +
                      (size_t)(threadIdx.x >> 5) * ROWS * kRowSumStride;
    float* s_ua = reinterpret_cast<float*>(smem + L.ua) + (threadIdx.x >> 5) * 16;   // its rows' u_A
    int64_t* s_off = reinterpret_cast<int64_t*>(smem + L.off);    // [2][G]
    int* s_cnt = reinterpret_cast<int*>(smem + L.cnt);            // [2][G]

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
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
    const int nloc = (int)(i1 - i0);   // W <= O < 2^31
    const int64_t AB = a.A * a.B;

    E* ring = reinterpret_cast<E*>(smem) + (size_t)warp * S * SLOT;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars) + warp * S;
    float* sscl = reinterpret_cast<float*>(smem + L.scl) + (size_t)warp * S * ROWS * 2;
    if (RING) {
        if (lane == 0) {
            for (int q = 0; q < S; ++q)
                mbar_init(&full[q], (MODE == LOAD_TMA ? 1u : 0u) + (CPA ? 32u : 0u));
            fence_mbar_init();
        }
        __syncwarp();
    }

    // ---- issue side: item position and the flat offset of its first element
    int64_t ii_o, ii_t, ii_ta, ii_tb, ii_flat;   // flat = (o*A + ar0)*B + tb*FB
    auto ii_tile = [&]() {
        ii_ta = ii_t / a.TB;
        ii_tb = ii_t - ii_ta * a.TB;
        ii_flat = (ii_o * a.A + ii_ta * FA + warp * ROWS) * a.B + ii_tb * FB;
    };
    ii_t = i0 / a.O;
    ii_o = i0 - ii_t * a.O;
    ii_tile();
    auto ii_next = [&]() {
        if (++ii_o == a.O) {
            ii_o = 0;
            ++ii_t;
            ii_tile();
        } else {
            ii_flat += AB;
        }
    };
    auto issue = [&](int slot) {
        const int64_t ar0 = ii_ta * FA + warp * ROWS;
        if (MODE == LOAD_TMA) {
            if (lane == 0) {
                fence_proxy_async();
                mbar_arrive_expect_tx(&full[slot], SLOT * sizeof(E));
                tma_load_3d(ring + (size_t)slot * SLOT, &tmap, (int)(ii_tb * FB), (int)ar0,
                            (int)ii_o, &full[slot]);
            }
        } else {
            const bool colok = ii_tb * FB + 4 * lane < a.B;
            const E* rowp = reinterpret_cast<const E*>(a.T) + ii_flat + 4 * lane;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const bool ok = colok && ar0 + r < a.A;
                cp_async<(int)sizeof(P4)>(ring + (size_t)slot * SLOT + r * FB + 4 * lane,
                                          ok ? (const void*)(rowp + r * a.B) : a.T, ok);
            }
        }
        if (F8) {
            // scales of the first and last 128-element group each row window touches
            if (lane < 2 * ROWS) {
                const int r = lane >> 1;
                const bool ok = ar0 + r < a.A;
                const int64_t last = min(ii_tb * FB + FB, a.B) - 1 - ii_tb * FB;
                const int64_t g = (ii_flat + r * a.B + ((lane & 1) ? last : 0)) >> 7;
                cp_async<4>(sscl + ((size_t)slot * ROWS + r) * 2 + (lane & 1),
                            ok ? (const void*)(a.scales + g) : (const void*)a.scales, ok);
            }
        }
        if (CPA) cp_async_arrive_noinc(&full[slot]);
    };

    // ---- consume side
    float2 acc[ROWS][2];
    float2 uB2[2];
    const int64_t t_first = i0 / a.O;
    int64_t cc_o = i0 - t_first * a.O, cc_t = t_first - 1;   // tile set up on first item
    int64_t ar0 = 0, b0 = 0, y2off = 0, sflat = 0;
    const float* wp = a.w + cc_o;
    float* y1p = nullptr;
    int ncol = 0;

    auto flush = [&](int64_t t) {
        const int seg = (int)(t - t_first);
        float* dst = a.hp + ((size_t)(c * 2 + seg) * FA) * FB;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            float4 q = make_float4(acc[r][0].x, acc[r][0].y, acc[r][1].x, acc[r][1].y);
            *reinterpret_cast<float4*>(dst + (size_t)(warp * ROWS + r) * FB + 4 * lane) = q;
        }
    };
    auto new_tile = [&](int64_t t) {
        const int64_t ta = t / a.TB, tb = t - (t / a.TB) * a.TB;
        ar0 = ta * FA + warp * ROWS;
        b0 = tb * FB + 4 * lane;
        y1p = a.y1p + (tb * a.O + cc_o) * a.A + ar0;
        y2off = (ta * a.O + cc_o) * a.B + tb * FB;
        sflat = (cc_o * a.A + ar0) * a.B + tb * FB;
        ncol = (int)min((int64_t)FB, a.B - tb * FB);
        float ub[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) ub[q] = b0 + q < a.B ? a.uB[b0 + q] : 0.f;
        uB2[0] = make_float2(ub[0], ub[1]);
        uB2[1] = make_float2(ub[2], ub[3]);
        __syncwarp();
        if (lane < ROWS) s_ua[lane] = ar0 + lane < a.A ? a.uA[ar0 + lane] : 0.f;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            acc[r][0] = make_float2(0.f, 0.f);
            acc[r][1] = make_float2(0.f, 0.f);
        }
    };

    // prologue: the first S-1 items in flight
    int si = 0;      // slot of the next issue
    int nis = 0;     // items issued
    if (RING) {
        for (; nis < S - 1 && nis < nloc; ++nis) {
            issue(si);
            ii_next();
            si = si + 1 == S ? 0 : si + 1;
        }
    }

    bool ok = true;
    int kfail = nloc;
    int cs = 0;          // slot being consumed
    uint32_t cph = 0;    // its phase parity
    int gbuf = 0, gj = 0;
    for (int k = 0; k < nloc; ++k) {
        if (RING && ok && nis < nloc) {
            issue(si);
            ii_next();
            si = si + 1 == S ? 0 : si + 1;
            ++nis;
        }
        if (k == 0 || cc_o == 0) {
            if (k > 0) flush(cc_t);
            ++cc_t;
            new_tile(cc_t);
        }
        const float wo = __ldg(wp);
        const float2 wo2 = make_float2(wo, wo);
        float y1[ROWS];
        float2 y2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (RING && ok) {
            // warp-uniform: once any lane gives up, the whole warp stops issuing
            const bool got = mbar_wait_bounded(&full[cs], cph, a.timeout_ns);
            if (!__all_sync(HOSCF_FULLMASK, got)) {
                if (lane == 0) atomicCAS(a.err, 0, (int)DEV_TIMEOUT);
                ok = false;
                kfail = k;
            }
        }
        // FP8: offset of the row window's first column within its scale group
        int g_lo = F8 && RING ? (int)(sflat & 127) : 0;
        const int g_step = (int)(a.B & 127);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            float v[4];
            if (RING) {
                unpack4e<E>(*reinterpret_cast<const P4*>(ring + (size_t)cs * SLOT + r * FB + 4 * lane), v);
                if (F8) {
                    const float* sp = sscl + ((size_t)cs * ROWS + r) * 2;
                    const float sc = ((g_lo + 4 * lane) & ~127) ? sp[1] : sp[0];
                    g_lo = (g_lo + g_step) & 127;
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] *= sc;
                }
            } else {
                const int64_t ar = ar0 + r;
                const E* rowp = reinterpret_cast<const E*>(a.T) + (cc_o * a.A + ar) * a.B;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t b = b0 + q;
                    v[q] = (ar < a.A && b < a.B) ? load1_global<E>(rowp + b) : 0.f;
                }
                if (F8 && ar < a.A && b0 < a.B) apply_scales(a.scales, (cc_o * a.A + ar) * a.B + b0, v);
            }
            const float2 v0 = make_float2(v[0], v[1]), v1 = make_float2(v[2], v[3]);
            acc[r][0] = ffma2(wo2, v0, acc[r][0]);
            acc[r][1] = ffma2(wo2, v1, acc[r][1]);
            const float ua = s_ua[r];
            const float2 ua2 = make_float2(ua, ua);
            y2[0] = ffma2(v0, ua2, y2[0]);
            y2[1] = ffma2(v1, ua2, y2[1]);
            const float2 dd = ffma2(v1, uB2[1], make_float2(v0.x * uB2[0].x, v0.y * uB2[0].y));
            y1[r] = dd.x + dd.y;
        }
        float* s_rs = RS_IN_SLOT ? reinterpret_cast<float*>(ring + (size_t)cs * SLOT) : s_rs_own;
        if (RING) {
            __syncwarp();   // every lane is done with slot cs (refilled at the next issue)
            if (++cs == S) {
                cs = 0;
                cph ^= 1u;
            }
        }
        // row sums -> y1 partial of this b-tile: the lanes' partials go through
        // a shared-memory transpose (row r, lane l at r*36 + l: conflict-free
        // both ways), then lanes 2r and 2r+1 each add 16 of row r's 32
        // partials with four 16-byte loads and combine with one shuffle.
#pragma unroll
        for (int r = 0; r < ROWS; ++r) s_rs[r * kRowSumStride + lane] = y1[r];
        __syncwarp();
        {
            const int row = lane >> 1;
            float ys = 0.f;
            if (row < ROWS) {
                const float4* src = reinterpret_cast<const float4*>(s_rs + row * kRowSumStride + 16 * (lane & 1));
                const float4 q0 = src[0], q1 = src[1], q2 = src[2], q3 = src[3];
                ys = ((q0.x + q0.y) + (q0.z + q0.w)) + ((q1.x + q1.y) + (q1.z + q1.w)) +
                     (((q2.x + q2.y) + (q2.z + q2.w)) + ((q3.x + q3.y) + (q3.z + q3.w)));
            }
            ys += __shfl_xor_sync(HOSCF_FULLMASK, ys, 1);
            if ((lane & 1) == 0 && row < ROWS && ar0 + row < a.A) y1p[row] = ys;
        }
        __syncwarp();   // transpose read before the slot is refilled / rewritten
        // column partials -> exchange ring; summed over the 8 warps every G items
        float* sy = s_y2 + ((size_t)(gbuf * G + gj) * 8 + warp) * FB;
        *reinterpret_cast<float4*>(sy + 4 * lane) = make_float4(y2[0].x, y2[0].y, y2[1].x, y2[1].y);
        if (tid == 0) {
            s_off[gbuf * G + gj] = y2off;
            s_cnt[gbuf * G + gj] = ncol;
        }
        if (gj == G - 1 || k == nloc - 1) {
            asm volatile("bar.sync 1, 256;" ::: "memory");
            const float* gb = s_y2 + (size_t)gbuf * G * 8 * FB;
            const int n = (gj + 1) * FB;
            for (int e = tid; e < n; e += 256) {
                const int jj = e >> 7, b = e & (FB - 1);
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
        // next outer index
        ++wp;
        y1p += a.A;
        y2off += a.B;
        sflat += AB;
        if (++cc_o == a.O) {
            cc_o = 0;
            wp = a.w;
        }
    }
    flush(cc_t);
    if constexpr (RING) {
        if (!ok) {
            // A wait gave up: the blocks are void and the code is in the device
            // status word, which the caller reads (hoscf_solve after each step,
            // hoscf_device_status for the asynchronous calls, the status output
            // of hoscf_ttvc_blocks_static).
            // Every copy already issued must still land before the CTA's shared
            // memory is released: wait for each, with a bound of at least 1 s
            // whatever the caller's limit.
            const uint64_t drain_ns = a.timeout_ns > 1000000000ull ? a.timeout_ns : 1000000000ull;
            for (int k = kfail; k < nis; ++k)
                mbar_wait_bounded(&full[k % S], (uint32_t)((k / S) & 1), drain_ns);
        }
    }
    if (CPA) cp_async_wait_all();
}

// H_{D,D+1}[a][b] = sum of the face partials of every CTA that touched the
// tile, in CTA order.
// All reductions of the streaming kernel's partials in one launch, over
// units of 128 outputs (two units per 256-thread CTA, grid-stride):
//  * face units (tile t, row rr): H_face[a][b] = sum of the face partials of
//    the CTAs whose item ranges meet tile t, in CTA order.  Per-tile split:
//    CTAs t P .. t P + P - 1.  Stream-K: only the first of them can have
//    started in tile t-1 (its partial sits in segment 1);
//  * y1 units: y1[i] = sum_{p < TB} y1p[p n1 + i], i < n1 = O A;
//  * y2 units: y2[i] = sum_{p < TA} y2p[p n2 + i], i < n2 = O B.
struct ReduceArgs {
    const float* hp;
    float* face;
    int64_t A, B, TB, O, W, P, TT;
    int FA, FB;
    const float* y1p;
    float* y1;
    int64_t n1, np1;
    const float* y2p;
    float* y2;
    int64_t n2, np2;
};

// sum_{p < n} x[p * stride]: four independent partial sums (loads in
// flight together), combined in a fixed order.
__device__ __forceinline__ float sum_strided(const float* __restrict__ x, size_t stride, int64_t n) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int64_t p = 0;
    for (; p + 4 <= n; p += 4) {
        const float v0 = __ldg(x + (size_t)p * stride), v1 = __ldg(x + (size_t)(p + 1) * stride),
                    v2 = __ldg(x + (size_t)(p + 2) * stride), v3 = __ldg(x + (size_t)(p + 3) * stride);
        a0 += v0;
        a1 += v1;
        a2 += v2;
        a3 += v3;
    }
    for (; p < n; ++p) a0 += __ldg(x + (size_t)p * stride);
    return (a0 + a1) + (a2 + a3);
}

// sum_{p < n} x[p * stride .. + 3] (16-byte aligned rows): up to eight
// loads in flight, four running sums (p mod 4) combined in the same fixed
// order as sum_strided.
__device__ __forceinline__ float4 sum_strided4(const float* __restrict__ x, size_t stride, int64_t n) {
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    int64_t p = 0;
    auto add = [](float4& a, const float4 v) {
        a.x += v.x;
        a.y += v.y;
        a.z += v.z;
        a.w += v.w;
    };
    // eight loads in flight, added in the order of two rounds of four
    for (; p + 8 <= n; p += 8) {
        float4 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __ldg(reinterpret_cast<const float4*>(x + (size_t)(p + i) * stride));
        add(a0, v[0]);
        add(a1, v[1]);
        add(a2, v[2]);
        add(a3, v[3]);
        add(a0, v[4]);
        add(a1, v[5]);
        add(a2, v[6]);
        add(a3, v[7]);
    }
    for (; p + 4 <= n; p += 4) {
        const float4 v0 = __ldg(reinterpret_cast<const float4*>(x + (size_t)p * stride));
        const float4 v1 = __ldg(reinterpret_cast<const float4*>(x + (size_t)(p + 1) * stride));
        const float4 v2 = __ldg(reinterpret_cast<const float4*>(x + (size_t)(p + 2) * stride));
        const float4 v3 = __ldg(reinterpret_cast<const float4*>(x + (size_t)(p + 3) * stride));
        add(a0, v0);
        add(a1, v1);
        add(a2, v2);
        add(a3, v3);
    }
    for (; p < n; ++p) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(x + (size_t)p * stride));
        a0.x += v.x; a0.y += v.y; a0.z += v.z; a0.w += v.w;
    }
    return make_float4((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y),
                       (a0.z + a1.z) + (a2.z + a3.z), (a0.w + a1.w) + (a2.w + a3.w));
}

__global__ void __launch_bounds__(256) reduce_pass_kernel(const ReduceArgs r) {
    const int col = threadIdx.x & 127;
    const int CU = r.FB / 128;                       // 128-column units per tile row
    const int64_t nuF = r.TT * r.FA * CU;
    // y1 / y2 units: 128 threads x 4 consecutive entries (16-byte loads, up
    // to eight partials in flight) when n % 4 == 0 and both arrays start
    // 16-byte aligned, else 128 x 1
    const bool v1 = (r.n1 & 3) == 0 &&
                    ((reinterpret_cast<uintptr_t>(r.y1p) | reinterpret_cast<uintptr_t>(r.y1)) & 15u) == 0;
    const bool v2 = (r.n2 & 3) == 0 &&
                    ((reinterpret_cast<uintptr_t>(r.y2p) | reinterpret_cast<uintptr_t>(r.y2)) & 15u) == 0;
    const int64_t e1 = v1 ? 512 : 128, e2 = v2 ? 512 : 128;
    const int64_t nu1 = (r.n1 + e1 - 1) / e1, nu2 = (r.n2 + e2 - 1) / e2;
    // face units: 4 rows x 128 columns, 4 consecutive columns per thread
    // (16-byte loads) when the tile is 128 wide and rows and partials are
    // 16-byte aligned; else one row of 128 columns
    const bool vF = (r.B & 3) == 0 &&
                    ((reinterpret_cast<uintptr_t>(r.hp) | reinterpret_cast<uintptr_t>(r.face)) & 15u) == 0;
    const int64_t FA4 = (r.FA + 3) / 4;
    const int64_t nuFv = vF ? r.TT * FA4 * CU : nuF;
    const int64_t total = nuFv + nu1 + nu2;
    for (int64_t u0 = blockIdx.x * 2 + (threadIdx.x >> 7); u0 < total; u0 += (int64_t)gridDim.x * 2) {
        if (vF && u0 < nuFv) {
            const int64_t t = u0 / (FA4 * CU);
            const int64_t rq = u0 - t * FA4 * CU;
            const int rr = (int)(rq / CU) * 4 + (col >> 5);
            const int cb = (int)(rq % CU) * 128 + (col & 31) * 4;
            const int64_t ta = t / r.TB, tb = t - (t / r.TB) * r.TB;
            const int64_t aa = ta * r.FA + rr, bb = tb * r.FB + cb;
            if (rr >= r.FA || aa >= r.A || bb >= r.B) continue;
            const int64_t c_lo = r.P > 0 ? t * r.P : (t * r.O) / r.W;
            const int64_t c_hi = r.P > 0 ? t * r.P + r.P - 1 : ((t + 1) * r.O - 1) / r.W;
            const size_t inner = (size_t)rr * r.FB + cb, tile = (size_t)r.FA * r.FB;
            const float4 first = __ldg(reinterpret_cast<const float4*>(
                r.hp + ((size_t)c_lo * 2 + (r.P == 0 && c_lo * r.W < t * r.O ? 1 : 0)) * tile + inner));
            const float4 rest =
                sum_strided4(r.hp + (size_t)(c_lo + 1) * 2 * tile + inner, 2 * tile, c_hi - c_lo);
            *reinterpret_cast<float4*>(r.face + aa * r.B + bb) =
                make_float4(first.x + rest.x, first.y + rest.y, first.z + rest.z, first.w + rest.w);
            continue;
        }
        const int64_t u = vF ? u0 - nuFv + nuF : u0;   // index in the unvectorised numbering
        if (u < nuF) {
            const int64_t t = u / ((int64_t)r.FA * CU);
            const int64_t rq = u - t * r.FA * CU;
            const int rr = (int)(rq / CU);
            const int cc = (int)(rq % CU) * 128 + col;
            const int64_t ta = t / r.TB, tb = t - (t / r.TB) * r.TB;
            const int64_t aa = ta * r.FA + rr, bb = tb * r.FB + cc;
            if (aa >= r.A || cc >= r.FB || bb >= r.B) continue;
            const int64_t c_lo = r.P > 0 ? t * r.P : (t * r.O) / r.W;
            const int64_t c_hi = r.P > 0 ? t * r.P + r.P - 1 : ((t + 1) * r.O - 1) / r.W;
            const size_t inner = (size_t)rr * r.FB + cc, tile = (size_t)r.FA * r.FB;
            const float first =
                r.hp[((size_t)c_lo * 2 + (r.P == 0 && c_lo * r.W < t * r.O ? 1 : 0)) * tile + inner];
            r.face[aa * r.B + bb] =
                first + sum_strided(r.hp + (size_t)(c_lo + 1) * 2 * tile + inner, 2 * tile, c_hi - c_lo);
        } else if (u < nuF + nu1) {
            if (v1) {
                const int64_t i = (u - nuF) * 512 + 4 * col;
                if (i >= r.n1) continue;
                *reinterpret_cast<float4*>(r.y1 + i) = sum_strided4(r.y1p + i, (size_t)r.n1, r.np1);
            } else {
                const int64_t i = (u - nuF) * 128 + col;
                if (i >= r.n1) continue;
                r.y1[i] = sum_strided(r.y1p + i, (size_t)r.n1, r.np1);
            }
        } else {
            if (v2) {
                const int64_t i = (u - nuF - nu1) * 512 + 4 * col;
                if (i >= r.n2) continue;
                *reinterpret_cast<float4*>(r.y2 + i) = sum_strided4(r.y2p + i, (size_t)r.n2, r.np2);
            } else {
                const int64_t i = (u - nuF - nu1) * 128 + col;
                if (i >= r.n2) continue;
                r.y2[i] = sum_strided(r.y2p + i, (size_t)r.n2, r.np2);
            }
        }
    }
}

// wx[m][o] = prod_{k != m} u_k[o_k]: the outer weight of o without mode m.
__global__ void outer_weights_excl_kernel(const float* __restrict__ u, OuterInfo oi, int64_t O,
                                          float* __restrict__ wx) {
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < O;
         o += (int64_t)gridDim.x * blockDim.x) {
        float f[kMaxOrder];
        for (int k = 0; k < oi.D; ++k) f[k] = u[oi.uoff[k] + outer_digit(oi, o, k)];
        for (int m = 0; m < oi.D; ++m) {
            float p = 1.f;
            for (int k = 0; k < oi.D; ++k)
                if (k != m) p *= f[k];
            wx[m * O + o] = p;
        }
    }
}

// Cross blocks H_{m,face}[i][col] = sum_{o: o_m = i} wx[m][o] y[o][col] for
// every outer mode m.  The outer indices with o_m = i are, in increasing
// order, o(q) = (q / st_m) * I_m st_m + i st_m + q % st_m for q < O / I_m.
// CTA (m, i, 32-column chunk): warp w sums a contiguous range of q with four
// independent accumulators; the 8 warp sums are added in warp order.
struct ModeOffs {
    int64_t off[kMaxOrder];
};

__global__ void __launch_bounds__(256) fold_cross_kernel(const float* __restrict__ y, int64_t C,
                                                         const float* __restrict__ wx, OuterInfo oi,
                                                         int64_t O, float* __restrict__ H,
                                                         const ModeOffs row_block_off) {
    __shared__ float part[8][32];
    // blockIdx.x enumerates (m, i) rows: rows of mode m start at sum_{k<m} I_k
    int m = 0;
    int64_t row = blockIdx.x;
    while (m < oi.D - 1 && row >= oi.dims[m]) {
        row -= oi.dims[m];
        ++m;
    }
    const int i = (int)row;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t Im = oi.dims[m];
    const int64_t stm = oi.st[m];
    const int64_t Q = O / Im;
    const int64_t col = blockIdx.y * 32 + lane;
    const bool colok = col < C;
    const float* wm = wx + m * O;
    const int64_t q0 = (Q * warp) / 8, q1 = (Q * (warp + 1)) / 8;
    int64_t s = q0 % stm;
    int64_t o = (q0 / stm) * Im * stm + i * stm + s;
    const int64_t jump = (Im - 1) * stm;   // from the end of one st_m run to the next
    auto step = [&]() {
        ++o;
        if (++s == stm) {
            s = 0;
            o += jump;
        }
    };
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int64_t q = q0;
    for (; q + 4 <= q1; q += 4) {
        int64_t oo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            oo[k] = o;
            step();
        }
        float yv[4], wv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            yv[k] = colok ? __ldg(y + oo[k] * C + col) : 0.f;
            wv[k] = __ldg(wm + oo[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] = fmaf(wv[k], yv[k], acc[k]);
    }
    for (; q < q1; ++q) {
        acc[0] = fmaf(__ldg(wm + o), colok ? __ldg(y + o * C + col) : 0.f, acc[0]);
        step();
    }
    part[warp][lane] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    __syncthreads();
    if (warp == 0 && colok) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += part[w][lane];
        H[row_block_off.off[m] + (int64_t)i * C + col] = t;
    }
}

// The same cross folds with 16-byte loads: lane l owns columns 4l .. 4l+3 of
// a 128-column chunk, four outer indices in flight per warp; y1 and y2 in one
// launch (blockIdx.z).  Needs C % 4 == 0 and 16-byte aligned y rows.
struct CrossArgs {
    const float* y[2];
    int64_t C[2];
    int64_t off[2][kMaxOrder];
};

__global__ void __launch_bounds__(256) fold_cross4_kernel(const CrossArgs ca,
                                                          const float* __restrict__ wx, OuterInfo oi,
                                                          int64_t O, float* __restrict__ H) {
    __shared__ float4 part[8][32];
    const int z = blockIdx.z;
    const float* __restrict__ y = z ? ca.y[1] : ca.y[0];
    const int64_t C = z ? ca.C[1] : ca.C[0];
    if ((int64_t)blockIdx.y * 128 >= C) return;
    int m = 0;
    int64_t row = blockIdx.x;
    while (m < oi.D - 1 && row >= oi.dims[m]) {
        row -= oi.dims[m];
        ++m;
    }
    const int i = (int)row;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t Im = oi.dims[m];
    const int64_t stm = oi.st[m];
    const int64_t Q = O / Im;
    const int64_t col = (int64_t)blockIdx.y * 128 + 4 * lane;
    const bool colok = col < C;
    const float* wm = wx + m * O;
    const int64_t q0 = (Q * warp) / 8, q1 = (Q * (warp + 1)) / 8;
    int64_t s = q0 % stm;
    int64_t o = (q0 / stm) * Im * stm + i * stm + s;
    const int64_t jump = (Im - 1) * stm;
    auto step = [&]() {
        ++o;
        if (++s == stm) {
            s = 0;
            o += jump;
        }
    };
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 acc[4] = {z4, z4, z4, z4};
    int64_t q = q0;
    for (; q + 4 <= q1; q += 4) {
        int64_t oo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            oo[k] = o;
            step();
        }
        float4 yv[4];
        float wv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            yv[k] = colok ? __ldg(reinterpret_cast<const float4*>(y + oo[k] * C + col)) : z4;
            wv[k] = __ldg(wm + oo[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[k].x = fmaf(wv[k], yv[k].x, acc[k].x);
            acc[k].y = fmaf(wv[k], yv[k].y, acc[k].y);
            acc[k].z = fmaf(wv[k], yv[k].z, acc[k].z);
            acc[k].w = fmaf(wv[k], yv[k].w, acc[k].w);
        }
    }
    for (; q < q1; ++q) {
        const float w = __ldg(wm + o);
        const float4 v = colok ? __ldg(reinterpret_cast<const float4*>(y + o * C + col)) : z4;
        acc[0].x = fmaf(w, v.x, acc[0].x);
        acc[0].y = fmaf(w, v.y, acc[0].y);
        acc[0].z = fmaf(w, v.z, acc[0].z);
        acc[0].w = fmaf(w, v.w, acc[0].w);
        step();
    }
    part[warp][lane] = make_float4((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x),
                                   (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y),
                                   (acc[0].z + acc[1].z) + (acc[2].z + acc[3].z),
                                   (acc[0].w + acc[1].w) + (acc[2].w + acc[3].w));
    __syncthreads();
    if (threadIdx.x < 128) {
        const int ln = threadIdx.x >> 2, e = threadIdx.x & 3;
        const int64_t cc = (int64_t)blockIdx.y * 128 + threadIdx.x;
        if (cc < C) {
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < 8; ++w) t += reinterpret_cast<const float*>(&part[w][ln])[e];
            H[(z ? ca.off[1][m] : ca.off[0][m]) + (int64_t)i * C + cc] = t;
        }
    }
}

// r[o] = sum_a y1[o][a] uA[a]   (one warp per o)
__global__ void fold_r_kernel(const float* __restrict__ y1, const float* __restrict__ uA, int64_t O,
                              int64_t A, float* __restrict__ r) {
    const int lane = threadIdx.x & 31;
    // 16-byte loads of y1 rows when A % 4 == 0 and y1 is 16-byte aligned
    const bool v4 = (A & 3) == 0 && (reinterpret_cast<uintptr_t>(y1) & 15u) == 0;
    for (int64_t o = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; o < O;
         o += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
        if (v4) {
            const float4* row = reinterpret_cast<const float4*>(y1 + o * A);
            for (int64_t q = lane; q < A / 4; q += 32) {
                const float4 v = __ldg(row + q);
                s = fmaf(v.x, __ldg(uA + 4 * q), s);
                s = fmaf(v.y, __ldg(uA + 4 * q + 1), s);
                s = fmaf(v.z, __ldg(uA + 4 * q + 2), s);
                s = fmaf(v.w, __ldg(uA + 4 * q + 3), s);
            }
        } else {
            for (int64_t aa = lane; aa < A; aa += 32) s = fmaf(y1[o * A + aa], uA[aa], s);
        }
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

__global__ void f16_to_f32_kernel(const uint16_t* __restrict__ src, float* __restrict__ dst,
                                  int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __half2float(__ushort_as_half(src[i]));
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
                                  cudaStream_t st, const KernelEvents* kev) {
    auto kern = ttvc_tiled_kernel<E, MODE, ROWS>;
    const size_t smem = 1024 + tiled_smem(MODE == LOAD_SCALAR ? 0 : p.nstage, p.group, ROWS,
                                          (int)sizeof(E), std::is_same<E, fp8_t>::value)
                                   .total;
    cudaError_t e = allow_max_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
    if (kev) cudaEventRecord(kev->begin, st);
    kern<<<p.grid, 256, smem, st>>>(map, a);
    if (kev) cudaEventRecord(kev->end, st);
    return cudaGetLastError();
}

template <typename E, int MODE>
static cudaError_t launch_tiled_rows(const PassPlan& p, const CUtensorMap& map, const TiledArgs& a,
                                     cudaStream_t st, const KernelEvents* kev) {
    if (p.rows == 8) return launch_tiled_k<E, MODE, 8>(p, map, a, st, kev);
    if constexpr (TiledOcc<E>::value == 1) {
        if (p.rows == 16) return launch_tiled_k<E, MODE, 16>(p, map, a, st, kev);
    }
    return launch_tiled_k<E, MODE, 13>(p, map, a, st, kev);
}

template <typename E>
static cudaError_t launch_tiled(const PassPlan& p, int mode, const CUtensorMap& map,
                                const TiledArgs& a, cudaStream_t st, const KernelEvents* kev) {
    if (mode == LOAD_TMA) return launch_tiled_rows<E, LOAD_TMA>(p, map, a, st, kev);
    if (mode == LOAD_ASYNC) return launch_tiled_rows<E, LOAD_ASYNC>(p, map, a, st, kev);
    return launch_tiled_rows<E, LOAD_SCALAR>(p, map, a, st, kev);
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
                      uint64_t timeout_ns, cudaStream_t st, Err& err, const KernelEvents* kev) {
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
        if (kev) cudaEventRecord(kev->begin, st);
        if (dtype == HOSCF_F32) {
            copy_kernel<<<grid_for(s.N, 256, 4096), 256, 0, st>>>((const float*)data, H, s.N);
        } else if (dtype == HOSCF_BF16) {
            bf16_to_f32_kernel<<<grid_for(s.N, 256, 4096), 256, 0, st>>>((const uint16_t*)data, H,
                                                                         s.N);
        } else if (dtype == HOSCF_F16) {
            f16_to_f32_kernel<<<grid_for(s.N, 256, 4096), 256, 0, st>>>((const uint16_t*)data, H,
                                                                        s.N);
        } else {
            fp8_to_f32_kernel<<<grid_for(s.N, 256, 4096), 256, 0, st>>>((const uint8_t*)data,
                                                                        scales, H, s.N);
        }
        if (kev) cudaEventRecord(kev->end, st);
        HOSCF_CK(cudaGetLastError());
        return HOSCF_OK;
    }
    if (p.small) {
        HOSCF_CK(run_small(s, p.sp, dtype, data, scales, u, H, ws, dev_err, timeout_ns, st, kev));
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
    a.nstage = p.nstage;
    a.group = p.group;
    a.P = p.P;

    if (p.narrow) {
        NarrowArgs na;
        na.T = data;
        na.scales = scales;
        na.O = s.O;
        na.A = s.A;
        na.B = s.B;
        na.items = p.items;
        na.W = p.W;
        na.P = p.P;
        na.w = wptr;
        na.uA = a.uA;
        na.uB = a.uB;
        na.hp = a.hp;
        na.y1p = a.y1p;
        na.y2p = a.y2p;
        na.err = dev_err;
        na.timeout_ns = timeout_ns;
        na.nstage = p.nstage;
        na.group = p.group;
        na.FA = p.FA;
        HOSCF_CK(launch_narrow(p, dtype, na, st, kev));
    } else {
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    bool use_tma = p.tma;
    if (use_tma) {
        EncodeTiledFn enc = get_encode_fn();
        const int es = elem_size(dtype);
        cuuint64_t gdim[3] = {(cuuint64_t)s.B, (cuuint64_t)s.A, (cuuint64_t)s.O};
        cuuint64_t gstr[2] = {(cuuint64_t)(s.B * es), (cuuint64_t)(s.A * s.B * es)};
        cuuint32_t box[3] = {(cuuint32_t)p.FB, (cuuint32_t)p.rows, 1};   // one warp's rows
        cuuint32_t estr[3] = {1, 1, 1};
        // Promote L2 fetches to 256 B only when rows start on 256-byte lines;
        // otherwise every row window would drag in a partial line twice.
        const int64_t pitch = s.B * es;
        const CUtensorMapL2promotion prom = pitch % 256 == 0   ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
                                            : pitch % 128 == 0 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                                               : CU_TENSOR_MAP_L2_PROMOTION_NONE;
        CUtensorMapDataType dt = dtype == HOSCF_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : dtype == HOSCF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : dtype == HOSCF_F16  ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_UINT8;
        if (!enc || (reinterpret_cast<uintptr_t>(data) & 15) != 0 ||
            enc(&map, dt, 3, const_cast<void*>(data), gdim, gstr, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, prom,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            use_tma = false;
    }
    const int mode = use_tma ? LOAD_TMA
                     : (p.vec && (reinterpret_cast<uintptr_t>(data) & 15) == 0) ? LOAD_ASYNC
                                                                                : LOAD_SCALAR;
    if (dtype == HOSCF_F32) {
        HOSCF_CK(launch_tiled<float>(p, mode, map, a, st, kev));
    } else if (dtype == HOSCF_BF16) {
        HOSCF_CK(launch_tiled<bf16_t>(p, mode, map, a, st, kev));
    } else if (dtype == HOSCF_F16) {
        HOSCF_CK(launch_tiled<f16_t>(p, mode, map, a, st, kev));
    } else {
        HOSCF_CK(launch_tiled<fp8_t>(p, mode, map, a, st, kev));
    }
    }
    // face block (d-2, d-1) and the row / column sums y1 (O x A), y2 (O x B):
    // for d == 3 these are H_{0,1} and H_{0,2} themselves
    float* y1 = s.d == 3 ? H + s.boff[block_index(3, 0, 1)] : reinterpret_cast<float*>(ws + p.off_y1);
    float* y2 = s.d == 3 ? H + s.boff[block_index(3, 0, 2)] : reinterpret_cast<float*>(ws + p.off_y2);
    // for d >= 4 a single partial (one column tile for y1, one row band for
    // y2) already is the sum, in the same [O][A] / [O][B] layout: the folds
    // read it in place instead of a copy
    const bool y1_direct = s.d > 3 && p.TB == 1;
    const bool y2_direct = s.d > 3 && p.TA == 1;
    if (y1_direct) y1 = a.y1p;
    if (y2_direct) y2 = a.y2p;
    {
        ReduceArgs ra;
        ra.hp = a.hp;
        ra.face = H + s.boff[block_index(s.d, s.d - 2, s.d - 1)];
        ra.A = s.A;
        ra.B = s.B;
        ra.TB = p.TB;
        ra.O = s.O;
        ra.W = p.W;
        ra.P = p.P;
        ra.TT = p.TT;
        ra.FA = p.FA;
        ra.FB = p.FB;
        ra.y1p = a.y1p;
        ra.y1 = y1;
        ra.n1 = y1_direct ? 0 : s.O * s.A;
        ra.np1 = p.TB;
        ra.y2p = a.y2p;
        ra.y2 = y2;
        ra.n2 = y2_direct ? 0 : s.O * s.B;
        ra.np2 = p.TA;
        const int64_t units = p.TT * p.FA * (p.FB / 128) + (ra.n1 + 127) / 128 + (ra.n2 + 127) / 128;
        const int64_t g = std::min<int64_t>((units + 1) / 2, 16 * (int64_t)std::max(1, p.nsm));
        reduce_pass_kernel<<<(unsigned)std::max<int64_t>(1, g), 256, 0, st>>>(ra);
        HOSCF_CK(cudaGetLastError());
    }
    if (s.d == 3) return HOSCF_OK;
    float* r = reinterpret_cast<float*>(ws + p.off_r);
    // cross blocks (m, d-2) from y1 and (m, d-1) from y2
    int64_t rows = 0;
    for (int k = 0; k < s.D; ++k) rows += s.dims[k];
    ModeOffs off1, off2;
    for (int m = 0; m < s.D; ++m) {
        off1.off[m] = s.boff[block_index(s.d, m, s.d - 2)];
        off2.off[m] = s.boff[block_index(s.d, m, s.d - 1)];
    }
    {
        float* wx = reinterpret_cast<float*>(ws + p.off_wx);
        outer_weights_excl_kernel<<<grid_for(s.O, 256, 4096), 256, 0, st>>>(u, oi, s.O, wx);
        const bool v4 = s.A % 4 == 0 && s.B % 4 == 0 &&
                        ((reinterpret_cast<uintptr_t>(y1) | reinterpret_cast<uintptr_t>(y2)) & 15u) == 0;
        if (v4) {
            CrossArgs ca;
            memset(&ca, 0, sizeof(ca));
            ca.y[0] = y1;
            ca.y[1] = y2;
            ca.C[0] = s.A;
            ca.C[1] = s.B;
            for (int m = 0; m < s.D; ++m) {
                ca.off[0][m] = off1.off[m];
                ca.off[1][m] = off2.off[m];
            }
            dim3 g((unsigned)rows, (unsigned)((std::max(s.A, s.B) + 127) / 128), 2);
            fold_cross4_kernel<<<g, 256, 0, st>>>(ca, wx, oi, s.O, H);
        } else {
            dim3 g1((unsigned)rows, (unsigned)((s.A + 31) / 32));
            fold_cross_kernel<<<g1, 256, 0, st>>>(y1, s.A, wx, oi, s.O, H, off1);
            dim3 g2((unsigned)rows, (unsigned)((s.B + 31) / 32));
            fold_cross_kernel<<<g2, 256, 0, st>>>(y2, s.B, wx, oi, s.O, H, off2);
        }
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
