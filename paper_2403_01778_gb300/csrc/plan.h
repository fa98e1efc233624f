// Host-side problem plans and workspace layout of the HOSCF library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/hoscf.h"

namespace hoscf {

constexpr int kMaxOrder = HOSCF_MAX_ORDER;
constexpr int kMaxBlocks = kMaxOrder * (kMaxOrder - 1) / 2;

// Shape facts shared by every stage.  Modes are 0-based; the tensor is
// viewed as [O][A][B] with A = I_{d-2}, B = I_{d-1} (the two fastest modes,
// the "face") and O = product of the D = d-2 leading ("outer") modes.
struct Shape {
    int d = 0;
    int64_t dims[kMaxOrder] = {0};
    int64_t N = 0, n_tot = 0, P = 0;
    int64_t moff[kMaxOrder + 1] = {0};   // factor offsets
    int64_t boff[kMaxBlocks + 1] = {0};  // packed block offsets
    int D = 0;
    int64_t O = 1, A = 1, B = 1;
    int64_t ost[kMaxOrder] = {0};        // outer strides: o = sum_k digit_k * ost[k]
};

// Packed index of block (m, n), m < n.
inline int block_index(int d, int m, int n) { return m * d - m * (m + 1) / 2 + (n - m - 1); }

bool make_shape(int d, const int64_t* dims, Shape& s);

// Small-face pass (B <= 32, A*B <= 1024): groups of K consecutive faces
// staged by bulk copies, contiguous outer ranges per CTA, in-CTA folds into a
// per-CTA patch, then one reduce over the patches.
constexpr int kSmallThreads = 256;
constexpr int kSmallMaxK = 32;     // faces per group
constexpr int kSmallMaxB = 32;     // face columns (row registers per thread)
constexpr int kSmallMaxNm = kMaxOrder - 3;                    // outer modes but the fastest
constexpr int kSmallMaxNq = kSmallMaxNm * (kSmallMaxNm - 1) / 2;

struct SmallPlanInfo {
    int G = 0;                 // CTAs
    int64_t L = 0;             // faces per CTA (a multiple of K)
    int K = 0;                 // faces per group
    int K1 = 0;                // faces per pass of the threads (K <= 2 K1)
    int nstage = 0;            // bulk-copy ring slots
    uint32_t stage_bytes = 0;  // bytes per slot (a multiple of 16)
    int occ = 0;               // CTAs per SM the plan was made for
    int Rmax[kMaxOrder] = {0};
    int64_t x1off[kMaxOrder] = {0}, x2off[kMaxOrder] = {0}, poff[kMaxBlocks] = {0};
    int npairs = 0;
    int pm[kMaxBlocks] = {0}, pn[kMaxBlocks] = {0};
    int64_t patch_floats = 0;
    int nsmax = 0;             // most runs of the fastest outer mode in one group
    int onebar = 0;            // one barrier per group (at most 4 outer modes)
    // shared-memory layout (bytes from a 128-byte aligned base)
    uint32_t o_bars = 0, o_ring = 0, o_uA = 0, o_uB = 0, o_y1 = 0, o_y2 = 0, o_r = 0, o_S = 0,
             o_meta = 0, o_first = 0, o_patch = 0, o_ur = 0, o_tab = 0;
    int NR = 0;                // runs of the fastest outer mode a range touches
    int uro[kMaxOrder] = {0};  // staged factor rows of outer mode m (offsets)
    uint32_t meta_words = 0;   // per metadata slot
    size_t smem = 0;
    size_t off_patch = 0, off_cover = 0;   // workspace offsets (bytes)
};

bool make_small_plan(const Shape& s, int dtype, int nsm, SmallPlanInfo& sp);

// Tiled pass configuration (face tiles of FA x FB, stream-K over
// (tile, outer index) items).
struct PassPlan {
    bool copy_only = false;   // d == 2: the single block is the tensor itself
    bool small = false;       // small-face path (see SmallPlanInfo)
    SmallPlanInfo sp;
    bool tma = false;
    bool vec = false;         // rows allow 4-element vector loads (B % 4 == 0)
    bool narrow = false;      // full-row kernel for BF16 / FP8 (see NarrowSmem)
    int slot_bytes = 0;       // narrow: bytes of one warp ring slot (rows + scales)
    int rows = 8;             // rows per consumer warp; FA = 8 * rows
    int FA = 64, FB = 128;
    int64_t TA = 1, TB = 1, TT = 1, items = 0, W = 0;
    int64_t P = 0;            // outer-index chunks per tile (0: stream-K split)
    int grid = 0;
    int nsm = 0;              // SMs the plan was made for
    int nstage = 0;           // slots of each warp's load ring (0: direct loads)
    int group = 0;            // items per column-sum exchange
    size_t smem = 0;
    // workspace offsets (bytes)
    size_t off_w = 0, off_hp = 0, off_y1p = 0, off_y2p = 0, off_y1 = 0, off_y2 = 0, off_r = 0,
           off_wx = 0;
    size_t bytes = 0;
};

bool make_pass_plan(const Shape& s, int dtype, int nsm, bool tma_ok, PassPlan& p);

#ifdef __CUDACC__
#define HOSCF_HD __host__ __device__
#else
#define HOSCF_HD
#endif

// Shared-memory layout of the tiled pass kernel, from a 1024-byte aligned
// base: each of the 8 warps owns S ring slots of rows x 128 elements, one
// mbarrier per slot, (FP8) two group scales per slot row and (FP8 or no
// ring) a rows x 36 float transpose for its row sums - otherwise the row
// sums go through the warp's just-consumed slot; then the per-warp u_A
// entries, the double-buffered column-sum
// exchange [2][G][8][128] floats and its item table (y2 offset, valid
// columns).
struct TiledSmem {
    size_t bars, scl, ysc, ua, y2, off, cnt, total;
};

constexpr int kRowSumStride = 36;   // floats per row of the row-sum transpose

HOSCF_HD inline TiledSmem tiled_smem(int S, int G, int rows, int es, bool fp8) {
    TiledSmem L;
    size_t o = (size_t)8 * S * rows * 128 * es;
    L.bars = o;
    o += (size_t)8 * S * 8;
    L.scl = o;
    o += fp8 ? (size_t)8 * S * rows * 2 * 4 : 0;
    o = (o + 15) & ~(size_t)15;
    // per warp: rows x kRowSumStride floats for the row-sum transpose, unless
    // the warp's just-consumed ring slot holds it (rows of >= 144 bytes)
    L.ysc = o;
    if (fp8 || S == 0 || 128 * es < kRowSumStride * 4) o += (size_t)8 * rows * kRowSumStride * 4;
    L.ua = o;    // per warp: its rows' factor entries u_{d-1}[a]
    o += (size_t)8 * 16 * 4;
    L.y2 = o;
    o += (size_t)2 * G * 8 * 128 * 4;
    L.off = o;
    o += (size_t)2 * G * 8;
    L.cnt = o;
    o += (size_t)2 * G * 4;
    L.total = o;
    return L;
}



// Shared-memory layout of the narrow-format kernel (BF16 / FP8 with
// 128 <= B <= 256, B % 8 == 0), from a 1024-byte aligned base: each of the 8
// warps owns S ring slots, each holding its rows x B elements of one outer
// index (one bulk copy, rounded out to 16-byte granules) and, for FP8, the
// scale groups those rows span (a second bulk copy); one mbarrier per slot;
// a rows x 36 float transpose per warp for its row sums; the per-warp u_A
// entries; the double-buffered column-sum exchange [2][G][8][256] floats and
// its item table.
struct NarrowSmem {
    size_t slot, data, bars, ysc, ua, y2, off, cnt, total;
};

// Rows per warp at most of the narrow kernel's two-CTAs-per-SM variant
// (registers <= 128); the one-CTA variant takes 13 or 16.
constexpr int kNarrowRowsOcc2 = 7;
#ifndef HOSCF_NARROW_OCC
#define HOSCF_NARROW_OCC 1   // CTAs per SM of the narrow kernel (1 or 2)
#endif

// A slot's data: 16 zero bytes (the pad lanes past the row end read), then
// the rows copied from the 16-byte granule below the band's first element
// (the copy is at most the band plus 30 bytes of rounding).
HOSCF_HD inline size_t narrow_slot_data(int rows, int64_t B, int es) {
    return ((size_t)(48 + rows * B * es) + 15) & ~(size_t)15;
}

HOSCF_HD inline size_t narrow_slot_bytes(int rows, int64_t B, int es, bool fp8) {
    // scale groups a band of rows * B flat elements can touch, plus the
    // 16-byte rounding of their copy on both ends
    const size_t ng = fp8 ? (size_t)(rows * B) / 128 + 2 + 8 : 0;
    return narrow_slot_data(rows, B, es) + (((ng * 4) + 15) & ~(size_t)15);
}

HOSCF_HD inline NarrowSmem narrow_smem(int S, int G, int rows, int64_t B, int es, bool fp8) {
    NarrowSmem L;
    L.slot = narrow_slot_bytes(rows, B, es, fp8);
    L.data = narrow_slot_data(rows, B, es);
    size_t o = (size_t)8 * S * L.slot;
    L.bars = o;
    o += (size_t)8 * S * 8;
    L.ysc = o;
    o += (size_t)8 * rows * kRowSumStride * 4;
    L.ua = o;
    o += (size_t)8 * 16 * 4;
    L.y2 = o;
    o += (size_t)2 * G * 8 * 256 * 4;
    L.off = o;
    o += (size_t)2 * G * 8;
    L.cnt = o;
    o += (size_t)2 * G * 4;
    L.total = o;
    return L;
}

// Eigen-step configuration (cooperative Lanczos over G CTAs).
struct EigPlan {
    int G = 1;
    int mmax = 64;
    int64_t cache_floats = 0;   // per-CTA shared-memory cache of J rows (floats)
    size_t smem = 0;            // dynamic shared memory of the Lanczos kernel
    size_t off_jr = 0, off_V = 0, off_Y = 0, off_part = 0, off_scal = 0, off_bar = 0;
    size_t bytes = 0;
};

bool make_eig_plan(const Shape& s, int nsm, int blocks_per_sm, int mmax, EigPlan& e);

// Factor offsets passed by value to small kernels.
struct ModeInfoArr {
    int64_t off[kMaxOrder + 1];
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace hoscf
