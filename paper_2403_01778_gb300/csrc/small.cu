// All-pairs TTVc for tensors whose face (the two fastest modes, A x B) is
// small (B <= 32, A*B <= 1024), e.g. 24x20x24x20x24x20 or 8^8 (the shapes of
// the paper's Sec. 6.2).
//
// The same factorisation as the tiled pass (eq. 3.3 split into a face block,
// row sums y1 = T_o u_B, column sums y2 = T_o^T u_A, r_o = <y1, u_A> and
// their outer-mode contractions), organised for faces too small to tile:
//
// * Each CTA owns a contiguous range of outer indices (faces), which is one
//   contiguous slab of the tensor.  It streams the slab in groups of K faces
//   through a ring of shared-memory slots filled by bulk copies
//   (cp.async.bulk, one elected thread, mbarrier transaction counts).
// * Element work: thread (k, r) reads row r of face k (vector loads) and
//   forms y1 and the face-block accumulation w_o T_o in registers; thread
//   (k, b) reads column (pair) b of face k and forms y2.  Packed FP32x2 FMAs.
// * Folds, two-level: the fastest outer mode c gets every face's y1, y2 and
//   r; the other outer modes only the run sums over c (faces that share all
//   other digits), sum_j u_c[j] y1(o_j), which carry the same information for
//   them.  All folds go into a shared-memory patch of the CTA (rows limited to
//   the digits its range covers), each patch entry updated by one thread in
//   face order, so the result is deterministic.
// * Every run the CTA's range touches has its patch offsets and factor
//   products in a table built once at the start; per group one warp derives
//   the per-face values (u_c[j], patch row, run) a group ahead from a
//   mode-c digit cursor (no 64-bit divisions in the loop).
// * The stages of consecutive groups overlap: one barrier per group up to 4
//   outer modes, two beyond (see the kernel).
// One reduce kernel then sums, for each output entry, the patches of the CTAs
// that cover it, in CTA order.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include "small_kernel.cuh"

namespace hoscf {

// Reduce: for every output entry, the patches of the CTAs whose digit ranges
// cover it, in CTA order.
struct SmallReduceArgs {
    int D, A, B, F, G, npairs;
    int dims[kMaxOrder];
    int Rmax[kMaxOrder];
    int pm[kMaxBlocks], pn[kMaxBlocks];
    int64_t x1off[kMaxOrder], x2off[kMaxOrder], poff[kMaxBlocks];
    int64_t patch_floats;
    int64_t hface;                 // packed offset of the face block
    int64_t hx1[kMaxOrder], hx2[kMaxOrder], hp[kMaxBlocks];
    int64_t seg[2 * kMaxOrder + kMaxBlocks + 2];   // output prefix: face, X1.., X2.., pairs..
    int nseg;
};

__global__ void small_reduce_kernel(const float* __restrict__ patch, const int* __restrict__ cover,
                                    SmallReduceArgs r, float* __restrict__ H) {
    // one warp per output entry; lanes stride over the CTAs, then a fixed
    // butterfly, so every entry is summed in the same order on every run
    const int lane = threadIdx.x & 31;
    const int64_t total = r.seg[r.nseg];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = wid; e < total; e += nwarps) {
        int sgi = 0;
        while (e >= r.seg[sgi + 1]) ++sgi;
        const int64_t loc = e - r.seg[sgi];
        float s = 0.f;
        int64_t dst;
        // each lane adds the CTAs lane, lane + 32, ... in that order; four of
        // them per round so that their loads are in flight together
        const int2* cv2 = reinterpret_cast<const int2*>(cover);
        if (sgi == 0) {   // face block
            int c = lane;
            for (; c + 96 < r.G; c += 128) {
                float v[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) v[t] = __ldg(patch + (size_t)(c + 32 * t) * r.patch_floats + loc);
#pragma unroll
                for (int t = 0; t < 4; ++t) s += v[t];
            }
            for (; c < r.G; c += 32) s += __ldg(patch + (size_t)c * r.patch_floats + loc);
            dst = r.hface + loc;
        } else if (sgi <= 2 * r.D) {
            const bool x1 = sgi <= r.D;
            const int m = x1 ? sgi - 1 : sgi - 1 - r.D;
            const int C = x1 ? r.A : r.B;
            const int i = (int)(loc / C), col = (int)(loc % C);
            const int64_t base = r.F + (x1 ? r.x1off[m] : r.x2off[m]) + col;
            auto entry = [&](int c, int2 cvv, float& v) {
                int rr = i - cvv.x;
                if (rr < 0) rr += r.dims[m];
                const bool in = rr < cvv.y;
                v = in ? __ldg(patch + (size_t)c * r.patch_floats + base + (int64_t)rr * C) : 0.f;
                return in;
            };
            int c = lane;
            for (; c + 96 < r.G; c += 128) {
                int2 cvv[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) cvv[t] = __ldg(cv2 + ((c + 32 * t) * r.D + m));
                float v[4];
                bool in[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) in[t] = entry(c + 32 * t, cvv[t], v[t]);
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (in[t]) s += v[t];
            }
            for (; c < r.G; c += 32) {
                float v;
                if (entry(c, __ldg(cv2 + (c * r.D + m)), v)) s += v;
            }
            dst = (x1 ? r.hx1[m] : r.hx2[m]) + loc;
        } else {
            const int p = sgi - 1 - 2 * r.D;
            const int m = r.pm[p], n = r.pn[p];
            const int i = (int)(loc / r.dims[n]), j = (int)(loc % r.dims[n]);
            const int Rn = r.Rmax[n];
            const int64_t base = r.F + r.poff[p];
            auto entry = [&](int c, int2 cm, int2 cn, float& v) {
                int rm = i - cm.x, rn = j - cn.x;
                if (rm < 0) rm += r.dims[m];
                if (rn < 0) rn += r.dims[n];
                const bool in = rm < cm.y && rn < cn.y;
                v = in ? __ldg(patch + (size_t)c * r.patch_floats + base + (int64_t)rm * Rn + rn) : 0.f;
                return in;
            };
            int c = lane;
            for (; c + 96 < r.G; c += 128) {
                int2 cm[4], cn[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    cm[t] = __ldg(cv2 + ((c + 32 * t) * r.D + m));
                    cn[t] = __ldg(cv2 + ((c + 32 * t) * r.D + n));
                }
                float v[4];
                bool in[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) in[t] = entry(c + 32 * t, cm[t], cn[t], v[t]);
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (in[t]) s += v[t];
            }
            for (; c < r.G; c += 32) {
                float v;
                if (entry(c, __ldg(cv2 + (c * r.D + m)), __ldg(cv2 + (c * r.D + n)), v)) s += v;
            }
            dst = r.hp[p] + loc;
        }
        s = warp_sum(s);
        if (lane == 0) H[dst] = s;
    }
}

// ---------------------------------------------------------------- host
static uint32_t small_magic(uint32_t d) {
    return d <= 1 ? 0u : (uint32_t)((1ull << 32) / d + 1);
}
static int small_es(int dtype) {
    return dtype == HOSCF_F32 ? 4 : (dtype == HOSCF_BF16 || dtype == HOSCF_F16) ? 2 : 1;
}
static uint32_t al16(uint64_t x) { return (uint32_t)((x + 15) & ~15ull); }

// Patch rows for a range of L faces, offsets and the shared-memory layout.
static bool small_layout(const Shape& s, int es, int64_t L, int S, SmallPlanInfo& sp) {
    const int A = (int)s.A, B = (int)s.B, D = s.D, K = sp.K;
    const int64_t F = s.A * s.B;
    int64_t off = 0;
    for (int m = 0; m < D; ++m)
        sp.Rmax[m] = (int)std::min<int64_t>(s.dims[m], (L + s.ost[m] - 1) / s.ost[m] + 1);
    // X1 / X2 blocks start on 16-byte boundaries (float4 folds when A and B
    // are multiples of 4)
    for (int m = 0; m < D; ++m) {
        sp.x1off[m] = off;
        off = (off + (int64_t)sp.Rmax[m] * A + 3) & ~3LL;
    }
    for (int m = 0; m < D; ++m) {
        sp.x2off[m] = off;
        off = (off + (int64_t)sp.Rmax[m] * B + 3) & ~3LL;
    }
    int np = 0;
    for (int m = 0; m < D; ++m)
        for (int n = m + 1; n < D; ++n) {
            sp.pm[np] = m;
            sp.pn[np] = n;
            sp.poff[np] = off;
            off += (int64_t)sp.Rmax[m] * sp.Rmax[n];
            ++np;
        }
    sp.npairs = np;
    sp.patch_floats = F + off;
    if (sp.patch_floats > (1LL << 30)) return false;
    const int C = (int)s.dims[D - 1];
    sp.nsmax = std::min(K, (K + C - 1) / C + 1);
    const int nm = D - 1, nq = nm * (nm - 1) / 2;
    sp.nstage = S;
    sp.stage_bytes = al16((uint64_t)K * F * es) + 16;
    uint64_t o = 0;
    sp.o_bars = (uint32_t)o;
    o = al16(o + 8ull * S);
    sp.o_ring = (uint32_t)o;
    o = al16(o + std::max<uint64_t>((uint64_t)S * sp.stage_bytes, 4ull * sp.K1 * F));
    sp.o_uA = (uint32_t)o;
    o = al16(o + 4ull * ((A + 3) & ~3));
    sp.o_uB = (uint32_t)o;
    o = al16(o + 4ull * kSmallMaxB);
    sp.o_y1 = (uint32_t)o;
    // y1 / y2 and metadata slots: 3 and 4 for the one-barrier schedule (at
    // most 4 outer modes), 2 and 3 for the two-barrier one
    const int ny = D <= 4 ? 3 : 2, nmeta = D <= 4 ? 4 : 3;
    sp.onebar = D <= 4 ? 1 : 0;
    o = al16(o + 4ull * ny * K * A);
    sp.o_y2 = (uint32_t)o;
    o = al16(o + 4ull * ny * K * B);
    sp.o_r = (uint32_t)o;
    o = al16(o + 8ull * K);
    sp.o_S = (uint32_t)o;
    o = al16(o + 8ull * sp.nsmax * (A + B));
    sp.meta_words = small_meta_words(K, sp.nsmax);
    sp.o_meta = (uint32_t)o;
    o = al16(o + 4ull * nmeta * sp.meta_words);
    // runs of mode c a range of L faces touches
    sp.NR = (int)((L + C - 2) / C + 1);
    sp.o_tab = (uint32_t)o;
    o = al16(o + 4ull * small_table_words(sp.NR, nm, nq));
    sp.o_first = (uint32_t)o;
    o = al16(o + 4ull * kMaxOrder);
    sp.o_patch = (uint32_t)o;
    o = al16(o + 4ull * (uint64_t)off);
    int64_t nur = 0;
    for (int m = 0; m < D; ++m) {
        sp.uro[m] = (int)nur;
        nur += sp.Rmax[m];
    }
    sp.o_ur = (uint32_t)o;
    o = al16(o + 4ull * (uint64_t)nur);
    sp.smem = o + 128;
    return true;
}

bool make_small_plan(const Shape& s, int dtype, int nsm, SmallPlanInfo& sp) {
    sp = SmallPlanInfo();
    if (s.d < 3 || s.D < 1) return false;
    const int64_t A = s.A, B = s.B, F = A * B;
    if (B > kSmallMaxB || F > 1024 || A > kSmallThreads) return false;
    // K1 faces per pass of the threads (thread per face row and per face
    // column), two passes per group where that stays within 32 faces
    const int K1 = (int)std::min<int64_t>(kSmallThreads / A, kSmallThreads / B);
    if (K1 < 1) return false;
    const int K = std::min(kSmallMaxK, 2 * K1);
    sp.K = K;
    sp.K1 = K1;
    const int es = small_es(dtype);
    const uint32_t sb = al16((uint64_t)K * F * es) + 16;
    nsm = std::max(1, nsm);
    // one wave of CTAs (2 per SM, else 1); more, with shorter ranges, when
    // the patch of a long range does not fit in shared memory
    // rows of at most 16 elements keep the kernel within 80 registers (3 CTAs
    // per SM); wider rows within 128 (2 CTAs)
    for (int occ = B <= 16 ? 3 : 2; occ >= 1; --occ) {
        const size_t cap = occ == 3 ? 73 * 1024 : occ == 2 ? 110 * 1024 : 220 * 1024;
        for (int64_t Gt = (int64_t)occ * nsm; ; Gt *= 2) {
            int64_t G = std::min<int64_t>(Gt, (s.O + K - 1) / K);
            G = std::max<int64_t>(G, 1);
            int64_t L = (s.O + G - 1) / G;
            L = (L + K - 1) / K * K;
            G = (s.O + L - 1) / L;
            SmallPlanInfo t = sp;
            // ring slots: what the rest leaves, 2 .. 8 and at most 96 KB
            bool fits = small_layout(s, es, L, 2, t) && t.smem <= cap;
            if (fits) {
                const int S = (int)std::max<int64_t>(
                    2, std::min<int64_t>({8, 2 + (int64_t)(cap - t.smem) / sb, 96 * 1024 / sb}));
                fits = small_layout(s, es, L, S, t) && t.smem <= cap;
            }
            if (fits) {
                t.G = (int)G;
                t.L = L;
                t.occ = occ;
                sp = t;
                return true;
            }
            if (L <= K || Gt > (1LL << 24)) break;
        }
    }
    return false;
}

cudaError_t run_small(const Shape& s, const SmallPlanInfo& sp, int dtype, const void* data,
                      const float* scales, const float* u, float* H, char* ws, int* dev_err,
                      uint64_t timeout_ns, cudaStream_t st, const KernelEvents* kev) {
    // row / column-pair vector loads need B % 4 == 0 and 16-byte aligned
    // faces and rows (then every slot's data starts 16-byte aligned)
    const int es = small_es(dtype);
    const bool vec = dtype != HOSCF_F8E4M3 && s.B % 4 == 0 &&
                     (reinterpret_cast<uintptr_t>(data) & 15u) == 0 && (s.A * s.B * es) % 16 == 0;
    const bool vec_cols = vec;
    SmallArgs a;
    memset(&a, 0, sizeof(a));
    a.T = data;
    a.scales = scales;
    a.u = u;
    a.patch = reinterpret_cast<float*>(ws + sp.off_patch);
    a.cover = reinterpret_cast<int*>(ws + sp.off_cover);
    a.err = dev_err;
    a.timeout_ns = timeout_ns ? timeout_ns : 2000000000ull;
    a.O = s.O;
    a.L = sp.L;
    a.A = (int)s.A;
    a.B = (int)s.B;
    a.F = (int)(s.A * s.B);
    a.D = s.D;
    a.K = sp.K;
    a.K1 = sp.K1;
    a.nsmax = sp.nsmax;
    a.C = (int)s.dims[s.D - 1];
    a.nstage = sp.nstage;
    a.stage_bytes = sp.stage_bytes;
    a.mag_ab = small_magic((uint32_t)(a.A + a.B));
    a.mag_nm = small_magic((uint32_t)std::max(1, s.D - 1));
    a.mag_c = small_magic((uint32_t)std::min<int64_t>(s.dims[s.D - 1], 1 << 15));
    a.v4 = (a.A % 4 == 0 && a.B % 4 == 0) ? 1 : 0;
    a.mag_ab4 = small_magic((uint32_t)std::max(1, (a.A + a.B) / 4));
    for (int k = 0; k < s.D; ++k) a.uro[k] = sp.uro[k];
    for (int k = 0; k < s.D; ++k) {
        a.dims[k] = (int)s.dims[k];
        a.st[k] = s.ost[k];
        a.uoff[k] = (int)s.moff[k];
        a.Rmax[k] = sp.Rmax[k];
        a.x1off[k] = (int)sp.x1off[k];
        a.x2off[k] = (int)sp.x2off[k];
    }
    a.uAoff = (int)s.moff[s.d - 2];
    a.uBoff = (int)s.moff[s.d - 1];
    const int c = s.D - 1;
    for (int p = 0; p < sp.npairs; ++p) {
        if (sp.pn[p] == c) {
            a.pcoff[sp.pm[p]] = (int)sp.poff[p];
        } else {
            a.qm[a.nq] = sp.pm[p];
            a.qn[a.nq] = sp.pn[p];
            a.qoff[a.nq] = (int)sp.poff[p];
            ++a.nq;
        }
    }
    a.patch_floats = sp.patch_floats;
    a.o_bars = sp.o_bars;
    a.o_ring = sp.o_ring;
    a.o_uA = sp.o_uA;
    a.o_uB = sp.o_uB;
    a.o_y1 = sp.o_y1;
    a.o_y2 = sp.o_y2;
    a.o_r = sp.o_r;
    a.o_S = sp.o_S;
    a.o_meta = sp.o_meta;
    a.o_first = sp.o_first;
    a.o_patch = sp.o_patch;
    a.o_ur = sp.o_ur;
    a.o_tab = sp.o_tab;
    a.NR = sp.NR;
    a.mag_bc = small_magic((uint32_t)(vec_cols ? a.B / 2 : a.B));
    {
        const int ncol = a.v4 ? (a.A + a.B) / 4 : a.A + a.B;
        int P = 1;
        while (P < ncol && P < 32) P <<= 1;
        a.pcol = P;
    }
    // measured: one barrier per group wins up to 4 outer modes
    // (24x20x24x20x24x20 -13 %), two barriers beyond (8^8, 16^4 8^3)
    a.onebar = sp.onebar;
    a.meta_words = sp.meta_words;

    cudaError_t e;
    if (dtype == HOSCF_F32)
        e = launch_small_f32(sp, a, vec, st, kev);
    else if (dtype == HOSCF_BF16)
        e = launch_small_bf16(sp, a, vec, st, kev);
    else if (dtype == HOSCF_F16)
        e = launch_small_f16(sp, a, vec, st, kev);
    else
        e = launch_small_bm<fp8_t, false>(sp, a, st, kev);
    if (e != cudaSuccess) return e;
    SmallReduceArgs r;
    memset(&r, 0, sizeof(r));
    r.D = s.D;
    r.A = a.A;
    r.B = a.B;
    r.F = a.F;
    r.G = sp.G;
    r.npairs = sp.npairs;
    for (int k = 0; k < s.D; ++k) {
        r.dims[k] = (int)s.dims[k];
        r.Rmax[k] = sp.Rmax[k];
        r.x1off[k] = sp.x1off[k];
        r.x2off[k] = sp.x2off[k];
        r.hx1[k] = s.boff[block_index(s.d, k, s.d - 2)];
        r.hx2[k] = s.boff[block_index(s.d, k, s.d - 1)];
    }
    for (int p = 0; p < sp.npairs; ++p) {
        r.pm[p] = sp.pm[p];
        r.pn[p] = sp.pn[p];
        r.poff[p] = sp.poff[p];
        r.hp[p] = s.boff[block_index(s.d, sp.pm[p], sp.pn[p])];
    }
    r.patch_floats = sp.patch_floats;
    r.hface = s.boff[block_index(s.d, s.d - 2, s.d - 1)];
    int g = 0;
    r.seg[0] = 0;
    r.seg[g + 1] = r.seg[g] + (int64_t)a.F;
    ++g;
    for (int k = 0; k < s.D; ++k, ++g) r.seg[g + 1] = r.seg[g] + s.dims[k] * s.A;
    for (int k = 0; k < s.D; ++k, ++g) r.seg[g + 1] = r.seg[g] + s.dims[k] * s.B;
    for (int p = 0; p < sp.npairs; ++p, ++g)
        r.seg[g + 1] = r.seg[g] + s.dims[sp.pm[p]] * s.dims[sp.pn[p]];
    r.nseg = g;
    const int64_t total = r.seg[g];
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(8192, (total * 32 + 255) / 256));
    small_reduce_kernel<<<blocks, 256, 0, st>>>(a.patch, a.cover, r, H);
    return cudaGetLastError();
}

}  // namespace hoscf
