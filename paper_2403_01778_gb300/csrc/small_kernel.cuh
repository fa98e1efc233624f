// Small-face pass kernel (see small.cu for the scheme): arguments, the
// kernel template and its launchers, instantiated per element type in
// small.cu (FP8), small_f32.cu and small_bf16.cu.
#pragma once
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hoscf {

struct SmallArgs {
    const void* T;
    const float* scales;      // FP8 only: one per 128 flat elements
    const float* u;
    float* patch;             // G x patch_floats
    int* cover;               // G x D x 2: first digit, row count
    int* err;
    uint64_t timeout_ns;
    int64_t O, L;
    int A, B, F, D, K, K1, C, nstage;   // K faces per group, K1 per pass of the threads
    int nsmax;
    uint32_t stage_bytes;
    uint32_t mag_ab, mag_nm, mag_c;   // t / (A+B), t / (D-1), t / C by multiply-high
    uint32_t mag_ab4;                 // t / ((A+B)/4)
    int v4;                           // A, B multiples of 4: folds by float4
    int uro[kMaxOrder];               // staged factor rows of outer mode m
    int dims[kMaxOrder];
    int64_t st[kMaxOrder];
    int uoff[kMaxOrder];
    int uAoff, uBoff;
    int Rmax[kMaxOrder];
    int x1off[kMaxOrder], x2off[kMaxOrder];
    int pcoff[kMaxOrder];                     // block (m, c) for m < c
    int nq;                                   // blocks (m, n) with n < c
    int qm[kSmallMaxNq], qn[kSmallMaxNq], qoff[kSmallMaxNq];
    int64_t patch_floats;
    uint32_t o_bars, o_ring, o_uA, o_uB, o_y1, o_y2, o_r, o_S, o_meta, o_first, o_patch, o_ur, o_tab;
    int NR;                           // runs of mode c in the run table
    uint32_t mag_bc;                  // t / (column tasks per face)
    int pcol;                         // run sums: column chunks per warp pass (power of 2)
    int onebar;                       // one barrier per group (see the kernel's schedules)
    uint32_t meta_words;
};

// n / d for n < 2^16, d < 2^16 by multiply-high with m = floor(2^32 / d) + 1
// (d >= 2; m = 0 stands for d = 1): the error term n (m d - 2^32) / (d 2^32)
// stays below 1/d, so the floor is exact.
__device__ __forceinline__ int sdiv(int n, uint32_t m) {
    return m ? (int)__umulhi((uint32_t)n, m) : n;
}

// ---------------------------------------------------------------- element loads
template <typename E>
__device__ __forceinline__ float lds_elem(const unsigned char* p);
template <>
__device__ __forceinline__ float lds_elem<float>(const unsigned char* p) {
    return *reinterpret_cast<const float*>(p);
}
template <>
__device__ __forceinline__ float lds_elem<bf16_t>(const unsigned char* p) {
    return __uint_as_float(static_cast<uint32_t>(*reinterpret_cast<const uint16_t*>(p)) << 16);
}
template <>
__device__ __forceinline__ float lds_elem<f16_t>(const unsigned char* p) {
    return __half2float(__ushort_as_half(*reinterpret_cast<const unsigned short*>(p)));
}
template <>
__device__ __forceinline__ float lds_elem<fp8_t>(const unsigned char* p) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)*p, __NV_E4M3);
    return __half2float(*reinterpret_cast<const __half*>(&h));
}

// four row elements 4c .. 4c+3 (zero past B when loaded one by one)
template <typename E, bool VEC>
__device__ __forceinline__ float4 lds_row4(const unsigned char* row, int c, int B) {
    if constexpr (VEC) {
        if constexpr (sizeof(E) == 4) {
            return *reinterpret_cast<const float4*>(row + 16 * c);
        } else if constexpr (std::is_same<E, f16_t>::value) {
            const uint2 v = *reinterpret_cast<const uint2*>(row + 8 * c);
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
            return make_float4(a.x, a.y, b.x, b.y);
        } else {
            const uint2 v = *reinterpret_cast<const uint2*>(row + 8 * c);
            return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u),
                               __uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
        }
    } else {
        constexpr int es = (int)sizeof(E);
        float4 r;
        r.x = 4 * c + 0 < B ? lds_elem<E>(row + (4 * c + 0) * es) : 0.f;
        r.y = 4 * c + 1 < B ? lds_elem<E>(row + (4 * c + 1) * es) : 0.f;
        r.z = 4 * c + 2 < B ? lds_elem<E>(row + (4 * c + 2) * es) : 0.f;
        r.w = 4 * c + 3 < B ? lds_elem<E>(row + (4 * c + 3) * es) : 0.f;
        return r;
    }
}

// two adjacent column elements (vector mode only)
template <typename E>
__device__ __forceinline__ float2 lds_pair(const unsigned char* p) {
    if constexpr (sizeof(E) == 4) {
        return *reinterpret_cast<const float2*>(p);
    } else if constexpr (std::is_same<E, f16_t>::value) {
        return __half22float2(*reinterpret_cast<const __half2*>(p));
    } else {
        const uint32_t v = *reinterpret_cast<const uint32_t*>(p);
        return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
    }
}

// ---------------------------------------------------------------- metadata
// Run table, built once per CTA: for every run of mode c (faces that share
// all other outer digits) that the CTA's range touches, the patch offsets of
// its rows in X1/X2 and in the pair blocks and its factor products.  NR runs
// per field.
struct RunTable {
    int* x1o;        // nm x NR: x1off[m] + row * A
    int* x2o;        // nm x NR: x2off[m] + row * B
    int* pco;        // nm x NR: block (m, c), start of the row
    float* qm;       // nm x NR: prod over the outer modes but m, c
    int* pqo;        // nq x NR: block (m, n), n < c, entry of the run
    float* qmn;      // nq x NR: prod over the outer modes but m, n, c
    float* p;        // NR: prod over the outer modes but c
    __device__ RunTable(int* base, int NR, int nm, int nq) {
        x1o = base;
        x2o = x1o + nm * NR;
        pco = x2o + nm * NR;
        qm = reinterpret_cast<float*>(pco + nm * NR);
        pqo = reinterpret_cast<int*>(qm + nm * NR);
        qmn = reinterpret_cast<float*>(pqo + nq * NR);
        p = qmn + nq * NR;
    }
};

inline uint32_t small_table_words(int NR, int nm, int nq) {
    return (uint32_t)NR * (uint32_t)(4 * nm + 2 * nq + 1);
}

// One slot per group: per face (K entries) the face-block weight w_o, the
// fold weight of mode c (the run's product), u_c[j], the patch row of mode c
// and the run (within the group); the first face of each run of the group;
// the run count and the table index of the group's first run.
struct MetaView {
    float* w;
    float* p;
    float* vc;
    int* jrow;
    int* seg;
    int* segstart;   // NS + 1
    int* hdr;        // runs in the group, table index of its first run
    __device__ MetaView(int* base, int K, int NS) {
        w = reinterpret_cast<float*>(base);
        p = w + K;
        vc = p + K;
        jrow = reinterpret_cast<int*>(vc + K);
        seg = jrow + K;
        segstart = seg + K;
        hdr = segstart + NS + 1;
    }
};

inline uint32_t small_meta_words(int K, int NS) { return (uint32_t)(5 * K + NS + 3); }

// index of the run of position jj = (first face's digit of mode c) + k
__device__ __forceinline__ int small_run(const SmallArgs& a, int jj) {
    return a.C >= 32 ? (jj >= a.C ? 1 : 0) : sdiv(jj, a.mag_c);
}

// n / d for a digit plus a carry (n < d + 32): one compare when d >= 32
__device__ __forceinline__ int small_carry(int n, int d, uint32_t mag) {
    return d >= 32 ? (n >= d ? 1 : 0) : sdiv(n, mag);
}

// Table entry of run r of the CTA's range [o_lo, ...): its first face is
// r C - first_c (run 0: face 0).
__device__ __forceinline__ void small_table_entry(const SmallArgs& a, const RunTable& tb, int NR,
                                                  int r, int64_t o_lo, const int* first,
                                                  const float* ur) {
    const int nm = a.D - 1;
    const int64_t o = o_lo + (r == 0 ? 0 : (int64_t)r * a.C - first[nm]);
    float v[kSmallMaxNm], pre[kSmallMaxNm + 1], suf[kSmallMaxNm + 1];
    int rr[kSmallMaxNm];
#pragma unroll
    for (int m = 0; m < kSmallMaxNm; ++m) {
        int row = 0;
        if (m < nm) {
            row = (int)((o / a.st[m]) % a.dims[m]) - first[m];
            if (row < 0) row += a.dims[m];
        }
        rr[m] = row;
        v[m] = m < nm ? ur[a.uro[m] + row] : 1.f;
    }
    pre[0] = 1.f;
#pragma unroll
    for (int m = 0; m < kSmallMaxNm; ++m) pre[m + 1] = pre[m] * v[m];
    suf[kSmallMaxNm] = 1.f;
#pragma unroll
    for (int m = kSmallMaxNm - 1; m >= 0; --m) suf[m] = suf[m + 1] * v[m];
    tb.p[r] = pre[kSmallMaxNm];
    const int Rc = a.Rmax[nm];
#pragma unroll
    for (int m = 0; m < kSmallMaxNm; ++m) {
        if (m < nm) {
            tb.x1o[m * NR + r] = a.x1off[m] + rr[m] * a.A;
            tb.x2o[m * NR + r] = a.x2off[m] + rr[m] * a.B;
            tb.pco[m * NR + r] = a.pcoff[m] + rr[m] * Rc;
            tb.qm[m * NR + r] = pre[m] * suf[m + 1];
        }
    }
    for (int q = 0; q < a.nq; ++q) {
        const int m = a.qm[q], n = a.qn[q];
        float mid = 1.f, pm = 1.f, sn = 1.f;
        int rm = 0, rn = 0;
#pragma unroll
        for (int k = 0; k < kSmallMaxNm; ++k) {
            if (k > m && k < n) mid *= v[k];
            if (k == m) { rm = rr[k]; pm = pre[k]; }
            if (k == n) { rn = rr[k]; sn = suf[k + 1]; }
        }
        tb.pqo[q * NR + r] = a.qoff[q] + rm * a.Rmax[n] + rn;
        tb.qmn[q * NR + r] = pm * mid * sn;
    }
}

// One warp: metadata of the group whose first face has digit c0 of mode c
// and lies in run run0 of the table.  Lane k handles face k.
__device__ __forceinline__ void small_meta(const SmallArgs& a, MetaView mv, const RunTable& tb,
                                           int c0, int run0, int first_c, const float* ur, int nfg,
                                           int lane) {
    const int nm = a.D - 1, C = a.C;
    const int sk = small_run(a, c0 + lane);
    const int j = c0 + lane - sk * C;
    int jr = j - first_c;
    if (jr < 0) jr += C;
    const int ns = small_run(a, c0 + nfg - 1) + 1;
    if (lane < nfg) {
        const float vcv = ur[a.uro[nm] + jr];
        const float pf = tb.p[run0 + sk];
        mv.w[lane] = pf * vcv;
        mv.p[lane] = pf;
        mv.vc[lane] = vcv;
        mv.jrow[lane] = jr;
        mv.seg[lane] = sk;
    }
    if (lane < ns) mv.segstart[lane] = lane == 0 ? 0 : lane * C - c0;
    if (lane == 0) {
        mv.segstart[ns] = nfg;
        mv.hdr[0] = ns;
        mv.hdr[1] = run0;
    }
}

// ---------------------------------------------------------------- folds
__device__ __forceinline__ float4 f4fma(float a, float4 y, float4 x) {
    return make_float4(fmaf(a, y.x, x.x), fmaf(a, y.y, x.y), fmaf(a, y.z, x.z), fmaf(a, y.w, x.w));
}

// Folds of one group into the patch: mode c gets every face's y1, y2 (T1);
// the other outer modes the run sums (U1); the pairs (m, c) every face's r
// (U2) and the pairs (m, n), n < c, the run sums of r (U3).  Each patch
// entry is updated by one thread, in face order; with A, B multiples of 4 a
// thread takes 4 adjacent columns.  Every warp takes one kind of task at a
// time (no divergence between kinds), from warp 6 down and warp 7 (which
// also builds the metadata) last.
__device__ __forceinline__ void small_folds(const SmallArgs& a, const MetaView& mv,
                                            const RunTable& tb, int NR, const float* y1s,
                                            const float* y2s, const float* Sg, const float* rs,
                                            const float* uB, float* patch, int nf, int warp,
                                            int lane) {
    const int A = a.A, B = a.B, AB = A + B, C = a.C, nm = a.D - 1;
    const bool v4 = a.v4 != 0;
    const int ncol = v4 ? AB >> 2 : AB;
    const uint32_t mcol = v4 ? a.mag_ab4 : a.mag_ab;
    const int kk = min(nf, C);
    const int n1 = kk * ncol;
    const bool outer = a.D >= 2;
    const int ns = outer ? mv.hdr[0] : 0;
    const int run0 = mv.hdr[1];
    const int u1 = outer ? nm * ncol : 0, u2 = outer ? nm * kk : 0, u3 = outer ? a.nq : 0;
    const int w1 = (n1 + 31) >> 5, w2 = w1 + ((u1 + 31) >> 5), w3 = w2 + ((u2 + 31) >> 5),
              w4 = w3 + ((u3 + 31) >> 5);
    for (int vw = warp == 7 ? 7 : 6 - warp; vw < w4; vw += 8) {
        if (vw < w1) {
            const int t = vw * 32 + lane;
            if (t < n1) {
                // faces k0, k0 + C, ... share the digit of mode c
                const int k0 = sdiv(t, mcol), cq = t - k0 * ncol;
                const int col = v4 ? 4 * cq : cq;
                const int jr = mv.jrow[k0];
                const bool x1 = col < A;
                float* X = x1 ? patch + a.x1off[nm] + jr * A + col
                              : patch + a.x2off[nm] + jr * B + (col - A);
                const float* y = x1 ? y1s + col : y2s + (col - A);
                const int ys = x1 ? A : B;
                if (v4) {
                    float4 x = *reinterpret_cast<const float4*>(X);
                    for (int k = k0; k < nf; k += C)
                        x = f4fma(mv.p[k], *reinterpret_cast<const float4*>(y + k * ys), x);
                    *reinterpret_cast<float4*>(X) = x;
                } else {
                    float x = *X;
                    for (int k = k0; k < nf; k += C) x = fmaf(mv.p[k], y[k * ys], x);
                    *X = x;
                }
            }
        } else if (vw < w2) {
            const int t = (vw - w1) * 32 + lane;
            if (t < u1) {
                const int m = sdiv(t, mcol), cq = t - m * ncol;
                const int col = v4 ? 4 * cq : cq;
                const bool x1 = col < A;
                const int* xo = (x1 ? tb.x1o : tb.x2o) + m * NR + run0;
                float* X = patch + (x1 ? col : col - A);
                const float* q = tb.qm + m * NR + run0;
                if (v4) {
                    for (int sg = 0; sg < ns; ++sg) {
                        float4* x = reinterpret_cast<float4*>(X + xo[sg]);
                        *x = f4fma(q[sg], *reinterpret_cast<const float4*>(Sg + sg * AB + col), *x);
                    }
                } else {
                    for (int sg = 0; sg < ns; ++sg) {
                        float* x = X + xo[sg];
                        *x = fmaf(q[sg], Sg[sg * AB + col], *x);
                    }
                }
            }
        } else if (vw < w3) {
            const int t = (vw - w2) * 32 + lane;
            if (t < u2) {
                const int k0 = sdiv(t, a.mag_nm), m = t - k0 * nm;
                for (int k = k0; k < nf; k += C) {
                    const int ri = m * NR + run0 + mv.seg[k];
                    float* x = patch + tb.pco[ri] + mv.jrow[k];
                    *x = fmaf(tb.qm[ri], rs[k], *x);
                }
            }
        } else {
            const int q = (vw - w3) * 32 + lane;
            if (q < u3) {
                // sum over the run of u_c[j] r_o = u_B . (run sum of y2)
                for (int sg = 0; sg < ns; ++sg) {
                    const float* S2 = Sg + sg * AB + A;
                    float s0 = 0.f, s1 = 0.f;
                    int b = 0;
                    for (; b + 2 <= B; b += 2) {
                        s0 = fmaf(uB[b], S2[b], s0);
                        s1 = fmaf(uB[b + 1], S2[b + 1], s1);
                    }
                    if (b < B) s0 = fmaf(uB[b], S2[b], s0);
                    const int ri = q * NR + run0 + sg;
                    float* x = patch + tb.pqo[ri];
                    *x = fmaf(tb.qmn[ri], s0 + s1, *x);
                }
            }
        }
    }
}

// Run sums over mode c (for the other outer modes) and r per face of one
// group (D >= 2).
__device__ __forceinline__ void small_runsums(const SmallArgs& a, const MetaView& mv,
                                      const float* y1s, const float* y2s, float* Sb,
                                      float* rb, const float* uB, int nf, int warp,
                                      int lane, int tid) {
    const int A = a.A, B = a.B, AB = A + B;
    const int ns = mv.hdr[0];
    const bool v4 = a.v4 != 0;
    const int ncol = v4 ? AB >> 2 : AB;
    float* Sg = Sb;
    float* rs = rb;
    // one warp per (run, block of P column chunks): lane = (face offset,
    // chunk); faces strided by 32 / P, then a fixed butterfly over the
    // face offsets
    const int P = a.pcol, FP = 32 / P;
    const int nblk = (ncol + P - 1) / P;
    const int fo = lane / P, cl = lane - fo * P;
    for (int wt = warp; wt < ns * nblk; wt += kSmallThreads / 32) {
        const int sg = wt / nblk, cq = (wt - sg * nblk) * P + cl;
        const int kb = mv.segstart[sg], ke = mv.segstart[sg + 1];
        const bool on = cq < ncol;
        const int col = v4 ? 4 * cq : cq;
        const bool x1 = col < A;
        const float* y = x1 ? y1s + col : y2s + (col - A);
        const int ys = x1 ? A : B;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (on) {
            for (int k = kb + fo; k < ke; k += FP) {
                const float vk = mv.vc[k];
                if (v4) {
                    acc = f4fma(vk, *reinterpret_cast<const float4*>(y + k * ys), acc);
                } else {
                    acc.x = fmaf(vk, y[k * ys], acc.x);
                }
            }
        }
        for (int off = 16; off >= P; off >>= 1) {
            acc.x += __shfl_xor_sync(HOSCF_FULLMASK, acc.x, off);
            if (v4) {
                acc.y += __shfl_xor_sync(HOSCF_FULLMASK, acc.y, off);
                acc.z += __shfl_xor_sync(HOSCF_FULLMASK, acc.z, off);
                acc.w += __shfl_xor_sync(HOSCF_FULLMASK, acc.w, off);
            }
        }
        if (on && fo == 0) {
            if (v4)
                *reinterpret_cast<float4*>(Sg + sg * AB + col) = acc;
            else
                Sg[sg * AB + col] = acc.x;
        }
    }
    // r per face (threads from the top)
    for (int k = kSmallThreads - 1 - tid; k < nf; k += kSmallThreads) {
        const float* y = y2s + k * B;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int b = 0;
        for (; b + 4 <= B; b += 4) {
            s0 = fmaf(uB[b], y[b], s0);
            s1 = fmaf(uB[b + 1], y[b + 1], s1);
            s2 = fmaf(uB[b + 2], y[b + 2], s2);
            s3 = fmaf(uB[b + 3], y[b + 3], s3);
        }
        for (; b < B; ++b) s0 = fmaf(uB[b], y[b], s0);
        rs[k] = (s0 + s1) + (s2 + s3);
    }
}

// ---------------------------------------------------------------- kernel
// Two schedules of a group's three stages (element work, run sums, folds).
// One barrier per group (up to 4 outer modes), iteration g running side by
// side
//   folds(g-2) | run sums and r per face (g-1) | metadata(g+1) (warp 7) |
//   wait slot, element work(g)                                       -- bar
//   refill the slot with group g+S
// or, with more outer modes (where the heavier fold tasks and the run sums
// would pile up on the same warps), two barriers per group:
//   folds(g-1) | metadata(g+1) | wait slot, element work(g)          -- bar
//   refill | run sums and r per face (g)                             -- bar
// (extra iterations drain the last groups).  Run sums and r are
// double-buffered; y1/y2 and the metadata take 3 and 4 slots in the first
// schedule, 2 and 3 in the second.
template <typename E, int BM, bool VEC, bool ONEBAR>
__global__ void __launch_bounds__(kSmallThreads, BM <= 16 ? 3 : 2) ttvc_small_kernel(const SmallArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + a.o_bars);
    unsigned char* ring = sm + a.o_ring;
    float* uA = reinterpret_cast<float*>(sm + a.o_uA);
    float* uB = reinterpret_cast<float*>(sm + a.o_uB);
    float* y1b = reinterpret_cast<float*>(sm + a.o_y1);   // 2 x K x A
    float* y2b = reinterpret_cast<float*>(sm + a.o_y2);   // 2 x K x B
    float* rb = reinterpret_cast<float*>(sm + a.o_r);     // 2 x K
    float* Sb = reinterpret_cast<float*>(sm + a.o_S);     // 2 x nsmax x (A+B)
    int* meta0 = reinterpret_cast<int*>(sm + a.o_meta);   // 3 slots
    int* first = reinterpret_cast<int*>(sm + a.o_first);
    float* patch = reinterpret_cast<float*>(sm + a.o_patch);
    float* ur = reinterpret_cast<float*>(sm + a.o_ur);    // factor rows the range covers
    const RunTable tb(reinterpret_cast<int*>(sm + a.o_tab), a.NR, a.D - 1, a.nq);

    constexpr int es = (int)sizeof(E);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t cta = blockIdx.x;
    const int64_t o_lo = cta * a.L;
    const int64_t o_hi = min(a.O, o_lo + a.L);
    const int A = a.A, B = a.B, F = a.F, D = a.D, K = a.K, K1 = a.K1, AB = A + B, S = a.nstage;
    const int nm = D - 1, NS = a.nsmax, NR = a.NR;
    const int ng = (int)((o_hi - o_lo + K - 1) / K);
    const E* Tp = reinterpret_cast<const E*>(a.T);
    const int64_t ploc = a.patch_floats - F;
    const int sbuf = NS * AB;

    // ---- set-up: barriers, factor rows, patch, covered digit ranges
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(full + s, 1);
        fence_mbar_init();
    }
    for (int i = tid; i < ((A + 3) & ~3); i += kSmallThreads) uA[i] = i < A ? a.u[a.uAoff + i] : 0.f;
    for (int i = tid; i < kSmallMaxB; i += kSmallThreads) uB[i] = i < B ? a.u[a.uBoff + i] : 0.f;
    for (int64_t i = tid; i < ploc; i += kSmallThreads) patch[i] = 0.f;
    if (tid < D) {
        const int m = tid;
        const int64_t q0 = o_lo / a.st[m], q1 = (o_hi - 1) / a.st[m];
        first[m] = (int)(q0 % a.dims[m]);
        const int64_t rows = (q1 - q0 + 1 < (int64_t)a.dims[m]) ? q1 - q0 + 1 : (int64_t)a.dims[m];
        a.cover[(cta * D + m) * 2 + 0] = first[m];
        a.cover[(cta * D + m) * 2 + 1] = (int)rows;
    }
    __syncthreads();
    // outer-mode factor values of the patch rows: ur[uro[m] + r] = u_m[first + r]
    for (int m = 0; m < D; ++m) {
        const int R = a.Rmax[m], fm = first[m], dm = a.dims[m];
        for (int r = tid; r < R; r += kSmallThreads) {
            int i = fm + r;
            if (i >= dm) i -= dm;
            ur[a.uro[m] + r] = a.u[a.uoff[m] + i];
        }
    }
    __syncthreads();
    // run table of the range
    {
        const int nruns = (int)((first[nm] + (o_hi - o_lo) - 1) / a.C) + 1;
        for (int r = tid; r < nruns; r += kSmallThreads) small_table_entry(a, tb, NR, r, o_lo, first, ur);
    }
    __syncthreads();

    auto issue = [&](int gi) {
        const int64_t f0 = o_lo + (int64_t)gi * K;
        const int nfg = (int)min((int64_t)K, o_hi - f0);
        const uintptr_t gb = reinterpret_cast<uintptr_t>(Tp + f0 * F);
        const uintptr_t gal = gb & ~(uintptr_t)15;
        const uint32_t head = (uint32_t)(gb - gal);
        const uint32_t bytes = (head + (uint32_t)nfg * (uint32_t)(F * es) + 15u) & ~15u;
        uint64_t* bar = full + gi % S;
        mbar_arrive_expect_tx(bar, bytes);
        bulk_load(ring + (size_t)(gi % S) * a.stage_bytes, reinterpret_cast<const void*>(gal), bytes,
                  bar);
    };
    if (tid == 0)
        for (int gi = 0; gi < S && gi < ng; ++gi) issue(gi);

    // mode-c digit and table run of the next group to describe (warp 7)
    const int first_c = first[nm];
    int c0 = first_c, run0 = 0;
    auto advance = [&]() {
        c0 += K;
        const int q = small_carry(c0, a.C, a.mag_c);
        c0 -= q * a.C;
        run0 += q;
    };
    if (warp == 7) {
        small_meta(a, MetaView(meta0, K, NS), tb, c0, run0, first_c, ur,
                   (int)min((int64_t)K, o_hi - o_lo), lane);
        advance();
    }

    // element-work roles: rows of faces rk0, rk0 + K1, ...; column (pairs)
    // from the top thread down
    const bool rowt = tid < K1 * A;
    const int rk0 = tid / A, rr = tid - (tid / A) * A;
    const int Bc = VEC ? B / 2 : B;
    float2 hacc[BM / 2];
#pragma unroll
    for (int i = 0; i < BM / 2; ++i) hacc[i] = make_float2(0.f, 0.f);
    __syncthreads();

    auto nf_of = [&](int gi) { return (int)min((int64_t)K, o_hi - o_lo - (int64_t)gi * K); };
    // element work of one group: rows (y1, face block) and columns (y2)
    auto element = [&](const MetaView& mv, float* y1s, float* y2s, int64_t f0, int nf, int s) {
        const unsigned char* data = ring + (size_t)s * a.stage_bytes +
                                    (reinterpret_cast<uintptr_t>(Tp + f0 * F) & 15u);
        if (rowt) {
            for (int rk = rk0; rk < nf; rk += K1) {
                const unsigned char* row = data + (size_t)(rk * F + rr * B) * es;
                const float w = mv.w[rk];
                const float2 w2 = make_float2(w, w);
                float s0 = 1.f, s1 = 1.f;
                int bnd = BM;
                if constexpr (std::is_same<E, fp8_t>::value) {
                    const int64_t e0 = (f0 + rk) * F + (int64_t)rr * B;
                    s0 = __ldg(a.scales + (e0 >> 7));
                    s1 = __ldg(a.scales + ((e0 + B - 1) >> 7));
                    bnd = 128 - (int)(e0 & 127);
                }
                float2 ya = make_float2(0.f, 0.f), yb = make_float2(0.f, 0.f);
    #pragma unroll
                for (int c = 0; c < BM / 4; ++c) {
                    float4 v = lds_row4<E, VEC>(row, c, B);
                    if constexpr (std::is_same<E, fp8_t>::value) {
                        v.x *= 4 * c + 0 < bnd ? s0 : s1;
                        v.y *= 4 * c + 1 < bnd ? s0 : s1;
                        v.z *= 4 * c + 2 < bnd ? s0 : s1;
                        v.w *= 4 * c + 3 < bnd ? s0 : s1;
                    }
                    const float4 ub = *reinterpret_cast<const float4*>(uB + 4 * c);
                    const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
                    ya = ffma2(v0, make_float2(ub.x, ub.y), ya);
                    yb = ffma2(v1, make_float2(ub.z, ub.w), yb);
                    hacc[2 * c] = ffma2(w2, v0, hacc[2 * c]);
                    hacc[2 * c + 1] = ffma2(w2, v1, hacc[2 * c + 1]);
                }
                y1s[rk * A + rr] = (ya.x + ya.y) + (yb.x + yb.y);
            }
        }
        {
            for (int ci = kSmallThreads - 1 - tid; ci < nf * Bc; ci += kSmallThreads) {
                const int ck = sdiv(ci, a.mag_bc), cb = ci - ck * Bc;
                if constexpr (VEC) {
                    const unsigned char* col = data + (size_t)(ck * F + 2 * cb) * es;
                    const int rs_b = B * es;
                    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
                    int r = 0;
                    for (; r + 4 <= A; r += 4) {
                        const float4 ua = *reinterpret_cast<const float4*>(uA + r);
                        const float2 t0 = lds_pair<E>(col + (r + 0) * rs_b);
                        const float2 t1 = lds_pair<E>(col + (r + 1) * rs_b);
                        const float2 t2 = lds_pair<E>(col + (r + 2) * rs_b);
                        const float2 t3 = lds_pair<E>(col + (r + 3) * rs_b);
                        acc0 = ffma2(t0, make_float2(ua.x, ua.x), acc0);
                        acc1 = ffma2(t1, make_float2(ua.y, ua.y), acc1);
                        acc0 = ffma2(t2, make_float2(ua.z, ua.z), acc0);
                        acc1 = ffma2(t3, make_float2(ua.w, ua.w), acc1);
                    }
                    for (; r < A; ++r) {
                        const float ua = uA[r];
                        acc0 = ffma2(lds_pair<E>(col + r * rs_b), make_float2(ua, ua), acc0);
                    }
                    *reinterpret_cast<float2*>(y2s + ck * B + 2 * cb) =
                        make_float2(acc0.x + acc1.x, acc0.y + acc1.y);
                } else {
                    const unsigned char* col = data + (size_t)(ck * F + cb) * es;
                    float acc0 = 0.f, acc1 = 0.f;
                    int r = 0;
                    for (; r + 2 <= A; r += 2) {
                        float t0 = lds_elem<E>(col + (size_t)r * B * es);
                        float t1 = lds_elem<E>(col + (size_t)(r + 1) * B * es);
                        if constexpr (std::is_same<E, fp8_t>::value) {
                            const int64_t e = (f0 + ck) * F + (int64_t)r * B + cb;
                            t0 *= __ldg(a.scales + (e >> 7));
                            t1 *= __ldg(a.scales + ((e + B) >> 7));
                        }
                        acc0 = fmaf(t0, uA[r], acc0);
                        acc1 = fmaf(t1, uA[r + 1], acc1);
                    }
                    if (r < A) {
                        float t = lds_elem<E>(col + (size_t)r * B * es);
                        if constexpr (std::is_same<E, fp8_t>::value)
                            t *= __ldg(a.scales + (((f0 + ck) * F + (int64_t)r * B + cb) >> 7));
                        acc0 = fmaf(t, uA[r], acc0);
                    }
                    y2s[ck * B + cb] = acc0 + acc1;
                }
            }
        }
    };

    if constexpr (ONEBAR) {
        // one barrier per group: folds(g-2) | run sums(g-1) | metadata(g+1) |
        // element work(g); y1/y2 in 3 slots, metadata in 4
        for (int g = 0; g < ng + 2; ++g) {
            const int s = g % S;
            const uint32_t par = (uint32_t)(g / S) & 1u;
            const int64_t f0 = o_lo + (int64_t)g * K;
            const int nf = g < ng ? nf_of(g) : 0;
            MetaView mv(meta0 + (g & 3) * a.meta_words, K, NS);
            float* y1s = y1b + (g % 3) * K * A;
            float* y2s = y2b + (g % 3) * K * B;
            if (g >= 2) {
                const int gf = g - 2;
                small_folds(a, MetaView(meta0 + (gf & 3) * a.meta_words, K, NS), tb, NR,
                            y1b + (gf % 3) * K * A, y2b + (gf % 3) * K * B, Sb + (gf & 1) * sbuf,
                            rb + (gf & 1) * K, uB, patch, nf_of(gf), warp, lane);
            }
            if (D >= 2 && g >= 1 && g - 1 < ng) {
                const int gr = g - 1;
                small_runsums(a, MetaView(meta0 + (gr & 3) * a.meta_words, K, NS),
                              y1b + (gr % 3) * K * A, y2b + (gr % 3) * K * B, Sb + (gr & 1) * sbuf,
                              rb + (gr & 1) * K, uB, nf_of(gr), warp, lane, tid);
            }
            if (warp == 7 && g + 1 < ng) {
                small_meta(a, MetaView(meta0 + ((g + 1) & 3) * a.meta_words, K, NS), tb, c0, run0,
                           first_c, ur, nf_of(g + 1), lane);
                advance();
            }
            const bool ok = g < ng ? mbar_wait_bounded(full + s, par, a.timeout_ns) : true;
            element(mv, y1s, y2s, f0, nf, s);
            if (__syncthreads_or(!ok)) {
                // a copy never completed: record it, wait (bounded) for the
                // copies still in flight into this CTA's slots, and leave
                if (tid == 0) {
                    atomicCAS(a.err, 0, (int)DEV_TIMEOUT);
                    for (int gi = g; gi < g + S && gi < ng; ++gi)
                        (void)mbar_wait_bounded(full + gi % S, (uint32_t)(gi / S) & 1u, a.timeout_ns);
                }
                __syncthreads();
                return;
            }
            if (tid == 0 && g + S < ng) issue(g + S);
        }
    } else {
        // two barriers per group: folds(g-1) | metadata(g+1) | element work(g)
        // -- bar -- run sums(g) -- bar; y1/y2 in 2 slots, metadata in 3
        for (int g = 0; g < ng; ++g) {
            const int s = g % S;
            const uint32_t par = (uint32_t)(g / S) & 1u;
            const int64_t f0 = o_lo + (int64_t)g * K;
            const int nf = nf_of(g);
            const int cur = g & 1, prv = cur ^ 1;
            MetaView mv(meta0 + (g % 3) * a.meta_words, K, NS);
            float* y1s = y1b + cur * K * A;
            float* y2s = y2b + cur * K * B;
            if (g > 0)
                small_folds(a, MetaView(meta0 + ((g + 2) % 3) * a.meta_words, K, NS), tb, NR,
                            y1b + prv * K * A, y2b + prv * K * B, Sb + prv * sbuf, rb + prv * K, uB,
                            patch, K, warp, lane);
            if (warp == 7 && g + 1 < ng) {
                small_meta(a, MetaView(meta0 + ((g + 1) % 3) * a.meta_words, K, NS), tb, c0, run0,
                           first_c, ur, nf_of(g + 1), lane);
                advance();
            }
            const bool ok = mbar_wait_bounded(full + s, par, a.timeout_ns);
            element(mv, y1s, y2s, f0, nf, s);
            if (__syncthreads_or(!ok)) {
                // a copy never completed: record it, wait (bounded) for the
                // copies still in flight into this CTA's slots, and leave
                if (tid == 0) {
                    atomicCAS(a.err, 0, (int)DEV_TIMEOUT);
                    for (int gi = g; gi < g + S && gi < ng; ++gi)
                        (void)mbar_wait_bounded(full + gi % S, (uint32_t)(gi / S) & 1u, a.timeout_ns);
                }
                __syncthreads();
                return;
            }
            if (tid == 0 && g + S < ng) issue(g + S);
            if (D >= 2)
                small_runsums(a, mv, y1s, y2s, Sb + cur * sbuf, rb + cur * K, uB, nf, warp, lane, tid);
            __syncthreads();
        }
        if (ng > 0) {
            const int gl = ng - 1, cl = gl & 1;
            small_folds(a, MetaView(meta0 + (gl % 3) * a.meta_words, K, NS), tb, NR, y1b + cl * K * A,
                        y2b + cl * K * B, Sb + cl * sbuf, rb + cl * K, uB, patch, nf_of(gl), warp, lane);
        }
    }

    // ---- face block partial: per-thread accumulators -> K1 x F scratch (the
    // ring, drained) -> sum over the K1 face slots in order
    __syncthreads();
    float* scr = reinterpret_cast<float*>(ring);
    if (rowt) {
#pragma unroll
        for (int i = 0; i < BM / 2; ++i) {
            if (2 * i < B) scr[rk0 * F + rr * B + 2 * i] = hacc[i].x;
            if (2 * i + 1 < B) scr[rk0 * F + rr * B + 2 * i + 1] = hacc[i].y;
        }
    }
    __syncthreads();
    float* out = a.patch + cta * a.patch_floats;
    for (int f = tid; f < F; f += kSmallThreads) {
        float sum = 0.f;
        for (int k = 0; k < K1; ++k) sum += scr[k * F + f];
        out[f] = sum;
    }
    for (int64_t i = tid; i < ploc; i += kSmallThreads) out[F + i] = patch[i];
}

template <typename E, int BM, bool VEC>
cudaError_t launch_small_k(const SmallPlanInfo& sp, const SmallArgs& a, cudaStream_t st,
                           const KernelEvents* kev) {
    auto k = a.onebar ? ttvc_small_kernel<E, BM, VEC, true> : ttvc_small_kernel<E, BM, VEC, false>;
    cudaError_t e = allow_max_dynamic_smem(k);
    if (e != cudaSuccess) return e;
    if (kev) cudaEventRecord(kev->begin, st);
    k<<<sp.G, kSmallThreads, sp.smem, st>>>(a);
    if (kev) cudaEventRecord(kev->end, st);
    return cudaGetLastError();
}

// Rows of B elements: exact B (a multiple of 4) with vector loads, else the
// next multiple of 8 with element loads.
template <typename E, bool VEC>
cudaError_t launch_small_bm(const SmallPlanInfo& sp, const SmallArgs& a, cudaStream_t st,
                            const KernelEvents* kev) {
    if constexpr (VEC) {
        switch (a.B / 4) {
            case 1: return launch_small_k<E, 4, true>(sp, a, st, kev);
            case 2: return launch_small_k<E, 8, true>(sp, a, st, kev);
            case 3: return launch_small_k<E, 12, true>(sp, a, st, kev);
            case 4: return launch_small_k<E, 16, true>(sp, a, st, kev);
            case 5: return launch_small_k<E, 20, true>(sp, a, st, kev);
            case 6: return launch_small_k<E, 24, true>(sp, a, st, kev);
            case 7: return launch_small_k<E, 28, true>(sp, a, st, kev);
            default: return launch_small_k<E, 32, true>(sp, a, st, kev);
        }
    } else {
        switch ((a.B + 7) / 8) {
            case 1: return launch_small_k<E, 8, false>(sp, a, st, kev);
            case 2: return launch_small_k<E, 16, false>(sp, a, st, kev);
            case 3: return launch_small_k<E, 24, false>(sp, a, st, kev);
            default: return launch_small_k<E, 32, false>(sp, a, st, kev);
        }
    }
}

cudaError_t launch_small_f32(const SmallPlanInfo& sp, const SmallArgs& a, bool vec, cudaStream_t st,
                             const KernelEvents* kev);
cudaError_t launch_small_bf16(const SmallPlanInfo& sp, const SmallArgs& a, bool vec, cudaStream_t st,
                              const KernelEvents* kev);
cudaError_t launch_small_f16(const SmallPlanInfo& sp, const SmallArgs& a, bool vec, cudaStream_t st,
                             const KernelEvents* kev);

}  // namespace hoscf
