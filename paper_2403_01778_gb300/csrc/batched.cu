// Batched form (no paper counterpart): many small independent tensors of
// orders 3 and 4, each solved by Algorithm 1 (HOSCF) inside one CTA of a
// single persistent launch.
//
// CTAs take tensors from an atomic work queue (the host orders the queue
// largest-first).  Per tensor and iteration, the CTA
//   1. builds every coupling block (eq. 3.3) in shared memory: faces
//      T[o][:][:] are staged one outer index o at a time and folded into the
//      face block, the row / column sums and their outer contractions; each
//      block entry is owned by one thread, so the sums are deterministic;
//   2. certifies the point (sigma = x^T J x, KKT residual, eq. 2.4) and, if
//      not converged, takes the largest-magnitude eigen step (Alg. 1 line 5)
//      by single-CTA Lanczos (FP32 vectors, FP64 scalars, full
//      reorthogonalisation), then normalises the blocks (lines 6-9);
// and at the end applies the sign fix of lines 12-15 and the gauge.
// Every wait is a __syncthreads of the CTA; the queue needs no spin waits.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"
#include "ritz.cuh"

namespace hoscf {

constexpr int kBatchMaxOrder = 4;
constexpr int kBatchLanczos = 32;
constexpr int kBatchDfScratch = 2 * 5 * 32;   // cta_df_sum of up to 5 values
constexpr int kBatchMinStage = 4096;          // floats per staging slot, at least

struct BatchItem {
    const float* T;
    const float* u0;
    float* u_out;
    int d;
    int dims[kBatchMaxOrder];
};

struct BatchOut {
    double sigma;
    double resid;
    int iters;
    int passes;
    int status;   // 0 ok, 4 not converged, 5 non-finite
    int pad;
};

struct BatchArgs {
    const BatchItem* items;
    const int* order;      // queue order (largest first)
    BatchOut* out;
    int count;
    int* counter;          // work-queue head, zeroed before launch
    double tol;
    int max_iter;
    double eig_tol;
    double eig_adapt;
    int mmax;
    int n_max, P_max, AB_max;
    int F_max;             // floats per staging slot (>= the largest face)
    int faces;             // at most this many faces per staged group (1 .. 32)
};

struct BShape {
    int d, n, P;
    int dims[kBatchMaxOrder];
    int moff[kBatchMaxOrder + 1];
    int boff[6];   // packed blocks (m<n lexicographic), up to d = 4
};

__device__ __forceinline__ int bidx(int d, int m, int n) { return m * d - m * (m + 1) / 2 + (n - m - 1); }

// Floats of each of the row-sum and column-sum regions: room for the sums of
// a group of faces (at least 1024, so groups of up to 32 faces of up to 32
// rows / columns fit).
HOSCF_HD inline int batch_ycap(int ab_max) { return std::max((ab_max + 3) & ~3, 1024); }

__device__ __forceinline__ int bmode(const BShape& s, int q) {
    int m = 0;
    while (m < s.d - 1 && q >= s.moff[m + 1]) ++m;
    return m;
}

// CTA-wide sums of NV double-float values (df_add: ~46 significant bits from
// FP32 instructions - FP64 issues slowly on this part, so no thread of the
// CTA does FP64 arithmetic here): a butterfly per warp, then thread v < NV
// adds the warp sums of value v in warp order and writes the total (FP64) to
// out[v] (shared); every thread may read out[] on return.  scratch holds
// 2 NV x 32 floats.
template <int NV>
__device__ void cta_df_sum(float (&h)[NV], float (&l)[NV], double* out, float* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const float bh = __shfl_xor_sync(HOSCF_FULLMASK, h[v], o);
            const float bl = __shfl_xor_sync(HOSCF_FULLMASK, l[v], o);
            df_add(h[v], l[v], bh);
            l[v] += bl;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            scratch[(2 * v) * 32 + warp] = h[v];
            scratch[(2 * v + 1) * 32 + warp] = l[v];
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < NV) {
        const int v = threadIdx.x;
        float th = 0.f, tl = 0.f;
        for (int w = 0; w < nw; ++w) {
            df_add(th, tl, scratch[(2 * v) * 32 + w]);
            tl += scratch[(2 * v + 1) * 32 + w];
        }
        out[v] = (double)th + (double)tl;
    }
    __syncthreads();
}

// All blocks of one tensor into H (shared memory), one pass over T.  Faces
// T[o][:][:] arrive in groups of K consecutive outer indices (K faces fill
// one staging slot, at most 32), double-buffered in shared memory by
// cp.async (group g + 1 lands while group g is folded; 16-byte copies when
// the group is 16-byte aligned, else 4-byte), two CTA barriers per group.
// Per group: the face block H_{d-2,d-1} += sum_k w_k T_k (each entry owned
// by one thread - or, for rows of 33-128, by one lane of the warp that also
// forms the row's sums - faces in order); the row sums y1_k[a] =
// T_k[a][:] . u_B by one warp per row (one thread per row for rows of at
// most 32); the column sums y2_k[b] = u_A . T_k[:][b] by one thread per
// (k, b), or - one big face per group - by groups of threads over
// interleaved rows, added in group order.  Every block entry is updated by
// one thread in face order: the blocks are deterministic.
__device__ void batch_blocks(const BShape& s, const float* __restrict__ T, const float* u, float* H,
                             float* faces, int fstride, float* y1, float* y2, int ycap, float* part,
                             float* red, int kmax) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int d = s.d;
    const int A = s.dims[d - 2], B = s.dims[d - 1], F = A * B;
    const int O = (d == 3) ? s.dims[0] : s.dims[0] * s.dims[1];
    const float* uA = u + s.moff[d - 2];
    const float* uB = u + s.moff[d - 1];
    const int K = max(1, min(min(kmax, fstride / F), min(ycap / A, ycap / B)));
    const int ngrp = (O + K - 1) / K;
    const bool v16 = ((K * F) & 3) == 0 && (F & 3) == 0 && (reinterpret_cast<uintptr_t>(T) & 15) == 0;
    // column-sum groups for one face per group: thread t -> column t % B,
    // rows t / B, t / B + ng, ...
    const int ng = max(1, nt / B);
    const int gb = tid % B, gg = tid / B;
    for (int i = tid; i < s.P; i += nt) H[i] = 0.f;
    float* Hf = H + s.boff[bidx(d, d - 2, d - 1)];
    // per group (double-buffered by group parity): the faces' outer weights
    // w_k and, for d = 4, their outer indices (i0, i1)
    __shared__ float s_wk[2][32];
    __shared__ int s_i0[2][32], s_i1[2][32];
    auto stage = [&](int g) {
        const int o0 = g * K, kk = min(K, O - o0);
        const float* src = T + (size_t)o0 * F;
        float* dst = faces + (size_t)(g & 1) * fstride;
        const int cnt = kk * F;
        if (v16) {
            for (int f4 = tid; f4 < (cnt >> 2); f4 += nt) cp_async<16>(dst + 4 * f4, src + 4 * f4, true);
        } else {
            for (int f = tid; f < cnt; f += nt) cp_async<4>(dst + f, src + f, true);
        }
        cp_async_commit();
    };
    // L2 prefetch of the groups PD ahead of the one being staged (the staging
    // ring holds two groups; the prefetch keeps ~128 KB more on the way, so
    // each copy finds its lines in L2 rather than waiting out the DRAM latency)
    const int gbytes = K * F * (int)sizeof(float);
    const int PD = max(1, min(8, (128 << 10) / max(gbytes, 1)));
    auto prefetch = [&](int g) {
        if (g >= ngrp) return;
        const int o0 = g * K, kk = min(K, O - o0);
        const char* src = reinterpret_cast<const char*>(T + (size_t)o0 * F);
        const int bytes = kk * F * (int)sizeof(float);
        for (int off = tid * 128; off < bytes; off += nt * 128) prefetch_l2(src + off);
    };
    for (int g = 1; g <= PD; ++g) prefetch(g);
    stage(0);
    for (int g = 0; g < ngrp; ++g) {
        if (g + 1 < ngrp) {
            prefetch(g + 1 + PD);
            stage(g + 1);
            cp_async_wait_group<1>();   // this thread's copies of group g have landed
        } else {
            cp_async_wait_group<0>();
        }
        const int o0 = g * K, kk = min(K, O - o0);
        const int par = g & 1;
        if (tid < kk) {
            const int o = o0 + tid;
            if (d == 3) {
                s_wk[par][tid] = u[o];
            } else {
                const int i0 = o / s.dims[1], i1 = o - i0 * s.dims[1];
                s_i0[par][tid] = i0;
                s_i1[par][tid] = i1;
                s_wk[par][tid] = u[i0] * u[s.moff[1] + i1];
            }
        }
        __syncthreads();               // everyone's copies of group g are visible (and H zeroed)
        const float* fb = faces + (size_t)(g & 1) * fstride;
        const float* wk = s_wk[par];
        if (B > 32 && B <= 128) {
            // one warp per face row a: its face-block entries (lane l holds
            // columns l + 32 c) stay in registers over the group's faces, and
            // each face's row sum y1[k][a] comes from the same loads; the
            // sums run in the same order as the separate loops below
            float ub[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int b = lane + 32 * c;
                ub[c] = b < B ? uB[b] : 0.f;
            }
            for (int a = warp; a < A; a += nw) {
                float* hr = Hf + (size_t)a * B;
                float h[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int b = lane + 32 * c;
                    h[c] = b < B ? hr[b] : 0.f;
                }
                for (int k = 0; k < kk; ++k) {
                    const float* fr = fb + (size_t)k * F + (size_t)a * B;
                    const float w = wk[k];
                    float t = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int b = lane + 32 * c;
                        if (b < B) {
                            const float x = fr[b];
                            h[c] = fmaf(w, x, h[c]);
                            t = fmaf(x, ub[c], t);
                        }
                    }
                    t = warp_sum(t);
                    if (lane == 0) y1[k * A + a] = t;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int b = lane + 32 * c;
                    if (b < B) hr[b] = h[c];
                }
            }
        } else {
            for (int f = tid; f < F; f += nt) {
                float h = Hf[f];
                for (int k = 0; k < kk; ++k) h = fmaf(wk[k], fb[k * F + f], h);
                Hf[f] = h;
            }
            if (B <= 32) {
                // short rows: one thread per row (rows B floats apart: distinct
                // banks for odd B; for even B each walks its row from column
                // row mod B)
                for (int row = tid; row < kk * A; row += nt) {
                    const float* fr = fb + (size_t)row * B;     // face row (k, a): k * F + a * B
                    int b = (B & 1) ? 0 : row % B;
                    float t = 0.f;
                    for (int c = 0; c < B; ++c) {
                        t = fmaf(fr[b], uB[b], t);
                        b = (b + 1 == B) ? 0 : b + 1;
                    }
                    y1[row] = t;
                }
            } else {
                for (int row = warp; row < kk * A; row += nw) {
                    const float* fr = fb + (size_t)row * B;
                    float t = 0.f;
                    for (int b = lane; b < B; b += 32) t = fmaf(fr[b], uB[b], t);
                    t = warp_sum(t);
                    if (lane == 0) y1[row] = t;
                }
            }
        }
        if (kk == 1) {
            if (gg < ng) {
                float t = 0.f;
                for (int a = gg; a < A; a += ng) t = fmaf(fb[a * B + gb], uA[a], t);
                part[gg * B + gb] = t;
            }
        } else {
            for (int kb = tid; kb < kk * B; kb += nt) {
                const int k = kb / B, b = kb - k * B;
                const float* fk = fb + (size_t)k * F + b;
                float t = 0.f;
                for (int a = 0; a < A; ++a) t = fmaf(fk[a * B], uA[a], t);
                y2[kb] = t;
            }
        }
        __syncthreads();               // y1, y2 (or the column partials) are complete
        if (kk == 1) {
            for (int b = tid; b < B; b += nt) {
                float t = 0.f;
                for (int q = 0; q < ng; ++q) t += part[q * B + b];
                y2[b] = t;   // order 3: read below only by the thread that wrote it
            }
            if (d == 4) __syncthreads();   // order 4: read below by other threads
        }
        if (d == 3) {
            // H01[o][a] = y1_k[a], H02[o][b] = y2_k[b]
            for (int ka = tid; ka < kk * A; ka += nt) H[s.boff[0] + (size_t)o0 * A + ka] = y1[ka];
            for (int kb = tid; kb < kk * B; kb += nt) H[s.boff[1] + (size_t)o0 * B + kb] = y2[kb];
        } else {
            // rows i0 = o / I_1, i1 = o % I_1 of H02, H12 (from y1) and H03, H13
            // (from y2); a thread owns one column of one of the four blocks
            // and walks the group's faces in order
            const int* gi0 = s_i0[par];
            const int* gi1 = s_i1[par];
            for (int e = tid; e < 2 * (A + B); e += nt) {
                const int which = e < 2 * A ? (e < A ? 0 : 1) : (e < 2 * A + B ? 2 : 3);
                const int len = which < 2 ? A : B;
                const int col = e - (which == 0 ? 0 : which == 1 ? A : which == 2 ? 2 * A : 2 * A + B);
                const float* yy = which < 2 ? y1 : y2;
                float* Hb = H + s.boff[bidx(4, (which & 1) ? 1 : 0, which < 2 ? 2 : 3)] + col;
                for (int k = 0; k < kk; ++k) {
                    const int i0 = gi0[k], i1 = gi1[k];
                    // H0n rows i0 take u_1[i1]; H1n rows i1 take u_0[i0]
                    const int rowi = (which & 1) ? i1 : i0;
                    const float wu = (which & 1) ? u[i0] : u[s.moff[1] + i1];
                    Hb[(size_t)rowi * len] = fmaf(wu, yy[k * len + col], Hb[(size_t)rowi * len]);
                }
            }
            // H01[i0][i1] = r_o = <y1_k, uA>, one warp per face
            for (int k = warp; k < kk; k += nw) {
                float r = 0.f;
                for (int a = lane; a < A; a += 32) r = fmaf(y1[k * A + a], uA[a], r);
                r = warp_sum(r);
                if (lane == 0) H[s.boff[0] + o0 + k] = r;
            }
        }
        // the next group's first barrier orders these reads of y1, y2, part and
        // the staging buffer before they are overwritten (the copy into this
        // buffer is issued after that barrier)
    }
    __syncthreads();
    (void)red;
}

// y = J v  (J = blocks / (d-1), symmetric, zero diagonal blocks); thread per row.
__device__ void batch_matvec(const BShape& s, const float* H, const float* v, float* y) {
    const float sc = 1.f / (float)(s.d - 1);
    for (int q = threadIdx.x; q < s.n; q += blockDim.x) {
        const int m = bmode(s, q);
        const int i = q - s.moff[m];
        float acc = 0.f;
        for (int nn = 0; nn < s.d; ++nn) {
            if (nn == m) continue;
            const float* vn = v + s.moff[nn];
            const int In = s.dims[nn];
            if (nn > m) {
                // row i of H_{m,nn}: the threads of a warp read rows In
                // floats apart - distinct banks for odd In; for even In each
                // walks its row from column i mod In (row stride In + 1)
                const float* row = H + s.boff[bidx(s.d, m, nn)] + (size_t)i * In;
                int j = (In & 1) ? 0 : i % In;
                for (int c = 0; c < In; ++c) {
                    acc = fmaf(row[j], vn[j], acc);
                    j = (j + 1 == In) ? 0 : j + 1;
                }
            } else {
                const int Im = s.dims[m];
                const float* blk = H + s.boff[bidx(s.d, nn, m)];
                for (int j = 0; j < In; ++j) acc = fmaf(blk[(size_t)j * Im + i], vn[j], acc);
            }
        }
        y[q] = acc * sc;
    }
}

struct BatchSmem {
    float* u;      // n
    float* H;      // P
    float* face;   // max(2 F', (mmax+1) n)   (two face buffers of F' = F rounded
                   // up to 4 floats; the Lanczos basis later)
    float* part;   // 1024 (column-sum partials of the face fold)
    float* y1;     // AB_max
    float* y2;     // AB_max
    float* w;      // n
    float* red;    // 64
    double* dred;  // 64: [0, 8) sums of cta_df_sum, [8, 12) FP64 scalars of thread 0
    double* alpha; // kMaxLanczos
    double* beta;  // kMaxLanczos
    double* sv;    // kMaxLanczos
    float* hs;     // kMaxLanczos + 8
    float* rscratch;   // 9 kMaxLanczos
    float* dfs;    // kBatchDfScratch: scratch of cta_df_sum
    float* fsc;    // 8: FP32 scalars of thread 0, broadcast
    float* svh;    // kBatchLanczos: the Ritz vector's coefficients, hi part
    float* svl;    // kBatchLanczos: and lo part (double-float)
};

__global__ void __launch_bounds__(1024) batched_hoscf_kernel(BatchArgs a) {
    extern __shared__ __align__(16) uint8_t sm_raw[];
    BatchSmem S;
    {
        double* dp = reinterpret_cast<double*>(sm_raw);
        S.dred = dp;
        S.alpha = S.dred + 64;
        S.beta = S.alpha + kMaxLanczos;
        S.sv = S.beta + kMaxLanczos;
        float* fp = reinterpret_cast<float*>(S.sv + kMaxLanczos);
        S.red = fp;
        S.hs = S.red + 64;
        S.rscratch = S.hs + kMaxLanczos + 8;
        S.dfs = S.rscratch + 9 * kMaxLanczos;
        S.fsc = S.dfs + kBatchDfScratch;
        S.svh = S.fsc + 8;
        S.svl = S.svh + kBatchLanczos;
        S.u = S.svl + kBatchLanczos;
        S.w = S.u + ((a.n_max + 3) & ~3);
        S.y1 = S.w + ((a.n_max + 3) & ~3);
        S.y2 = S.y1 + batch_ycap(a.AB_max);
        S.H = S.y2 + batch_ycap(a.AB_max);
        S.face = S.H + ((a.P_max + 3) & ~3);
        const int basis = max(2 * ((a.F_max + 3) & ~3), (a.mmax + 1) * a.n_max);
        S.part = S.face + ((basis + 3) & ~3);
    }
    __shared__ int s_item;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    while (true) {
        if (tid == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int qi = s_item;
        __syncthreads();
        if (qi >= a.count) break;
        const int t = a.order[qi];
        const BatchItem it = a.items[t];
        BShape sh;
        sh.d = it.d;
        sh.moff[0] = 0;
        for (int k = 0; k < it.d; ++k) {
            sh.dims[k] = it.dims[k];
            sh.moff[k + 1] = sh.moff[k] + it.dims[k];
        }
        sh.n = sh.moff[it.d];
        {
            int b = 0, off = 0;
            for (int m = 0; m < it.d; ++m)
                for (int n2 = m + 1; n2 < it.d; ++n2) {
                    sh.boff[b++] = off;
                    off += it.dims[m] * it.dims[n2];
                }
            sh.P = off;
        }
        const int d = sh.d, n = sh.n;
        // FP64 arithmetic only in thread 0 (or one warp): every scalar is
        // formed there and broadcast through shared memory (S.dred[8..12),
        // S.fsc, s_ctl); the sums are double-float (cta_df_sum)
        __shared__ int s_ctl;
        int status = 0;
        // normalise the initial guess per block
        {
            float hh[kBatchMaxOrder] = {0.f, 0.f, 0.f, 0.f}, ll[kBatchMaxOrder] = {0.f, 0.f, 0.f, 0.f};
            for (int q = tid; q < n; q += nt) {
                const int m = bmode(sh, q);
                const float x = it.u0[q];
#pragma unroll
                for (int v = 0; v < kBatchMaxOrder; ++v)
                    if (v == m) df_add_prod(hh[v], ll[v], x, x);
            }
            cta_df_sum<kBatchMaxOrder>(hh, ll, S.dred, S.dfs);
            if (tid == 0) {
                int st = 0;
                for (int m = 0; m < d; ++m) {
                    const double ss = S.dred[m];
                    const bool ok = ss > 0.0 && isfinite(ss);
                    S.fsc[4 + m] = ok ? (float)rsqrt_nr(ss) : 0.f;
                    if (!ok) st = 5;
                }
                s_ctl = st;
            }
            __syncthreads();
            status = s_ctl;
            for (int q = tid; q < n; q += nt) S.u[q] = it.u0[q] * S.fsc[4 + bmode(sh, q)];
        }
        __syncthreads();
        int iters = 0, passes = 0;
        double sigma = 0.0, resid = INFINITY;   // thread 0's values are the results
        // x = u / sqrt(d) (the scale of x is immaterial to rho and the
        // relative residual; sqrt(d) enters the residual below)
        const float xs = d == 4 ? 0.5f : 0.577350269f;
        while (status == 0) {
            batch_blocks(sh, it.T, S.u, S.H, S.face, (a.F_max + 3) & ~3, S.y1, S.y2, batch_ycap(a.AB_max),
                         S.part, S.red, a.faces);
            ++passes;
            // ---- certificate at x: rho = x^T J x / x^T x, KKT residual (eq. 2.4)
            float* V = S.face;   // (mmax+1) x n basis
            float* Y = S.w;
            for (int q = tid; q < n; q += nt) V[q] = S.u[q] * xs;
            __syncthreads();
            batch_matvec(sh, S.H, V, Y);
            __syncthreads();
            {
                float hh[2] = {0.f, 0.f}, ll[2] = {0.f, 0.f};
                for (int q = tid; q < n; q += nt) {
                    df_add_prod(hh[0], ll[0], V[q], Y[q]);
                    df_add_prod(hh[1], ll[1], V[q], V[q]);
                }
                cta_df_sum<2>(hh, ll, S.dred, S.dfs);
            }
            if (tid == 0) {
                const double xy = S.dred[0], xx = S.dred[1];
                const bool bad = !(xx > 0.0) || !isfinite(xx) || !isfinite(xy);
                const double rho = bad ? 0.0 : xy * rcp_nr(xx);
                S.dred[8] = rho;
                S.fsc[0] = (float)rho;
                S.fsc[1] = (float)(rho - (double)S.fsc[0]);
                S.fsc[2] = bad ? 0.f : (float)rsqrt_nr(xx);
                s_ctl = bad ? 1 : 0;
            }
            __syncthreads();
            // w = (y - rho x) / |x| (rho split hi + lo: the two FMAs leave only
            // the final rounding, so the cancellation costs nothing), which is
            // the first Lanczos residual; v0 = x / |x|
            {
                const float rho_h = S.fsc[0], rho_l = S.fsc[1], finv = S.fsc[2];
                float hh[1] = {0.f}, ll[1] = {0.f};
                for (int q = tid; q < n; q += nt) {
                    const float x = V[q];
                    const float w = fmaf(-rho_l, x, fmaf(-rho_h, x, Y[q])) * finv;
                    df_add_prod(hh[0], ll[0], w, w);
                    Y[q] = w;
                    V[q] = x * finv;
                }
                cta_df_sum<1>(hh, ll, S.dred, S.dfs);
            }
            if (tid == 0) {
                const double rho = S.dred[8];
                const double sw = fmax(S.dred[0], 0.0);
                const double b0 = sw > 0.0 ? sw * rsqrt_nr(sw) : 0.0;
                const double sqrt_d = d == 4 ? 2.0 : 1.7320508075688772;
                sigma = rho;
                resid = (rho != 0.0) ? sqrt_d * b0 * rcp_nr(fabs(rho)) : INFINITY;
                int st = 0;
                if (s_ctl || !isfinite(rho) || !isfinite(b0))
                    st = 5;
                else if (resid <= a.tol)
                    st = 1;
                else if (iters >= a.max_iter)
                    st = 4;
                s_ctl = st;
                // inexact eigen steps: the Ritz tolerance follows the residual
                double etol = a.eig_tol;
                if (a.eig_adapt > 0.0) etol = fmax(etol, fmin(1e-3, a.eig_adapt * resid));
                S.dred[9] = etol;
                S.alpha[0] = rho;
                S.beta[0] = (double)(float)b0;
                S.fsc[3] = (float)b0;
            }
            __syncthreads();
            {
                const int st = s_ctl;
                if (st == 1) break;
                if (st) {
                    status = st;
                    break;
                }
            }
            ++iters;
            // ---- Lanczos for the largest-magnitude eigenpair (warm start at x)
            const double etol = S.dred[9];
            float beta_f = S.fsc[3];
            int k = 1;
            bool done = false;
            const int mmax = min(a.mmax, n);
            for (int j = 1; !done; ++j) {
                // V[j] = w / beta ; y = J V[j]
                const bool last_basis = (j >= mmax) || !(beta_f > 1e-30f);
                if (!last_basis) {
                    const float ib = 1.f / beta_f;
                    for (int q = tid; q < n; q += nt) V[(size_t)j * n + q] = Y[q] * ib;
                    __syncthreads();
                    batch_matvec(sh, S.H, V + (size_t)j * n, Y);
                    __syncthreads();
                    // CGS with a second pass under cancellation (FP32 vectors)
                    for (int pass2 = 0; pass2 < 2; ++pass2) {
                        for (int i = warp; i <= j + 1; i += (nt >> 5)) {
                            float sdot = 0.f;
                            if (i <= j) {
                                for (int q = lane; q < n; q += 32) sdot = fmaf(V[(size_t)i * n + q], Y[q], sdot);
                            } else {
                                for (int q = lane; q < n; q += 32) sdot = fmaf(Y[q], Y[q], sdot);
                            }
                            sdot = warp_sum(sdot);
                            if (lane == 0) S.hs[i] = sdot;
                        }
                        __syncthreads();
                        float ssq = 0.f;
                        for (int i = 0; i <= j; ++i) ssq = fmaf(S.hs[i], S.hs[i], ssq);
                        const float yy = S.hs[j + 1];
                        const float b2 = yy - ssq;
                        for (int q = tid; q < n; q += nt) {
                            float wv = Y[q];
                            for (int i = 0; i <= j; ++i) wv = fmaf(-S.hs[i], V[(size_t)i * n + q], wv);
                            Y[q] = wv;
                        }
                        if (tid == 0) S.alpha[j] = (pass2 == 0 ? 0.0 : S.alpha[j]) + S.hs[j];
                        __syncthreads();
                        beta_f = sqrtf(fmaxf(b2, 0.f));
                        if (pass2 == 0 && b2 >= 0.25f * yy) break;
                    }
                    if (tid == 0) S.beta[j] = beta_f;
                    k = j + 1;
                    __syncthreads();
                }
                const bool last = last_basis || k >= mmax || !(beta_f > 1e-30f);
                if (k >= 2 && (k <= 6 || (k & 1) == 0 || last)) {
                    // FP32 pair to decide; the FP64 refinement only once accepted
                    __shared__ int s_acc;
                    if (warp == 0) {
                        RitzOut rr = ritz_extreme_fp32(S.alpha, S.beta, k, beta_f, S.rscratch, etol, last);
                        const bool acc = rr.resid <= etol * fabs(rr.theta) || last;
                        if (acc) ritz_refine_fp64(S.alpha, S.beta, k, beta_f, S.sv, S.rscratch);
                        if (lane == 0) s_acc = acc ? 1 : 0;
                    }
                    __syncthreads();
                    if (s_acc) done = true;
                } else if (last) {
                    if (tid == 0) S.sv[0] = 1.0;
                    __syncthreads();
                    done = true;
                }
            }
            // Ritz vector x = V s (double-float coefficients and sums), sign-
            // aligned with x, blocks normalised (Alg. 1 lines 6-9)
            if (tid < k) {
                const double sv = S.sv[tid];
                const float h = (float)sv;
                S.svh[tid] = h;
                S.svl[tid] = (float)(sv - (double)h);
            }
            __syncthreads();
            {
                float hh[kBatchMaxOrder + 1] = {0.f, 0.f, 0.f, 0.f, 0.f};
                float ll[kBatchMaxOrder + 1] = {0.f, 0.f, 0.f, 0.f, 0.f};
                for (int q = tid; q < n; q += nt) {
                    float xh = 0.f, xl = 0.f;
                    for (int i = 0; i < k; ++i) {
                        const float v = V[(size_t)i * n + q];
                        df_add_prod(xh, xl, S.svh[i], v);
                        xl = fmaf(S.svl[i], v, xl);
                    }
                    const float x = xh + xl;
                    Y[q] = x;
                    const int m = bmode(sh, q);
#pragma unroll
                    for (int v = 0; v < kBatchMaxOrder; ++v)
                        if (v == m) df_add_prod(hh[v], ll[v], x, x);
                    df_add_prod(hh[kBatchMaxOrder], ll[kBatchMaxOrder], x, V[q]);
                }
                cta_df_sum<kBatchMaxOrder + 1>(hh, ll, S.dred, S.dfs);
            }
            if (tid == 0) {
                for (int m = 0; m < d; ++m) {
                    const double ss = S.dred[m];
                    S.fsc[4 + m] = ss > 0.0 ? (float)rsqrt_nr(ss) : 0.f;
                }
                S.fsc[3] = S.dred[kBatchMaxOrder] < 0.0 ? -1.f : 1.f;
            }
            __syncthreads();
            {
                const float sgn = S.fsc[3];
                for (int q = tid; q < n; q += nt) S.u[q] = sgn * Y[q] * S.fsc[4 + bmode(sh, q)];
            }
            __syncthreads();
        }
        // ---- sign fix (Alg. 1 lines 12-15) and gauge, then write out
        __shared__ int s_flip;
        if (tid == 0) s_flip = (sigma < 0.0) ? 1 : 0;
        __syncthreads();
        for (int m = 1; m < d; ++m) {
            // largest |u| entry of mode m (lowest index on ties) made positive:
            // a lane scan in index order, then a warp arg-max
            if (warp == 0) {
                float best = -1.f;
                int bi = sh.moff[m];
                for (int q = sh.moff[m] + lane; q < sh.moff[m + 1]; q += 32)
                    if (fabsf(S.u[q]) > best) {
                        best = fabsf(S.u[q]);
                        bi = q;
                    }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(HOSCF_FULLMASK, best, o);
                    const int oi = __shfl_xor_sync(HOSCF_FULLMASK, bi, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                if (lane == 0) S.red[0] = (S.u[bi] < 0.f) ? 1.f : 0.f;
            }
            __syncthreads();
            if (S.red[0] != 0.f) {
                for (int q = sh.moff[m] + tid; q < sh.moff[m + 1]; q += nt) S.u[q] = -S.u[q];
                if (tid == 0) s_flip ^= 1;
            }
            __syncthreads();
        }
        for (int q = tid; q < n; q += nt) {
            const bool m0 = q < sh.moff[1];
            it.u_out[q] = (m0 && s_flip) ? -S.u[q] : S.u[q];
        }
        if (tid == 0) {
            BatchOut bo;
            bo.sigma = fabs(sigma);
            bo.resid = resid;
            bo.iters = iters;
            bo.passes = passes;
            bo.status = status;
            bo.pad = 0;
            a.out[t] = bo;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host
static size_t batch_smem(int n_max, int P_max, int F_max, int AB_max, int mmax) {
    const int basis = std::max(2 * ((F_max + 3) & ~3), (mmax + 1) * n_max);
    return sizeof(double) * (64 + 3 * kMaxLanczos) +
           sizeof(float) * (64 + kMaxLanczos + 8 + 9 * kMaxLanczos + kBatchDfScratch + 8 +
                            2 * kBatchLanczos + 2 * ((n_max + 3) & ~3) +
                            2 * batch_ycap(AB_max) + ((P_max + 3) & ~3) + ((basis + 3) & ~3) + 1024) +
           64;
}

struct BatchDev {
    BatchItem* items;
    int* order;
    BatchOut* out;
    int* counter;
};

hoscf_status run_batched(int count, const hoscf_tensor_desc* T, const float* const* u0,
                         float* const* u_out, const hoscf_opts& o, int threads, char* ws,
                         size_t ws_bytes, int nsm, cudaStream_t st, double* sigma_out,
                         hoscf_info* infos, void* pinned, size_t pinned_bytes,
                         BatchGraphCache& cache, Err& err) {
    // validate and describe the batch
    std::vector<BatchItem> items((size_t)count);
    std::vector<int64_t> sizes((size_t)count);
    int n_max = 1, P_max = 1, F_max = 1, AB_max = 1;
    for (int t = 0; t < count; ++t) {
        const hoscf_tensor_desc& D = T[t];
        if (D.order < 3 || D.order > kBatchMaxOrder || D.dtype != HOSCF_F32 || !D.data || !D.dims ||
            !u0[t] || !u_out[t]) {
            err.code = HOSCF_EINVAL;
            snprintf(err.msg, sizeof(err.msg), "batch item %d: need an FP32 tensor of order 3..4", t);
            return err.code;
        }
        BatchItem it;
        memset(&it, 0, sizeof(it));
        it.T = static_cast<const float*>(D.data);
        it.u0 = u0[t];
        it.u_out = u_out[t];
        it.d = D.order;
        int64_t N = 1, n = 0, P = 0;
        for (int k = 0; k < D.order; ++k) {
            if (D.dims[k] < 1 || D.dims[k] > 4096) {
                err.code = HOSCF_EINVAL;
                snprintf(err.msg, sizeof(err.msg), "batch item %d: dims must be 1..4096", t);
                return err.code;
            }
            it.dims[k] = (int)D.dims[k];
            N *= D.dims[k];
            n += D.dims[k];
        }
        for (int m = 0; m < D.order; ++m)
            for (int k = m + 1; k < D.order; ++k) P += D.dims[m] * D.dims[k];
        const int64_t A = D.dims[D.order - 2], B = D.dims[D.order - 1];
        n_max = std::max<int>(n_max, (int)n);
        P_max = std::max<int>(P_max, (int)P);
        F_max = std::max<int>(F_max, (int)(A * B));
        AB_max = std::max<int>(AB_max, (int)std::max(A, B));
        items[(size_t)t] = it;
        sizes[(size_t)t] = N;
    }
    const int mmax = std::min(kBatchLanczos, std::max(2, o.eig_max_steps));
    // each of the two staging slots holds at least kBatchMinStage floats when
    // that fits, so batches of small faces stage many faces per group
    int F_stage = std::max(F_max, kBatchMinStage);
    size_t smem = batch_smem(n_max, P_max, F_stage, AB_max, mmax);
    if (smem > 220 * 1024) {
        F_stage = F_max;
        smem = batch_smem(n_max, P_max, F_stage, AB_max, mmax);
    }
    if (smem > 220 * 1024) {
        err.code = HOSCF_EUNSUPPORTED;
        snprintf(err.msg, sizeof(err.msg), "batch tensors too large for one CTA (%zu bytes)", smem);
        return err.code;
    }
    std::vector<int> order((size_t)count);
    for (int t = 0; t < count; ++t) order[(size_t)t] = t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return sizes[(size_t)x] > sizes[(size_t)y]; });
    // device copies of the descriptors (workspace), via the pinned buffer
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t q = off;
        off = align_up(off + bytes, 256);
        return q;
    };
    const size_t o_items = take(sizeof(BatchItem) * count);
    const size_t o_order = take(sizeof(int) * count);
    const size_t o_out = take(sizeof(BatchOut) * count);
    const size_t o_cnt = take(256);
    if (off > ws_bytes || off > pinned_bytes) {
        err.code = HOSCF_ENOMEM;
        snprintf(err.msg, sizeof(err.msg), "batch descriptors need %zu bytes", off);
        return err.code;
    }
    char* hp = static_cast<char*>(pinned);
    memcpy(hp + o_items, items.data(), sizeof(BatchItem) * count);
    memcpy(hp + o_order, order.data(), sizeof(int) * count);
    memset(hp + o_cnt, 0, 256);
    BatchArgs a;
    memset(&a, 0, sizeof(a));   // padding too: the graph key hashes these bytes
    a.items = reinterpret_cast<BatchItem*>(ws + o_items);
    a.order = reinterpret_cast<int*>(ws + o_order);
    a.out = reinterpret_cast<BatchOut*>(ws + o_out);
    a.count = count;
    a.counter = reinterpret_cast<int*>(ws + o_cnt);
    a.tol = o.tol;
    a.max_iter = o.max_iter;
    a.eig_tol = o.eig_tol > 0 ? o.eig_tol : 1e-10;
    a.eig_adapt = o.eig_adapt;
    a.mmax = mmax;
    a.faces = o.batch_faces > 0 ? std::min(32, o.batch_faces) : 32;
    a.n_max = n_max;
    a.P_max = P_max;
    a.F_max = F_stage;
    a.AB_max = AB_max;
    cudaError_t e = allow_max_dynamic_smem(batched_hoscf_kernel);
    int per_sm = 1;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_hoscf_kernel, threads, smem);
    const int grid = std::max(1, std::min(count, nsm * std::max(1, per_sm)));
    // the whole batch is one CUDA graph: descriptors in, the persistent
    // kernel, results out; a repeated batch replays the instantiated graph
    uint64_t key = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) key = (key ^ c[i]) * 1099511628211ull;
    };
    mix(&a, sizeof(a));
    mix(hp, o_out);
    mix(&grid, sizeof(grid));
    mix(&threads, sizeof(threads));
    mix(&smem, sizeof(smem));
    mix(&st, sizeof(st));
    const void* hpp = hp;
    const void* wsp = ws;
    mix(&hpp, sizeof(hpp));
    mix(&wsp, sizeof(wsp));
    if (key == 0) key = 1;
    int slot = -1;
    for (int i = 0; i < BatchGraphCache::kSlots; ++i)
        if (cache.exec[i] && cache.key[i] == key) slot = i;
    if (e == cudaSuccess && slot < 0) {
        // capture this batch; it replaces the least recently used entry
        slot = 0;
        for (int i = 1; i < BatchGraphCache::kSlots; ++i)
            if (!cache.exec[i] || (cache.exec[slot] && cache.used[i] < cache.used[slot])) slot = i;
        if (cache.exec[slot]) cudaGraphExecDestroy(cache.exec[slot]);
        cache.exec[slot] = nullptr;
        cache.key[slot] = 0;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemcpyAsync(ws, hp, o_out, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(ws + o_cnt, hp + o_cnt, 256, cudaMemcpyHostToDevice, st);
            batched_hoscf_kernel<<<grid, threads, smem, st>>>(a);
            cudaMemcpyAsync(hp + o_out, ws + o_out, sizeof(BatchOut) * count,
                            cudaMemcpyDeviceToHost, st);
            e = cudaStreamEndCapture(st, &graph);
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&cache.exec[slot], graph, 0);
            if (e == cudaSuccess) {
                cache.key[slot] = key;
                ++cache.captures;
            } else {
                cache.exec[slot] = nullptr;
            }
        }
        if (graph) cudaGraphDestroy(graph);
    }
    if (e == cudaSuccess) {
        cache.used[slot] = ++cache.clock;
        e = cudaGraphLaunch(cache.exec[slot], st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err.code = HOSCF_ECUDA;
        snprintf(err.msg, sizeof(err.msg), "batched solve: %s", cudaGetErrorString(e));
        return err.code;
    }
    const BatchOut* res = reinterpret_cast<const BatchOut*>(hp + o_out);
    hoscf_status worst = HOSCF_OK;
    for (int t = 0; t < count; ++t) {
        sigma_out[t] = res[t].sigma;
        if (infos) {
            infos[t].iters = res[t].iters;
            infos[t].passes = res[t].passes;
            infos[t].passes_refine = 0;
            infos[t].rqi_accepts = 0;
            infos[t].resid = res[t].resid;
            infos[t].resid_4_1 = NAN;
            infos[t].sigma_raw = res[t].sigma;
        }
        const hoscf_status sst = res[t].status == 0 ? HOSCF_OK
                                 : res[t].status == 4 ? HOSCF_NOT_CONVERGED : HOSCF_NONFINITE;
        if (sst == HOSCF_NONFINITE || (sst == HOSCF_NOT_CONVERGED && worst == HOSCF_OK)) worst = sst;
    }
    if (worst != HOSCF_OK) {
        err.code = worst;
        snprintf(err.msg, sizeof(err.msg), "some batch items did not converge");
    }
    return worst;
}

}  // namespace hoscf
