// Eigen step of HOSCF: the largest-magnitude eigenpair of J(x) (Algorithm 1
// line 5), the block normalisation of lines 6-9, the KKT certificate of the
// point the blocks were built at (eq. 2.4 / eq. 4.1), and the final sign fix
// of lines 12-15.
//
// J is never formed densely.  `Jr` holds the rows of the full symmetric block
// matrix with its zero diagonal blocks dropped (row q of mode m is the
// concatenation of A_{m,n} rows for n > m and A_{n,m}^T rows for n < m), so a
// mat-vec is a set of independent contiguous row dot products.
//
// Lanczos runs as one cooperative kernel over G CTAs: rows are split across
// CTAs, every step does one mat-vec and one full (classical Gram-Schmidt)
// reorthogonalisation against the whole basis (FP32 rows kept by each CTA),
// with two exchanges between CTAs (the dot products' partials, the next
// basis vector), both as epoch-tagged words whose reads are the waits.
// Scalars (dot products, the tridiagonal matrix, Ritz values) are reduced in
// a fixed order and recomputed identically by every CTA, so all CTAs take the
// same decisions without another barrier.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"
#include "ritz.cuh"

namespace hoscf {

constexpr int kEigThreads = 256;
constexpr int kEigWarps = kEigThreads / 32;

struct EigArgs {
    const float* Jr;        // 2P floats
    int d;
    int n;
    int64_t moff[kMaxOrder + 1];
    int64_t jroff[kMaxOrder + 1];   // Jr offset of the first row of each mode
    float scale;            // 1 / (d - 1)
    const double* x0;       // start vector (n), or NULL: start = u0 / sqrt(d)
    const float* u0;
    double* V;              // workspace: the two epoch-tagged basis-vector slots
    double* Y;              // n: the start's exchange of y = J x0 (as floats)
    double* part;           // [2][G][pstride] epoch-tagged dot partials, then the
                            // FP64 partials of the certificate and the final sums
    int pstride;
    double* scal;           // outputs (see EigScal)
    double* x_out;          // n or NULL
    float* u_out;           // n or NULL
    double* lambda_out;     // 1 or NULL
    int mmax;
    double eig_tol;
    int check;              // 1: certify the start point first, stop if r <= kkt_tol
    double kkt_tol;
    int64_t cache_floats;   // shared floats holding this CTA's Jr rows (0: read from L2)
    double adapt;           // > 0: inexact eigen steps (see hoscf_opts.eig_adapt)
    int rqi;                // 1: solve (J - rho I) y = x0 in the Krylov space instead
                            //    (rho = Rayleigh quotient of x0; iHOSCF, Sec. 4.4)
                            // 2: solve A y = x0 (adjoint; A = operator below), y returned
                            //    unnormalised in x_out
    float shift_add;        // operator: y = scale * Jr v + shift_add * v
    const float* proj_u;    // non-NULL: operator projected blockwise orthogonal to these unit
                            //    vectors (the tangent space of the factors)
    int hopm;               // 1: after the certificate return the blocks of J x0 normalised
                            //    (the Jacobi-HOPM update g_n / ||g_n||) instead of an eigenpair
    unsigned* bar;
    int* err;
    uint64_t timeout_ns;
};

__device__ __forceinline__ int mode_of(const EigArgs& a, int q) {
    int m = 0;
    while (m < a.d - 1 && q >= a.moff[m + 1]) ++m;
    return m;
}

__device__ __forceinline__ int64_t row_len(const EigArgs& a, int m) {
    return a.n - (a.moff[m + 1] - a.moff[m]);
}

// y[q] = (1/(d-1)) * Jr_row(q) . v  for the rows of this CTA, one warp per
// row, FP32 (lane sums, then a butterfly).  Rows come from the shared-memory
// cache when it holds them; on the first call (fill) they are read from L2 and
// copied into the cache.  Also returns the squared row norms (||J||_F) when
// sq != NULL (FP32 per row, accumulated in FP64 per CTA).
__device__ void matvec_rows(const EigArgs& a, const float* __restrict__ vf, int r0, int r1,
                            float* cache, const int64_t* crow, bool fill, double* sq,
                            float* yrow) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float sqacc = 0.f;
    for (int q = r0 + warp; q < r1; q += kEigWarps) {
        const int m = mode_of(a, q);
        const int64_t Im = a.moff[m + 1] - a.moff[m];
        const int64_t len = a.n - Im;
        const float* grow = a.Jr + a.jroff[m] + (int64_t)(q - a.moff[m]) * len;
        float* srow = cache ? cache + crow[q - r0] : nullptr;
        const bool from_smem = cache && !fill;
        const int lo = (int)a.moff[m];
        float f = 0.f, s2 = 0.f;
        // row columns: J columns [0, lo) then [lo + Im, n)
        const float* vhi = vf + Im;   // column j + Im for Jr index j >= lo
        if (from_smem) {
            for (int j = lane; j < lo; j += 32) f = fmaf(srow[j], vf[j], f);
            for (int j = lo + lane; j < (int)len; j += 32) f = fmaf(srow[j], vhi[j], f);
        } else {
            // four independent loads in flight per lane (rows stream from L2)
            int j = lane;
            for (; j + 96 < (int)len; j += 128) {
                float h[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) h[t] = __ldg(grow + j + 32 * t);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int jj = j + 32 * t;
                    if (srow) srow[jj] = h[t];
                    f = fmaf(h[t], jj < lo ? vf[jj] : vhi[jj], f);
                    s2 = fmaf(h[t], h[t], s2);
                }
            }
            for (; j < (int)len; j += 32) {
                const float h = __ldg(grow + j);
                if (srow) srow[j] = h;
                f = fmaf(h, j < lo ? vf[j] : vhi[j], f);
                s2 = fmaf(h, h, s2);
            }
        }
        f = warp_sum(f);
        if (lane == 0) yrow[q - r0] = f * a.scale + a.shift_add * vf[q];
        if (sq) {
            s2 = warp_sum(s2);
            sqacc += s2;
        }
    }
    if (sq && lane == 0) atomicAdd(sq, (double)sqacc);   // shared-memory scratch, per CTA
}

// Copies this CTA's rows of Jr into the shared-memory cache (rows of one mode
// are contiguous in Jr and in the cache, so each mode segment is one block
// copy).  Where source and destination share their 16-byte phase the middle
// goes by cp.async (16 bytes, no register round trip, every copy of the
// thread in flight at once) and is NOT waited for here: the caller overlaps
// other loads, then calls fill_cache_wait.  Elsewhere the copy is done with
// register loads, 16 in flight per thread.
__device__ void fill_cache_rows(const EigArgs& a, int r0, int r1, float* cache,
                                const int64_t* crow) {
    constexpr int T = kEigThreads;
    for (int q = r0; q < r1;) {
        const int m = mode_of(a, q);
        const int qe = min(r1, (int)a.moff[m + 1]);
        const int64_t len = a.n - (a.moff[m + 1] - a.moff[m]);
        const float* __restrict__ src = a.Jr + a.jroff[m] + (int64_t)(q - a.moff[m]) * len;
        float* dst = cache + crow[q - r0];
        const int64_t cnt = (int64_t)(qe - q) * len;
        // scalar head up to a 16-byte boundary of the source, 16-byte copies
        // for the middle, scalar tail
        const int64_t head = min(cnt, (int64_t)((16 - (reinterpret_cast<uintptr_t>(src) & 15)) & 15) / 4);
        const int64_t nv = (cnt - head) / 4;
        for (int64_t i = threadIdx.x; i < head; i += T) dst[i] = __ldcg(src + i);
        const float4* __restrict__ src4 = reinterpret_cast<const float4*>(src + head);
        float* d4 = dst + head;
        if ((reinterpret_cast<uintptr_t>(d4) & 15) == 0) {
            for (int64_t v = threadIdx.x; v < nv; v += T) cp_async<16>(d4 + 4 * v, src4 + v, true);
        } else {
            constexpr int kFillBatch = 16;
            for (int64_t v0 = threadIdx.x; v0 < nv; v0 += kFillBatch * T) {
                float4 h[kFillBatch];
#pragma unroll
                for (int t = 0; t < kFillBatch; ++t)
                    if (v0 + t * T < nv) h[t] = __ldcg(src4 + v0 + t * T);
#pragma unroll
                for (int t = 0; t < kFillBatch; ++t) {
                    if (v0 + t * T < nv) {
                        float* o = d4 + 4 * (v0 + t * T);
                        o[0] = h[t].x;
                        o[1] = h[t].y;
                        o[2] = h[t].z;
                        o[3] = h[t].w;
                    }
                }
            }
        }
        for (int64_t i = head + 4 * nv + threadIdx.x; i < cnt; i += T) dst[i] = __ldcg(src + i);
        q = qe;
    }
}

// Waits for the fill's copies, then adds the squared cached entries of this
// CTA (nfl floats from the cache start, 16-byte aligned) to *sq (FP32 per
// thread, FP64 per CTA: ||Jr||_F^2).
__device__ void fill_cache_wait(const float* cache, int64_t nfl, double* sq) {
    cp_async_wait_all();
    __syncthreads();
    float s2a = 0.f, s2b = 0.f;
    const float4* c4 = reinterpret_cast<const float4*>(cache);
    const int64_t n4 = (reinterpret_cast<uintptr_t>(cache) & 15) == 0 ? nfl / 4 : 0;
    for (int64_t v = threadIdx.x; v < n4; v += kEigThreads) {
        const float4 h = c4[v];
        s2a = fmaf(h.x, h.x, fmaf(h.y, h.y, s2a));
        s2b = fmaf(h.z, h.z, fmaf(h.w, h.w, s2b));
    }
    for (int64_t i = 4 * n4 + threadIdx.x; i < nfl; i += kEigThreads) s2a = fmaf(cache[i], cache[i], s2a);
    const float s2 = warp_sum(s2a + s2b);
    if ((threadIdx.x & 31) == 0) atomicAdd(sq, (double)s2);   // shared-memory scratch, per CTA
    __syncthreads();
}

// The same mat-vec from the shared-memory cache of this CTA's rows: warp w
// takes a contiguous chunk of rows and walks it in groups of up to four rows
// of one mode (same column pattern), so each vector element read from
// shared memory feeds four independent FMA chains; a reduce-scatter then
// sums the four rows over the lanes with six shuffles.
// With vec4 (every mode offset a multiple of 4, so every row, its column
// runs and the vector are 16-byte aligned) the loads are 16 bytes wide.
// Warps w0 .. w0 + nw - 1 take part (all by default); every row's sum is the
// same whichever warp computes it.
__device__ void matvec_rows_cached(const EigArgs& a, const float* __restrict__ vf, int r0, int r1,
                                   const float* __restrict__ cache, const int64_t* crow,
                                   float* yrow, bool vec4, int w0 = 0, int nw = kEigWarps) {
    const int warp = (int)(threadIdx.x >> 5) - w0, lane = threadIdx.x & 31;
    const int RW = (r1 - r0 + nw - 1) / nw;
    const int qb = r0 + warp * RW, qe = min(r1, qb + RW);
    for (int q = qb; q < qe;) {
        const int m = mode_of(a, q);
        const int cnt = min(4, min(qe, (int)a.moff[m + 1]) - q);
        const int64_t Im = a.moff[m + 1] - a.moff[m];
        const int len = (int)(a.n - Im);
        const int lo = (int)a.moff[m];
        const float* vhi = vf + Im;
        const float* rp[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) rp[i] = cache + crow[q + min(i, cnt - 1) - r0];
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (vec4) {
            auto fma4 = [](float4 r, float4 v, float acc) {
                return fmaf(r.w, v.w, fmaf(r.z, v.z, fmaf(r.y, v.y, fmaf(r.x, v.x, acc))));
            };
            const float4* v4 = reinterpret_cast<const float4*>(vf);
            const float4* vh4 = reinterpret_cast<const float4*>(vhi);
            const int lo4 = lo >> 2, len4 = len >> 2;
            for (int j = lane; j < lo4; j += 32) {
                const float4 v = v4[j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    acc[i] = fma4(reinterpret_cast<const float4*>(rp[i])[j], v, acc[i]);
            }
            for (int j = lo4 + lane; j < len4; j += 32) {
                const float4 v = vh4[j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    acc[i] = fma4(reinterpret_cast<const float4*>(rp[i])[j], v, acc[i]);
            }
        } else {
            for (int j = lane; j < lo; j += 32) {
                const float v = vf[j];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] = fmaf(rp[i][j], v, acc[i]);
            }
            for (int j = lo + lane; j < len; j += 32) {
                const float v = vhi[j];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] = fmaf(rp[i][j], v, acc[i]);
            }
        }
        // reduce-scatter: lanes with bit 4 set keep rows 2,3, bit 3 picks the odd row
        const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
        const float s0 = (up16 ? acc[2] : acc[0]) +
                         __shfl_xor_sync(HOSCF_FULLMASK, up16 ? acc[0] : acc[2], 16);
        const float s1 = (up16 ? acc[3] : acc[1]) +
                         __shfl_xor_sync(HOSCF_FULLMASK, up16 ? acc[1] : acc[3], 16);
        float t = (up8 ? s1 : s0) + __shfl_xor_sync(HOSCF_FULLMASK, up8 ? s0 : s1, 8);
        t += __shfl_xor_sync(HOSCF_FULLMASK, t, 4);
        t += __shfl_xor_sync(HOSCF_FULLMASK, t, 2);
        t += __shfl_xor_sync(HOSCF_FULLMASK, t, 1);
        const int row = (up16 ? 2 : 0) + (up8 ? 1 : 0);
        if ((lane & 7) == 0 && row < cnt)
            yrow[q + row - r0] = t * a.scale + a.shift_add * vf[q + row];
        q += cnt;
    }
}

// out[i] = sum_{c < G} pb[c * ps + i] for i < cnt, every CTA computing the
// same values in the same order.  Lanes take 32 consecutive indices (one
// contiguous segment of a CTA's row per warp load), warps take every
// kEigWarps-th CTA with up to 16 loads per lane issued before any add, and
// the kEigWarps warp sums are added in warp order by warp 0.  scratch holds
// 2 * kEigWarps * 32 values (two buffers, so chunks of 32 indices need one
// CTA barrier each).
template <typename T>
__device__ void reduce_partials(const T* pb, int ps, int G, int cnt, T* out, T* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i0 = 0, h = 0; i0 < cnt; i0 += 32, h ^= 1) {
        const int i = i0 + lane;
        T s = 0;
        if (i < cnt) {
            for (int c0 = warp; c0 < G; c0 += 16 * kEigWarps) {
                T v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int c = c0 + u * kEigWarps;
                    v[u] = c < G ? __ldcg(pb + (size_t)c * ps + i) : T(0);
                }
#pragma unroll
                for (int u = 0; u < 16; ++u) s += v[u];
            }
        }
        T* sc = scratch + h * (kEigWarps * 32);
        sc[warp * 32 + lane] = s;
        __syncthreads();
        if (warp == 0 && i < cnt) {
            T t = sc[lane];
            for (int w = 1; w < kEigWarps; ++w) t += sc[w * 32 + lane];
            out[i] = t;
        }
    }
    __syncthreads();
}

// FP64 form of reduce_partials for cnt <= 32 values, laid out for the fewest
// FP64 instructions (an FP64 instruction occupies the pipe for ~64 cycles
// on this part whatever its active lanes): each value has L lanes (L the
// largest power of two with L * cnt <= 32); lane s of value i in warp w adds
// the partials of CTAs w + 8 (s + L t), t = 0, 1, ...; a butterfly adds the
// L lane sums and warp 0 adds the 8 warp sums in warp order.  Every CTA
// computes the same values in the same order.
__device__ void reduce_partials_d(const double* pb, int ps, int G, int cnt, double* out,
                                  double* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int L = 32;
    while (L > 1 && L * cnt > 32) L >>= 1;
    const int i = lane / L, sub = lane - i * L;
    const int stride = kEigWarps * L;
    const int nt = (G + stride - 1) / stride;   // terms per lane (uniform)
    double s = 0.0;
    if (i < cnt) {
        const int c0 = warp + kEigWarps * sub;
        for (int t0 = 0; t0 < nt; t0 += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + (t0 + u) * stride;
                v[u] = (t0 + u < nt && c < G) ? __ldcg(pb + (size_t)c * ps + i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (t0 + u < nt) s += v[u];
        }
    }
    for (int o = L >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(HOSCF_FULLMASK, s, o);
    if (sub == 0 && i < cnt) scratch[warp * 32 + i] = s;
    __syncthreads();
    if (warp == 0 && lane < cnt) {
        double t = scratch[lane];
        for (int w = 1; w < kEigWarps; ++w) t += scratch[w * 32 + lane];
        out[lane] = t;
    }
    __syncthreads();
}

// CTA-wide sums of NV double-float values (every thread passes its own
// partial; every thread gets the totals in FP64 in out[0..NV), a shared
// array): a butterfly per warp, then thread v adds the warp sums of value v
// in warp order.  The same values give the same sums in every CTA.
template <int NV>
__device__ void df_block_sum(float (&h)[NV], float (&l)[NV], double* out, float* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
            scratch[(2 * v) * kEigWarps + warp] = h[v];
            scratch[(2 * v + 1) * kEigWarps + warp] = l[v];
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < NV) {
        const int v = threadIdx.x;
        float th = 0.f, tl = 0.f;
        for (int w = 0; w < kEigWarps; ++w) {
            df_add(th, tl, scratch[(2 * v) * kEigWarps + w]);
            tl += scratch[(2 * v + 1) * kEigWarps + w];
        }
        out[v] = (double)th + (double)tl;
    }
    __syncthreads();
}

// Epoch-tagged publication for the per-step exchanges of the Lanczos kernel:
// a 32-bit value and a 32-bit epoch in one 8-byte word, written with a single
// relaxed store, so a reader that sees the expected epoch holds the matching
// value (one single-copy-atomic access) - the data read is the wait, and no
// release fence or arrival counter is needed.  Epochs start at 1 in every
// launch (the J-row build zeroes the tagged buffers before it).
__device__ __forceinline__ void tag_put(unsigned long long* p, float v, unsigned ep) {
    const unsigned long long w = ((unsigned long long)ep << 32) | (unsigned long long)__float_as_uint(v);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long tag_ld(const unsigned long long* p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

// Wait (bounded) until each of the N words w[u] = *p[u] (already loaded
// once) carries epoch ep; the pending ones are reloaded together, so a round
// costs one memory latency however many are pending.  Words with null
// pointers count as ready.  On a give-up the error word is set and false
// returned.
template <int N>
__device__ __forceinline__ bool tag_wait_all(const unsigned long long* const (&p)[N],
                                             unsigned long long (&w)[N], unsigned ep, int* err,
                                             uint64_t limit_ns) {
    auto pending = [&]() {
        bool any = false;
#pragma unroll
        for (int u = 0; u < N; ++u) any |= p[u] && (unsigned)(w[u] >> 32) != ep;
        return any;
    };
    if (!pending()) return true;
    const uint64_t t0 = global_timer_ns();
    for (unsigned rounds = 1;; ++rounds) {
#pragma unroll
        for (int u = 0; u < N; ++u)
            if (p[u] && (unsigned)(w[u] >> 32) != ep) w[u] = tag_ld(p[u]);
        if (!pending()) return true;
        if ((rounds & 15u) == 0 && (*(volatile int*)err || global_timer_ns() - t0 > limit_ns)) {
            atomicCAS(err, 0, (int)DEV_TIMEOUT);
            return false;
        }
    }
}

// reduce_partials over epoch-tagged partials: out[i] = sum_c value of pb[c *
// ps + i] once every one carries epoch ep (same order as reduce_partials).
// Returns false (CTA-uniform) when a wait gave up.
__device__ bool reduce_partials_tagged(const unsigned long long* pb, int ps, int G, int cnt,
                                       unsigned ep, float* out, float* scratch, int* err,
                                       uint64_t limit_ns) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool ok = true;
    for (int i0 = 0, h = 0; i0 < cnt; i0 += 32, h ^= 1) {
        const int i = i0 + lane;
        float s = 0.f;
        if (i < cnt) {
            for (int c0 = warp; c0 < G; c0 += 16 * kEigWarps) {
                const unsigned long long* pp[16];
                unsigned long long w[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int c = c0 + u * kEigWarps;
                    pp[u] = c < G ? pb + (size_t)c * ps + i : nullptr;
                    w[u] = pp[u] ? tag_ld(pp[u]) : 0ull;
                }
                if (ok) ok = tag_wait_all<16>(pp, w, ep, err, limit_ns);
#pragma unroll
                for (int u = 0; u < 16; ++u) s += pp[u] ? __uint_as_float((unsigned)w[u]) : 0.f;
            }
        }
        float* sc = scratch + h * (kEigWarps * 32);
        sc[warp * 32 + lane] = s;
        __syncthreads();
        if (warp == 0 && i < cnt) {
            float t = sc[lane];
            for (int w2 = 1; w2 < kEigWarps; ++w2) t += sc[w2 * 32 + lane];
            out[i] = t;
        }
    }
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// Convergence checks of the Ritz pair: every step early on (a good warm start
// converges in a few steps), sparser later.
__device__ __forceinline__ bool check_now(int k) {
    return k >= 2 && (k <= 6 || (k <= 16 && (k & 1) == 0) || (k & 3) == 0);
}

// Grid-wide barrier; a single-CTA launch only needs __syncthreads.
__device__ __forceinline__ bool eig_sync(const EigArgs& a, int G, unsigned& epoch) {
    if (G == 1) {
        __syncthreads();
        return true;
    }
    return grid_barrier(a.bar, G, epoch, a.err, a.timeout_ns);
}

// Lanczos with full reorthogonalisation.  Each CTA owns rows [r0, r1) of J:
// its rows of Jr (shared-memory cache), its rows of the Lanczos basis and of
// the work vector, all in shared memory.  Only the current Lanczos vector and
// the per-CTA dot-product partials cross CTAs, through L2.
//
// Precision: the certificate of the start point (sigma = x^T J x, the KKT
// residual, ||J||_F) and the final normalisation are FP64; the Lanczos
// vectors, mat-vecs and Gram-Schmidt are FP32 with a second Gram-Schmidt pass
// whenever cancellation appears; the tridiagonal matrix and the Ritz value
// are FP64.  J itself is FP32 (the blocks), so FP32 vectors lose nothing that
// the blocks had, and GB300's FP64 rate (1/64 of FP32) would make FP64 vector
// work the bottleneck.
__global__ void __launch_bounds__(kEigThreads, 1) lanczos_kernel(EigArgs a) {
    const int G = gridDim.x;
    const int c = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n;
    const int R = (n + G - 1) / G;
    const int r0 = min(n, c * R), r1 = min(n, r0 + R);
    const int nr = r1 - r0;
    const int M1 = a.mmax + 1;
    unsigned bar_epoch = 0;   // grid barriers passed (see grid_barrier)

    extern __shared__ __align__(16) uint8_t sm_raw[];
    double* hd = reinterpret_cast<double*>(sm_raw);                       // 16 (FP64 scalars)
    double* alpha = hd + 16;                                              // kMaxLanczos
    double* beta = alpha + kMaxLanczos;                                   // kMaxLanczos
    double* sv = beta + kMaxLanczos;                                      // kMaxLanczos
    double* xrow = sv + kMaxLanczos;                                      // R (Ritz vector rows)
    int64_t* crow = reinterpret_cast<int64_t*>(xrow + R);                 // R + 2
    float* hsum = reinterpret_cast<float*>(crow + R + 2);                 // kMaxLanczos + 16
    float* Vl = hsum + kMaxLanczos + 16;                                  // M1 x R
    float* Yl = Vl + (((size_t)M1 * R + 3) & ~size_t(3));                 // R
    float* vf = Yl + ((R + 3) & ~3);                                      // n (padded)
    float* rscratch = vf + ((n + 3) & ~3);                                // 9 * kMaxLanczos
    float* jcache = rscratch + 9 * kMaxLanczos;                           // cache_floats

    // shared-memory row cache for this CTA's rows of Jr, if it fits: row
    // q - r0 starts at crow[q - r0] = sum over the rows r0..q-1 of their
    // lengths (n - I_m for a row of mode m)
    auto rows_before = [&](int q) {
        int64_t off = 0;
        for (int m = 0; m < a.d; ++m) {
            const int lo = max(r0, (int)a.moff[m]), hi = min(q, (int)a.moff[m + 1]);
            if (hi > lo) off += (int64_t)(hi - lo) * row_len(a, m);
        }
        return off;
    };
    for (int t = tid; t <= nr; t += kEigThreads) crow[t] = rows_before(r0 + t);
    if (tid == 0) hd[0] = 0.0;
    __syncthreads();
    float* cache = (rows_before(r1) <= a.cache_floats) ? jcache : nullptr;
    // 16-byte vector exchange and mat-vec loads: every mode offset (hence n,
    // every row length and every cached row start) a multiple of 4 floats
    bool vec4 = ((reinterpret_cast<uintptr_t>(a.V) | reinterpret_cast<uintptr_t>(vf) |
                  reinterpret_cast<uintptr_t>(jcache)) & 15) == 0;
    int64_t min_len = a.n;
    for (int m = 0; m <= a.d; ++m) vec4 = vec4 && (a.moff[m] & 3) == 0;
    for (int m = 0; m < a.d; ++m) min_len = min(min_len, row_len(a, m));
    // 16-byte mat-vec loads pay off on long rows only (>= 8 per lane); on
    // short ones the ragged lane split costs more than they save
    const bool vec4_mv = vec4 && min_len >= 1024;
    if (cache) fill_cache_rows(a, r0, r1, cache, crow);   // completed below, after the start vector
    __shared__ double s_znorm;   // |z| of the last tridiagonal solve (solve modes)
    __shared__ double s_rp[2 * kEigWarps * 32];   // cross-warp sums of reduce_partials
    double* const rp_d = s_rp;
    float* const rp_f = reinterpret_cast<float*>(s_rp);

    const int ps = a.pstride;
    int phase = 0;
    // partial buffers: FP32 for the Lanczos dots, FP64 for the certificate
    float* pf = reinterpret_cast<float*>(a.part);
    double* pdd = a.part + (size_t)2 * G * ps;   // after the two FP32 buffers (sized in doubles)
    auto pbuf = [&]() { return pf + (size_t)(phase & 1) * G * ps; };
    // epoch-tagged per-step exchanges (see tag_put): the dot partials in two
    // alternating [G][ps] buffers over the partial region, the basis vectors
    // in two alternating slots over the V workspace
    unsigned long long* const tpart = reinterpret_cast<unsigned long long*>(a.part);
    auto tpbuf = [&]() { return tpart + (size_t)(phase & 1) * G * ps; };
    unsigned ep_dots = 0;
    // the current vector is exchanged as FP32 through a ping-pong buffer in
    // global memory (the V workspace): slot (j & 1)
    unsigned long long* const tvec = reinterpret_cast<unsigned long long*>(a.V);
    auto tslot = [&](int j) { return tvec + (size_t)(j & 1) * ((n + 3) & ~3); };

    // ---- start vector (unnormalised), FP32: every CTA reads the whole input
    // itself (no exchange), u0 / sqrt(d) when no x0 is given (only the
    // direction matters); my rows also start the basis
    {
        const float rsd = rsqrtf((float)a.d);
        for (int i = tid; i < n; i += kEigThreads) {
            const float v = a.x0 ? (float)__ldg(a.x0 + i) : __ldg(a.u0 + i) * rsd;
            vf[i] = v;
            if (i >= r0 && i < r1) Vl[i - r0] = v;
        }
    }
    if (cache) fill_cache_wait(cache, crow[nr], &hd[0]);

    int k = 0;
    // the last off-diagonal beta_k: FP32 in every thread (FP64 only where a
    // single warp needs it), FP64 for the start's b0
    double beta_last = 0.0;
    float beta_f = 0.f;
    RitzOut ro;
    ro.theta = 0.0;
    ro.resid = 0.0;
    bool done = false;
    bool hopm_out = false;
    bool have_vec = true;    // vf already holds the next vector (x0; v1, formed by the start)
    double r41_b0 = 0.0, r41_rho = 0.0;   // the start's b0 and rho, for eq. 4.1's residual
    // every CTA gets the whole basis vector v_jj (published with epoch jj)
    // into vf; threads t0 .. t0 + nt - 1 take part, eight words in flight
    // each; false if a wait gave up
    auto read_vec = [&](int jj, int t0, int nt) -> bool {
        const unsigned long long* src = tslot(jj);
        const int t = tid - t0;
        bool ok = true;
        for (int q0 = t; q0 < n; q0 += 8 * nt) {
            const unsigned long long* pp[8];
            unsigned long long w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                pp[u] = q0 + u * nt < n ? src + q0 + u * nt : nullptr;
                w[u] = pp[u] ? tag_ld(pp[u]) : 0ull;
            }
            if (ok) ok = tag_wait_all<8>(pp, w, (unsigned)jj, a.err, a.timeout_ns);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (pp[u]) vf[q0 + u * nt] = __uint_as_float((unsigned)w[u]);
        }
        return ok;
    };
    // set when warps 1..7 already read the next vector and formed its
    // mat-vec during the previous step's Ritz check (see below)
    bool pre = false;
    float gs2_frac = 0.25f;   // second Gram-Schmidt pass when b2 < gs2_frac * yy (set at the start)
    for (int j = 0; j < a.mmax && !done; ++j) {
        if (!pre) {
            const bool okv = have_vec ? true : read_vec(j, 0, kEigThreads);
            have_vec = false;
            if (!__syncthreads_and(okv ? 1 : 0)) return;   // an exchange wait gave up
            if (cache)
                matvec_rows_cached(a, vf, r0, r1, cache, crow, Yl, vec4_mv);
            else
                matvec_rows(a, vf, r0, r1, nullptr, crow, false, j == 0 ? &hd[0] : nullptr, Yl);
        }
        pre = false;
        __syncthreads();
        if (j == 0) {
            // FP64 certificate of the start point x0 (unnormalised):
            // rho = x.y / x.x, ||y - rho x||^2, ||Jr||_F^2 -> one reduction
            if (a.proj_u) {
                // project y = A v0 onto the tangent space: y_n -= (u_n . y_n) u_n
                __shared__ double mu_s[kMaxOrder];
                for (int m = warp; m < a.d; m += kEigWarps) {
                    const int lo = max(r0, (int)a.moff[m]), hi = min(r1, (int)a.moff[m + 1]);
                    double t = 0.0;
                    for (int q = lo + lane; q < hi; q += 32) t += (double)a.proj_u[q] * (double)Yl[q - r0];
                    t = warp_sum_d(t);
                    if (lane == 0) pdd[(size_t)24 * G + (size_t)c * kMaxOrder + m] = t;
                }
                if (!eig_sync(a, G, bar_epoch)) return;
                reduce_partials_d(pdd + (size_t)24 * G, kMaxOrder, G, a.d, mu_s, rp_d);
                for (int q = tid; q < nr; q += kEigThreads) {
                    const int m = mode_of(a, q + r0);
                    Yl[q] = (float)((double)Yl[q] - mu_s[m] * (double)a.proj_u[q + r0]);
                }
                __syncthreads();
            }
            // y = J x0: every CTA publishes its rows (and its ||Jr||^2 partial)
            // and, after one grid barrier, forms the certificate and the first
            // Lanczos vector over the whole vector itself - in double-float,
            // identically in every CTA, so no second exchange is needed.
            float* ydst = reinterpret_cast<float*>(a.Y);
            for (int q = tid; q < nr; q += kEigThreads) {
                ydst[r0 + q] = Yl[q];
                if (a.hopm) xrow[q] = (double)Yl[q];
            }
            if (tid == 0) pdd[(size_t)c * 4 + 3] = hd[0];
            if (!eig_sync(a, G, bar_epoch)) return;
            __shared__ double s_df[3];
            __shared__ float s_dfs[6 * kEigWarps];
            {
                // x.y, x.x, y.y (x = x0 in vf)
                float hh[3] = {0.f, 0.f, 0.f}, ll[3] = {0.f, 0.f, 0.f};
                for (int i = tid; i < n; i += kEigThreads) {
                    const float xi = vf[i], yi = __ldcg(ydst + i);
                    df_add_prod(hh[0], ll[0], xi, yi);
                    df_add_prod(hh[1], ll[1], xi, xi);
                    df_add_prod(hh[2], ll[2], yi, yi);
                }
                df_block_sum<3>(hh, ll, s_df, s_dfs);
            }
            // FP64 scalar work once per CTA (FP64 is a narrow pipe on this
            // part), the results broadcast through shared memory; every CTA
            // computes the same values, so every decision below is uniform
            __shared__ double s_sc[4];   // rho, 1/|x0|, b0, r
            __shared__ float s_f[4];     // rho split hi + lo, 1/|x0|, b0 (FP32)
            __shared__ int s_flag;       // 0 go on, 1 non-finite, 2 start point certified
            if (tid == 0) {
                const double xy = s_df[0], xx = s_df[1], yy = s_df[2];
                hd[2] = xx;   // |x0|^2, the scale of the solve modes' result
                const bool bad = !(xx > 0.0) || !isfinite(xx) || !isfinite(yy);
                s_flag = bad ? 1 : 0;
                const double rho = bad ? 0.0 : xy * rcp_nr(xx);
                s_sc[0] = rho;
                s_sc[1] = bad ? 0.0 : rsqrt_nr(xx);
                s_f[0] = (float)rho;
                s_f[1] = (float)(rho - (double)s_f[0]);
                s_f[2] = (float)s_sc[1];
            }
            __syncthreads();
            if (s_flag) {
                if (tid == 0) atomicCAS(a.err, 0, (int)DEV_NONFINITE);
                return;
            }
            const double rho = s_sc[0];
            // w = (y - rho x) / |x0| (the two FMAs leave only the final
            // rounding, so cancellation costs nothing) and ||w||^2, the KKT
            // residual's sum of squares; w replaces x0 in vf, v0 = x0 / |x0|
            // replaces my rows of x0 in the basis
            const float rho_h = s_f[0], rho_l = s_f[1], finv = s_f[2];
            {
                float hh[1] = {0.f}, ll[1] = {0.f};
                for (int i = tid; i < n; i += kEigThreads) {
                    const float xi = vf[i], yi = __ldcg(ydst + i);
                    const float wi = fmaf(-rho_l, xi, fmaf(-rho_h, xi, yi)) * finv;
                    df_add_prod(hh[0], ll[0], wi, wi);
                    vf[i] = wi;
                }
                for (int q = tid; q < nr; q += kEigThreads) Vl[q] *= finv;
                df_block_sum<1>(hh, ll, s_df, s_dfs);
            }
            __shared__ float s_b0f;
            if (tid == 0) {
                const double h5 = fmax(s_df[0], 0.0);
                const double b0 = h5 > 0.0 ? h5 * rsqrt_nr(h5) : 0.0;
                const double dd = (double)a.d;
                const double r = (rho != 0.0) ? dd * rsqrt_nr(dd) * b0 * rcp_nr(fabs(rho)) : INFINITY;
                s_sc[2] = b0;
                s_sc[3] = r;
                // inexact eigen steps: the Ritz tolerance follows the residual
                s_sc[0] = (a.adapt > 0.0 && rho != 0.0) ? fmax(a.eig_tol, fmin(1e-3, a.adapt * r))
                                                        : a.eig_tol;
                s_flag = (!isfinite(rho) || !isfinite(b0)) ? 1
                         : (a.check && rho != 0.0 && r <= a.kkt_tol) ? 2 : 0;
                s_b0f = (float)b0;
                if (c == 0) {
                    a.scal[SC_SIGMA] = rho;
                    a.scal[SC_KKT] = r;
                    a.scal[SC_CONVERGED] = 0.0;
                }
            }
            __syncthreads();
            const double b0 = s_sc[2], tol_adapted = s_sc[0];
            r41_b0 = b0;
            r41_rho = rho;
            if (s_flag == 1) {
                if (tid == 0) atomicCAS(a.err, 0, (int)DEV_NONFINITE);
                return;
            }
            if (s_flag == 2) {
                // the start point is certified: no eigen step; ||J||_F for the
                // residual of eq. 4.1 from the CTAs' partials
                reduce_partials_d(pdd + 3, 4, G, 1, hd + 4, rp_d);
                if (c == 0 && tid == 0) {
                    const double jfro = (hd[4] > 0.0 ? hd[4] * rsqrt_nr(hd[4]) : 0.0) * (double)a.scale;
                    a.scal[SC_R41] = b0 * rcp_nr(jfro + fabs(rho));
                    a.scal[SC_JFRO] = jfro;
                    a.scal[SC_CONVERGED] = 1.0;
                    a.scal[SC_LAMBDA] = rho;
                    a.scal[SC_STEPS] = 0.0;
                    a.scal[SC_RITZRES] = b0;
                }
                return;
            }
            if (a.hopm) {
                // Jacobi-HOPM: y = J x0 has blocks g_n / sqrt(d) (g_n = A x_{k!=n} u^(k))
                ro.theta = rho;
                ro.resid = b0;
                hopm_out = true;
                break;
            }
            a.eig_tol = tol_adapted;
            gs2_frac = fminf(0.25f, __fdividef(6e-6f, (float)tol_adapted));
            if (tid == 0) {
                alpha[0] = rho;
                beta[0] = b0;
                // the FP32 tridiagonal of the Ritz checks, kept one entry per step
                rscratch[0] = (float)rho;
                rscratch[kMaxLanczos] = s_b0f;
                rscratch[2 * kMaxLanczos] = s_b0f * s_b0f;
            }
            beta_last = b0;
            beta_f = s_b0f;
            // v1 = w / b0, whole in vf for the next mat-vec, my rows in the basis
            const float ib = 1.0f / beta_f;
            for (int i = tid; i < n; i += kEigThreads) vf[i] *= ib;
            have_vec = true;
            k = 1;
        } else {
            // partial dots over my rows: h_i = V[i].y (i <= j), yy, and with a
            // projection mu_n = u_n . y_n (the basis already lies in the tangent
            // space, so h_i is unchanged by projecting y)
            const int nproj = a.proj_u ? a.d : 0;
            const int cnt = j + 2 + nproj;
            for (int i = warp; i < cnt; i += kEigWarps) {
                float s = 0.f;
                if (i <= j) {
                    for (int q = lane; q < nr; q += 32) s = fmaf(Vl[(size_t)i * R + q], Yl[q], s);
                } else if (i == j + 1) {
                    for (int q = lane; q < nr; q += 32) s = fmaf(Yl[q], Yl[q], s);
                } else {
                    const int m = i - j - 2;
                    const int lo = max(r0, (int)a.moff[m]), hi = min(r1, (int)a.moff[m + 1]);
                    for (int q = lo + lane; q < hi; q += 32) s = fmaf(a.proj_u[q], Yl[q - r0], s);
                }
                s = warp_sum(s);
                if (lane == 0) tag_put(tpbuf() + (size_t)c * ps + i, s, ep_dots + 1);
            }
            ++ep_dots;
            if (!reduce_partials_tagged(tpbuf(), ps, G, cnt, ep_dots, hsum, rp_f, a.err, a.timeout_ns))
                return;
            ++phase;
            if (nproj) {
                float mu2 = 0.f;
                for (int m = 0; m < a.d; ++m) mu2 = fmaf(hsum[j + 2 + m], hsum[j + 2 + m], mu2);
                for (int q = tid; q < nr; q += kEigThreads) {
                    const int m = mode_of(a, q + r0);
                    Yl[q] = fmaf(-hsum[j + 2 + m], a.proj_u[q + r0], Yl[q]);
                }
                if (tid == 0) hsum[j + 1] -= mu2;
                __syncthreads();
            }
            // full classical Gram-Schmidt against V[0..j]
            float ssq = 0.f;
            for (int i = 0; i <= j; ++i) ssq = fmaf(hsum[i], hsum[i], ssq);
            const float yy = hsum[j + 1];
            float b2 = yy - ssq;
            for (int q = tid; q < nr; q += kEigThreads) {
                float w = Yl[q];
                for (int i = 0; i <= j; ++i) w = fmaf(-hsum[i], Vl[(size_t)i * R + q], w);
                Yl[q] = w;
            }
            const float h1 = hsum[j];
            float h2 = 0.f;
            bool two = false;
            // Cancellation leaves b2 = yy - ssq with an error of ~eps32 yy, so
            // beta (and the basis' orthogonality, ~eps32 sqrt(yy / b2)) carry a
            // relative error of ~eps32 yy / b2.  A second Gram-Schmidt pass with
            // the exact norm is taken when that error could reach 1 % of the
            // Ritz tolerance: yy / b2 > 4 for tight tolerances (<= 2.4e-5), up to
            // ~170 at the loosest (1e-3) of the inexact early eigen steps.
            if (b2 < gs2_frac * yy) {
                // heavy cancellation: second Gram-Schmidt pass with exact norm
                __syncthreads();
                for (int i = warp; i < j + 2; i += kEigWarps) {
                    float s = 0.f;
                    if (i <= j) {
                        for (int q = lane; q < nr; q += 32) s = fmaf(Vl[(size_t)i * R + q], Yl[q], s);
                    } else {
                        for (int q = lane; q < nr; q += 32) s = fmaf(Yl[q], Yl[q], s);
                    }
                    s = warp_sum(s);
                    if (lane == 0) tag_put(tpbuf() + (size_t)c * ps + i, s, ep_dots + 1);
                }
                ++ep_dots;
                if (!reduce_partials_tagged(tpbuf(), ps, G, j + 2, ep_dots, hsum, rp_f, a.err,
                                            a.timeout_ns))
                    return;
                ++phase;
                float ssq2 = 0.f;
                for (int i = 0; i <= j; ++i) ssq2 = fmaf(hsum[i], hsum[i], ssq2);
                b2 = hsum[j + 1] - ssq2;
                h2 = hsum[j];
                two = true;
                for (int q = tid; q < nr; q += kEigThreads) {
                    float w = Yl[q];
                    for (int i = 0; i <= j; ++i) w = fmaf(-hsum[i], Vl[(size_t)i * R + q], w);
                    Yl[q] = w;
                }
            }
            beta_f = sqrtf(fmaxf(b2, 0.f));
            if (tid == 0) {
                const double aj = two ? (double)h1 + (double)h2 : (double)h1;
                alpha[j] = aj;
                beta[j] = (double)beta_f;
                rscratch[j] = (float)aj;
                rscratch[kMaxLanczos + j] = beta_f;
                rscratch[2 * kMaxLanczos + j] = beta_f * beta_f;
            }
            k = j + 1;
        }
        __syncthreads();
        // convergence test on the largest-magnitude Ritz pair
        const bool last = (k == a.mmax) || (k == n) || !(beta_f > 1e-30f);
        const bool chk = check_now(k) || last;
        // The next basis vector goes out (epoch-tagged) before a check, so the
        // check (one warp, identical in every CTA) overlaps the other CTAs'
        // progress; with the rows cached, warps 1..7 meanwhile read the next
        // vector and form its mat-vec (kept unless the check stops).
        const bool pub_early = chk && !last && !a.rqi;
        const bool ovl = pub_early && k >= 2 && cache != nullptr;
        auto publish = [&]() {
            const float inv = 1.0f / beta_f;
            unsigned long long* dst = tslot(j + 1);
            for (int q = tid; q < nr; q += kEigThreads) {
                const float v = Yl[q] * inv;
                Vl[(size_t)(j + 1) * R + q] = v;
                tag_put(dst + r0 + q, v, (unsigned)(j + 1));
            }
        };
        if (pub_early) publish();
        if (chk) {
            __shared__ RitzOut s_ro;
            __shared__ int s_acc;
            bool okx = true;
            if (a.rqi) {
                if (tid == 0) {
                    float* w = rscratch;
                    const double rel = tridiag_shifted_solve(
                        alpha, beta, k, a.rqi == 1 ? alpha[0] : 0.0, sv, w, w + kMaxLanczos,
                        w + 2 * kMaxLanczos, w + 3 * kMaxLanczos, w + 4 * kMaxLanczos,
                        reinterpret_cast<int*>(w + 5 * kMaxLanczos), &s_znorm);
                    s_ro.theta = alpha[0];
                    s_ro.resid = (double)beta_f * rel;   // relative Galerkin residual of the solve
                }
            } else if (k >= 2) {
                // FP32 pair to decide; the FP64 refinement only once accepted
                if (warp == 0) {
                    const double bk = (double)beta_f;
                    RitzOut t = ritz_extreme_core(k, bk, rscratch, a.eig_tol, last);
                    const bool acc = t.resid <= a.eig_tol * fabs(t.theta) || last;
                    if (acc) t = ritz_refine_fp64(alpha, beta, k, bk, sv, rscratch);
                    if (lane == 0) {
                        s_ro = t;
                        s_acc = acc ? 1 : 0;
                    }
                } else if (ovl) {
                    okx = read_vec(j + 1, 32, kEigThreads - 32);
                    asm volatile("bar.sync 2, %0;" ::"r"(kEigThreads - 32) : "memory");
                    matvec_rows_cached(a, vf, r0, r1, cache, crow, Yl, vec4_mv, 1, kEigWarps - 1);
                }
            } else if (tid == 0) {
                sv[0] = 1.0;
                s_ro.theta = alpha[0];
                s_ro.resid = beta_last;
            }
            if (!__syncthreads_and(okx ? 1 : 0)) return;   // an exchange wait gave up
            ro = s_ro;
            if (!a.rqi && k >= 2) {
                if (s_acc) done = true;
            } else {
                const double scale_t = a.rqi ? 1.0 : fabs(ro.theta);
                if (ro.resid <= a.eig_tol * scale_t || last) done = true;
            }
        }
        if (ovl) {
            pre = !done;
        } else if (!done && !pub_early) {
            if (j == 0) {
                // every CTA formed the whole v1 itself (the start block)
                __syncthreads();
                for (int q = tid; q < nr; q += kEigThreads) Vl[(size_t)R + q] = vf[r0 + q];
            } else {
                publish();   // the next read waits for it
            }
        }
    }
    // ---- Ritz vector x = V[0..k-1] s for my rows (FP64 accumulation); block
    // norms and the sign reference <x, v0>
    const int d = a.d;
    if (a.rqi == 2) {
        // linear solve: y = |b| |z| V (z / |z|), returned as is
        const double sc = sqrt(hd[2]) * s_znorm;
        for (int q = tid; q < nr; q += kEigThreads) {
            double x = 0.0;
            for (int i = 0; i < k; ++i) x += sv[i] * (double)Vl[(size_t)i * R + q];
            if (a.x_out) a.x_out[r0 + q] = x * sc;
        }
        if (c == 0 && tid == 0) {
            a.scal[SC_LAMBDA] = ro.theta;
            a.scal[SC_STEPS] = (double)k;
            a.scal[SC_RITZRES] = ro.resid;
            a.scal[SC_CONVERGED] = (ro.resid <= a.eig_tol && isfinite(sc)) ? 1.0 : 0.0;
        }
        return;
    }
    if (!hopm_out) {
        for (int q = tid; q < nr; q += kEigThreads) {
            double x = 0.0;
            for (int i = 0; i < k; ++i) x += sv[i] * (double)Vl[(size_t)i * R + q];
            xrow[q] = x;
        }
    }
    __syncthreads();
    auto xval = [&](int q) -> double { return xrow[q]; };
    // partials: [0..d-1] block norms^2, [d] x . v0
    for (int i = warp; i < d + 1; i += kEigWarps) {
        double s = 0.0;
        if (i < d) {
            const int lo = max(r0, (int)a.moff[i]), hi = min(r1, (int)a.moff[i + 1]);
            for (int q = lo + lane; q < hi; q += 32) s += xval(q - r0) * xval(q - r0);
        } else {
            for (int q = lane; q < nr; q += 32) s += xval(q) * (double)Vl[q];
        }
        s = warp_sum_d(s);
        if (lane == 0) pdd[(size_t)8 * G + (size_t)c * (kMaxOrder + 2) + i] = s;
    }
    // [d + 1]: this CTA's ||Jr||^2 (for ||J||_F in eq. 4.1's residual)
    if (tid == 0) pdd[(size_t)8 * G + (size_t)c * (kMaxOrder + 2) + d + 1] = hd[0];
    if (!eig_sync(a, G, bar_epoch)) return;
    reduce_partials_d(pdd + (size_t)8 * G, kMaxOrder + 2, G, d + 2, hd + 6, rp_d);
    // the scale factors once per CTA (lanes of warp 0), then one multiply per
    // entry: x_out = sgn x / |x|, u_out = sgn x_n / |x_n| per block
    const double* bn = hd + 6;
    __shared__ double s_xs[kMaxOrder + 1];   // [0..d-1] block factors, [d] whole-vector factor
    if (warp == 0) {
        const double sgn = (!hopm_out && bn[d] < 0.0) ? -1.0 : 1.0;   // HOPM keeps g's sign
        double v = 0.0;   // lanes 0..d-1: block norms^2; lane d: their sum
        if (lane < d) v = bn[lane];
        if (lane == d)
            for (int m = 0; m < d; ++m) v += bn[m];
        if (lane <= d) s_xs[lane] = v > 0.0 ? sgn * rsqrt_nr(v) : 0.0;
    }
    __syncthreads();
    for (int q = r0 + tid; q < r1; q += kEigThreads) {
        const double x = xval(q - r0);
        if (a.x_out) a.x_out[q] = x * s_xs[d];
        if (a.u_out) a.u_out[q] = (float)(x * s_xs[mode_of(a, q)]);
    }
    if (c == 0 && tid == 0) {
        const double j2 = hd[6 + d + 1];
        const double jfro = (j2 > 0.0 ? j2 * rsqrt_nr(j2) : 0.0) * (double)a.scale;
        a.scal[SC_R41] = r41_b0 * rcp_nr(jfro + fabs(r41_rho));
        a.scal[SC_JFRO] = jfro;
        a.scal[SC_LAMBDA] = ro.theta;
        a.scal[SC_STEPS] = (double)k;
        a.scal[SC_RITZRES] = ro.resid;
        if (a.lambda_out) *a.lambda_out = ro.theta;
    }
}

// ---------------------------------------------------------------- Jr build
// Jr rows from the packed blocks: block (m,n) goes to rows of mode m as is
// and to rows of mode n transposed (32x32 smem tiles, coalesced both ways).
struct JrBuildArgs {
    int d, nblk;
    int64_t n;
    int64_t dims[kMaxOrder];
    int64_t moff[kMaxOrder + 1];
    int64_t jroff[kMaxOrder + 1];
    int64_t boff[kMaxBlocks + 1];
    int bm[kMaxBlocks], bn[kMaxBlocks];
    int64_t tstart[kMaxBlocks + 1];   // tile prefix
    // the Lanczos kernel's epoch-tagged exchange buffers, cleared for the
    // launch that follows (epochs start at 1)
    unsigned long long* z0;
    int64_t nz0;
    unsigned long long* z1;
    int64_t nz1;
};

__device__ __forceinline__ void clear_tagged(const JrBuildArgs& a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = t; i < a.nz0; i += nt) a.z0[i] = 0ull;
    for (int64_t i = t; i < a.nz1; i += nt) a.z1[i] = 0ull;
}

__global__ void build_jr_kernel(const float* __restrict__ H, float* __restrict__ Jr, JrBuildArgs a,
                                unsigned* bar) {
    __shared__ float tile[32][33];
    if (blockIdx.x == 0 && threadIdx.x == 0 && bar) *bar = 0u;   // for the next Lanczos launch
    clear_tagged(a);
    const int64_t tix = blockIdx.x;
    int b = 0;
    while (tix >= a.tstart[b + 1]) ++b;
    const int m = a.bm[b], nn = a.bn[b];
    const int64_t Im = a.dims[m], In = a.dims[nn];
    const int64_t tj_count = (In + 31) / 32;
    const int64_t loc = tix - a.tstart[b];
    const int64_t ti = loc / tj_count, tj = loc % tj_count;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    const float* blk = H + a.boff[b];
    const int64_t lenm = a.n - Im, lenn = a.n - In;
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = ti * 32 + r, jj = tj * 32 + tx;
        float v = 0.f;
        if (i < Im && jj < In) {
            v = blk[i * In + jj];
            // row (moff[m] + i), column (moff[nn] + jj) of J; drop the m block
            Jr[a.jroff[m] + i * lenm + (a.moff[nn] - Im) + jj] = v;
        }
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t jj = tj * 32 + r, i = ti * 32 + tx;
        if (i < Im && jj < In) {
            // row (moff[nn] + jj), column (moff[m] + i), m < nn so no shift
            Jr[a.jroff[nn] + jj * lenn + a.moff[m] + i] = tile[tx][r];
        }
    }
}

// The same with 64 x 64 tiles and 16-byte loads and stores, for blocks whose
// sides are multiples of 4 (every row of H and of Jr, and every tile column
// offset, 16-byte aligned): each thread moves four float4 in and eight out,
// the transposed copy through a [64][65] shared tile.
__global__ void __launch_bounds__(256) build_jr_vec4_kernel(const float* __restrict__ H,
                                                            float* __restrict__ Jr, JrBuildArgs a,
                                                            unsigned* bar) {
    __shared__ float tile[64][65];
    if (blockIdx.x == 0 && threadIdx.x == 0 && bar) *bar = 0u;   // for the next Lanczos launch
    clear_tagged(a);
    const int64_t tix = blockIdx.x;
    int b = 0;
    while (tix >= a.tstart[b + 1]) ++b;
    const int m = a.bm[b], nn = a.bn[b];
    const int64_t Im = a.dims[m], In = a.dims[nn];
    const int64_t tj_count = (In + 63) / 64;
    const int64_t loc = tix - a.tstart[b];
    const int64_t i0 = (loc / tj_count) * 64, j0 = (loc % tj_count) * 64;
    const int c4 = threadIdx.x & 15, r16 = threadIdx.x >> 4;   // float4 column, row within 16
    const float* blk = H + a.boff[b];
    const int64_t lenm = a.n - Im, lenn = a.n - In;
    float* dst_direct = Jr + a.jroff[m] + (a.moff[nn] - Im);
    float* dst_trans = Jr + a.jroff[nn] + a.moff[m];
    const int64_t jj = j0 + 4 * c4;
    float4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = i0 + r16 + 16 * k;
        v[k] = (i < Im && jj < In) ? __ldcg(reinterpret_cast<const float4*>(blk + i * In + jj))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = r16 + 16 * k;
        const int64_t i = i0 + r;
        if (i < Im && jj < In) *reinterpret_cast<float4*>(dst_direct + i * lenm + jj) = v[k];
        tile[r][4 * c4 + 0] = v[k].x;
        tile[r][4 * c4 + 1] = v[k].y;
        tile[r][4 * c4 + 2] = v[k].z;
        tile[r][4 * c4 + 3] = v[k].w;
    }
    __syncthreads();
    const int64_t ii = i0 + 4 * c4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = r16 + 16 * k;   // row of the transposed tile: column j0 + r of the block
        const int64_t j = j0 + r;
        if (j < In && ii < Im) {
            const float4 w = make_float4(tile[4 * c4 + 0][r], tile[4 * c4 + 1][r],
                                         tile[4 * c4 + 2][r], tile[4 * c4 + 3][r]);
            *reinterpret_cast<float4*>(dst_trans + j * lenn + ii) = w;
        }
    }
}

// ---------------------------------------------------------------- small kernels
// Per-mode norms of u (FP64) into out[0..d-1]; one CTA.
__global__ void mode_norms_kernel(const float* __restrict__ u, int d, ModeInfoArr mi, double* out) {
    __shared__ double red[32];
    for (int m = 0; m < d; ++m) {
        double s = 0.0;
        for (int64_t q = mi.off[m] + threadIdx.x; q < mi.off[m + 1]; q += blockDim.x) {
            const double v = u[q];
            s += v * v;
        }
        s = warp_sum_d(s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            out[m] = t;
        }
        __syncthreads();
    }
}

__global__ void scale_modes_kernel(const float* __restrict__ u, int d, ModeInfoArr mi,
                                   const double* __restrict__ nrm2, float* __restrict__ out) {
    const int64_t n = mi.off[d];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        int m = 0;
        while (m < d - 1 && q >= mi.off[m + 1]) ++m;
        out[q] = (float)((double)u[q] / sqrt(nrm2[m]));
    }
}

// Alg. 1 lines 12-15 (sign of sigma) plus the sign gauge: for n >= 1 the
// largest-|.| entry of u^(n) (lowest index on ties) is made positive, the
// flip carried by u^(0).  One CTA; sigma in/out in FP64.
__global__ void final_fix_kernel(float* __restrict__ u, int d, ModeInfoArr mi, double* sigma) {
    __shared__ float bv[32];
    __shared__ int bi[32];
    __shared__ int flips;
    if (threadIdx.x == 0) flips = (*sigma < 0.0) ? 1 : 0;
    __syncthreads();
    for (int m = 1; m < d; ++m) {
        float best = -1.f;
        int bidx = 0x7fffffff;
        for (int64_t q = mi.off[m] + threadIdx.x; q < mi.off[m + 1]; q += blockDim.x) {
            const float v = fabsf(u[q]);
            if (v > best || (v == best && (int)q < bidx)) {
                best = v;
                bidx = (int)q;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(HOSCF_FULLMASK, best, o);
            const int oi = __shfl_xor_sync(HOSCF_FULLMASK, bidx, o);
            if (ov > best || (ov == best && oi < bidx)) {
                best = ov;
                bidx = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            bv[threadIdx.x >> 5] = best;
            bi[threadIdx.x >> 5] = bidx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float b = bv[0];
            int ix = bi[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (bv[w] > b || (bv[w] == b && bi[w] < ix)) {
                    b = bv[w];
                    ix = bi[w];
                }
            bi[0] = ix;
        }
        __syncthreads();
        const bool neg = u[bi[0]] < 0.f;
        __syncthreads();
        if (neg) {
            for (int64_t q = mi.off[m] + threadIdx.x; q < mi.off[m + 1]; q += blockDim.x) u[q] = -u[q];
            if (threadIdx.x == 0) flips ^= 1;
        }
        __syncthreads();
    }
    if (flips)
        for (int64_t q = mi.off[0] + threadIdx.x; q < mi.off[1]; q += blockDim.x) u[q] = -u[q];
    if (threadIdx.x == 0) *sigma = fabs(*sigma);
}

// ASVD sub-step epilogue (Sec. 1): the eigen step of the two-mode problem
// J2 = [[0, B], [B^T, 0]] returned the normalised blocks (a, b') of an
// eigenvector for lambda = +-s_1.  For lambda < 0 the vector is (a, -b), so b'
// is negated to give a^T B b = +s_1; the pair is then negated together when
// <a, u_m> + <b, u_n> < 0 (u the current point).  The next iterate is the
// current one with modes m and n replaced.  One CTA; the dot product is an
// FP64 sum in a fixed order.
__global__ void asvd_pair_fix_kernel(const float* __restrict__ ucur, int64_t n_tot, int64_t om,
                                     int64_t im, int64_t on, int64_t in,
                                     const float* __restrict__ pair, const double* __restrict__ lambda,
                                     float* __restrict__ unext) {
    __shared__ double red[32];
    __shared__ int s_flip;
    const float sb = (*lambda < 0.0) ? -1.f : 1.f;
    double acc = 0.0;
    for (int64_t q = threadIdx.x; q < im + in; q += blockDim.x) {
        const float v = q < im ? pair[q] : sb * pair[q];
        const float w = q < im ? ucur[om + q] : ucur[on + (q - im)];
        acc += (double)v * (double)w;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(HOSCF_FULLMASK, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        s_flip = t < 0.0 ? 1 : 0;
    }
    __syncthreads();
    const float fa = s_flip ? -1.f : 1.f;
    for (int64_t q = threadIdx.x; q < n_tot; q += blockDim.x) {
        float v = ucur[q];
        if (q >= om && q < om + im) v = fa * pair[q - om];
        if (q >= on && q < on + in) v = fa * sb * pair[im + (q - on)];
        unext[q] = v;
    }
}

// ---------------------------------------------------------------- host
static size_t lanczos_smem_base(int64_t n, int R, int mmax) {
    return sizeof(double) * (size_t)(16 + 3 * kMaxLanczos) + sizeof(double) * (size_t)R +
           sizeof(int64_t) * (size_t)(R + 2) +
           sizeof(float) * (size_t)(kMaxLanczos + 16) + sizeof(float) * (((size_t)(mmax + 1) * R + 3) & ~size_t(3)) +
           sizeof(float) * (size_t)((R + 3) & ~3) + sizeof(float) * (size_t)((n + 3) & ~3) +
           sizeof(float) * 9 * kMaxLanczos + 256;
}

constexpr size_t kEigSmemCap = 220 * 1024;

// Rows of Jr owned by a CTA when the n rows are split over G CTAs: the cache
// size is the largest such row block.
static int64_t max_rows_floats(const Shape& s, int G) {
    const int64_t n = s.n_tot;
    const int64_t R = (n + G - 1) / G;
    int64_t best = 0;
    for (int c = 0; c < G; ++c) {
        const int64_t r0 = std::min(n, c * R), r1 = std::min(n, r0 + R);
        int64_t f = 0;
        for (int m = 0; m < s.d; ++m) {
            const int64_t lo = std::max(r0, s.moff[m]), hi = std::min(r1, s.moff[m + 1]);
            if (hi > lo) f += (hi - lo) * (n - s.dims[m]);
        }
        best = std::max(best, f);
    }
    return best;
}

int lanczos_blocks_per_sm(int64_t n_tot) {
    (void)n_tot;
    return 1;   // the kernel sizes its shared-memory row cache to own the SM
}

bool make_eig_plan(const Shape& s, int nsm, int blocks_per_sm, int mmax, EigPlan& e) {
    (void)blocks_per_sm;
    e = EigPlan();
    if (mmax < 2) mmax = 2;
    if (mmax > kMaxLanczos) mmax = kMaxLanczos;
    e.mmax = mmax;
    // One CTA when the whole of J fits in its shared memory (no grid
    // barriers at all); otherwise the fewest CTAs (from ~32 rows each) whose
    // row blocks of J fit, up to one per SM.
    int64_t G = 1;
    {
        const size_t base1 = lanczos_smem_base(s.n_tot, (int)s.n_tot, mmax);
        if (base1 + sizeof(float) * 2 * (size_t)s.P > kEigSmemCap)
            G = std::min<int64_t>(std::max<int64_t>(2, (s.n_tot + 31) / 32), nsm);
    }
    int64_t cache = 0;
    for (;; ++G) {
        const int64_t R = (s.n_tot + G - 1) / G;
        const size_t base = lanczos_smem_base(s.n_tot, (int)R, mmax);
        if (base > kEigSmemCap) {
            if (G >= nsm) return false;
            continue;
        }
        const int64_t need = max_rows_floats(s, (int)G);
        if (base + sizeof(float) * (size_t)need <= kEigSmemCap) {
            cache = need;
            break;
        }
        if (G >= nsm) {
            cache = 0;   // rows do not fit: stream them from L2 every step
            break;
        }
    }
    e.G = (int)G;
    e.cache_floats = cache;
    e.smem = lanczos_smem_base(s.n_tot, (int)((s.n_tot + G - 1) / G), mmax) +
             sizeof(float) * (size_t)((cache + 3) & ~int64_t(3));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    e.off_jr = take(sizeof(float) * 2 * (size_t)s.P);
    // the basis workspace also holds the two epoch-tagged vector slots
    e.off_V = take(sizeof(double) * std::max((size_t)(mmax + 1) * s.n_tot,
                                             (size_t)2 * ((s.n_tot + 3) & ~(int64_t)3)));
    e.off_Y = take(sizeof(double) * (size_t)s.n_tot);
    e.off_part = take(sizeof(double) * 2 * (size_t)e.G * (mmax + 8 + kMaxOrder) +
                      sizeof(double) * 40 * (size_t)e.G);
    e.bytes = off;
    return true;
}

static void jr_offsets(const Shape& s, int64_t* jroff) {
    jroff[0] = 0;
    for (int m = 0; m < s.d; ++m) jroff[m + 1] = jroff[m] + s.dims[m] * (s.n_tot - s.dims[m]);
}

cudaError_t launch_build_jr(const Shape& s, const float* H, float* Jr, unsigned* bar,
                            unsigned long long* zero0, int64_t nzero0, unsigned long long* zero1,
                            int64_t nzero1, cudaStream_t st) {
    JrBuildArgs a;
    memset(&a, 0, sizeof(a));
    a.z0 = zero0;
    a.nz0 = nzero0;
    a.z1 = zero1;
    a.nz1 = nzero1;
    a.d = s.d;
    a.n = s.n_tot;
    for (int k = 0; k < s.d; ++k) a.dims[k] = s.dims[k];
    for (int k = 0; k <= s.d; ++k) a.moff[k] = s.moff[k];
    jr_offsets(s, a.jroff);
    int b = 0;
    for (int m = 0; m < s.d; ++m)
        for (int n = m + 1; n < s.d; ++n) {
            a.bm[b] = m;
            a.bn[b] = n;
            a.boff[b] = s.boff[b];
            a.tstart[b + 1] = a.tstart[b] + ((s.dims[m] + 31) / 32) * ((s.dims[n] + 31) / 32);
            ++b;
        }
    a.nblk = b;
    // 16-byte path: every dimension a multiple of 4 and both buffers aligned
    bool v4 = ((reinterpret_cast<uintptr_t>(H) | reinterpret_cast<uintptr_t>(Jr)) & 15) == 0;
    for (int k = 0; k < s.d; ++k) v4 = v4 && s.dims[k] % 4 == 0;
    if (v4) {
        int64_t t4 = 0;
        for (int q = 0; q < b; ++q) {
            a.tstart[q] = t4;
            t4 += ((s.dims[a.bm[q]] + 63) / 64) * ((s.dims[a.bn[q]] + 63) / 64);
        }
        a.tstart[b] = t4;
        build_jr_vec4_kernel<<<(unsigned)t4, 256, 0, st>>>(H, Jr, a, bar);
        return cudaGetLastError();
    }
    const int64_t tiles = a.tstart[b];
    build_jr_kernel<<<(unsigned)tiles, 256, 0, st>>>(H, Jr, a, bar);
    return cudaGetLastError();
}

cudaError_t launch_lanczos(const Shape& s, const LanczosLaunch& l, cudaStream_t st) {
    EigArgs a;
    memset(&a, 0, sizeof(a));
    a.Jr = l.Jr;
    a.d = s.d;
    a.n = (int)s.n_tot;
    for (int k = 0; k <= s.d; ++k) a.moff[k] = s.moff[k];
    jr_offsets(s, a.jroff);
    a.scale = 1.0f / (float)(s.d - 1);
    a.hopm = l.hopm;
    a.x0 = l.x0;
    a.u0 = l.u0;
    a.V = l.V;
    a.Y = l.Y;
    a.part = l.part;
    a.pstride = l.mmax + 8 + kMaxOrder;
    a.scal = l.scal;
    a.x_out = l.x_out;
    a.u_out = l.u_out;
    a.lambda_out = l.lambda_out;
    a.mmax = l.mmax;
    a.eig_tol = l.eig_tol;
    a.check = l.check;
    a.kkt_tol = l.kkt_tol;
    a.bar = l.bar;
    a.err = l.err;
    a.timeout_ns = l.timeout_ns;
    a.cache_floats = l.cache_floats;
    a.adapt = l.adapt;
    a.rqi = l.rqi;
    a.shift_add = l.shift_add;
    a.proj_u = l.proj_u;
    if (l.scale_override != 0.f) a.scale = l.scale_override;
    const size_t sm = l.smem;
    cudaError_t e = allow_max_dynamic_smem(lanczos_kernel);
    if (e != cudaSuccess) return e;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)lanczos_kernel, dim3(l.G), dim3(kEigThreads),
                                       args, sm, st);
}

static ModeInfoArr mode_info(const Shape& s) {
    ModeInfoArr mi;
    memset(&mi, 0, sizeof(mi));
    for (int k = 0; k <= s.d; ++k) mi.off[k] = s.moff[k];
    return mi;
}

cudaError_t launch_mode_norms(const Shape& s, const float* u, double* out, cudaStream_t st) {
    mode_norms_kernel<<<1, 256, 0, st>>>(u, s.d, mode_info(s), out);
    return cudaGetLastError();
}

cudaError_t launch_scale_modes(const Shape& s, const float* u, const double* nrm2, float* out,
                               cudaStream_t st) {
    const int64_t n = s.n_tot;
    scale_modes_kernel<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, st>>>(
        u, s.d, mode_info(s), nrm2, out);
    return cudaGetLastError();
}

cudaError_t launch_asvd_pair_fix(const float* ucur, int64_t n_tot, int64_t om, int64_t im,
                                 int64_t on, int64_t in, const float* pair, const double* lambda,
                                 float* unext, cudaStream_t st) {
    asvd_pair_fix_kernel<<<1, 256, 0, st>>>(ucur, n_tot, om, im, on, in, pair, lambda, unext);
    return cudaGetLastError();
}

cudaError_t launch_final_fix(const Shape& s, float* u, double* sigma, cudaStream_t st) {
    final_fix_kernel<<<1, 256, 0, st>>>(u, s.d, mode_info(s), sigma);
    return cudaGetLastError();
}

}  // namespace hoscf
