// All-pairs TTVc for tensors whose face (the two fastest modes, A x B) is
// small (A*B <= 1024), e.g. 24x20x24x20x24x20 or 8^8 (paper Sec. 6.2 shapes).
//
// The same factorisation as the tiled pass (eq. 3.3 split into a face block,
// row sums y1, column sums y2 and their outer-mode contractions), but nothing
// of size N/A or N/B goes back to memory: each CTA streams a contiguous range
// of outer indices, one face per warp, keeps the face accumulator in
// registers, and folds y1, y2 and r_o = <y1, u_A> straight into a
// shared-memory patch of every other block (rows limited to the digits its
// range covers).  Warps of a group of 8 faces hand their per-face results to
// the CTA through shared memory and the fold walks them in warp order, so the
// result is deterministic.  One reduce kernel then sums, for each output
// entry, the patches of the CTAs that cover it, in CTA order.
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

struct SmallArgs {
    const void* T;
    int64_t O;
    int A, B, F, Bp, D;
    int dims[kMaxOrder];      // outer mode sizes
    int64_t st[kMaxOrder];    // outer strides
    int uoff[kMaxOrder];      // factor offsets of outer modes
    int npairs;
    int pm[kMaxBlocks], pn[kMaxBlocks];
    const float* u;
    int uAoff, uBoff;
    int64_t L;                // outer indices per CTA
    int G;
    int Rmax[kMaxOrder];      // patch rows per outer mode
    int64_t x1off[kMaxOrder], x2off[kMaxOrder], poff[kMaxBlocks];
    int64_t patch_floats;     // per CTA: F + X1 + X2 + pairs
    float* patch;             // G x patch_floats
    int* cover;               // G x D x 2: first digit, row count
    const float* scales;      // FP8 only: one per 128 flat elements
};

template <typename E>
__device__ __forceinline__ float ld_elem(const E* p);
template <>
__device__ __forceinline__ float ld_elem<float>(const float* p) { return __ldcs(p); }
template <>
__device__ __forceinline__ float ld_elem<bf16_t>(const bf16_t* p) {
    return __uint_as_float(static_cast<uint32_t>(__ldcs(reinterpret_cast<const unsigned short*>(p))) << 16);
}
template <>
__device__ __forceinline__ float ld_elem<fp8_t>(const fp8_t* p) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw(
        (__nv_fp8_storage_t)__ldcs(reinterpret_cast<const unsigned char*>(p)), __NV_E4M3);
    return __half2float(*reinterpret_cast<const __half*>(&h));
}

constexpr int kSmallWarps = 8;

template <typename E, int JF>
__global__ void __launch_bounds__(256) ttvc_small_kernel(const SmallArgs a) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t c = blockIdx.x;
    const int64_t o_lo = c * a.L;
    const int64_t o_hi = min(a.O, o_lo + a.L);
    const int A = a.A, B = a.B, F = a.F, Bp = a.Bp, D = a.D;
    extern __shared__ __align__(16) float sm[];
    float* uA = sm;                                        // A
    float* uB = uA + ((A + 3) & ~3);                       // B
    float* scratch = uB + ((B + 3) & ~3);                  // 8 x A*Bp (per-warp face)
    const int tile = A * Bp;
    float* gy1 = scratch + (size_t)kSmallWarps * tile;     // 8 x A
    float* gy2 = gy1 + kSmallWarps * A;                    // 8 x B
    float* gr = gy2 + kSmallWarps * B;                     // 8
    float* gpi = gr + kSmallWarps;                         // 8 x D
    float* gpi2 = gpi + kSmallWarps * kMaxOrder;           // 8 x npairs
    int* grow = reinterpret_cast<int*>(gpi2 + kSmallWarps * kMaxBlocks);   // 8 x D
    int* first = grow + kSmallWarps * kMaxOrder;           // D
    float* patch = reinterpret_cast<float*>(first + kMaxOrder);   // X1, X2, pairs (local part)
    const int64_t ploc = a.patch_floats - F;               // local patch floats (no face)

    for (int i = tid; i < A; i += blockDim.x) uA[i] = a.u[a.uAoff + i];
    for (int i = tid; i < B; i += blockDim.x) uB[i] = a.u[a.uBoff + i];
    for (int64_t i = tid; i < ploc; i += blockDim.x) patch[i] = 0.f;
    if (tid < D) {
        const int m = tid;
        const int64_t q0 = o_lo / a.st[m], q1 = (o_hi - 1) / a.st[m];
        first[m] = (int)(q0 % a.dims[m]);
        const int64_t rows = (q1 - q0 + 1 < (int64_t)a.dims[m]) ? q1 - q0 + 1 : (int64_t)a.dims[m];
        a.cover[(c * D + m) * 2 + 0] = first[m];
        a.cover[(c * D + m) * 2 + 1] = (int)rows;
    }
    // smem position of each of my face elements (row pitch Bp avoids bank conflicts)
    int sidx[JF];
#pragma unroll
    for (int j = 0; j < JF; ++j) {
        const int f = lane + 32 * j;
        sidx[j] = f < F ? (f / B) * Bp + (f % B) : -1;
    }
    float hacc[JF];
#pragma unroll
    for (int j = 0; j < JF; ++j) hacc[j] = 0.f;
    __syncthreads();
    float* my = scratch + (size_t)warp * tile;
    const E* Tp = reinterpret_cast<const E*>(a.T);

    for (int64_t og = o_lo; og < o_hi; og += kSmallWarps) {
        const int64_t o = og + warp;
        if (o < o_hi) {
            // outer digits and factor values (lane k < D owns mode k)
            int dig = 0;
            float val = 1.f;
            if (lane < D) {
                dig = (int)((o / a.st[lane]) % a.dims[lane]);
                val = __ldg(a.u + a.uoff[lane] + dig);
            }
            float v[kMaxOrder];
            float wo = 1.f;
#pragma unroll
            for (int k = 0; k < kMaxOrder; ++k) {
                v[k] = __shfl_sync(HOSCF_FULLMASK, val, k);
                if (k < D) wo *= v[k];
            }
            const E* face = Tp + (size_t)o * F;
            float t[JF];
#pragma unroll
            for (int j = 0; j < JF; ++j) {
                t[j] = sidx[j] >= 0 ? ld_elem<E>(face + lane + 32 * j) : 0.f;
                if (std::is_same<E, fp8_t>::value && sidx[j] >= 0)
                    t[j] *= __ldg(a.scales + ((o * F + lane + 32 * j) >> 7));
            }
#pragma unroll
            for (int j = 0; j < JF; ++j) {
                hacc[j] = fmaf(wo, t[j], hacc[j]);
                if (sidx[j] >= 0) my[sidx[j]] = t[j];
            }
            __syncwarp();
            float rpart = 0.f;
            for (int r = lane; r < A; r += 32) {
                float s = 0.f;
                const float* row = my + r * Bp;
                for (int b = 0; b < B; ++b) s = fmaf(row[b], uB[b], s);
                gy1[warp * A + r] = s;
                rpart = fmaf(s, uA[r], rpart);
            }
            for (int b = lane; b < B; b += 32) {
                float s = 0.f;
                for (int r = 0; r < A; ++r) s = fmaf(my[r * Bp + b], uA[r], s);
                gy2[warp * B + b] = s;
            }
            rpart = warp_sum(rpart);
            if (lane == 0) gr[warp] = rpart;
            if (lane < D) {
                float p = 1.f;
#pragma unroll
                for (int k = 0; k < kMaxOrder; ++k)
                    if (k < D && k != lane) p *= v[k];
                gpi[warp * kMaxOrder + lane] = p;
                int rr = dig - first[lane];
                if (rr < 0) rr += a.dims[lane];
                grow[warp * kMaxOrder + lane] = rr;
            }
            for (int p = lane; p < a.npairs; p += 32) {
                const int m = a.pm[p], n = a.pn[p];
                float q = 1.f;
#pragma unroll
                for (int k = 0; k < kMaxOrder; ++k)
                    if (k < D && k != m && k != n) q *= v[k];
                gpi2[warp * kMaxBlocks + p] = q;
            }
        }
        __syncthreads();
        // fold the group's faces into the patch, in warp order
        const int nw = (o_hi - og < kSmallWarps) ? (int)(o_hi - og) : kSmallWarps;
        for (int idx = tid; idx < D * A; idx += blockDim.x) {
            const int m = idx / A, col = idx - (idx / A) * A;
            float* X = patch + a.x1off[m] + col;
            for (int w = 0; w < nw; ++w) {
                const int rr = grow[w * kMaxOrder + m];
                X[rr * A] = fmaf(gpi[w * kMaxOrder + m], gy1[w * A + col], X[rr * A]);
            }
        }
        for (int idx = tid; idx < D * B; idx += blockDim.x) {
            const int m = idx / B, col = idx - (idx / B) * B;
            float* X = patch + a.x2off[m] + col;
            for (int w = 0; w < nw; ++w) {
                const int rr = grow[w * kMaxOrder + m];
                X[rr * B] = fmaf(gpi[w * kMaxOrder + m], gy2[w * B + col], X[rr * B]);
            }
        }
        for (int p = tid; p < a.npairs; p += blockDim.x) {
            const int m = a.pm[p], n = a.pn[p];
            float* X = patch + a.poff[p];
            const int Rn = a.Rmax[n];
            for (int w = 0; w < nw; ++w) {
                const int rm = grow[w * kMaxOrder + m], rn = grow[w * kMaxOrder + n];
                X[rm * Rn + rn] = fmaf(gpi2[w * kMaxBlocks + p], gr[w], X[rm * Rn + rn]);
            }
        }
        __syncthreads();
    }
    // face partial: warp accumulators -> scratch (8 x F) -> sum in warp order
#pragma unroll
    for (int j = 0; j < JF; ++j) {
        const int f = lane + 32 * j;
        if (f < F) scratch[(size_t)warp * F + f] = hacc[j];
    }
    __syncthreads();
    float* out = a.patch + c * a.patch_floats;
    for (int f = tid; f < F; f += blockDim.x) {
        float s = 0.f;
        for (int w = 0; w < kSmallWarps; ++w) s += scratch[(size_t)w * F + f];
        out[f] = s;
    }
    for (int64_t i = tid; i < ploc; i += blockDim.x) out[F + i] = patch[i];
}

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
        if (sgi == 0) {   // face block
            for (int c = lane; c < r.G; c += 32) s += __ldg(patch + (size_t)c * r.patch_floats + loc);
            dst = r.hface + loc;
        } else if (sgi <= 2 * r.D) {
            const bool x1 = sgi <= r.D;
            const int m = x1 ? sgi - 1 : sgi - 1 - r.D;
            const int C = x1 ? r.A : r.B;
            const int i = (int)(loc / C), col = (int)(loc % C);
            const int64_t base = r.F + (x1 ? r.x1off[m] : r.x2off[m]) + col;
            for (int c = lane; c < r.G; c += 32) {
                const int2 cv = __ldg(reinterpret_cast<const int2*>(cover) + (c * r.D + m));
                int rr = i - cv.x;
                if (rr < 0) rr += r.dims[m];
                if (rr < cv.y) s += __ldg(patch + (size_t)c * r.patch_floats + base + (int64_t)rr * C);
            }
            dst = (x1 ? r.hx1[m] : r.hx2[m]) + loc;
        } else {
            const int p = sgi - 1 - 2 * r.D;
            const int m = r.pm[p], n = r.pn[p];
            const int i = (int)(loc / r.dims[n]), j = (int)(loc % r.dims[n]);
            const int Rn = r.Rmax[n];
            for (int c = lane; c < r.G; c += 32) {
                const int2 cm = __ldg(reinterpret_cast<const int2*>(cover) + (c * r.D + m));
                const int2 cn = __ldg(reinterpret_cast<const int2*>(cover) + (c * r.D + n));
                int rm = i - cm.x, rn = j - cn.x;
                if (rm < 0) rm += r.dims[m];
                if (rn < 0) rn += r.dims[n];
                if (rm < cm.y && rn < cn.y)
                    s += __ldg(patch + (size_t)c * r.patch_floats + r.F + r.poff[p] + (int64_t)rm * Rn + rn);
            }
            dst = r.hp[p] + loc;
        }
        s = warp_sum(s);
        if (lane == 0) H[dst] = s;
    }
}

// ---------------------------------------------------------------- host
static int small_jf(int F) {
    const int need = (F + 31) / 32;
    int jf = 1;
    while (jf < need) jf <<= 1;
    return jf;
}

static size_t small_smem(const Shape& s, const SmallPlanInfo& sp) {
    const int A = (int)s.A, B = (int)s.B, Bp = (int)(s.B | 1);
    return sizeof(float) * (((A + 3) & ~3) + ((B + 3) & ~3) + (size_t)kSmallWarps * A * Bp +
                            kSmallWarps * A + kSmallWarps * B + kSmallWarps +
                            kSmallWarps * kMaxOrder + kSmallWarps * kMaxBlocks) +
           sizeof(int) * (kSmallWarps * kMaxOrder + kMaxOrder) +
           sizeof(float) * (size_t)(sp.patch_floats - s.A * s.B) + 64;
}

bool make_small_plan(const Shape& s, int nsm, SmallPlanInfo& sp) {
    sp = SmallPlanInfo();
    if (s.d < 3) return false;
    const int64_t F = s.A * s.B;
    if (F > 1024) return false;
    const int D = s.D;
    // candidate CTA counts: a few waves of the SMs, at least one group of faces each
    for (int64_t target = 8LL * nsm; target >= 1; target /= 2) {
        int64_t G = std::min<int64_t>(target, (s.O + kSmallWarps - 1) / kSmallWarps);
        G = std::max<int64_t>(G, 1);
        int64_t L = (s.O + G - 1) / G;
        L = (L + kSmallWarps - 1) / kSmallWarps * kSmallWarps;
        G = (s.O + L - 1) / L;
        int64_t off = 0;
        for (int m = 0; m < D; ++m) {
            const int64_t st = s.ost[m];
            sp.Rmax[m] = (int)std::min<int64_t>(s.dims[m], (L + st - 1) / st + 1);
        }
        for (int m = 0; m < D; ++m) {
            sp.x1off[m] = off;
            off += (int64_t)sp.Rmax[m] * s.A;
        }
        for (int m = 0; m < D; ++m) {
            sp.x2off[m] = off;
            off += (int64_t)sp.Rmax[m] * s.B;
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
        sp.G = (int)G;
        sp.L = L;
        sp.smem = small_smem(s, sp);
        if (sp.smem <= 200 * 1024) return true;
    }
    return false;
}

template <typename E>
static cudaError_t launch_small_t(const Shape& s, const SmallPlanInfo& sp, const SmallArgs& a,
                                  cudaStream_t st, const KernelEvents* kev) {
    const int jf = small_jf((int)(s.A * s.B));
    void (*k)(const SmallArgs) = nullptr;
    switch (jf) {
        case 1: k = ttvc_small_kernel<E, 1>; break;
        case 2: k = ttvc_small_kernel<E, 2>; break;
        case 4: k = ttvc_small_kernel<E, 4>; break;
        case 8: k = ttvc_small_kernel<E, 8>; break;
        case 16: k = ttvc_small_kernel<E, 16>; break;
        default: k = ttvc_small_kernel<E, 32>; break;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp.smem);
    if (e != cudaSuccess) return e;
    if (kev) cudaEventRecord(kev->begin, st);
    k<<<sp.G, 256, sp.smem, st>>>(a);
    if (kev) cudaEventRecord(kev->end, st);
    return cudaGetLastError();
}

cudaError_t run_small(const Shape& s, const SmallPlanInfo& sp, int dtype, const void* data,
                      const float* scales, const float* u, float* H, char* ws, cudaStream_t st,
                      const KernelEvents* kev) {
    SmallArgs a;
    memset(&a, 0, sizeof(a));
    a.T = data;
    a.O = s.O;
    a.A = (int)s.A;
    a.B = (int)s.B;
    a.F = (int)(s.A * s.B);
    a.Bp = (int)(s.B | 1);
    a.D = s.D;
    for (int k = 0; k < s.D; ++k) {
        a.dims[k] = (int)s.dims[k];
        a.st[k] = s.ost[k];
        a.uoff[k] = (int)s.moff[k];
        a.Rmax[k] = sp.Rmax[k];
        a.x1off[k] = sp.x1off[k];
        a.x2off[k] = sp.x2off[k];
    }
    a.npairs = sp.npairs;
    for (int p = 0; p < sp.npairs; ++p) {
        a.pm[p] = sp.pm[p];
        a.pn[p] = sp.pn[p];
        a.poff[p] = sp.poff[p];
    }
    a.u = u;
    a.uAoff = (int)s.moff[s.d - 2];
    a.uBoff = (int)s.moff[s.d - 1];
    a.L = sp.L;
    a.G = sp.G;
    a.patch_floats = sp.patch_floats;
    a.patch = reinterpret_cast<float*>(ws + sp.off_patch);
    a.cover = reinterpret_cast<int*>(ws + sp.off_cover);
    a.scales = scales;
    cudaError_t e = dtype == HOSCF_F32    ? launch_small_t<float>(s, sp, a, st, kev)
                    : dtype == HOSCF_BF16 ? launch_small_t<bf16_t>(s, sp, a, st, kev)
                                          : launch_small_t<fp8_t>(s, sp, a, st, kev);
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
