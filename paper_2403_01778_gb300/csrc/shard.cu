// Sharded pass (the multi-GPU form of the block construction, Alg. 1 line 4):
// a rank holds the slab of rows [row0, row0 + rows) of mode 1 and runs the
// ordinary pass over it.  Its blocks are scattered into the packed layout of
// the whole tensor: a block A_{1,n} gets the slab's rows at rows row0.. and
// zeros elsewhere (the rows of A_{1,n} are the mode-1 indices, eq. 3.3), a
// block A_{m,n} with m, n >= 2 gets the slab's partial sum (a sum over the
// mode-1 indices).  The elementwise sum over all slabs is then exactly the
// whole tensor's blocks, so one SUM all-reduce does both the reduction of the
// shared blocks and the gather of the A_{1,n} rows.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hoscf {

namespace {

struct ScatterArgs {
    int nblk = 0;
    int64_t full_off[kMaxBlocks];    // block offsets in the whole tensor's layout
    int64_t slab_off[kMaxBlocks];    // block offsets in the slab's layout
    int64_t rows[kMaxBlocks];        // rows of the block in the whole layout
    int64_t cols[kMaxBlocks];
    int64_t row0[kMaxBlocks];        // first row the slab fills (0 for m >= 2)
    int64_t srows[kMaxBlocks];       // rows the slab fills
};

// blockIdx.y = block; a grid-stride loop over the block's entries writes
// every entry once (slab value or zero).
__global__ void shard_scatter_kernel(const float* __restrict__ Hs, float* __restrict__ H,
                                     ScatterArgs a) {
    const int b = blockIdx.y;
    const int64_t n = a.rows[b] * a.cols[b];
    const int64_t lo = a.row0[b] * a.cols[b];
    const int64_t hi = lo + a.srows[b] * a.cols[b];
    const float* src = Hs + a.slab_off[b];
    float* dst = H + a.full_off[b];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = (q >= lo && q < hi) ? src[q - lo] : 0.f;
}

}  // namespace

cudaError_t launch_shard_scatter(const Shape& full, const Shape& slab, int64_t row0,
                                 const float* Hs, float* H, cudaStream_t st) {
    ScatterArgs a;
    memset(&a, 0, sizeof(a));
    int b = 0;
    int64_t biggest = 1;
    for (int m = 0; m < full.d; ++m)
        for (int n = m + 1; n < full.d; ++n, ++b) {
            a.full_off[b] = full.boff[b];
            a.slab_off[b] = slab.boff[b];
            a.rows[b] = full.dims[m];
            a.cols[b] = full.dims[n];
            a.row0[b] = m == 0 ? row0 : 0;
            a.srows[b] = slab.dims[m];
            biggest = std::max(biggest, a.rows[b] * a.cols[b]);
        }
    a.nblk = b;
    const unsigned gx = (unsigned)std::min<int64_t>(1024, (biggest + 255) / 256);
    shard_scatter_kernel<<<dim3(gx, (unsigned)b), 256, 0, st>>>(Hs, H, a);
    return cudaGetLastError();
}

}  // namespace hoscf
