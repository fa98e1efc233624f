// Host launchers of the HOSCF kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "plan.h"

namespace hoscf {

// A pair of events recorded around a pass's streaming kernel (measurement).
struct KernelEvents {
    cudaEvent_t begin = nullptr, end = nullptr;
};

// narrow.cu: the streaming kernel for BF16 / FP8 with full-row tiles
struct NarrowArgs {
    const void* T;
    const float* scales;   // FP8 only: one per 128 flat elements
    int64_t O, A, B;
    int64_t items, W, P;   // (tile, outer index) items as the tiled kernel, one column tile
    const float* w;        // O outer weights
    const float* uA;       // factor of mode d-2 (length A)
    const float* uB;       // factor of mode d-1 (length B)
    float* hp;             // grid x 2 x FA x 256 face partials
    float* y1p;            // O x A
    float* y2p;            // TA x O x B
    int* err;
    uint64_t timeout_ns;
    int nstage;            // ring slots per warp
    int group;             // items per column-sum exchange
    int FA;                // rows per tile (split over the 8 warps)
};
cudaError_t launch_narrow(const PassPlan& p, int dtype, const NarrowArgs& a, cudaStream_t st,
                          const KernelEvents* kev);

// ttvc.cu
hoscf_status run_ttvc(const Shape& s, const PassPlan& p, int dtype, const void* data,
                      const float* scales, const float* u, float* H, char* ws, int* dev_err,
                      uint64_t timeout_ns, cudaStream_t st, Err& err,
                      const KernelEvents* kev = nullptr);

// batched.cu
// Instantiated graphs of the batched solve, one small cache per handle: a
// batch signature (descriptors, launch shape, buffers, stream) maps to the
// graph captured for it; the least recently used entry is replaced.
struct BatchGraphCache {
    static constexpr int kSlots = 4;
    uint64_t key[kSlots] = {};
    cudaGraphExec_t exec[kSlots] = {};
    uint64_t used[kSlots] = {};
    uint64_t clock = 0;
    int captures = 0;          // graphs captured over the handle's life (measurement)
    void release() {
        for (int i = 0; i < kSlots; ++i) {
            if (exec[i]) cudaGraphExecDestroy(exec[i]);
            exec[i] = nullptr;
            key[i] = 0;
        }
    }
};

hoscf_status run_batched(int count, const hoscf_tensor_desc* T, const float* const* u0,
                         float* const* u_out, const hoscf_opts& o, int threads, char* ws,
                         size_t ws_bytes, int nsm, cudaStream_t st, double* sigma_out,
                         hoscf_info* infos, void* pinned, size_t pinned_bytes,
                         BatchGraphCache& cache, Err& err);

// backward.cu
cudaError_t launch_tangent_project(const Shape& s, const float* u, const float* w, double* b,
                                   double* bnorm2, cudaStream_t st);
cudaError_t launch_grad_write(const Shape& s, const float* u, const double* a, double c,
                              float* coef, float* out, cudaStream_t st,
                              const KernelEvents* kev = nullptr);

// quant.cu
cudaError_t launch_quantize(const float* x, int64_t n, int dtype, void* q, float* scales,
                            cudaStream_t st);

// defl.cu
cudaError_t launch_deflate(const Shape& s, float* H, const float* u, const float* uprev,
                           const double* sigma, int R, double* dots, cudaStream_t st);
cudaError_t launch_sumsq(int dtype, const void* data, const float* scales, int64_t n,
                         double* part, int nparts, double* out, cudaStream_t st);

// small.cu
cudaError_t run_small(const Shape& s, const SmallPlanInfo& sp, int dtype, const void* data,
                      const float* scales, const float* u, float* H, char* ws, int* dev_err,
                      uint64_t timeout_ns, cudaStream_t st, const KernelEvents* kev = nullptr);

// eig.cu
struct LanczosLaunch {
    const float* Jr;
    const double* x0;
    const float* u0;
    double* V;
    double* Y;
    double* part;
    double* scal;
    double* x_out;
    float* u_out;
    double* lambda_out;
    int mmax;
    int G;
    double eig_tol;
    int check;
    double kkt_tol;
    unsigned* bar;
    int* err;
    uint64_t timeout_ns;
    int64_t cache_floats;
    size_t smem;
    double adapt;   // > 0: eig_tol = max(eig_tol, min(1e-3, adapt * r)) after the certificate
    int rqi = 0;    // 1: Rayleigh-quotient solve instead of the eigenpair; 2: plain solve
    float shift_add = 0.f;        // operator: scale * Jr v + shift_add * v
    const float* proj_u = nullptr;   // project the operator onto the factors' tangent space
    float scale_override = 0.f;   // non-zero: mat-vec scale instead of 1/(d-1)
    int hopm = 0;                 // 1: return the Jacobi-HOPM update instead of an eigenpair
};

enum EigScal {
    SC_LAMBDA = 0,     // chosen Ritz value (eigenvalue of J)
    SC_SIGMA = 1,      // Rayleigh quotient of the start vector (sigma at the certified point)
    SC_KKT = 2,        // sqrt(d) ||J x - rho x|| / |rho|  (KKT residual when x is balanced)
    SC_R41 = 3,        // ||J x - rho x|| / (||J||_F + |rho|)  (eq. 4.1 at the start point)
    SC_STEPS = 4,
    SC_CONVERGED = 5,  // 1 when the start point met kkt_tol (no eigen step taken)
    SC_RITZRES = 6,
    SC_JFRO = 7,
    SC_COUNT = 8
};

int lanczos_blocks_per_sm(int64_t n_tot);
// Also zeroes the grid-barrier counter `bar` and the nzero0 / nzero1 words
// of the epoch-tagged exchange buffers of the Lanczos launch that follows on
// the same stream.
cudaError_t launch_build_jr(const Shape& s, const float* H, float* Jr, unsigned* bar,
                            unsigned long long* zero0, int64_t nzero0, unsigned long long* zero1,
                            int64_t nzero1, cudaStream_t st);
cudaError_t launch_lanczos(const Shape& s, const LanczosLaunch& l, cudaStream_t st);
cudaError_t launch_mode_norms(const Shape& s, const float* u, double* out, cudaStream_t st);
cudaError_t launch_scale_modes(const Shape& s, const float* u, const double* nrm2, float* out,
                               cudaStream_t st);
cudaError_t launch_final_fix(const Shape& s, float* u, double* sigma, cudaStream_t st);
// shard.cu: scatter a slab's blocks (rows [row0, row0 + slab.dims[0]) of
// mode 1) into the whole tensor's packed layout, zeros elsewhere.
cudaError_t launch_shard_scatter(const Shape& full, const Shape& slab, int64_t row0,
                                 const float* Hs, float* H, cudaStream_t st);
// ASVD: sign rule for the top singular pair of block (m, n) and the next
// iterate (the current one with modes m and n replaced).
cudaError_t launch_asvd_pair_fix(const float* ucur, int64_t n_tot, int64_t om, int64_t im,
                                 int64_t on, int64_t in, const float* pair, const double* lambda,
                                 float* unext, cudaStream_t st);

}  // namespace hoscf
