// C ABI of the HOSCF library (declared in include/hoscf.h): handle,
// workspace, argument checks and the host-side iteration driver.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

using namespace hoscf;

constexpr int kProfKinds = 4;      // measurement aid: pass kernel, gradient write, adjoint solve, eigen step

struct hoscf_handle {
    int device = 0;
    int nsm = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    double* h_pinned = nullptr;   // small pinned readback buffer
    void* pinned_big = nullptr;   // descriptor / result staging of the batched solve
    size_t pinned_big_bytes = 0;
    cudaStream_t own = nullptr;   // private stream (graph capture)
    // greedy rank-R: the terms found so far (factors, device) whose rank-one
    // tensors every pass subtracts from the blocks (sigmas in the workspace head)
    const float* defl_u = nullptr;
    int defl_count = 0;
    // measurement aid: while enabled, events around (0) the streaming kernel
    // of each hoscf_ttvc_blocks call, (1) the gradient write of each
    // hoscf_backward call, (2) its adjoint solve (the pass at the solution
    // and the Lanczos solve)
    bool prof_on = false;
    size_t prof_n[kProfKinds] = {0, 0, 0, 0};
    std::vector<KernelEvents> prof[kProfKinds];
    BatchGraphCache graphs;       // batched solve: instantiated graphs of recent batches
    char msg[512] = {0};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

hoscf_status fail(hoscf_handle* h, hoscf_status code, const char* fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->msg, sizeof(h->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

hoscf_status cuda_fail(hoscf_handle* h, cudaError_t e, const char* what) {
    return fail(h, HOSCF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return cuda_fail(h, _e, #call);     \
    } while (0)

constexpr size_t kProfMax = 65536;   // timed calls kept by the measurement aid

// Fixed head of the workspace: device error word, grid barrier, scalars.
constexpr size_t kHeadBytes = 8192;
constexpr size_t kOffErr = 0;        // int
constexpr size_t kOffBar = 64;       // grid-barrier arrival counter (unsigned)
constexpr size_t kOffScal = 256;     // 32 doubles
constexpr size_t kOffNorms = 1024;   // up to 16 doubles
constexpr int kMaxGreedy = 32;       // greedy terms: sigmas + <u^(s)_k, u_k> in the head
constexpr size_t kOffDeflSigma = 1280;                               // kMaxGreedy doubles
constexpr size_t kOffDeflDots = kOffDeflSigma + 8 * kMaxGreedy;      // kMaxGreedy x 8 doubles
constexpr size_t kOffSumsq = 4096;                                   // 1 + kSumsqParts doubles
constexpr int kSumsqParts = 256;
static_assert(kOffDeflDots + 8 * kMaxGreedy * 8 <= kOffSumsq, "workspace head overflow");
static_assert(kOffSumsq + 8 * (1 + kSumsqParts) <= kHeadBytes, "workspace head overflow");

struct Layout {
    Shape s;
    PassPlan pp;
    EigPlan ep;
    size_t off_pass = 0, off_eig = 0, off_H = 0, off_H2 = 0, off_ua = 0, off_ub = 0, off_uc = 0,
           off_x = 0, off_x2 = 0, off_extra = 0;
    size_t total = 0;
};

hoscf_status ensure_ws(hoscf_handle* h, size_t bytes) {
    if (bytes <= h->ws_bytes) return HOSCF_OK;
    int pending = 0;   // a failure recorded by earlier asynchronous calls survives the move
    if (h->ws) {
        // nothing may still run on the old workspace when it is freed
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(&pending, h->ws + kOffErr, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "workspace move");
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&h->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, HOSCF_ENOMEM, "workspace allocation of %zu bytes failed: %s", want,
                    cudaGetErrorString(e));
    }
    h->ws_bytes = want;
    // the head (status word, barrier counter, scalars) starts at zero
    e = cudaMemset(h->ws, 0, kHeadBytes);
    if (e == cudaSuccess && pending)
        e = cudaMemcpy(h->ws + kOffErr, &pending, sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "workspace set-up");
    return HOSCF_OK;
}

bool dims_valid(int order, const int64_t* dims) {
    if (order < 2 || order > HOSCF_MAX_ORDER || !dims) return false;
    for (int k = 0; k < order; ++k)
        if (dims[k] < 1) return false;
    return true;
}

hoscf_status check_desc(hoscf_handle* h, const hoscf_tensor_desc* T) {
    if (!T) return fail(h, HOSCF_EINVAL, "tensor descriptor is NULL");
    if (!dims_valid(T->order, T->dims)) return fail(h, HOSCF_EINVAL, "order must be 2..%d and dims >= 1", HOSCF_MAX_ORDER);
    if (!T->data) return fail(h, HOSCF_EINVAL, "tensor data is NULL");
    if (T->dtype != HOSCF_F32 && T->dtype != HOSCF_BF16 && T->dtype != HOSCF_F8E4M3 &&
        T->dtype != HOSCF_F16)
        return fail(h, HOSCF_EINVAL, "unknown dtype %d", (int)T->dtype);
    if (T->dtype == HOSCF_F8E4M3 && !T->scales) return fail(h, HOSCF_EINVAL, "FP8 tensor needs scales");
    if ((reinterpret_cast<uintptr_t>(T->data) & 15) != 0)
        return fail(h, HOSCF_EINVAL, "tensor data must be 16-byte aligned");
    return HOSCF_OK;
}

// Workspace for one shape.  `dtype2` (>= 0) is a second tensor dtype whose
// pass must fit in the same pass region (precision form: low-precision tensor
// plus its FP32 refinement copy).
hoscf_status plan_all(hoscf_handle* h, int order, const int64_t* dims, int dtype, bool pass,
                      bool eig, int mmax, Layout& L, int dtype2 = -1, size_t extra = 0) {
    if (!make_shape(order, dims, L.s)) return fail(h, HOSCF_EINVAL, "invalid shape");
    size_t off = kHeadBytes;
    if (pass) {
        make_pass_plan(L.s, dtype, h->nsm, true, L.pp);
        size_t need = L.pp.bytes;
        if (dtype2 >= 0) {
            PassPlan p2;
            make_pass_plan(L.s, dtype2, h->nsm, true, p2);
            need = std::max(need, p2.bytes);
        }
        L.off_pass = off;
        off = align_up(off + need, 256);
    }
    if (eig) {
        if (!make_eig_plan(L.s, h->nsm, lanczos_blocks_per_sm(L.s.n_tot), mmax, L.ep))
            return fail(h, HOSCF_EINVAL, "eigen plan failed");
        L.off_eig = off;
        off = align_up(off + L.ep.bytes, 256);
    }
    L.off_H = off;
    off = align_up(off + sizeof(float) * (size_t)L.s.P, 256);
    L.off_H2 = off;
    off = align_up(off + sizeof(float) * (size_t)L.s.P, 256);
    L.off_ua = off;
    off = align_up(off + sizeof(float) * (size_t)L.s.n_tot, 256);
    L.off_ub = off;
    off = align_up(off + sizeof(float) * (size_t)L.s.n_tot, 256);
    L.off_uc = off;
    off = align_up(off + sizeof(float) * (size_t)L.s.n_tot, 256);
    L.off_x = off;
    off = align_up(off + sizeof(double) * (size_t)L.s.n_tot, 256);
    L.off_x2 = off;
    off = align_up(off + sizeof(double) * (size_t)L.s.n_tot, 256);
    L.off_extra = off;
    off = align_up(off + extra, 256);
    L.total = off;
    return ensure_ws(h, L.total);
}

int* dev_err(hoscf_handle* h) { return reinterpret_cast<int*>(h->ws + kOffErr); }

hoscf_status reset_dev_state(hoscf_handle* h, cudaStream_t st) {
    CK(cudaMemsetAsync(h->ws, 0, 256, st));
    return HOSCF_OK;
}

// The asynchronous entry points clear only the grid-barrier state: a failure
// an earlier asynchronous call recorded in the device status word stays there
// until hoscf_device_status reads it.
hoscf_status reset_barrier_state(hoscf_handle* h, cudaStream_t st) {
    CK(cudaMemsetAsync(h->ws + kOffBar, 0, 256 - kOffBar, st));
    return HOSCF_OK;
}

uint64_t timeout_of(const hoscf_opts* o) {
    return (o && o->timeout_ns > 0) ? (uint64_t)o->timeout_ns : 2000000000ull;
}

hoscf_status dev_status(hoscf_handle* h, int code) {
    if (code == DEV_OK) return HOSCF_OK;
    if (code == DEV_TIMEOUT) return fail(h, HOSCF_TIMEOUT, "a device-side wait exceeded its time limit");
    if (code == DEV_NONFINITE) return fail(h, HOSCF_NONFINITE, "non-finite value met on the device");
    return fail(h, HOSCF_ECUDA, "device error code %d", code);
}

// Measurement aid: the next event pair of list `which` while recording is
// on (nullptr otherwise, or once kProfMax pairs are taken).
hoscf_status prof_slot(hoscf_handle* h, int which, const KernelEvents** out) {
    *out = nullptr;
    if (!h->prof_on || h->prof_n[which] >= kProfMax) return HOSCF_OK;
    std::vector<KernelEvents>& list = h->prof[which];
    if (h->prof_n[which] == list.size()) {
        KernelEvents e;
        CK(cudaEventCreate(&e.begin));
        CK(cudaEventCreate(&e.end));
        list.push_back(e);
    }
    *out = &list[h->prof_n[which]++];
    return HOSCF_OK;
}

// Eigen step launcher (shared by hoscf_eig_step and the solve driver).
hoscf_status eig_launch(hoscf_handle* h, const Layout& L, const float* H, const double* x0,
                        const float* u0, double* x_out, float* u_out, double* lambda_out,
                        const hoscf_opts* o, int check, double kkt_tol, cudaStream_t st,
                        double adapt = 0.0, int rqi = 0, float shift_add = 0.f,
                        const float* proj_u = nullptr, float scale_override = 0.f,
                        double tol_override = 0.0, int hopm = 0) {
    char* eb = h->ws + L.off_eig;
    float* Jr = reinterpret_cast<float*>(eb + L.ep.off_jr);
    const KernelEvents* kev = nullptr;
    hoscf_status ps = prof_slot(h, 3, &kev);
    if (ps) return ps;
    if (kev) cudaEventRecord(kev->begin, st);
    // the Lanczos kernel's epoch-tagged buffers: [2][G][pstride] dot partials
    // over the partial region, two basis-vector slots over the V region
    const int64_t pstride = (int64_t)L.ep.mmax + 8 + kMaxOrder;
    cudaError_t e = launch_build_jr(
        L.s, H, Jr, reinterpret_cast<unsigned*>(h->ws + kOffBar),
        reinterpret_cast<unsigned long long*>(eb + L.ep.off_part), 2 * (int64_t)L.ep.G * pstride,
        reinterpret_cast<unsigned long long*>(eb + L.ep.off_V), 2 * ((L.s.n_tot + 3) & ~(int64_t)3), st);
    if (e != cudaSuccess) return cuda_fail(h, e, "build_jr");
    LanczosLaunch ll;
    ll.Jr = Jr;
    ll.x0 = x0;
    ll.u0 = u0;
    ll.V = reinterpret_cast<double*>(eb + L.ep.off_V);
    ll.Y = reinterpret_cast<double*>(eb + L.ep.off_Y);
    ll.part = reinterpret_cast<double*>(eb + L.ep.off_part);
    ll.scal = reinterpret_cast<double*>(h->ws + kOffScal);
    ll.x_out = x_out;
    ll.u_out = u_out;
    ll.lambda_out = lambda_out;
    ll.mmax = L.ep.mmax;
    ll.G = L.ep.G;
    ll.eig_tol = (o && o->eig_tol > 0) ? o->eig_tol : 1e-10;
    ll.check = check;
    ll.kkt_tol = kkt_tol;
    ll.bar = reinterpret_cast<unsigned*>(h->ws + kOffBar);
    ll.err = dev_err(h);
    ll.timeout_ns = timeout_of(o);
    ll.cache_floats = L.ep.cache_floats;
    ll.adapt = adapt;
    ll.rqi = rqi;
    ll.shift_add = shift_add;
    ll.proj_u = proj_u;
    ll.scale_override = scale_override;
    ll.hopm = hopm;
    if (tol_override > 0.0) ll.eig_tol = tol_override;
    ll.smem = L.ep.smem;
    e = launch_lanczos(L.s, ll, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "lanczos");
    if (kev) cudaEventRecord(kev->end, st);
    return HOSCF_OK;
}

}  // namespace

// ====================================================================== ABI
// Failure-path self-test kernels: waits that nothing can ever satisfy.
__global__ void selftest_mbar_kernel(int* err, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // no thread ever arrives on `bar` and no copy targets it
    const bool got = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!got && threadIdx.x == 0) atomicCAS(err, 0, (int)DEV_TIMEOUT);
}

__global__ void selftest_grid_kernel(unsigned* state, int* err, uint64_t limit_ns) {
    // one arrival short of the count: the barrier can never open
    unsigned epoch = 0;
    grid_barrier(state, gridDim.x + 1, epoch, err, limit_ns);
}

extern "C" {

hoscf_status hoscf_create(hoscf_handle** out, int device) {
    if (!out) return HOSCF_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HOSCF_EINVAL;
    }
    hoscf_handle* h = new (std::nothrow) hoscf_handle();
    if (!h) return HOSCF_ENOMEM;
    h->device = device;
    DeviceGuard g(device);
    if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete h;
        return HOSCF_ECUDA;
    }
    if (cudaMallocHost(&h->h_pinned, 64 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return HOSCF_ENOMEM;
    }
    *out = h;
    return HOSCF_OK;
}

hoscf_status hoscf_destroy(hoscf_handle* h) {
    if (!h) return HOSCF_EINVAL;
    {
        DeviceGuard g(h->device);
        if (h->ws) cudaFree(h->ws);
        if (h->h_pinned) cudaFreeHost(h->h_pinned);
        if (h->pinned_big) cudaFreeHost(h->pinned_big);
        h->graphs.release();
        if (h->own) cudaStreamDestroy(h->own);
        for (auto& list : h->prof)
            for (KernelEvents& e : list) {
                cudaEventDestroy(e.begin);
                cudaEventDestroy(e.end);
            }
    }
    delete h;
    return HOSCF_OK;
}

const char* hoscf_last_error(const hoscf_handle* h) { return h ? h->msg : "null handle"; }

hoscf_status hoscf_opts_default(hoscf_opts* o) {
    if (!o) return HOSCF_EINVAL;
    memset(o, 0, sizeof(*o));
    o->tol = 1e-6;
    o->max_iter = 200;
    o->variant = HOSCF_VARIANT_HOSCF;
    o->eig_tol = 1e-10;
    o->eig_max_steps = 64;
    o->eig_adapt = 1e-3;
    o->refine = nullptr;
    o->switch_tol = 1e-3;
    o->switch_predict = 1;
    o->timeout_ns = 2000000000;   // 2 s per bounded device wait
    o->batch_threads = 0;
    o->batch_faces = 0;
    return HOSCF_OK;
}

hoscf_status hoscf_workspace_size(int order, const int64_t* dims, int dtype, size_t* bytes) {
    if (!bytes || !dims_valid(order, dims)) return HOSCF_EINVAL;
    Shape s;
    if (!make_shape(order, dims, s)) return HOSCF_EINVAL;
    int nsm = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    PassPlan pp, p32;
    EigPlan ep;
    make_pass_plan(s, dtype, nsm, true, pp);
    make_pass_plan(s, HOSCF_F32, nsm, true, p32);   // a refinement copy is FP32
    make_eig_plan(s, nsm, 1, 64, ep);
    size_t t = kHeadBytes + align_up(std::max(pp.bytes, p32.bytes), 256) + align_up(ep.bytes, 256) +
               2 * align_up(sizeof(float) * s.P, 256) + 3 * align_up(sizeof(float) * s.n_tot, 256) +
               2 * align_up(sizeof(double) * s.n_tot, 256);
    *bytes = t;
    return HOSCF_OK;
}

hoscf_status hoscf_ttvc_blocks(hoscf_handle* h, const hoscf_tensor_desc* T, const float* u,
                               float* H, void* stream) {
    if (!h) return HOSCF_EINVAL;
    hoscf_status st = check_desc(h, T);
    if (st) return st;
    if (!u || !H) return fail(h, HOSCF_EINVAL, "u and H must be non-NULL device pointers");
    DeviceGuard g(h->device);
    Layout L;
    st = plan_all(h, T->order, T->dims, T->dtype, true, false, 64, L);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Err err;
    const KernelEvents* kev = nullptr;
    st = prof_slot(h, 0, &kev);
    if (st) return st;
    st = run_ttvc(L.s, L.pp, T->dtype, T->data, T->scales, u, H, h->ws + L.off_pass, dev_err(h),
                  2000000000ull, s, err, kev);
    if (st) return fail(h, st, "%s", err.msg);
    return HOSCF_OK;
}

hoscf_status hoscf_device_status(hoscf_handle* h, void* stream) {
    if (!h) return HOSCF_EINVAL;
    DeviceGuard g(h->device);
    if (!h->ws) return HOSCF_OK;                  // nothing has run on this handle
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(h->h_pinned + 32, h->ws + kOffErr, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int code;
    memcpy(&code, h->h_pinned + 32, sizeof(int));
    if (code == 0) return HOSCF_OK;
    CK(cudaMemsetAsync(h->ws + kOffErr, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    return dev_status(h, code);
}

hoscf_status hoscf_profile_enable(hoscf_handle* h, int enable) {
    if (!h) return HOSCF_EINVAL;
    h->prof_on = enable != 0;
    if (h->prof_on)
        for (size_t& n : h->prof_n) n = 0;
    return HOSCF_OK;
}

hoscf_status hoscf_profile_read(hoscf_handle* h, int which, int* count, double* total_ms) {
    if (!h || !count || !total_ms || which < 0 || which >= kProfKinds) return HOSCF_EINVAL;
    DeviceGuard g(h->device);
    double tot = 0.0;
    for (size_t i = 0; i < h->prof_n[which]; ++i) {
        float ms = 0.f;
        CK(cudaEventSynchronize(h->prof[which][i].end));
        CK(cudaEventElapsedTime(&ms, h->prof[which][i].begin, h->prof[which][i].end));
        tot += ms;
    }
    *count = (int)h->prof_n[which];
    *total_ms = tot;
    return HOSCF_OK;
}

hoscf_status hoscf_eig_step(hoscf_handle* h, int order, const int64_t* dims, const float* H,
                            const double* x_prev, double* x_out, float* u_out, double* lambda_out,
                            const hoscf_opts* opts, void* stream) {
    if (!h) return HOSCF_EINVAL;
    if (!dims_valid(order, dims)) return fail(h, HOSCF_EINVAL, "order must be 2..%d and dims >= 1", HOSCF_MAX_ORDER);
    if (!H || !x_prev || !x_out || !lambda_out) return fail(h, HOSCF_EINVAL, "NULL pointer argument");
    DeviceGuard g(h->device);
    hoscf_opts o;
    hoscf_opts_default(&o);
    if (opts) o = *opts;
    Layout L;
    hoscf_status st = plan_all(h, order, dims, HOSCF_F32, false, true,
                               std::min(std::max(o.eig_max_steps, 2), 128), L);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    st = reset_barrier_state(h, s);
    if (st) return st;
    return eig_launch(h, L, H, x_prev, nullptr, x_out, u_out, lambda_out, &o, 0, 0.0, s,
                      o.eig_adapt);
}

hoscf_status hoscf_rqi_step(hoscf_handle* h, int order, const int64_t* dims, const float* H,
                            const float* u, double* x_out, float* u_out, double* rho_out,
                            const hoscf_opts* opts, void* stream) {
    if (!h) return HOSCF_EINVAL;
    if (!dims_valid(order, dims)) return fail(h, HOSCF_EINVAL, "order must be 2..%d and dims >= 1", HOSCF_MAX_ORDER);
    if (!H || !u || !u_out) return fail(h, HOSCF_EINVAL, "NULL pointer argument");
    DeviceGuard g(h->device);
    hoscf_opts o;
    hoscf_opts_default(&o);
    if (opts) o = *opts;
    Layout L;
    hoscf_status st = plan_all(h, order, dims, HOSCF_F32, false, true,
                               std::min(std::max(o.eig_max_steps, 2), 128), L);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    st = reset_barrier_state(h, s);
    if (st) return st;
    // start x~ = u / sqrt(d) (the kernel's balanced start from factors), shift
    // = the Rayleigh quotient alpha_0, no certificate shortcut
    return eig_launch(h, L, H, nullptr, u, x_out, u_out, rho_out, &o, 0, 0.0, s, 0.0, 1);
}

// HOSCF / iHOSCF / comparison variants (hoscf_solve), optionally with the
// tensor sharded over ranks by slabs of mode 1 (hoscf_solve_sharded): then T
// is this rank's slab, every pass is the slab pass scattered into the whole
// tensor's block layout followed by the caller's SUM reduction over ranks,
// and everything after the pass (certificate, eigen step, final fix) runs
// on the whole blocks, identically on every rank.
static hoscf_status solve_core(hoscf_handle* h, const hoscf_tensor_desc* T, const hoscf_shard* sh,
                               const float* u0, const hoscf_opts* opts, float* u_out,
                               double* sigma_out, hoscf_info* info, void* stream) {
    if (!h) return HOSCF_EINVAL;
    hoscf_status st = check_desc(h, T);
    if (st) return st;
    if (!u0 || !u_out || !sigma_out) return fail(h, HOSCF_EINVAL, "NULL pointer argument");
    hoscf_opts o;
    hoscf_opts_default(&o);
    if (opts) o = *opts;
    if (o.max_iter < 0 || !(o.tol >= 0)) return fail(h, HOSCF_EINVAL, "bad tol / max_iter");
    if (o.variant != HOSCF_VARIANT_HOSCF && o.variant != HOSCF_VARIANT_IHOSCF &&
        o.variant != HOSCF_VARIANT_IHOSCF_PREV && o.variant != HOSCF_VARIANT_JACOBI_HOPM &&
        o.variant != HOSCF_VARIANT_ASVD)
        return fail(h, HOSCF_EINVAL, "unknown variant %d", o.variant);
    if (o.variant == HOSCF_VARIANT_ASVD && T->order > 3)
        return fail(h, HOSCF_EUNSUPPORTED, "ASVD is built for orders 2 and 3");
    const hoscf_tensor_desc* Tr = o.refine;
    if (Tr) {
        st = check_desc(h, Tr);
        if (st) return st;
        if (Tr->dtype != HOSCF_F32 || Tr->order != T->order)
            return fail(h, HOSCF_EINVAL, "refine tensor must be FP32 of the same shape");
        for (int k = 0; k < T->order; ++k)
            if (Tr->dims[k] != T->dims[k]) return fail(h, HOSCF_EINVAL, "refine tensor shape differs");
    }
    // the whole tensor's dims (a shard holds rows [row0, row0 + I_1') of mode 1)
    int64_t fdims[HOSCF_MAX_ORDER];
    for (int k = 0; k < T->order; ++k) fdims[k] = T->dims[k];
    if (sh) {
        if (sh->row0 < 0 || sh->dim0 < 1 || sh->row0 + T->dims[0] > sh->dim0)
            return fail(h, HOSCF_EINVAL, "slab rows [%lld, %lld) outside mode 1 of size %lld",
                        (long long)sh->row0, (long long)(sh->row0 + T->dims[0]), (long long)sh->dim0);
        fdims[0] = sh->dim0;
    }
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Layout L;
    const int mmax = std::min(std::max(o.eig_max_steps, 2), 128);
    // ASVD: the eigen step of each two-mode sub-problem (one block, J2 =
    // [[0, A_mn], [A_mn^T, 0]]) runs in the extra region, after its input and
    // output pair buffers and its eigenvalue
    const bool asvd = o.variant == HOSCF_VARIANT_ASVD;
    Layout Lpair[3];
    size_t extra = 0, off_pin = 0, off_pout = 0, off_lam = 0, off_peig = 0;
    if (asvd) {
        int64_t ntot = 0;
        for (int k = 0; k < T->order; ++k) ntot += fdims[k];
        off_pin = 0;
        off_pout = align_up(sizeof(float) * (size_t)ntot, 256);
        off_lam = off_pout + align_up(sizeof(float) * (size_t)ntot, 256);
        off_peig = off_lam + 256;
        size_t peig = 0;
        int b = 0;
        for (int m = 0; m < T->order; ++m)
            for (int n = m + 1; n < T->order; ++n, ++b) {
                const int64_t dd[2] = {fdims[m], fdims[n]};
                if (!make_shape(2, dd, Lpair[b].s) ||
                    !make_eig_plan(Lpair[b].s, h->nsm, 1, mmax, Lpair[b].ep))
                    return fail(h, HOSCF_EINVAL, "ASVD eigen plan failed");
                peig = std::max(peig, Lpair[b].ep.bytes);
            }
        extra = off_peig + peig;
    }
    // shard: the slab pass (its scratch, its packed blocks, its factors) in
    // the extra region after the ASVD buffers
    Shape Ss;
    PassPlan pps, pps_lo;
    size_t off_shard = 0, off_sh_H = 0, off_sh_u = 0;
    if (sh) {
        if (!make_shape(T->order, T->dims, Ss)) return fail(h, HOSCF_EINVAL, "invalid slab shape");
        make_pass_plan(Ss, Tr ? HOSCF_F32 : T->dtype, h->nsm, true, pps);
        pps_lo = pps;
        if (Tr) make_pass_plan(Ss, T->dtype, h->nsm, true, pps_lo);
        off_shard = align_up(extra, 256);
        off_sh_H = align_up(std::max(pps.bytes, pps_lo.bytes), 256);
        off_sh_u = off_sh_H + align_up(sizeof(float) * (size_t)Ss.P, 256);
        extra = off_shard + off_sh_u + align_up(sizeof(float) * (size_t)Ss.n_tot, 256);
    }
    // the pass region must fit both the low-precision and the FP32 pass
    st = plan_all(h, T->order, fdims, Tr ? HOSCF_F32 : T->dtype, sh == nullptr, true, mmax, L,
                  Tr && !sh ? T->dtype : -1, extra);
    if (st) return st;
    for (Layout& lp : Lpair) lp.off_eig = L.off_extra + off_peig;
    PassPlan pp_lo = L.pp;
    if (Tr && !sh) make_pass_plan(L.s, T->dtype, h->nsm, true, pp_lo);
    const Shape& S = L.s;
    float* H = reinterpret_cast<float*>(h->ws + L.off_H);
    float* ua = reinterpret_cast<float*>(h->ws + L.off_ua);
    float* ub = reinterpret_cast<float*>(h->ws + L.off_ub);
    double* norms = reinterpret_cast<double*>(h->ws + kOffNorms);
    double* scal = reinterpret_cast<double*>(h->ws + kOffScal);
    st = reset_dev_state(h, s);
    if (st) return st;
    // normalise the initial guess (eq. 3.4); zero / non-finite blocks are errors
    CK(launch_mode_norms(S, u0, norms, s));
    CK(cudaMemcpyAsync(h->h_pinned, norms, sizeof(double) * S.d, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < S.d; ++k)
        if (!(h->h_pinned[k] > 0.0) || !std::isfinite(h->h_pinned[k]))
            return fail(h, HOSCF_EINVAL, "initial guess block %d is zero or non-finite", k);
    CK(launch_scale_modes(S, u0, norms, ua, s));

    const uint64_t tmo = timeout_of(&o);
    int iters = 0, passes = 0, passes_ref = 0, accepts = 0;
    double sigma = 0.0, resid = INFINITY, r41 = NAN;
    bool use_ref = false;
    double lo_min = INFINITY;   // precision form: lowest residual so far and
    int since_min = 0;          // the iterations since it was reached
    constexpr int kStallIters = 64;
    hoscf_status result = HOSCF_NOT_CONVERGED;
    // three factor buffers (current point, eigen step, RQI candidate) and two
    // block buffers, so a rejected RQI step never costs a repeated pass
    float* ucur = ua;
    float* unext = ub;
    float* uy = reinterpret_cast<float*>(h->ws + L.off_uc);
    float* Hcur = H;
    float* Hoth = reinterpret_cast<float*>(h->ws + L.off_H2);
    Err err;

    auto do_pass = [&](const float* u, float* Hdst) -> hoscf_status {
        const hoscf_tensor_desc* TT = use_ref ? Tr : T;
        if (sh) {
            // this rank's slab: its factor rows, its pass, the scatter into
            // the whole layout, then the SUM over ranks (the caller's collective)
            char* base = h->ws + L.off_extra + off_shard;
            float* us = reinterpret_cast<float*>(base + off_sh_u);
            float* Hs = reinterpret_cast<float*>(base + off_sh_H);
            const int64_t rows = Ss.dims[0];
            CK(cudaMemcpyAsync(us, u + sh->row0, sizeof(float) * rows, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(us + rows, u + S.moff[1], sizeof(float) * (S.n_tot - S.moff[1]),
                               cudaMemcpyDeviceToDevice, s));
            const PassPlan& pq = use_ref ? pps : (Tr ? pps_lo : pps);
            hoscf_status q = run_ttvc(Ss, pq, TT->dtype, TT->data, TT->scales, us, Hs, base,
                                      dev_err(h), tmo, s, err);
            if (q) return fail(h, q, "%s", err.msg);
            CK(launch_shard_scatter(S, Ss, sh->row0, Hs, Hdst, s));
            if (sh->reduce(Hdst, S.P, stream, sh->user) != 0)
                return fail(h, HOSCF_ECUDA, "the block reduction over ranks failed");
        } else {
            const PassPlan& pp = use_ref ? L.pp : (Tr ? pp_lo : L.pp);
            hoscf_status q = run_ttvc(S, pp, TT->dtype, TT->data, TT->scales, u, Hdst,
                                      h->ws + L.off_pass, dev_err(h), tmo, s, err);
            if (q) return fail(h, q, "%s", err.msg);
        }
        if (h->defl_count > 0) {
            // greedy rank-R: blocks of the deflated tensor at u
            cudaError_t e = launch_deflate(S, Hdst, u, h->defl_u,
                                           reinterpret_cast<double*>(h->ws + kOffDeflSigma),
                                           h->defl_count,
                                           reinterpret_cast<double*>(h->ws + kOffDeflDots), s);
            if (e != cudaSuccess) return cuda_fail(h, e, "deflate");
        }
        ++passes;
        if (use_ref) ++passes_ref;
        return HOSCF_OK;
    };
    // certificate at u (+ the eigen step or the RQI solve into u_res unless u
    // is certified); scalars are read back synchronously
    auto do_step = [&](const float* Hsrc, const float* u, float* u_res, int rqi, double* out,
                       int check = 1) -> hoscf_status {
        // Jacobi-HOPM takes its update from the certificate's mat-vec; ASVD
        // needs only the certificate here (its step is the pair's eigen step)
        const int hopm_mode = (o.variant == HOSCF_VARIANT_JACOBI_HOPM || asvd) && rqi == 0 ? 1 : 0;
        hoscf_status q = eig_launch(h, L, Hsrc, nullptr, u, nullptr, u_res, nullptr, &o, check,
                                    o.tol, s, o.eig_adapt, rqi, 0.f, nullptr, 0.f, 0.0, hopm_mode);
        if (q) return q;
        cudaError_t e = cudaMemcpyAsync(h->h_pinned, scal, sizeof(double) * SC_COUNT,
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "readback");
        e = cudaMemcpyAsync(h->h_pinned + 32, h->ws + kOffErr, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "readback");
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "iteration");
        int code;
        memcpy(&code, h->h_pinned + 32, sizeof(int));
        if (code) return dev_status(h, code);
        memcpy(out, h->h_pinned, sizeof(double) * SC_COUNT);
        if (!std::isfinite(out[SC_SIGMA]) || std::isnan(out[SC_KKT]))
            return fail(h, HOSCF_NONFINITE, "non-finite sigma or residual");
        return HOSCF_OK;
    };

    double sc[SC_COUNT], sk[SC_COUNT], sy[SC_COUNT];
    double prev_resid = INFINITY, prev2_resid = INFINITY;
    st = do_pass(ucur, Hcur);
    if (st) return st;
    while (true) {
        // certify the current point; unless certified, take the eigen step
        st = do_step(Hcur, ucur, unext, 0, sc);
        if (st) return st;
        sigma = sc[SC_SIGMA];
        resid = sc[SC_KKT];
        r41 = sc[SC_R41];
        // precision form: move to the FP32 tensor once the residual reaches
        // switch_tol, stops decreasing, or is predicted to reach switch_tol
        // at the next iterate (the observed contraction r_k / r_{k-1} applied
        // once more) - so that the pass at that iterate is already an FP32
        // pass.  The low-precision certificate itself has no floor (it
        // certifies the low-precision tensor, whose fixed point the iteration
        // approaches), so a slow decrease is progress, not a floor; the KKT
        // residual need not fall monotonically either (slowly converging
        // problems show humps of tens of iterations), so "stops decreasing"
        // means no new lowest residual for kStallIters iterations - or half
        // of max_iter spent, so that the FP32 passes keep their share.
        if (resid < lo_min) {
            lo_min = resid;
            since_min = 0;
        } else {
            ++since_min;
        }
        const bool stalled = Tr && !use_ref && (since_min >= kStallIters || 2 * iters >= o.max_iter);
        // the prediction applies the last contraction once more
        // (switch_predict 1), or the slower of the last two (2), so that a
        // single fast first step on a slowly converging problem does not end
        // the narrow passes early
        bool predicted = false;
        if (Tr && !use_ref && o.switch_predict == 1 && iters > 0 && prev_resid > 0.0 &&
            std::isfinite(prev_resid))
            predicted = resid * (resid / prev_resid) <= o.switch_tol;
        if (Tr && !use_ref && o.switch_predict == 2 && iters > 1 && prev_resid > 0.0 &&
            prev2_resid > 0.0 && std::isfinite(prev2_resid))
            predicted = resid * std::max(resid / prev_resid, prev_resid / prev2_resid) <= o.switch_tol;
        prev2_resid = prev_resid;
        prev_resid = resid;
        if (Tr && !use_ref &&
            (resid <= o.switch_tol || stalled || predicted || sc[SC_CONVERGED] != 0.0)) {
            // precision form: the low-precision tensor has done its part; the
            // remaining passes and the certificate use the FP32 tensor
            use_ref = true;
            // (ASVD's step is not the certificate's by-product: it re-certifies
            // the current point on the FP32 tensor and steps from there)
            if (!asvd && sc[SC_CONVERGED] == 0.0 && iters < o.max_iter) {
                ++iters;
                std::swap(ucur, unext);
            }
            st = do_pass(ucur, Hcur);
            if (st) return st;
            continue;
        }
        if (sc[SC_CONVERGED] != 0.0) {
            result = HOSCF_OK;
            break;
        }
        if (iters >= o.max_iter) break;
        ++iters;
        if (asvd) {
            // fixed mode f = 1, 2, 3, 1, ... (d = 3); the free pair (m, n)
            int m = 0, n = 1;
            if (S.d == 3) {
                const int f = (iters - 1) % 3;
                m = f == 0 ? 1 : 0;
                n = f == 2 ? 1 : 2;
            }
            const int b = m == 0 ? n - 1 : 2;      // lexicographic pair index (d <= 3)
            float* pin = reinterpret_cast<float*>(h->ws + L.off_extra + off_pin);
            float* pout = reinterpret_cast<float*>(h->ws + L.off_extra + off_pout);
            double* lam = reinterpret_cast<double*>(h->ws + L.off_extra + off_lam);
            const int64_t im = S.dims[m], in = S.dims[n];
            CK(cudaMemcpyAsync(pin, ucur + S.moff[m], sizeof(float) * im, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(pin + im, ucur + S.moff[n], sizeof(float) * in, cudaMemcpyDeviceToDevice, s));
            st = eig_launch(h, Lpair[b], Hcur + S.boff[b], nullptr, pin, nullptr, pout, lam, &o, 0,
                            0.0, s, o.eig_adapt);
            if (st) return st;
            CK(launch_asvd_pair_fix(ucur, S.n_tot, S.moff[m], im, S.moff[n], in, pout, lam, unext, s));
            std::swap(ucur, unext);
            st = do_pass(ucur, Hcur);
            if (st) return st;
            continue;
        }
        if (o.variant == HOSCF_VARIANT_HOSCF || o.variant == HOSCF_VARIANT_JACOBI_HOPM) {
            std::swap(ucur, unext);
            st = do_pass(ucur, Hcur);
            if (st) return st;
            continue;
        }
        if (o.variant == HOSCF_VARIANT_IHOSCF) {
            // RQI with J built at the new point x_k (Sec. 4.4, read with the
            // matrix of the point the eigen step just returned)
            st = do_pass(unext, Hoth);                 // J(x_k)
            if (st) return st;
            st = do_step(Hoth, unext, uy, 1, sk);      // certify x_k, then solve for y
            if (st) return st;
            if (sk[SC_CONVERGED] != 0.0) {
                std::swap(ucur, unext);
                std::swap(Hcur, Hoth);
                sigma = sk[SC_SIGMA];
                resid = sk[SC_KKT];
                r41 = sk[SC_R41];
                result = HOSCF_OK;
                break;
            }
            st = do_pass(uy, Hcur);                    // J(y)
            if (st) return st;
            st = do_step(Hcur, uy, ucur, 0, sy);       // certificate of y (eig result unused)
            if (st) return st;
            if (sy[SC_CONVERGED] != 0.0 || std::fabs(sy[SC_SIGMA]) >= std::fabs(sk[SC_SIGMA])) {
                ++accepts;                             // keep y: Hcur holds J(y)
                std::swap(ucur, uy);
                if (sy[SC_CONVERGED] != 0.0) {
                    sigma = sy[SC_SIGMA];
                    resid = sy[SC_KKT];
                    r41 = sy[SC_R41];
                    result = HOSCF_OK;
                    break;
                }
            } else {                                   // keep x_k: its blocks are in Hoth
                std::swap(ucur, unext);
                std::swap(Hcur, Hoth);
            }
            continue;
        }
        // HOSCF_VARIANT_IHOSCF_PREV: RQI with J_{k-1} (the matrix just used)
        st = do_step(Hcur, unext, uy, 1, sk, 0);       // rho from J_{k-1} at x~_k
        if (st) return st;
        st = do_pass(uy, Hoth);
        if (st) return st;
        st = do_step(Hoth, uy, unext, 0, sy);
        if (st) return st;
        if (sy[SC_CONVERGED] != 0.0 || std::fabs(sy[SC_SIGMA]) >= std::fabs(sigma)) {
            ++accepts;
            std::swap(ucur, uy);
            std::swap(Hcur, Hoth);
            if (sy[SC_CONVERGED] != 0.0) {
                sigma = sy[SC_SIGMA];
                resid = sy[SC_KKT];
                r41 = sy[SC_R41];
                result = HOSCF_OK;
                break;
            }
        } else {
            // restore x_k with one extra pass; its eigen step was overwritten
            // above, so recompute from J_{k-1}
            st = do_step(Hcur, ucur, unext, 0, sc);
            if (st) return st;
            std::swap(ucur, unext);
            st = do_pass(ucur, Hcur);
            if (st) return st;
        }
    }
    // final sign fix (Alg. 1 lines 12-15) and gauge, into u_out
    CK(cudaMemcpyAsync(u_out, ucur, sizeof(float) * S.n_tot, cudaMemcpyDeviceToDevice, s));
    h->h_pinned[0] = sigma;
    CK(cudaMemcpyAsync(norms, h->h_pinned, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(launch_final_fix(S, u_out, norms, s));
    CK(cudaMemcpyAsync(h->h_pinned + 1, norms, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *sigma_out = h->h_pinned[1];
    if (info) {
        info->iters = iters;
        info->passes = passes;
        info->passes_refine = passes_ref;
        info->rqi_accepts = accepts;
        info->resid = resid;
        info->resid_4_1 = r41;
        info->sigma_raw = sigma;
    }
    if (result == HOSCF_NOT_CONVERGED)
        fail(h, HOSCF_NOT_CONVERGED, "not converged after %d iterations (r = %.3e)", iters, resid);
    return result;
}

hoscf_status hoscf_solve(hoscf_handle* h, const hoscf_tensor_desc* T, const float* u0,
                         const hoscf_opts* opts, float* u_out, double* sigma_out,
                         hoscf_info* info, void* stream) {
    return solve_core(h, T, nullptr, u0, opts, u_out, sigma_out, info, stream);
}

hoscf_status hoscf_solve_sharded(hoscf_handle* h, const hoscf_tensor_desc* T,
                                 const hoscf_shard* shard, const float* u0,
                                 const hoscf_opts* opts, float* u_out, double* sigma_out,
                                 hoscf_info* info, void* stream) {
    if (!h) return HOSCF_EINVAL;
    if (!shard || !shard->reduce) return fail(h, HOSCF_EINVAL, "shard descriptor or reduce callback missing");
    return solve_core(h, T, shard, u0, opts, u_out, sigma_out, info, stream);
}

hoscf_status hoscf_ttvc_blocks_slab(hoscf_handle* h, const hoscf_tensor_desc* T, int64_t row0,
                                    int64_t dim0, const float* u, float* H, void* stream) {
    if (!h) return HOSCF_EINVAL;
    hoscf_status st = check_desc(h, T);
    if (st) return st;
    if (!u || !H) return fail(h, HOSCF_EINVAL, "u and H must be non-NULL device pointers");
    if (row0 < 0 || dim0 < 1 || row0 + T->dims[0] > dim0)
        return fail(h, HOSCF_EINVAL, "slab rows outside mode 1");
    int64_t fdims[HOSCF_MAX_ORDER];
    for (int k = 0; k < T->order; ++k) fdims[k] = T->dims[k];
    fdims[0] = dim0;
    Shape Sf;
    if (!make_shape(T->order, fdims, Sf)) return fail(h, HOSCF_EINVAL, "invalid shape");
    DeviceGuard g(h->device);
    Layout L;   // the slab: pass scratch, its blocks (off_H) and its factors (off_ua)
    st = plan_all(h, T->order, T->dims, T->dtype, true, false, 64, L);
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float* us = reinterpret_cast<float*>(h->ws + L.off_ua);
    float* Hs = reinterpret_cast<float*>(h->ws + L.off_H);
    const int64_t rows = T->dims[0];
    CK(cudaMemcpyAsync(us, u + row0, sizeof(float) * rows, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(us + rows, u + dim0, sizeof(float) * (Sf.n_tot - dim0),
                       cudaMemcpyDeviceToDevice, s));
    Err err;
    st = run_ttvc(L.s, L.pp, T->dtype, T->data, T->scales, us, Hs, h->ws + L.off_pass, dev_err(h),
                  2000000000ull, s, err);
    if (st) return fail(h, st, "%s", err.msg);
    CK(launch_shard_scatter(Sf, L.s, row0, Hs, H, s));
    return HOSCF_OK;
}

hoscf_status hoscf_solve_batched(hoscf_handle* h, int count, const hoscf_tensor_desc* T,
                                 const float* const* u0, const hoscf_opts* opts,
                                 float* const* u_out, double* sigma_out, hoscf_info* infos,
                                 void* stream) {
    if (!h) return HOSCF_EINVAL;
    if (count < 0 || (count > 0 && (!T || !u0 || !u_out || !sigma_out)))
        return fail(h, HOSCF_EINVAL, "bad batch arguments");
    if (count == 0) return HOSCF_OK;
    hoscf_opts o;
    hoscf_opts_default(&o);
    if (opts) o = *opts;
    const int threads = o.batch_threads == 0 ? 512 : o.batch_threads;
    if (threads != 256 && threads != 512 && threads != 1024)
        return fail(h, HOSCF_EINVAL, "batch_threads must be 256, 512 or 1024");
    if (o.batch_faces < 0 || o.batch_faces > 32)
        return fail(h, HOSCF_EINVAL, "batch_faces must be 0 .. 32");
    DeviceGuard g(h->device);
    // descriptors + results: ~100 bytes per tensor, staged through pinned
    // memory; the workspace head (status word, barrier state) is left alone
    const size_t need = 4096 + (size_t)count * 128;
    hoscf_status st = ensure_ws(h, kHeadBytes + need);
    if (st) return st;
    if (h->pinned_big_bytes < need) {
        // captured graphs copy through the old staging buffer: drop them first
        CK(cudaDeviceSynchronize());
        h->graphs.release();
        if (h->pinned_big) cudaFreeHost(h->pinned_big);
        h->pinned_big = nullptr;
        h->pinned_big_bytes = 0;
        if (cudaMallocHost(&h->pinned_big, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, HOSCF_ENOMEM, "pinned staging of %zu bytes failed", need);
        }
        h->pinned_big_bytes = need;
    }
    if (!h->own) CK(cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking));
    CK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    Err err;
    st = run_batched(count, T, u0, u_out, o, threads, h->ws + kHeadBytes, h->ws_bytes - kHeadBytes,
                     h->nsm, h->own, sigma_out, infos, h->pinned_big, h->pinned_big_bytes,
                     h->graphs, err);
    if (st) return fail(h, st, "%s", err.msg);
    return HOSCF_OK;
}

hoscf_status hoscf_backward(hoscf_handle* h, const hoscf_tensor_desc* T, const float* u,
                            double sigma, double grad_sigma, const float* grad_u, float* grad_T,
                            void* stream) {
    if (!h) return HOSCF_EINVAL;
    hoscf_status st = check_desc(h, T);
    if (st) return st;
    if (T->dtype != HOSCF_F32) return fail(h, HOSCF_EINVAL, "backward needs an FP32 tensor");
    if (!u || !grad_T) return fail(h, HOSCF_EINVAL, "NULL pointer argument");
    if (!std::isfinite(sigma) || !std::isfinite(grad_sigma))
        return fail(h, HOSCF_NONFINITE, "non-finite sigma or grad_sigma");
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Layout L;
    {
        Shape s0;
        if (!make_shape(T->order, T->dims, s0)) return fail(h, HOSCF_EINVAL, "invalid shape");
        // extra region: the write's per-outer-index coefficients (2 O floats)
        st = plan_all(h, T->order, T->dims, HOSCF_F32, true, true, 128, L, -1,
                      sizeof(float) * 2 * (size_t)s0.O);
    }
    if (st) return st;
    const Shape& S = L.s;
    st = reset_dev_state(h, s);
    if (st) return st;
    float* H = reinterpret_cast<float*>(h->ws + L.off_H);
    double* b = reinterpret_cast<double*>(h->ws + L.off_x);
    double* av = reinterpret_cast<double*>(h->ws + L.off_x2);
    double* bn2 = reinterpret_cast<double*>(h->ws + kOffNorms);
    double* scal = reinterpret_cast<double*>(h->ws + kOffScal);
    Err err;
    const double* aptr = nullptr;
    hoscf_status result = HOSCF_OK;
    if (grad_u) {
        // adjoint: P (H - sigma I) P a = P w on the factors' tangent space
        CK(launch_tangent_project(S, u, grad_u, b, bn2, s));
        CK(cudaMemcpyAsync(h->h_pinned, bn2, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double bnorm2 = h->h_pinned[0];
        if (!std::isfinite(bnorm2)) return fail(h, HOSCF_NONFINITE, "non-finite grad_u");
        if (bnorm2 > 0.0) {
            const KernelEvents* kadj = nullptr;
            st = prof_slot(h, 2, &kadj);
            if (st) return st;
            if (kadj) CK(cudaEventRecord(kadj->begin, s));
            st = run_ttvc(S, L.pp, HOSCF_F32, T->data, nullptr, u, H, h->ws + L.off_pass,
                          dev_err(h), 2000000000ull, s, err);
            if (st) return fail(h, st, "%s", err.msg);
            hoscf_opts o;
            hoscf_opts_default(&o);
            o.eig_max_steps = 128;
            st = eig_launch(h, L, H, b, nullptr, av, nullptr, nullptr, &o, 0, 0.0, s, 0.0, 2,
                            (float)(-sigma), u, 1.0f, 1e-6);
            if (st) return st;
            if (kadj) CK(cudaEventRecord(kadj->end, s));
            CK(cudaMemcpyAsync(h->h_pinned, scal, sizeof(double) * SC_COUNT,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(h->h_pinned + 32, h->ws + kOffErr, sizeof(int),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            int code;
            memcpy(&code, h->h_pinned + 32, sizeof(int));
            if (code) return dev_status(h, code);
            if (!std::isfinite(h->h_pinned[SC_RITZRES]))
                return fail(h, HOSCF_NONFINITE, "adjoint system singular to working precision");
            if (h->h_pinned[SC_CONVERGED] == 0.0) {
                result = HOSCF_NOT_CONVERGED;
                fail(h, HOSCF_NOT_CONVERGED, "adjoint solve stopped at relative residual %.3e",
                     h->h_pinned[SC_RITZRES]);
            }
            aptr = av;
        }
    }
    float* coef = reinterpret_cast<float*>(h->ws + L.off_extra);
    const KernelEvents* kw = nullptr;
    st = prof_slot(h, 1, &kw);
    if (st) return st;
    CK(launch_grad_write(S, u, aptr, grad_sigma, coef, grad_T, s, kw));
    CK(cudaStreamSynchronize(s));
    return result;
}

hoscf_status hoscf_solve_greedy(hoscf_handle* h, const hoscf_tensor_desc* T, int R,
                                const float* u0, const hoscf_opts* opts, float* u_out,
                                double* sigma_out, hoscf_info* info, double* res_out,
                                void* stream) {
    if (!h) return HOSCF_EINVAL;
    hoscf_status st = check_desc(h, T);
    if (st) return st;
    if (R < 1 || R > kMaxGreedy) return fail(h, HOSCF_EINVAL, "R must be 1..%d", kMaxGreedy);
    if (!u0 || !u_out || !sigma_out) return fail(h, HOSCF_EINVAL, "NULL pointer argument");
    Shape S;
    if (!make_shape(T->order, T->dims, S)) return fail(h, HOSCF_EINVAL, "bad shape");
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the deflation state lives only for the duration of this call
    struct Reset {
        hoscf_handle* h;
        ~Reset() {
            h->defl_u = nullptr;
            h->defl_count = 0;
        }
    } reset{h};
    st = ensure_ws(h, kHeadBytes);
    if (st) return st;
    hoscf_status result = HOSCF_OK;
    for (int r = 0; r < R; ++r) {
        h->defl_u = u_out;        // rows 0 .. r-1 hold the terms found so far
        h->defl_count = r;
        if (r > 0)
            CK(cudaMemcpyAsync(h->ws + kOffDeflSigma, sigma_out, sizeof(double) * r,
                               cudaMemcpyHostToDevice, s));
        double sig = 0.0;
        st = hoscf_solve(h, T, u0 + (size_t)r * S.n_tot, opts, u_out + (size_t)r * S.n_tot, &sig,
                         info ? &info[r] : nullptr, stream);
        if (st != HOSCF_OK && st != HOSCF_NOT_CONVERGED) return st;
        if (st == HOSCF_NOT_CONVERGED) result = HOSCF_NOT_CONVERGED;
        sigma_out[r] = sig;
    }
    if (res_out) {
        // ||A^(r+1)||^2 = ||A^(r)||^2 - sigma_r^2 (<A^(r), B^(r)> = sigma_r^2 at a
        // KKT point); ||A||_F from the tensor the certificates use
        const hoscf_tensor_desc* TA = (opts && opts->refine) ? opts->refine : T;
        double* part = reinterpret_cast<double*>(h->ws + kOffSumsq) + 1;
        double* tot = reinterpret_cast<double*>(h->ws + kOffSumsq);
        CK(launch_sumsq(TA->dtype, TA->data, TA->scales, S.N, part, kSumsqParts, tot, s));
        CK(cudaMemcpyAsync(h->h_pinned, tot, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double a2 = h->h_pinned[0];
        double acc = 0.0;
        res_out[0] = 1.0;
        for (int r = 0; r < R; ++r) {
            acc += sigma_out[r] * sigma_out[r];
            res_out[r + 1] = a2 > 0.0 ? std::sqrt(std::max(0.0, a2 - acc) / a2) : 0.0;
        }
    }
    return result;
}

hoscf_status hoscf_selftest_timeout(hoscf_handle* h, int kind, int64_t timeout_ns, void* stream) {
    if (!h || kind < 0 || kind > 2 || timeout_ns <= 0 || timeout_ns > 10000000000ll)
        return HOSCF_EINVAL;
    DeviceGuard g(h->device);
    const size_t need = kHeadBytes;
    hoscf_status st = ensure_ws(h, need);
    if (st) return st;
    if (!h->own) CK(cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking));
    cudaStream_t s = h->own;
    st = reset_dev_state(h, s);
    if (st) return st;
    if (kind == 2) {
        // asynchronous form: the wait runs on the caller's stream and its
        // timeout is left in the status word for hoscf_device_status
        selftest_mbar_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
            dev_err(h), (uint64_t)timeout_ns);
        CK(cudaGetLastError());
        return HOSCF_OK;
    }
    if (kind == 0) {
        selftest_mbar_kernel<<<1, 32, 0, s>>>(dev_err(h), (uint64_t)timeout_ns);
    } else {
        selftest_grid_kernel<<<2, 64, 0, s>>>(reinterpret_cast<unsigned*>(h->ws + kOffBar),
                                             dev_err(h), (uint64_t)timeout_ns);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_pinned + 32, h->ws + kOffErr, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int code;
    memcpy(&code, h->h_pinned + 32, sizeof(int));
    st = reset_dev_state(h, s);   // leave the barrier state clean for the next launch
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    if (code) return dev_status(h, code);
    return fail(h, HOSCF_ECUDA, "self-test wait did not report its timeout");
}

hoscf_status hoscf_quantize(hoscf_handle* h, const float* x, int64_t n, int dtype, void* q,
                            float* scales, void* stream) {
    if (!h) return HOSCF_EINVAL;
    if (n < 0 || (n > 0 && (!x || !q))) return fail(h, HOSCF_EINVAL, "bad quantize arguments");
    if (dtype != HOSCF_BF16 && dtype != HOSCF_F8E4M3 && dtype != HOSCF_F16)
        return fail(h, HOSCF_EINVAL, "quantize dtype must be BF16, F16 or F8E4M3");
    if (dtype == HOSCF_F8E4M3 && n > 0 && !scales) return fail(h, HOSCF_EINVAL, "FP8 needs scales");
    DeviceGuard g(h->device);
    CK(launch_quantize(x, n, dtype, q, scales, reinterpret_cast<cudaStream_t>(stream)));
    return HOSCF_OK;
}

}  // extern "C"
