// hoscf_ttvc_blocks_static: the all-pairs TTVc pass for callers that cannot
// allocate device memory (see include/hoscf.h).  It runs exactly the pass
// that hoscf_ttvc_blocks runs, with its scratch taken from one file-scope
// device array instead of a handle workspace.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "plan.h"

namespace {

constexpr size_t kHead = 256;   // device error word lives here; must start at zero

// Scratch shared by every call on a device.  Every GPU that loads this library
// holds it (HOSCF_STATIC_SCRATCH_BYTES) until the process exits.
static __device__ __align__(256) char g_scratch[HOSCF_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
char* g_scratch_dev[kMaxDevices] = {nullptr};

// Host code cannot use g_scratch's name as a device address (it is a host
// stand-in); the real address is looked up with the device current.  The
// lookup is repeated on every call whose stream is not capturing, so a
// context that was destroyed and created again (cudaDeviceReset, a primary
// context released and retained by the host application) never leaves a
// stale address behind; while a stream captures, the address found by an
// earlier call on that device is used.
hoscf_status scratch_for_current_device(cudaStream_t st, char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return HOSCF_ECUDA;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return HOSCF_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_dev[dev]) {
        if (cap != cudaStreamCaptureStatusNone) return HOSCF_EINVAL;   // no set-up during capture
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HOSCF_ECUDA;
        }
        g_scratch_dev[dev] = static_cast<char*>(p);
    }
    *out = g_scratch_dev[dev];
    return HOSCF_OK;
}

}  // namespace

extern "C" hoscf_status hoscf_ttvc_blocks_static(const hoscf_tensor_desc* T, const float* u,
                                                 float* H, int* status, void* stream) {
    using namespace hoscf;
    if (!T || !u || !H || !T->data || !T->dims) return HOSCF_EINVAL;
    if (T->order < 2 || T->order > HOSCF_MAX_ORDER) return HOSCF_EINVAL;
    if (T->dtype != HOSCF_F32 && T->dtype != HOSCF_BF16 && T->dtype != HOSCF_F16) return HOSCF_EINVAL;
    if ((reinterpret_cast<uintptr_t>(T->data) & 15) != 0) return HOSCF_EINVAL;
    Shape s;
    if (!make_shape(T->order, T->dims, s)) return HOSCF_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return HOSCF_ECUDA;
    }
    PassPlan pp;
    make_pass_plan(s, T->dtype, nsm, true, pp);
    if (kHead + pp.bytes > (size_t)HOSCF_STATIC_SCRATCH_BYTES) return HOSCF_EINVAL;  // too large
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    char* base = nullptr;
    hoscf_status st = scratch_for_current_device(cs, &base);
    if (st) return st;
    int* dev_err = reinterpret_cast<int*>(base);
    if (cudaMemsetAsync(dev_err, 0, sizeof(int), cs) != cudaSuccess) {
        cudaGetLastError();
        return HOSCF_ECUDA;
    }
    Err err;
    st = run_ttvc(s, pp, T->dtype, T->data, T->scales, u, H, base + kHead, dev_err,
                  2000000000ull, cs, err);
    if (st) return st;
    // the pass's device status word (0, or the code of a wait that gave up)
    // goes to the caller's word, in stream order after the pass
    if (status && cudaMemcpyAsync(status, dev_err, sizeof(int), cudaMemcpyDeviceToDevice, cs) != cudaSuccess) {
        cudaGetLastError();
        return HOSCF_ECUDA;
    }
    return HOSCF_OK;
}
