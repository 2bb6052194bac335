// gbs_cumulants_noalloc: the click-cumulant table for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the table:
// code that runs inside an allocator or memory-pool callback, plugins whose
// host application owns every device allocation, and runtimes that forbid
// allocation after start-up. They can pass the input and the output but not a
// workspace. This entry point runs the same kernels as gbs_cumulants (GBS_FP64)
// with every scratch buffer (packed 2x2 blocks, lower-order P0 table,
// per-block Schur-complement slots, status word and work counters) placed in
// one file-scope device array of fixed size, reserved on each GPU that loads
// the library and held until the process exits.
#include <cstdio>
#include <mutex>

#include "gbs.h"
#include "gbs_common.cuh"
#include "gbs_fwd.cuh"

namespace gbs {
int record_error(int code, const char *msg);
}

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)GBS_NOALLOC_SCRATCH_MB << 20;

// The scratch array. Host code must not pass its name to a kernel: in host code
// the name is a host-side stand-in, not a device address. The device address
// comes from cudaGetSymbolAddress, looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set up on first use).
int scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gbs::record_error(GBS_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return gbs::record_error(GBS_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
            return gbs::record_error(GBS_ERR_CUDA, msg);
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GBS_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int gbs_cumulants_noalloc(const double *V, int M, int kmax, double *kappa_out, void *cuda_stream) {
    if (!gbs::valid_mk(M, kmax)) return gbs::record_error(GBS_ERR_INVALID_ARG, gbs::shape_message(M, kmax).c_str());
    if (!V || !kappa_out) return gbs::record_error(GBS_ERR_INVALID_ARG, "V and kappa_out must be non-NULL");
    if (((uintptr_t)V & 7) || ((uintptr_t)kappa_out & 7))
        return gbs::record_error(GBS_ERR_INVALID_ARG, "V and kappa_out must be 8-byte aligned");
    if (!on_device(V) || !on_device(kappa_out))
        return gbs::record_error(GBS_ERR_INVALID_ARG, "V and kappa_out must be CUDA device (or managed) memory");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return gbs::record_error(GBS_ERR_CUDA, "no CUDA device is current");
    // one scratch slot per multiprocessor: the default 512-thread schedule runs
    // at most one CTA per multiprocessor
    const gbs::WsLayout L = gbs::ws_layout(M, kmax, sms, 1);
    if (L.total > kNoallocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "M=%d kmax=%d needs %zu bytes of scratch; the allocation-free entry point holds %zu "
                 "(use gbs_cumulants with a caller workspace)",
                 M, kmax, L.total, kNoallocScratchBytes);
        return gbs::record_error(GBS_ERR_WORKSPACE, msg);
    }
    void *ws = nullptr;
    int rc = scratch_address(&ws);
    if (rc != GBS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    char *w = static_cast<char *>(ws);
    // the status word and the work counters must start at zero on every call
    cudaError_t e = cudaMemsetAsync(w + L.status_off, 0, 256, st);
    if (e != cudaSuccess) return gbs::record_error(GBS_ERR_CUDA, "cudaMemsetAsync on the scratch failed");
    gbs::FwdArgs a{};
    a.V = V;
    a.M = M;
    a.kmax = kmax;
    a.mode = gbs::MODE_KAPPA;
    a.precision = GBS_FP64;
    a.A = reinterpret_cast<double *>(w + L.A_off);
    a.Af = reinterpret_cast<float *>(a.A + 4 * (size_t)M * M);
    a.p0 = reinterpret_cast<double *>(w + L.p0_off);
    a.out = kappa_out;
    a.status = reinterpret_cast<unsigned *>(w + L.status_off);
    a.counters = a.status + 8;
    a.scratch = reinterpret_cast<double *>(w + L.scratch_off);
    a.slot_doubles = L.slot_doubles;
    a.slots = L.slots;
    a.sms = sms;
    a.ev = nullptr;
    a.variant = 0;
    e = gbs::launch_forward(a, st);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "kernel launch: %s", cudaGetErrorString(e));
        return gbs::record_error(GBS_ERR_CUDA, msg);
    }
    return gbs::record_error(GBS_OK, "");
}

extern "C" int gbs_noalloc_status(void *cuda_stream) {
    void *ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != GBS_OK) return rc;
    // the status word sits at the start of the scratch array (workspace layout offset 0)
    return gbs_stream_status(ws, cuda_stream);
}
