// Host side of the libgbs C ABI (include/gbs.h): argument validation, workspace
// layout and kernel launches. No function here allocates device memory.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "gbs.h"
#include "gbs_common.cuh"
#include "gbs_fwd.cuh"
#include "gbs_bwd.cuh"
#include "gbs_batch.cuh"
#include "gbs_tune.cuh"

namespace {

thread_local char g_err[512] = "";

// Profiling events (gbs_timing): ev[0..1] around packing, ev[d+1] after order d.
bool g_timing = false;
bool g_timing_used = false;
cudaEvent_t g_ev[GBS_MAX_ORDER + 2];
bool g_ev_ready = false;
// Backward-pass events: ev[0] before the P0 recomputation, ev[i] after phase i.
bool g_bwd_timing_used = false;
cudaEvent_t g_bev[5];
bool g_bev_ready = false;

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int ok() {
    g_err[0] = '\0';
    return GBS_OK;
}

using gbs::valid_mk;
static_assert(GBS_MAX_ORDER == 5 && GBS_MAX_MODES == 1024 && GBS_MAX_MODES_K3 == 4096,
              "valid_mk (gbs_fwd.cuh) spells out the limits of gbs.h");

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

// True if p is memory the current device can dereference (device or managed).
bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Workspace of a range call: the forward layout, then the lower orders of the
// mode's table (the output slice holds only order kmax).
size_t range_low_off(const gbs::WsLayout &L) { return L.total; }
size_t range_total(const gbs::WsLayout &L, int M, int kmax) {
    return L.total + ((sizeof(double) * (size_t)gbs::order_offset(M, kmax) + 255) & ~(size_t)255);
}

int check_common(const double *V, int M, int kmax, const void *out, int precision, void *ws, size_t ws_bytes,
                 gbs::WsLayout &L, int &sms, bool range = false) {
    if (!valid_mk(M, kmax)) return fail(GBS_ERR_INVALID_ARG, "%s", gbs::shape_message(M, kmax).c_str());
    if (precision != GBS_FP64 && precision != GBS_FP32_REFINED)
        return fail(GBS_ERR_INVALID_ARG, "precision must be GBS_FP64 (0) or GBS_FP32_REFINED (1); got %d", precision);
    if (!V || !out || !ws) return fail(GBS_ERR_INVALID_ARG, "V, output and workspace must be non-NULL");
    if (((uintptr_t)V & 7) || ((uintptr_t)out & 7))
        return fail(GBS_ERR_INVALID_ARG, "V and the output must be 8-byte aligned");
    if ((uintptr_t)ws & 255) return fail(GBS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (!is_device_ptr(V) || !is_device_ptr(out) || !is_device_ptr(ws))
        return fail(GBS_ERR_INVALID_ARG, "V, output and workspace must be CUDA device (or managed) memory");
    sms = device_sms();
    if (sms <= 0) return fail(GBS_ERR_CUDA, "no CUDA device is current");
    L = gbs::ws_layout(M, kmax, sms);
    const size_t need = range ? range_total(L, M, kmax) : L.total;
    if (ws_bytes < need)
        return fail(GBS_ERR_WORKSPACE, "workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
    return GBS_OK;
}

// Top-element range [c_lo, c_hi) of a range call; c_hi < 0 = whole tables.
struct Range {
    int c_lo = 0, c_hi = -1;
    bool on() const { return c_hi >= 0; }
};

int run_forward(int mode, const double *V, int M, int kmax, double *out, int precision, void *ws, size_t ws_bytes,
                void *stream, const double *mean = nullptr, Range range = Range{}) {
    gbs::WsLayout L;
    int sms = 0;
    if (range.on() && (range.c_lo < 0 || range.c_lo > range.c_hi || range.c_hi > M))
        return fail(GBS_ERR_INVALID_ARG, "need 0 <= c_lo <= c_hi <= M; got c_lo=%d c_hi=%d M=%d", range.c_lo,
                    range.c_hi, M);
    int rc = check_common(V, M, kmax, out, precision, ws, ws_bytes, L, sms, range.on());
    if (rc != GBS_OK) return rc;
    if (mean && (((uintptr_t)mean & 7) || !is_device_ptr(mean)))
        return fail(GBS_ERR_INVALID_ARG, "mean must be 8-byte aligned CUDA device (or managed) memory");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(ws);
    if (gbs::fault_injected("forward_memset"))
        return fail(GBS_ERR_CUDA, "cudaMemsetAsync: injected failure (GBS_FAULT_INJECT=forward_memset)");
    cudaError_t e = cudaMemsetAsync(w + L.status_off, 0, 256, st);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    gbs::FwdArgs a{};
    a.V = V;
    a.mean = mean;
    a.M = M;
    a.kmax = kmax;
    a.mode = mode;
    a.precision = precision;
    a.A = reinterpret_cast<double *>(w + L.A_off);
    a.Af = reinterpret_cast<float *>(a.A + 4 * (size_t)M * M);
    a.p0f = reinterpret_cast<float *>(w + L.p0f_off);
    a.p0 = (mode == gbs::MODE_P0 && !range.on()) ? out : reinterpret_cast<double *>(w + L.p0_off);
    a.out = range.on() ? reinterpret_cast<double *>(w + range_low_off(L)) : out;
    if (range.on()) {
        a.top = out;
        a.top_base = gbs::order_offset(M, kmax) + gbs::binom(range.c_lo, kmax);
        a.c_lo = range.c_lo;
        a.c_hi = range.c_hi;
    }
    a.status = reinterpret_cast<unsigned *>(w + L.status_off);
    a.counters = a.status + 8;
    a.scratch = reinterpret_cast<double *>(w + L.scratch_off);
    a.slot_doubles = L.slot_doubles;
    a.slots = L.slots;
    a.sms = sms;
    a.ev = nullptr;
    const gbs::TreeCfg cfg = gbs::tuned_cfg(sms, M, kmax, precision);
    a.grain = cfg.grain;
    a.ccap = cfg.ccap;
    a.variant = cfg.variant;
    if (g_timing) {
        if (!g_ev_ready) {
            for (auto &ev : g_ev)
                if ((e = cudaEventCreate(&ev)) != cudaSuccess)
                    return fail(GBS_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
            g_ev_ready = true;
        }
        a.ev = g_ev;
        g_timing_used = true;
    }
    e = mean ? gbs::launch_forward_displaced(a, st) : gbs::launch_forward(a, st);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return ok();
}

}  // namespace

namespace gbs {
// Sets the message gbs_last_error() returns on this host thread; for entry
// points defined in other translation units of the library.
int record_error(int code, const char *msg) { return code == GBS_OK ? ok() : fail(code, "%s", msg); }

std::string shape_message(int M, int kmax) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "need 1 <= kmax <= min(M, %d) and M <= %d (kmax >= 4) or %d (kmax <= 3); got M=%d kmax=%d",
             GBS_MAX_ORDER, GBS_MAX_MODES, GBS_MAX_MODES_K3, M, kmax);
    return buf;
}
}  // namespace gbs

extern "C" {

uint64_t gbs_table_size(int M, int kmax) {
    if (!valid_mk(M, kmax)) return 0;
    return gbs::order_offset(M, kmax + 1);
}

uint64_t gbs_order_offset(int M, int d) {
    if (M < 1 || M > GBS_MAX_MODES_K3 || d < 1 || d > GBS_MAX_ORDER || d > M) return 0;
    return gbs::order_offset(M, d);
}

uint64_t gbs_rank(const int *modes, int d) {
    if (!modes || d < 1 || d > GBS_MAX_ORDER) return UINT64_MAX;
    uint64_t r = 0;
    for (int i = 0; i < d; ++i) {
        if (modes[i] < 0 || modes[i] >= GBS_MAX_MODES_K3 || (i > 0 && modes[i] <= modes[i - 1])) return UINT64_MAX;
        r += gbs::binom(modes[i], i + 1);
    }
    return r;
}

int gbs_unrank(uint64_t r, int d, int *modes_out) {
    if (!modes_out || d < 1 || d > GBS_MAX_ORDER) return fail(GBS_ERR_INVALID_ARG, "bad d or NULL output");
    if (r >= gbs::binom(GBS_MAX_MODES_K3, d)) return fail(GBS_ERR_INVALID_ARG, "rank out of range");
    for (int k = d; k >= 1; --k) {
        // largest c with C(c, k) <= r, by bisection over [k-1, GBS_MAX_MODES_K3)
        int lo = k - 1, hi = GBS_MAX_MODES_K3;
        while (hi - lo > 1) {
            const int mid = (lo + hi) / 2;
            if (gbs::binom(mid, k) <= r) lo = mid;
            else hi = mid;
        }
        modes_out[k - 1] = lo;
        r -= gbs::binom(lo, k);
    }
    return ok();
}

size_t gbs_workspace_bytes(int M, int kmax, int precision) {
    if (!valid_mk(M, kmax) || (precision != GBS_FP64 && precision != GBS_FP32_REFINED)) return 0;
    const int sms = device_sms();
    return gbs::ws_layout(M, kmax, sms > 0 ? sms : 1).total;
}

const char *gbs_last_error(void) { return g_err; }

int gbs_timing(int on) {
    g_timing = on != 0;
    return ok();
}

int gbs_timing_read(float *ms_out) {
    if (!ms_out) return fail(GBS_ERR_INVALID_ARG, "NULL output");
    if (!g_ev_ready || !g_timing_used) return fail(GBS_ERR_INVALID_ARG, "no timed call has been made");
    cudaError_t e = cudaEventSynchronize(g_ev[GBS_MAX_ORDER + 1]);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
    for (int i = 0; i <= GBS_MAX_ORDER; ++i) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, g_ev[i], g_ev[i + 1]);
        if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "cudaEventElapsedTime: %s", cudaGetErrorString(e));
        ms_out[i] = ms;
    }
    return ok();
}

int gbs_timing_read_backward(float *ms_out) {
    if (!ms_out) return fail(GBS_ERR_INVALID_ARG, "NULL output");
    if (!g_bev_ready || !g_bwd_timing_used) return fail(GBS_ERR_INVALID_ARG, "no timed backward call has been made");
    cudaError_t e = cudaEventSynchronize(g_bev[4]);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "cudaEventSynchronize: %s", cudaGetErrorString(e));
    for (int i = 0; i < 4; ++i) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, g_bev[i], g_bev[i + 1]);
        if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "cudaEventElapsedTime: %s", cudaGetErrorString(e));
        ms_out[i] = ms;
    }
    return ok();
}

int gbs_stream_status(const void *workspace, void *cuda_stream) {
    if (!workspace) return fail(GBS_ERR_INVALID_ARG, "NULL workspace");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
    unsigned s = 0;
    e = cudaMemcpy(&s, workspace, sizeof s, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "reading the status word: %s", cudaGetErrorString(e));
    return gbs_status_code(s);
}

int gbs_status_code(unsigned s) {
    if (s & gbs::ST_TIMEOUT) return fail(GBS_ERR_TIMEOUT, "a bounded device wait gave up");
    if (s & gbs::ST_NOT_POSDEF)
        return fail(GBS_ERR_NOT_POSDEF, "a reduced covariance (V_T + I)/2 is not positive definite");
    if (s & gbs::ST_BAD_INDEX) return fail(GBS_ERR_INVALID_ARG, "a device index check failed");
    return ok();
}

size_t gbs_backward_workspace_bytes(int M, int kmax) {
    if (!valid_mk(M, kmax) || M > GBS_MAX_MODES) return 0;
    const int sms = device_sms();
    return gbs::bwd_layout(M, kmax, sms > 0 ? sms : 1).total;
}

int gbs_cumulants_backward(const double *V, int M, int kmax, const double *grad_kappa, double *grad_V,
                           void *workspace, size_t ws_bytes, void *cuda_stream) {
    if (!valid_mk(M, kmax) || M > GBS_MAX_MODES)
        return fail(GBS_ERR_INVALID_ARG, "need 1 <= M <= %d and 1 <= kmax <= min(M, %d); got M=%d kmax=%d",
                    GBS_MAX_MODES, GBS_MAX_ORDER, M, kmax);
    if (!V || !grad_kappa || !grad_V || !workspace)
        return fail(GBS_ERR_INVALID_ARG, "V, grad_kappa, grad_V and workspace must be non-NULL");
    if (((uintptr_t)V & 7) || ((uintptr_t)grad_kappa & 7) || ((uintptr_t)grad_V & 7) || ((uintptr_t)workspace & 255))
        return fail(GBS_ERR_INVALID_ARG, "arrays must be 8-byte aligned and the workspace 256-byte aligned");
    if (!is_device_ptr(V) || !is_device_ptr(grad_kappa) || !is_device_ptr(grad_V) || !is_device_ptr(workspace))
        return fail(GBS_ERR_INVALID_ARG, "all arrays must be CUDA device (or managed) memory");
    const int sms = device_sms();
    if (sms <= 0) return fail(GBS_ERR_CUDA, "no CUDA device is current");
    const gbs::BwdLayout L = gbs::bwd_layout(M, kmax, sms);
    if (ws_bytes < L.total)
        return fail(GBS_ERR_WORKSPACE, "workspace too small: %zu bytes given, %zu needed", ws_bytes, L.total);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    char *w = static_cast<char *>(workspace);
    cudaError_t e = cudaMemsetAsync(w + L.fwd.status_off, 0, 256, st);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    gbs::BwdArgs b{};
    b.M = M;
    b.kmax = kmax;
    gbs::FwdArgs &a = b.fwd;
    a.V = V;
    a.M = M;
    a.kmax = kmax;
    a.mode = gbs::MODE_P0;
    a.precision = GBS_FP32_REFINED;  // the P0 recomputation (launch_backward)
    {
        const gbs::TreeCfg cfg = gbs::tuned_cfg(sms, M, kmax, GBS_FP32_REFINED);
        a.grain = cfg.grain;
        a.ccap = cfg.ccap;
        a.variant = cfg.variant;
    }
    a.A = reinterpret_cast<double *>(w + L.fwd.A_off);
    a.Af = reinterpret_cast<float *>(a.A + 4 * (size_t)M * M);
    a.status = reinterpret_cast<unsigned *>(w + L.fwd.status_off);
    a.counters = a.status + 8;
    a.scratch = reinterpret_cast<double *>(w + L.fwd.scratch_off);
    a.slot_doubles = L.fwd.slot_doubles;
    a.slots = L.fwd.slots;
    a.sms = sms;
    a.ev = nullptr;
    b.gk = grad_kappa;
    b.gV = grad_V;
    b.p0 = reinterpret_cast<double *>(w + L.p0_off);
    b.h = reinterpret_cast<double *>(w + L.h_off);
    b.gp0 = reinterpret_cast<double *>(w + L.gp0_off);
    b.inv = reinterpret_cast<double *>(w + L.inv_off);
    b.ev = nullptr;
    if (g_timing) {
        if (!g_bev_ready) {
            for (auto &ev : g_bev)
                if ((e = cudaEventCreate(&ev)) != cudaSuccess)
                    return fail(GBS_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
            g_bev_ready = true;
        }
        b.ev = g_bev;
        g_bwd_timing_used = true;
    }
    e = gbs::launch_backward(b, st);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return ok();
}

static int check_batch(const gbs_instance *inst, int n, int precision) {
    if (!inst || n < 1 || n > (1 << 20)) return fail(GBS_ERR_INVALID_ARG, "need a host array of 1..2^20 instances");
    if (precision != GBS_FP64 && precision != GBS_FP32_REFINED)
        return fail(GBS_ERR_INVALID_ARG, "precision must be GBS_FP64 (0) or GBS_FP32_REFINED (1); got %d", precision);
    for (int i = 0; i < n; ++i) {
        if (!valid_mk(inst[i].M, inst[i].kmax) || inst[i].M > GBS_MAX_MODES)
            return fail(GBS_ERR_INVALID_ARG, "instance %d: need 1 <= M <= %d and 1 <= kmax <= min(M, %d)", i,
                        GBS_MAX_MODES, GBS_MAX_ORDER);
        if (!inst[i].V || !inst[i].kappa_out || ((uintptr_t)inst[i].V & 7) || ((uintptr_t)inst[i].kappa_out & 7))
            return fail(GBS_ERR_INVALID_ARG, "instance %d: V and kappa_out must be non-NULL and 8-byte aligned", i);
    }
    return GBS_OK;
}

size_t gbs_batched_workspace_bytes(const gbs_instance *inst, int n, int precision) {
    if (check_batch(inst, n, precision) != GBS_OK) return 0;
    const int sms = device_sms();
    return gbs::batched_workspace_bytes(inst, n, precision, sms > 0 ? sms : 1);
}

int gbs_batched_plan(const gbs_instance *inst, int n, int precision, void *workspace, size_t ws_bytes,
                     void *cuda_stream) {
    int rc = check_batch(inst, n, precision);
    if (rc != GBS_OK) return rc;
    if (!workspace || ((uintptr_t)workspace & 255) || !is_device_ptr(workspace))
        return fail(GBS_ERR_INVALID_ARG, "workspace must be 256-byte aligned device memory");
    for (int i = 0; i < n; ++i)
        if (!is_device_ptr(inst[i].V) || !is_device_ptr(inst[i].kappa_out))
            return fail(GBS_ERR_INVALID_ARG, "instance %d: V and kappa_out must be device memory", i);
    const int sms = device_sms();
    if (sms <= 0) return fail(GBS_ERR_CUDA, "no CUDA device is current");
    size_t needed = 0;
    rc = gbs::batched_plan(inst, n, precision, static_cast<char *>(workspace), ws_bytes, sms,
                           static_cast<cudaStream_t>(cuda_stream), needed);
    if (rc == GBS_ERR_WORKSPACE)
        return fail(rc, "workspace too small: %zu bytes given, %zu needed", ws_bytes, needed);
    if (rc != GBS_OK) return fail(rc, "copying the batch plan failed");
    return ok();
}

int gbs_cumulants_batched(int precision, void *workspace, void *cuda_stream) {
    if (precision != GBS_FP64 && precision != GBS_FP32_REFINED)
        return fail(GBS_ERR_INVALID_ARG, "precision must be GBS_FP64 (0) or GBS_FP32_REFINED (1); got %d", precision);
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(GBS_ERR_INVALID_ARG, "workspace must be 256-byte aligned device memory");
    bool planned = false;
    cudaError_t e = gbs::launch_batched(static_cast<char *>(workspace), precision,
                                        static_cast<cudaStream_t>(cuda_stream), planned);
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "batched launch: %s", cudaGetErrorString(e));
    if (!planned)
        return fail(GBS_ERR_INVALID_ARG,
                    "the workspace holds no batch plan of this precision: call gbs_batched_plan first");
    return ok();
}

int gbs_batched_schedule(const void *workspace, int *schedule_out) {
    if (!workspace || !schedule_out) return fail(GBS_ERR_INVALID_ARG, "NULL workspace or output");
    if (!gbs::batched_schedule(workspace, schedule_out))
        return fail(GBS_ERR_INVALID_ARG, "the workspace holds no batch plan: call gbs_batched_plan first");
    return ok();
}

int gbs_batched_autotune(const gbs_instance *inst, int n, int precision, void *workspace, size_t ws_bytes,
                         void *cuda_stream, float *best_ms_out) {
    int rc = check_batch(inst, n, precision);
    if (rc != GBS_OK) return rc;
    if (!workspace || ((uintptr_t)workspace & 255) || !is_device_ptr(workspace))
        return fail(GBS_ERR_INVALID_ARG, "workspace must be 256-byte aligned device memory");
    for (int i = 0; i < n; ++i)
        if (!is_device_ptr(inst[i].V) || !is_device_ptr(inst[i].kappa_out))
            return fail(GBS_ERR_INVALID_ARG, "instance %d: V and kappa_out must be device memory", i);
    const int sms = device_sms();
    if (sms <= 0) return fail(GBS_ERR_CUDA, "no CUDA device is current");
    const size_t need = gbs::batched_workspace_bytes(inst, n, precision, sms);
    if (ws_bytes < need) return fail(GBS_ERR_WORKSPACE, "workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
    gbs::TreeCfg best;
    float ms = 0.f;
    int tried = 0;
    rc = gbs::batched_autotune(inst, n, precision, static_cast<char *>(workspace), ws_bytes, sms,
                               static_cast<cudaStream_t>(cuda_stream), best, ms, tried);
    if (rc != GBS_OK) return fail(rc, "batched autotuning failed");
    if (best_ms_out) *best_ms_out = ms;
    return ok();
}

int gbs_covariance(const double *U_re, const double *U_im, const double *r, const double *eta, int M,
                   double *V_out, void *cuda_stream) {
    if (M < 1 || M > GBS_MAX_MODES_K3) return fail(GBS_ERR_INVALID_ARG, "need 1 <= M <= %d", GBS_MAX_MODES_K3);
    const void *ptrs[] = {U_re, U_im, r, eta, V_out};
    for (const void *p : ptrs)
        if (!p || ((uintptr_t)p & 7) || !is_device_ptr(p))
            return fail(GBS_ERR_INVALID_ARG, "all arrays must be non-NULL, 8-byte aligned device memory");
    cudaError_t e = gbs::launch_covariance(U_re, U_im, r, eta, M, V_out, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return ok();
}

int gbs_covariance_backward(const double *U_re, const double *U_im, const double *r, const double *eta, int M,
                            const double *V, const double *grad_V, double *grad_r, double *grad_eta,
                            void *cuda_stream) {
    if (M < 1 || M > GBS_MAX_MODES_K3) return fail(GBS_ERR_INVALID_ARG, "need 1 <= M <= %d", GBS_MAX_MODES_K3);
    const void *ptrs[] = {U_re, U_im, r, eta, V, grad_V, grad_r, grad_eta};
    for (const void *p : ptrs)
        if (!p || ((uintptr_t)p & 7) || !is_device_ptr(p))
            return fail(GBS_ERR_INVALID_ARG, "all arrays must be non-NULL, 8-byte aligned device memory");
    cudaError_t e = gbs::launch_covariance_bwd(U_re, U_im, r, eta, M, V, grad_V, grad_r, grad_eta,
                                               static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return fail(GBS_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return ok();
}

int gbs_autotune(const double *V, int M, int kmax, double *kappa_out, int precision, void *workspace,
                 size_t ws_bytes, void *cuda_stream, float *best_ms_out) {
    gbs::WsLayout L;
    int sms = 0;
    int rc = check_common(V, M, kmax, kappa_out, precision, workspace, ws_bytes, L, sms);
    if (rc != GBS_OK) return rc;
    char *w = static_cast<char *>(workspace);
    gbs::FwdArgs a{};
    a.V = V;
    a.M = M;
    a.kmax = kmax;
    a.mode = gbs::MODE_KAPPA;
    a.precision = precision;
    a.A = reinterpret_cast<double *>(w + L.A_off);
    a.Af = reinterpret_cast<float *>(a.A + 4 * (size_t)M * M);
    a.p0f = reinterpret_cast<float *>(w + L.p0f_off);
    a.p0 = reinterpret_cast<double *>(w + L.p0_off);
    a.out = kappa_out;
    a.status = reinterpret_cast<unsigned *>(w + L.status_off);
    a.counters = a.status + 8;
    a.scratch = reinterpret_cast<double *>(w + L.scratch_off);
    a.slot_doubles = L.slot_doubles;
    a.slots = L.slots;
    a.sms = sms;
    a.ev = nullptr;
    gbs::TreeCfg best;
    float ms = 0.f;
    int tried = 0;
    rc = gbs::autotune(a, static_cast<cudaStream_t>(cuda_stream), best, ms, tried);
    if (rc != GBS_OK) return fail(rc, "autotuning launch failed");
    if (best_ms_out) *best_ms_out = ms;
    return ok();
}

int gbs_schedule(int M, int kmax, int precision, int *schedule_out) {
    if (!schedule_out) return fail(GBS_ERR_INVALID_ARG, "schedule_out is NULL");
    if (!valid_mk(M, kmax)) return fail(GBS_ERR_INVALID_ARG, "%s", gbs::shape_message(M, kmax).c_str());
    if (precision != GBS_FP64 && precision != GBS_FP32_REFINED)
        return fail(GBS_ERR_INVALID_ARG, "precision must be GBS_FP64 or GBS_FP32_REFINED");
    const int sms = device_sms();
    if (sms <= 0) return fail(GBS_ERR_CUDA, "no current CUDA device");
    const gbs::TreeCfg cfg = gbs::tuned_cfg(sms, M, kmax, precision);
    schedule_out[0] = gbs::effective_variant(cfg.variant, M, precision);
    schedule_out[1] = cfg.grain > 0 ? cfg.grain : gbs::kDefaultCfg.grain;
    schedule_out[2] = cfg.ccap > 0 && cfg.ccap <= gbs::kMaxChildren ? cfg.ccap : gbs::kDefaultCfg.ccap;
    if (schedule_out[0] == 9 && schedule_out[2] > gbs::kNoSlotCC) schedule_out[2] = gbs::kNoSlotCC;
    return ok();
}

int gbs_vacuum_probs(const double *V, int M, int kmax, double *p0_out, int precision, void *workspace,
                     size_t ws_bytes, void *cuda_stream) {
    return run_forward(gbs::MODE_P0, V, M, kmax, p0_out, precision, workspace, ws_bytes, cuda_stream);
}

int gbs_click_moments(const double *V, int M, int kmax, double *mu_out, int precision, void *workspace,
                      size_t ws_bytes, void *cuda_stream) {
    return run_forward(gbs::MODE_MU, V, M, kmax, mu_out, precision, workspace, ws_bytes, cuda_stream);
}

int gbs_cumulants(const double *V, int M, int kmax, double *kappa_out, int precision, void *workspace,
                  size_t ws_bytes, void *cuda_stream) {
    return run_forward(gbs::MODE_KAPPA, V, M, kmax, kappa_out, precision, workspace, ws_bytes, cuda_stream);
}

int gbs_spin_correlators(const double *V, int M, int kmax, double *c_out, int precision, void *workspace,
                         size_t ws_bytes, void *cuda_stream) {
    return run_forward(gbs::MODE_SPINC, V, M, kmax, c_out, precision, workspace, ws_bytes, cuda_stream);
}

int gbs_spin_cumulants(const double *V, int M, int kmax, double *kappa_out, int precision, void *workspace,
                       size_t ws_bytes, void *cuda_stream) {
    return run_forward(gbs::MODE_SPINK, V, M, kmax, kappa_out, precision, workspace, ws_bytes, cuda_stream);
}

size_t gbs_range_workspace_bytes(int M, int kmax, int precision) {
    if (!valid_mk(M, kmax) || (precision != GBS_FP64 && precision != GBS_FP32_REFINED)) return 0;
    const int sms = device_sms();
    return range_total(gbs::ws_layout(M, kmax, sms > 0 ? sms : 1), M, kmax);
}

uint64_t gbs_range_entries(int M, int kmax, int c_lo, int c_hi) {
    if (!valid_mk(M, kmax) || c_lo < 0 || c_lo > c_hi || c_hi > M) return 0;
    return gbs::binom(c_hi, kmax) - gbs::binom(c_lo, kmax);
}

int gbs_range_split(int M, int kmax, int n_parts, int *bounds_out) {
    if (!valid_mk(M, kmax)) return fail(GBS_ERR_INVALID_ARG, "%s", gbs::shape_message(M, kmax).c_str());
    if (n_parts < 1 || n_parts > M || !bounds_out)
        return fail(GBS_ERR_INVALID_ARG, "need 1 <= n_parts <= M and a host array of n_parts + 1 ints");
    const uint64_t total = gbs::binom(M, kmax);
    bounds_out[0] = 0;
    int c = 0;
    for (int i = 1; i < n_parts; ++i) {
        // smallest c with C(c, kmax) >= i * total / n_parts (128-bit product: no overflow)
        const uint64_t goal = (uint64_t)(((unsigned __int128)total * (unsigned)i) / (unsigned)n_parts);
        while (c < M && gbs::binom(c, kmax) < goal) ++c;
        bounds_out[i] = c;
    }
    bounds_out[n_parts] = M;
    return ok();
}

int gbs_table_range(const double *V, int M, int kmax, int table, int c_lo, int c_hi, double *out, int precision,
                    void *workspace, size_t ws_bytes, void *cuda_stream) {
    if (table < GBS_TABLE_P0 || table > GBS_TABLE_SPIN_CUMULANT)
        return fail(GBS_ERR_INVALID_ARG, "table must be one of the gbs_table values; got %d", table);
    if (c_hi < 0) return fail(GBS_ERR_INVALID_ARG, "need 0 <= c_lo <= c_hi <= M; got c_hi=%d", c_hi);
    Range r;
    r.c_lo = c_lo;
    r.c_hi = c_hi;
    return run_forward(table, V, M, kmax, out, precision, workspace, ws_bytes, cuda_stream, nullptr, r);
}

int gbs_displaced_tables(const double *V, const double *mean, int M, int kmax, int table, double *out,
                         void *workspace, size_t ws_bytes, void *cuda_stream) {
    if (!mean) return fail(GBS_ERR_INVALID_ARG, "mean must be non-NULL (use the zero-mean entry points otherwise)");
    if (table < GBS_TABLE_P0 || table > GBS_TABLE_SPIN_CUMULANT)
        return fail(GBS_ERR_INVALID_ARG, "table must be one of the gbs_table values; got %d", table);
    static_assert(GBS_TABLE_P0 == gbs::MODE_P0 && GBS_TABLE_CLICK_MOMENT == gbs::MODE_MU &&
                      GBS_TABLE_CLICK_CUMULANT == gbs::MODE_KAPPA && GBS_TABLE_SPIN_CORRELATOR == gbs::MODE_SPINC &&
                      GBS_TABLE_SPIN_CUMULANT == gbs::MODE_SPINK,
                  "table numbering follows the kernel modes");
    return run_forward(table, V, M, kmax, out, GBS_FP64, workspace, ws_bytes, cuda_stream, mean);
}

}  // extern "C"
