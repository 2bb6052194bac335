// Pipe-throughput probe (gbs_pipe_peaks): the sustained FMA rate of the FP64
// and FP32 pipes of the current GPU, the denominators of the arithmetic
// rooflines reported beside the kernels.
//
// Every thread runs kChains independent multiply-add chains for a fixed number
// of iterations, with enough resident warps per multiprocessor to hide the
// pipes' latency, so the rate is set by the pipe alone. Thread 0 of each block
// also reads the SM cycle counter and the global nanosecond timer at its start
// and end, which gives the SM clock the probe ran at.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "gbs.h"

namespace gbs {
int record_error(int code, const char *msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe(T x, T y, int iters, T *sink, unsigned long long *clk) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
    unsigned long long c0 = 0, t0 = 0;
    if (threadIdx.x == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if constexpr (sizeof(T) == 4) a[c] = __fmaf_rn(a[c], x, y);
            else a[c] = __fma_rn(a[c], x, y);
        }
    }
    T s = a[0];
#pragma unroll
    for (int c = 1; c < kChains; ++c) s += a[c];
    if (s == (T)-1.2345) sink[threadIdx.x] = s;  // keeps the chains live; never true for these inputs
    if (threadIdx.x == 0) {
        unsigned long long t1;
        const unsigned long long c1 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        clk[2 * blockIdx.x] = c1 - c0;
        clk[2 * blockIdx.x + 1] = t1 - t0;
    }
}

// Runs one probe: FMAs per second over the whole GPU and the median SM clock (MHz)
// seen by its blocks. scratch: device buffer of at least 2 * blocks words + 256 doubles.
template <typename T>
int run_probe(int sms, int iters, cudaStream_t st, void *scratch, double &fma_per_s, double &mhz) {
    const int blocks = sms * kBlocksPerSm;
    T *sink = reinterpret_cast<T *>(scratch);
    unsigned long long *clk = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(scratch) + 2048);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GBS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GBS_ERR_CUDA;
    }
    // a short warm-up launch (clocks ramp up), then the timed one
    fma_probe<T><<<blocks, kThreads, 0, st>>>((T)0.999, (T)1e-4, iters / 8 + 1, sink, clk);
    cudaEventRecord(e0, st);
    fma_probe<T><<<blocks, kThreads, 0, st>>>((T)0.999, (T)1e-4, iters, sink, clk);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0.f) return GBS_ERR_CUDA;
    std::vector<unsigned long long> h(2 * (size_t)blocks);
    if (cudaMemcpy(h.data(), clk, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GBS_ERR_CUDA;
    std::vector<double> f;
    for (int b = 0; b < blocks; ++b)
        if (h[2 * b + 1] > 0) f.push_back(1e3 * (double)h[2 * b] / (double)h[2 * b + 1]);
    std::sort(f.begin(), f.end());
    mhz = f.empty() ? 0.0 : f[f.size() / 2];
    fma_per_s = (double)blocks * kThreads * kChains * (double)iters / (1e-3 * ms);
    return GBS_OK;
}

}  // namespace

extern "C" int gbs_pipe_peaks(double *out, void *scratch, void *cuda_stream) {
    if (!out || !scratch) return gbs::record_error(GBS_ERR_INVALID_ARG, "NULL output or scratch");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return gbs::record_error(GBS_ERR_CUDA, "no CUDA device is current");
    if (sms * kBlocksPerSm * 2 * 8 + 2048 > GBS_PIPE_PEAKS_SCRATCH)
        return gbs::record_error(GBS_ERR_WORKSPACE, "more multiprocessors than the probe's scratch covers");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double f64 = 0, f32 = 0, mhz64 = 0, mhz32 = 0;
    // about 40 ms each on a 152-SM GB300
    int rc = run_probe<double>(sms, 1 << 14, st, scratch, f64, mhz64);
    if (rc == GBS_OK) rc = run_probe<float>(sms, 1 << 20, st, scratch, f32, mhz32);
    if (rc != GBS_OK) return gbs::record_error(rc, "probe launch failed");
    out[0] = 2.0 * f64;
    out[1] = 2.0 * f32;
    out[2] = mhz64 > 0 ? f64 / (sms * mhz64 * 1e6) : 0.0;
    out[3] = mhz32 > 0 ? f32 / (sms * mhz32 * 1e6) : 0.0;
    out[4] = mhz64;
    out[5] = mhz32;
    return gbs::record_error(GBS_OK, "");
}
