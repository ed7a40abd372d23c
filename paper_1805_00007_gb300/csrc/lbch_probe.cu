// lbch_probe.cu -- fused multiply-add throughput of the device in FP32 or FP64 (a measurement helper for
// the arithmetic rooflines reported beside the step; the paper has no counterpart).
#include <cuda_runtime.h>

#include <cstdio>

#include "lbch.h"

__attribute__((visibility("hidden"))) void lbch_set_last_error(const char* msg);

namespace {

constexpr int kChains = 8;   // independent dependency chains per thread
constexpr int kThreads = 256;

// Every thread runs kChains chains of `iters` FMAs x <- x a + b; the sum is stored only if it takes a value
// it never takes, so the work is kept and nothing is written.
template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T* sink, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    if (s == T(-1.25e30)) sink[0] = s;
}

template <typename T>
cudaError_t time_probe(cudaStream_t st, int blocks, int iters, T* sink, float* ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        fma_probe_kernel<T><<<blocks, kThreads, 0, st>>>(sink, iters, T(0.999), T(1e-4));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

template <typename T>
cudaError_t probe(cudaStream_t st, double* out)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<T>, kThreads, 0);
    if (e != cudaSuccess) return e;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    T* sink = nullptr;
    e = cudaMalloc(&sink, sizeof(T));
    if (e != cudaSuccess) return e;
    // a short run sizes the measured one to about 20 ms; the faster of three measured runs counts
    float ms = 0.0f;
    int iters = 256;
    e = time_probe<T>(st, blocks, iters, sink, &ms);
    if (e == cudaSuccess && ms > 0.0f) {
        const double scale = 20.0 / (double)ms;
        iters = (int)(iters * (scale < 1.0 ? 1.0 : (scale > 4.0e5 ? 4.0e5 : scale)));
    }
    float best = 0.0f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
        e = time_probe<T>(st, blocks, iters, sink, &ms);
        if (e == cudaSuccess && (rep == 0 || ms < best)) best = ms;
    }
    cudaFree(sink);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
    *out = flops / (best * 1e-3);
    return cudaSuccess;
}

}  // namespace

extern "C" lbch_status lb_ch_alu_peak(int prec, void* stream, double* flop_per_s)
{
    if (!flop_per_s || (prec != LBCH_F32 && prec != LBCH_F64)) {
        lbch_set_last_error("lb_ch_alu_peak: prec must be LBCH_F32 or LBCH_F64, and the output non-NULL");
        return LBCH_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = prec == LBCH_F64 ? probe<double>(st, flop_per_s) : probe<float>(st, flop_per_s);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "lb_ch_alu_peak: %s", cudaGetErrorString(e));
        lbch_set_last_error(msg);
        return LBCH_ECUDA;
    }
    return LBCH_OK;
}
