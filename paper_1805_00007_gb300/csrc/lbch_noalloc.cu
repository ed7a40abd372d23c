// lbch_noalloc.cu -- field statistics without any device allocation.
//
// lb_ch_observe reduces phi through per-block partial sums that live in device memory the handle
// allocated at lb_ch_init.  Some callers cannot allocate device memory at the point where they need
// these numbers: code running while another framework owns the device memory pool, or plugins that
// may only touch buffers handed to them.  lb_ch_field_stats_noalloc serves them: it reduces a field the
// caller owns into an output the caller owns, and keeps its partial sums in a fixed, file-scope
// device array instead of allocated memory.
//
// The partial sums are written to a static __device__ array of LBCH_NOALLOC_MAX_BLOCKS x 6 doubles
// (48 KiB) that every GPU which loads this library holds until the process exits.  Host code never
// uses the array's name as an address: at the first call on a device, with that device current, the
// entry point asks the runtime for the array's device address (cudaGetSymbolAddress) and caches it per
// device.  That first call should therefore happen before any stream capture.  All calls share the
// array; each call overwrites the slots it uses before reading them, so nothing needs clearing, but
// calls whose kernels overlap on the GPU (on different streams, say) race on it.
#include "lbch.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

namespace {

constexpr int NA_NT = 256;   // threads per block
constexpr int NA_NV = 6;     // sum phi, sum (phi - phi0)^2, sum phi0^2, max, min, non-finite count

__device__ __align__(256) double g_noalloc_partials[LBCH_NOALLOC_MAX_BLOCKS * NA_NV];

__device__ __forceinline__ void na_combine(double* a, const double* b)
{
    a[0] += b[0]; a[1] += b[1]; a[2] += b[2];
    a[3] = fmax(a[3], b[3]); a[4] = fmin(a[4], b[4]); a[5] += b[5];
}

// Reduce the 6 values of every thread of the block into thread 0 (warp shuffles, then one warp).
__device__ void na_block_reduce(double* v)
{
    __shared__ double sh[NA_NT / 32][NA_NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        double t[NA_NV];
        for (int k = 0; k < NA_NV; k++) t[k] = __shfl_down_sync(0xffffffffu, v[k], o);
        na_combine(v, t);
    }
    if (lane == 0)
        for (int k = 0; k < NA_NV; k++) sh[w][k] = v[k];
    __syncthreads();
    if (w == 0) {
        double t[NA_NV] = {0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
        if (lane < NA_NT / 32)
            for (int k = 0; k < NA_NV; k++) t[k] = sh[lane][k];
        for (int o = 16; o > 0; o >>= 1) {
            double u[NA_NV];
            for (int k = 0; k < NA_NV; k++) u[k] = __shfl_down_sync(0xffffffffu, t[k], o);
            na_combine(t, u);
        }
        for (int k = 0; k < NA_NV; k++) v[k] = t[k];
    }
}

// Pass 1: block b reduces the nodes b, b + nblocks, ... (in units of NA_NT) into partials[b].
__global__ void __launch_bounds__(NA_NT) na_partials_kernel(const double* phi, const double* phi0, int nx, int ny,
                                                            int pitch, double* partials)
{
    double v[NA_NV] = {0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    const long long N = (long long)nx * ny;
    for (long long k = (long long)blockIdx.x * NA_NT + threadIdx.x; k < N; k += (long long)gridDim.x * NA_NT) {
        int y = (int)(k / nx), x = (int)(k - (long long)y * nx);
        long long gi = (long long)y * pitch + x;
        double p = phi[gi], p0 = phi0[gi];
        if (!isfinite(p)) { v[5] += 1.0; continue; }
        v[0] += p; v[1] += (p - p0) * (p - p0); v[2] += p0 * p0;
        v[3] = fmax(v[3], p); v[4] = fmin(v[4], p);
    }
    na_block_reduce(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < NA_NV; k++) partials[(long long)blockIdx.x * NA_NV + k] = v[k];
}

// Pass 2: one block reduces the partials in a fixed order into the caller's output.
__global__ void __launch_bounds__(NA_NT) na_final_kernel(const double* partials, int nblocks, double* out)
{
    double v[NA_NV] = {0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += NA_NT) na_combine(v, partials + (long long)b * NA_NV);
    na_block_reduce(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < NA_NV; k++) out[k] = v[k];
}

// Device address of the partials array, looked up once per device (with that device current).
constexpr int kMaxDevices = 64;
double* g_partials_addr[kMaxDevices] = {nullptr};

}  // namespace

// Records the message that lb_ch_last_error() returns (defined with the rest of the runtime).
void lbch_set_last_error(const char* msg);

namespace {
lbch_status na_fail(lbch_status s, const char* msg)
{
    lbch_set_last_error(msg);
    return s;
}
}  // namespace

extern "C" {

lbch_status lb_ch_field_stats_noalloc(const double* phi, const double* phi0, int nx, int ny, int pitch,
                                      double* out, void* stream)
{
    char msg[256];
    if (!phi || !phi0 || !out) return na_fail(LBCH_EINVAL, "phi, phi0 and out must be device pointers");
    if (nx < 1 || ny < 1 || pitch < nx) {
        snprintf(msg, sizeof msg, "need nx, ny >= 1 and pitch >= nx (got %d, %d, %d)", nx, ny, pitch);
        return na_fail(LBCH_EINVAL, msg);
    }
    if ((long long)nx * ny > LBCH_NOALLOC_MAX_NODES) {
        snprintf(msg, sizeof msg, "field of %lld nodes exceeds the maximum of %lld nodes", (long long)nx * ny,
                 (long long)LBCH_NOALLOC_MAX_NODES);
        return na_fail(LBCH_EINVAL, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return na_fail(LBCH_ECUDA, "no usable current device");
    if (!g_partials_addr[dev]) {
        // set-up on this device: the device address of the static partials array
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            cudaGetLastError();
            return na_fail(LBCH_ECUDA, msg);
        }
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    long long N = (long long)nx * ny;
    int nblocks = (int)((N + NA_NT * 8 - 1) / (NA_NT * 8));
    if (nblocks > LBCH_NOALLOC_MAX_BLOCKS) nblocks = LBCH_NOALLOC_MAX_BLOCKS;
    if (nblocks < 1) nblocks = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    na_partials_kernel<<<nblocks, NA_NT, 0, s>>>(phi, phi0, nx, ny, pitch, g_partials_addr[dev]);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        na_final_kernel<<<1, NA_NT, 0, s>>>(g_partials_addr[dev], nblocks, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "kernel launch: %s", cudaGetErrorString(e));
        return na_fail(LBCH_ECUDA, msg);
    }
    return LBCH_OK;
}

}  // extern "C"
