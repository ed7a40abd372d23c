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
// uses the array's name as an address: the first call in a CUDA context (with that context's device
// current) asks the runtime for the array's device address (cudaGetSymbolAddress) and caches it under the
// context's unique ID, under a lock, so concurrent first calls from several host threads are safe and a
// context created later (after cudaDeviceReset, say) gets its own lookup.  That first call should
// happen before any stream capture.  All calls share the array; each call overwrites the slots it uses
// before reading them, so nothing needs clearing, but calls whose kernels overlap on the GPU (on
// different streams, say) race on it.
#include "lbch.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

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

// Device address of the partials array in each CUDA context it has been looked up in.  The key is the
// context's unique ID (cuCtxGetId), not its handle or the device ordinal: an address belongs to the context
// it was taken in, and a context created later (after cudaDeviceReset, say) may reuse an old handle value
// but never an old ID.
typedef int (*CtxGetCurrentFn)(void**);                      // cuCtxGetCurrent
typedef int (*CtxGetIdFn)(void*, unsigned long long*);        // cuCtxGetId
constexpr int kMaxContexts = 64;
struct AddrEntry { unsigned long long ctx_id; double* addr; };
AddrEntry g_addr[kMaxContexts];
int g_n_addr = 0;
std::mutex g_addr_mu;

void* driver_fn(const char* name)
{
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return p;
    return nullptr;
}

// The partials array's address in the current context (set-up on first use in that context).
cudaError_t partials_addr(double** out)
{
    static CtxGetCurrentFn get_ctx = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        get_ctx = reinterpret_cast<CtxGetCurrentFn>(driver_fn("cuCtxGetCurrent"));
        get_id = reinterpret_cast<CtxGetIdFn>(driver_fn("cuCtxGetId"));
    });
    *out = nullptr;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_ctx || !get_id || get_ctx(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) {
        // nothing to key on: look the address up on every call instead of caching it
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        *out = static_cast<double*>(p);
        return e;
    }
    std::lock_guard<std::mutex> lock(g_addr_mu);
    for (int i = 0; i < g_n_addr; i++)
        if (g_addr[i].ctx_id == id) { *out = g_addr[i].addr; return cudaSuccess; }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    if (g_n_addr < kMaxContexts) g_addr[g_n_addr++] = AddrEntry{id, static_cast<double*>(p)};
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

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
    if (e != cudaSuccess) return na_fail(LBCH_ECUDA, "no usable current device");
    double* partials = nullptr;
    e = partials_addr(&partials);  // set-up in this context: the device address of the static array
    if (e != cudaSuccess || !partials) {
        snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return na_fail(LBCH_ECUDA, msg);
    }
    cudaGetLastError();  // a launch error reported below is then this call's, not an earlier one left pending
    long long N = (long long)nx * ny;
    int nblocks = (int)((N + NA_NT * 8 - 1) / (NA_NT * 8));
    if (nblocks > LBCH_NOALLOC_MAX_BLOCKS) nblocks = LBCH_NOALLOC_MAX_BLOCKS;
    if (nblocks < 1) nblocks = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    na_partials_kernel<<<nblocks, NA_NT, 0, s>>>(phi, phi0, nx, ny, pitch, partials);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        na_final_kernel<<<1, NA_NT, 0, s>>>(partials, nblocks, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "kernel launch: %s", cudaGetErrorString(e));
        return na_fail(LBCH_ECUDA, msg);
    }
    return LBCH_OK;
}

}  // extern "C"
