// lbch_api.cu -- host runtime of the C ABI declared in include/lbch.h.
//
// Owns the device state of a handle (ping-pong population planes and phi, the instance table, the step
// counter, reduction scratch), derives the model constants from the parameters (Eqs. betakappa, rho,
// F2-1, the mobility relation after Eq. phit3 and the Peclet number of Sec. III.A), launches the step
// kernel -- replayed from CUDA graphs of 64 steps -- and the reductions behind lb_ch_observe.
#include "lbch.h"
#include "lbch_kernels.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

using namespace lbch;

namespace {

thread_local char g_msg[512] = "";

lbch_status fail(lbch_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return s;
}

lbch_status cuda_fail(cudaError_t e, const char* what)
{
    cudaGetLastError();  // clear a sticky-free error so later calls on this thread are not confused
    return fail(e == cudaErrorMemoryAllocation ? LBCH_ENOMEM : LBCH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

constexpr int kGraphChunk = 64;  // steps per captured graph (even, so the ping-pong parity is preserved)

// Tile shapes of the step kernel per precision (output nodes per block; 256 threads).
constexpr int TX64 = 32, TY64 = 8;
constexpr int TX32 = 32, TY32 = 16;
constexpr int NT = 256;

}  // namespace

struct lbch_handle {
    int device = 0;
    int prec = LBCH_F64;
    int n_inst = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<InstDev> inst;
    InstDev* d_inst = nullptr;
    long long plane = 0;        // elements per population plane (all instances, padded)
    long long nodes = 0;        // lattice nodes (all instances, unpadded)
    int total_tiles = 0;
    int n_planes = 9;           // stored population planes
    size_t g_elem = 8, phi_elem = 8;
    void* g[2] = {nullptr, nullptr};
    void* phi[2] = {nullptr, nullptr};
    double* phi0 = nullptr;     // initial field, double, pitched like phi
    Ctl* ctl = nullptr;
    double* partials = nullptr; // reduction scratch: n_inst * chunks * RED_NV doubles
    double* result = nullptr;   // n_inst * RED_NV doubles
    int chunks = 0;
    long long n = 0;            // host mirror of the step index
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double* h_stage = nullptr;  // pinned host staging for observations
    size_t h_stage_bytes = 0;
};

namespace {

template <typename C, typename S, typename P, int TX, int TY>
cudaError_t launch_step_t(lbch_handle* h, int parity)
{
    using L = TileSmem<TX, TY, C>;
    auto kern = ch_step_kernel<C, S, P, TX, TY, NT>;
    StepArgs<S, P> a;
    a.inst = h->d_inst;
    a.n_inst = h->n_inst;
    a.total_tiles = h->total_tiles;
    a.plane = h->plane;
    a.g_in = static_cast<const S*>(h->g[parity]);
    a.g_out = static_cast<S*>(h->g[parity ^ 1]);
    a.phi_in = static_cast<const P*>(h->phi[parity]);
    a.phi_out = static_cast<P*>(h->phi[parity ^ 1]);
    a.ctl = h->ctl;
    kern<<<h->total_tiles, NT, L::bytes, h->stream>>>(a);
    return cudaGetLastError();
}

// Allow the step kernel of this handle's precision its dynamic shared memory (on the current device).
template <typename C, typename S, typename P, int TX, int TY>
cudaError_t prepare_step_t()
{
    return cudaFuncSetAttribute(ch_step_kernel<C, S, P, TX, TY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TileSmem<TX, TY, C>::bytes);
}

cudaError_t prepare_step(int prec)
{
    switch (prec) {
    case LBCH_F64: return prepare_step_t<double, double, double, TX64, TY64>();
    case LBCH_F32: return prepare_step_t<float, float, float, TX32, TY32>();
    default: return prepare_step_t<float, __half, float, TX32, TY32>();
    }
}

cudaError_t launch_step(lbch_handle* h, int parity)
{
    switch (h->prec) {
    case LBCH_F64: return launch_step_t<double, double, double, TX64, TY64>(h, parity);
    case LBCH_F32: return launch_step_t<float, float, float, TX32, TY32>(h, parity);
    default: return launch_step_t<float, __half, float, TX32, TY32>(h, parity);
    }
}

void tile_shape(int prec, int& tx, int& ty)
{
    if (prec == LBCH_F64) { tx = TX64; ty = TY64; } else { tx = TX32; ty = TY32; }
}

lbch_status check_params(const lbch_params& p, int k)
{
    if (p.nx < 4 || p.ny < 4 || p.nx > (1 << 20) || p.ny > (1 << 20))
        return fail(LBCH_EINVAL, "instance %d: nx, ny must be in [4, 2^20] (got %d x %d)", k, p.nx, p.ny);
    if (!(p.tau > 0.5)) return fail(LBCH_EINVAL, "instance %d: tau must exceed 1/2", k);
    if (p.model != 1 && p.model != 2) return fail(LBCH_EINVAL, "instance %d: model must be 1 or 2", k);
    if (p.vel < 0 || p.vel > 5) return fail(LBCH_EINVAL, "instance %d: unknown velocity field %d", k, p.vel);
    if (p.walls != 0 && p.walls != 1) return fail(LBCH_EINVAL, "instance %d: walls must be 0 or 1", k);
    if (p.phiA == p.phiB) return fail(LBCH_EINVAL, "instance %d: phiA == phiB", k);
    if (!(p.W > 0.0) || !(p.sigma >= 0.0)) return fail(LBCH_EINVAL, "instance %d: need W > 0, sigma >= 0", k);
    if (!(p.M > 0.0) && !(p.Pe > 0.0 && p.Ustar > 0.0 && p.sigma > 0.0))
        return fail(LBCH_EINVAL, "instance %d: give M > 0, or Pe > 0 and Ustar > 0", k);
    if ((p.vel == LBCH_VEL_VORTEX || p.vel == LBCH_VEL_DEFORM || p.vel == LBCH_VEL_REV_SHEAR) && !(p.Tper > 0.0))
        return fail(LBCH_EINVAL, "instance %d: time-dependent flow needs Tper > 0", k);
    if (p.vel == LBCH_VEL_ROTATION && !(p.half > 0.0)) return fail(LBCH_EINVAL, "instance %d: rotation needs half > 0", k);
    return LBCH_OK;
}

// Derived constants of the model for one instance.
void derive(const lbch_params& p, InstDev& d)
{
    const double cs2 = 1.0 / 3.0;
    const double dphi = std::fabs(p.phiA - p.phiB);
    d.beta = 12.0 * p.sigma / (p.W * dphi * dphi * dphi * dphi);      // Eq. betakappa
    d.kappa = 3.0 * p.sigma * p.W / (2.0 * dphi * dphi);
    double M = p.M > 0.0 ? p.M
                         : p.Ustar * p.W / (p.Pe * d.beta * (p.phiA - p.phiB) * (p.phiA - p.phiB));  // Pe, Sec. III.A
    d.eta = M / (cs2 * (p.tau - 0.5));                                  // M = c_s^2 eta (tau - 1/2)
    d.a = (p.rhoA - p.rhoB) / (p.phiA - p.phiB);                        // Eq. rho
    d.b = (p.rhoB * p.phiA - p.phiB * p.rhoA) / (p.phiA - p.phiB);
    d.K = (p.tau - 1.0 / 6.0 - p.tau * p.tau) / (p.tau - 0.5);          // Eq. F2-1
    d.tau = p.tau;
    d.phiA = p.phiA; d.phiB = p.phiB;
    d.U0 = p.U0; d.ux0 = p.ux0; d.uy0 = p.uy0; d.xc = p.xc; d.yc = p.yc; d.half = p.half;
    d.Tper = p.Tper; d.shear = p.shear;
    d.walls = p.walls; d.model = p.model; d.vel = p.vel; d.nvort = p.nvort;
}

void release(lbch_handle* h)
{
    for (int k = 0; k < 2; k++) {
        if (h->graph[k]) cudaGraphExecDestroy(h->graph[k]);
        if (h->g[k]) cudaFree(h->g[k]);
        if (h->phi[k]) cudaFree(h->phi[k]);
    }
    if (h->d_inst) cudaFree(h->d_inst);
    if (h->phi0) cudaFree(h->phi0);
    if (h->ctl) cudaFree(h->ctl);
    if (h->partials) cudaFree(h->partials);
    if (h->result) cudaFree(h->result);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

lbch_status stage(lbch_handle* h, size_t bytes)
{
    if (h->h_stage_bytes >= bytes) return LBCH_OK;
    if (h->h_stage) cudaFreeHost(h->h_stage);
    h->h_stage = nullptr;
    h->h_stage_bytes = 0;
    CK(cudaMallocHost(&h->h_stage, bytes));
    h->h_stage_bytes = bytes;
    return LBCH_OK;
}

lbch_status run_reduce(lbch_handle* h)
{
    int parity = (int)(h->n & 1);
    dim3 grid(h->chunks, h->n_inst);
    if (h->prec == LBCH_F64)
        reduce_partials_kernel<double><<<grid, RED_NT, 0, h->stream>>>(h->d_inst, (const double*)h->phi[parity], h->phi0, h->partials, h->chunks);
    else
        reduce_partials_kernel<float><<<grid, RED_NT, 0, h->stream>>>(h->d_inst, (const float*)h->phi[parity], h->phi0, h->partials, h->chunks);
    CK(cudaGetLastError());
    reduce_final_kernel<<<h->n_inst, RED_NT, 0, h->stream>>>(h->partials, h->chunks, h->result);
    CK(cudaGetLastError());
    return LBCH_OK;
}

}  // namespace

extern "C" {

lbch_status lb_ch_init(const lbch_params* params, int n_inst, const double* phi0, int prec, void* stream,
                       lbch_handle** out)
{
    if (!out) return fail(LBCH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || !phi0 || n_inst < 1) return fail(LBCH_EINVAL, "params/phi0 NULL or n_inst < 1");
    if (prec != LBCH_F64 && prec != LBCH_F32 && prec != LBCH_F16S) return fail(LBCH_EINVAL, "unknown precision %d", prec);
    for (int k = 0; k < n_inst; k++) {
        lbch_status s = check_params(params[k], k);
        if (s != LBCH_OK) return s;
    }
    lbch_handle* h = new (std::nothrow) lbch_handle();
    if (!h) return fail(LBCH_ENOMEM, "host allocation failed");
    h->prec = prec;
    h->n_inst = n_inst;
    h->g_elem = prec == LBCH_F64 ? 8 : (prec == LBCH_F32 ? 4 : 2);
    h->phi_elem = prec == LBCH_F64 ? 8 : 4;
    h->n_planes = prec == LBCH_F16S ? 8 : 9;
    int tx, ty;
    tile_shape(prec, tx, ty);

    // instance table: rows padded to 32 elements, each instance's block aligned to 64 elements
    h->inst.resize(n_inst);
    long long off = 0;
    int tiles = 0;
    for (int k = 0; k < n_inst; k++) {
        const lbch_params& p = params[k];
        InstDev& d = h->inst[k];
        std::memset(&d, 0, sizeof d);
        derive(p, d);
        d.nx = p.nx;
        d.ny = p.ny;
        d.pitch = (p.nx + 31) / 32 * 32;
        d.off = off;
        d.tiles_x = (p.nx + tx - 1) / tx;
        d.tiles_y = (p.ny + ty - 1) / ty;
        d.tile_begin = tiles;
        tiles += d.tiles_x * d.tiles_y;
        off += ((long long)d.pitch * p.ny + 63) / 64 * 64;
        h->nodes += (long long)p.nx * p.ny;
    }
    h->plane = off;
    h->total_tiles = tiles;

    auto bail = [&](lbch_status s) { release(h); delete h; return s; };
    cudaError_t e;
#define CKI(call)                                                    \
    do {                                                             \
        e = (call);                                                  \
        if (e != cudaSuccess) return bail(cuda_fail(e, #call));      \
    } while (0)
    CKI(cudaGetDevice(&h->device));
    CKI(prepare_step(prec));
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        CKI(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    size_t gbytes = (size_t)h->plane * h->n_planes * h->g_elem;
    size_t pbytes = (size_t)h->plane * h->phi_elem;
    for (int k = 0; k < 2; k++) {
        CKI(cudaMalloc(&h->g[k], gbytes));
        CKI(cudaMalloc(&h->phi[k], pbytes));
    }
    CKI(cudaMalloc(&h->phi0, (size_t)h->plane * sizeof(double)));
    CKI(cudaMalloc(&h->d_inst, sizeof(InstDev) * n_inst));
    CKI(cudaMalloc(&h->ctl, sizeof(Ctl)));
    long long max_nodes = 0;
    for (auto& d : h->inst) max_nodes = std::max(max_nodes, (long long)d.nx * d.ny);
    h->chunks = (int)std::min<long long>(1024, (max_nodes + RED_NT * 8 - 1) / (RED_NT * 8));
    if (h->chunks < 1) h->chunks = 1;
    CKI(cudaMalloc(&h->partials, sizeof(double) * RED_NV * (size_t)h->chunks * n_inst));
    CKI(cudaMalloc(&h->result, sizeof(double) * RED_NV * (size_t)n_inst));

    // upload the initial field, pitched, through pinned staging
    lbch_status s = stage(h, (size_t)h->plane * sizeof(double));
    if (s != LBCH_OK) return bail(s);
    std::memset(h->h_stage, 0, (size_t)h->plane * sizeof(double));
    const double* src = phi0;
    for (int k = 0; k < n_inst; k++) {
        const InstDev& d = h->inst[k];
        for (int j = 0; j < d.ny; j++)
            std::memcpy(h->h_stage + d.off + (long long)j * d.pitch, src + (long long)j * d.nx, sizeof(double) * d.nx);
        src += (long long)d.nx * d.ny;
    }
    CKI(cudaMemcpyAsync(h->phi0, h->h_stage, (size_t)h->plane * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CKI(cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(InstDev) * n_inst, cudaMemcpyHostToDevice, h->stream));
    CKI(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
    for (int k = 0; k < 2; k++) {
        CKI(cudaMemsetAsync(h->g[k], 0, gbytes, h->stream));
        CKI(cudaMemsetAsync(h->phi[k], 0, pbytes, h->stream));
    }
    int nb = (int)((h->plane + 255) / 256);
    switch (prec) {
    case LBCH_F64:
        init_kernel<double, double, double><<<nb, 256, 0, h->stream>>>(h->d_inst, n_inst, h->phi0, h->plane,
                                                                     (double*)h->g[0], (double*)h->phi[0], h->plane);
        break;
    case LBCH_F32:
        init_kernel<float, float, float><<<nb, 256, 0, h->stream>>>(h->d_inst, n_inst, h->phi0, h->plane,
                                                                  (float*)h->g[0], (float*)h->phi[0], h->plane);
        break;
    default:
        init_kernel<float, __half, float><<<nb, 256, 0, h->stream>>>(h->d_inst, n_inst, h->phi0, h->plane,
                                                                   (__half*)h->g[0], (float*)h->phi[0], h->plane);
    }
    CKI(cudaGetLastError());
    CKI(cudaStreamSynchronize(h->stream));  // the pinned staging buffer is reused after this point
#undef CKI
    *out = h;
    return LBCH_OK;
}

lbch_status lb_ch_step(lbch_handle* h, long nsteps)
{
    if (!h || nsteps < 0) return fail(LBCH_EINVAL, "NULL handle or negative step count");
    static const bool no_graph = std::getenv("LBCH_NO_GRAPH") != nullptr;
    while (nsteps > 0) {
        int parity = (int)(h->n & 1);
        if (!no_graph && nsteps >= kGraphChunk) {
            if (!h->graph[parity]) {
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = cudaSuccess;
                for (int s = 0; s < kGraphChunk && e == cudaSuccess; s++) e = launch_step(h, parity ^ (s & 1));
                cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
                if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "step launch during capture"); }
                if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&h->graph[parity], g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) { h->graph[parity] = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
            }
            CK(cudaGraphLaunch(h->graph[parity], h->stream));
            h->n += kGraphChunk;
            nsteps -= kGraphChunk;
        } else {
            CK(launch_step(h, parity));
            h->n += 1;
            nsteps -= 1;
        }
    }
    return LBCH_OK;
}

lbch_status lb_ch_observe(lbch_handle* h, int inst, int what, double* out)
{
    if (!h || !out) return fail(LBCH_EINVAL, "NULL handle or output");
    if (inst < 0 || inst >= h->n_inst) return fail(LBCH_EINVAL, "instance %d out of range", inst);
    if (what == LBCH_OBS_STEP) {
        *out = (double)h->n;
        return LBCH_OK;
    }
    if (what == LBCH_OBS_PHI) {
        const InstDev& d = h->inst[inst];
        int parity = (int)(h->n & 1);
        lbch_status s = stage(h, (size_t)d.nx * d.ny * sizeof(double));
        if (s != LBCH_OK) return s;
        const char* base = static_cast<const char*>(h->phi[parity]) + (size_t)d.off * h->phi_elem;
        CK(cudaMemcpy2DAsync(h->h_stage, (size_t)d.nx * h->phi_elem, base, (size_t)d.pitch * h->phi_elem,
                             (size_t)d.nx * h->phi_elem, d.ny, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        long long N = (long long)d.nx * d.ny;
        bool finite = true;
        if (h->phi_elem == 8) {
            std::memcpy(out, h->h_stage, sizeof(double) * N);
        } else {
            const float* f = reinterpret_cast<const float*>(h->h_stage);
            for (long long k = 0; k < N; k++) out[k] = (double)f[k];
        }
        for (long long k = 0; k < N; k++) finite = finite && std::isfinite(out[k]);
        return finite ? LBCH_OK : fail(LBCH_ENONFINITE, "phi holds non-finite values");
    }
    if (what < LBCH_OBS_MASS || what > LBCH_OBS_MIN) return fail(LBCH_EINVAL, "unknown observable %d", what);
    lbch_status s = run_reduce(h);
    if (s != LBCH_OK) return s;
    double r[RED_NV];
    CK(cudaMemcpyAsync(r, h->result + (size_t)inst * RED_NV, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    switch (what) {
    case LBCH_OBS_MASS: *out = r[0]; break;
    case LBCH_OBS_ERR_L2: *out = std::sqrt(r[1] / r[2]); break;
    case LBCH_OBS_MAX: *out = r[3]; break;
    default: *out = r[4]; break;
    }
    return r[5] > 0.0 ? fail(LBCH_ENONFINITE, "phi holds %.0f non-finite values", r[5]) : LBCH_OK;
}

lbch_status lb_ch_observe_all(lbch_handle* h, int what, double* out)
{
    if (!h || !out) return fail(LBCH_EINVAL, "NULL handle or output");
    if (what < LBCH_OBS_MASS || what > LBCH_OBS_MIN) return fail(LBCH_EINVAL, "observable %d is not a scalar", what);
    lbch_status s = run_reduce(h);
    if (s != LBCH_OK) return s;
    std::vector<double> r((size_t)RED_NV * h->n_inst);
    CK(cudaMemcpyAsync(r.data(), h->result, sizeof(double) * r.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    bool nonfinite = false;
    for (int k = 0; k < h->n_inst; k++) {
        const double* v = &r[(size_t)k * RED_NV];
        switch (what) {
        case LBCH_OBS_MASS: out[k] = v[0]; break;
        case LBCH_OBS_ERR_L2: out[k] = std::sqrt(v[1] / v[2]); break;
        case LBCH_OBS_MAX: out[k] = v[3]; break;
        default: out[k] = v[4]; break;
        }
        nonfinite = nonfinite || v[5] > 0.0;
    }
    return nonfinite ? fail(LBCH_ENONFINITE, "phi holds non-finite values") : LBCH_OK;
}

lbch_status lb_ch_free(lbch_handle* h)
{
    if (!h) return LBCH_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    return LBCH_OK;
}

const char* lb_ch_strerror(lbch_status s)
{
    switch (s) {
    case LBCH_OK: return "ok";
    case LBCH_EINVAL: return "invalid argument";
    case LBCH_ENOMEM: return "out of device memory";
    case LBCH_ECUDA: return "CUDA error";
    case LBCH_ETIMEOUT: return "device wait timed out";
    case LBCH_ENONFINITE: return "non-finite order parameter";
    default: return "unknown status";
    }
}

const char* lb_ch_last_error(void) { return g_msg; }

lbch_status lb_ch_info(lbch_handle* h, double* out)
{
    if (!h || !out) return fail(LBCH_EINVAL, "NULL handle or output");
    // algorithmic HBM bytes per lattice update: read + write of the stored populations and of phi
    double bytes = 2.0 * (h->n_planes * (double)h->g_elem + (double)h->phi_elem);
    out[0] = (double)h->nodes;
    out[1] = bytes;
    out[2] = (double)h->total_tiles;
    out[3] = (double)h->n;
    return LBCH_OK;
}

void* lb_ch_stream(lbch_handle* h) { return h ? (void*)h->stream : nullptr; }

}  // extern "C"
