// lbch_api.cu -- host runtime of the C ABI declared in include/lbch.h.
//
// Owns the device state of a handle: ping-pong population and phi arrays in the padded image layout,
// the instance table, the separable velocity tables, the TMA tensor maps, the step counter and the
// reduction scratch.  It derives the model constants from the parameters (Eqs. betakappa, rho, F2-1,
// the mobility relation after Eq. phit3 and the Peclet number of Sec. III.A), launches the persistent
// step kernel -- replayed from CUDA graphs of 64 steps -- and the reductions behind lb_ch_observe.
#include "lbch.h"
#include "lbch_adjoint.cuh"
#include "lbch_internal.h"
#include "lbch_kernels.cuh"
#include "lbch_ns.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
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
    cudaGetLastError();  // clear a non-sticky error so later calls on this thread start clean
    return fail(e == cudaErrorMemoryAllocation ? LBCH_ENOMEM : LBCH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// An NVTX range over one entry point, for profilers that record NVTX (nothing is recorded otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

// Steps per captured graph (a multiple of 4, so that a graph of two-step launches holds an even number of
// launches and ends in the buffer it starts from).  A call of many steps replays graphs of kGraphBig steps
// and finishes with graphs of kGraphChunk: a launch that follows a graph cannot overlap its tail (the
// programmatic dependence holds only within a graph), so fewer, longer graphs leave fewer such gaps.
constexpr int kGraphChunk = 64;
constexpr int kGraphBig = 512;
static_assert(kGraphChunk % 4 == 0 && kGraphBig % kGraphChunk == 0, "graph sizes");

// Tile shapes the step kernel is built for (output nodes per tile; 256 threads per CTA).  lb_ch_tune
// times them on the handle's own problem and keeps the fastest; the first one is the default.  Every
// TX divides 32 and every TY divides 16, so one storage layout serves all shapes.
constexpr int NT = 256;
// FP64 32 x 16 with 736 threads: 128 tiles at 256^2, at most one per SM, and the least recomputed halo of
// the shapes that fit that count (the FP64 step is bound by the FP64 pipe, so the halo's share counts);
// 736 threads take each phase in one pass (0.3 to 0.7 % faster than 512 at 1024^2 to 4096^2).
// FP64 32 x 14 with 672 threads: 152 tiles at 256^2, one per SM, with a little less halo per SM than
// 32 x 16; 672 threads take every phase in one pass (mu and D on the tile + 2 are 648 nodes; with 576
// threads a second pass of three warps left the FP64 pipe short: 25.2 against 24.65 us per step).  (Only for FP64: its per-tile copy of
// the Y tables starts at row y0, which is 16-byte aligned for 8-byte entries and even y0 only.)
constexpr Shape kShapes64[5] = {{32, 8, 256}, {16, 8, 256}, {32, 8, 512}, {32, 16, 736}, {32, 14, 672}};
constexpr Shape kShapesF[4] = {{32, 16, 256}, {32, 8, 256}, {16, 8, 256}, {32, 16, 768}};
inline int n_shapes(int prec) { return prec == LBCH_F64 ? 5 : 4; }
inline Shape shape_of(int prec, int k) { return prec == LBCH_F64 ? kShapes64[k] : kShapesF[k]; }


typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

cudaError_t lbch_kernel_smem(const void* kern, int device, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> set;  // (kernel, device) -> the bytes allowed so far
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(kern, device);
    auto it = set.find(key);
    if (it != set.end() && it->second >= smem) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) set[key] = smem;
    return e;
}

cudaError_t lbch_kernel_fit(const void* kern, int device, int threads, size_t smem, int* per_sm, int* sms)
{
    struct Key {
        const void* kern;
        int device, threads;
        size_t smem;
        bool operator<(const Key& o) const
        {
            return kern != o.kern ? kern < o.kern
                 : device != o.device ? device < o.device : threads != o.threads ? threads < o.threads : smem < o.smem;
        }
    };
    static std::mutex mu;
    static std::map<Key, int> fits;
    static std::map<int, int> sm_count;
    std::lock_guard<std::mutex> lock(mu);
    auto s = sm_count.find(device);
    if (s == sm_count.end()) {
        int n = 0;
        const cudaError_t e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        s = sm_count.emplace(device, n).first;
    }
    *sms = s->second;
    const Key key{kern, device, threads, smem};
    auto it = fits.find(key);
    if (it == fits.end()) {
        int n = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem);
        if (e != cudaSuccess) return e;
        it = fits.emplace(key, n).first;
    }
    *per_sm = it->second;
    return cudaSuccess;
}

// Used by the allocation-free entry point (another translation unit) to report its failures through
// lb_ch_last_error(); not exported.
__attribute__((visibility("hidden"))) void lbch_set_last_error(const char* msg)
{
    snprintf(g_msg, sizeof g_msg, "%s", msg);
}


namespace {


template <typename C, typename S, typename P, int TX, int TY, int NTT, bool TAU1>
cudaError_t launch_step_v(lbch_handle* h, int parity)
{
    using L = StepShape<C, S, P, TX, TY>;
    const lbch_handle::PerShape& ps = h->ps[h->shape];
    StepArgs<C, S, P> a;
    a.inst = h->d_inst;
    a.tile_begin = ps.d_tile_begin;
    a.tabs = tables<C>(h);
    a.n_inst = h->n_inst;
    a.total_tiles = ps.total_tiles;
    a.pitch = h->pitch;
    a.debug_skip = h->debug_skip;
    a.g_out = static_cast<S*>(h->g[parity ^ 1]);
    a.phi_out = static_cast<P*>(h->phi[parity ^ 1]);
    a.lo_out = h->lo[parity ^ 1];
    a.ctl = h->ctl;
    a.H_in = static_cast<const C*>(h->H[parity]);
    a.H_out = static_cast<C*>(h->H[parity ^ 1]);
    a.H_plane = (long long)h->rows * h->pitch;
    a.t_off = h->t_off;
    a.t_adv = h->t_adv;
    a.need_time = h->need_time;
    // a programmatic dependent of the previous launch in the stream (the kernel waits on it before it
    // touches memory that launch writes), so its launch and prologue overlap the previous step's tail
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ps.grid);
    cfg.blockDim = dim3(NTT);
    cfg.dynamicSmemBytes = L::BYTES;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = h->no_pdl ? 0 : 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ch_step_kernel<C, S, P, TX, TY, NTT, TAU1>, ps.tm_g[parity], ps.tm_phi[parity],
                              ps.tm_lo[parity], a);
}

template <typename C, typename S, typename P, int TX, int TY, int NTT = NT>
cudaError_t launch_step_t(lbch_handle* h, int parity)
{
    // at tau_g = 1 the tile kernel drops the populations too (exact, as in the row sweep)
    return (h->tau1 && !h->force_general) ? launch_step_v<C, S, P, TX, TY, NTT, true>(h, parity)
                                          : launch_step_v<C, S, P, TX, TY, NTT, false>(h, parity);
}

// The row-sweep kernel steps the handle (its shape index then names a sweep configuration), without the
// populations when every instance has tau_g = 1; the tile kernel only when a test asks for it.  When the
// two-step kernel is selected (and applies), it takes the steps two at a time and the one-step kernel
// takes an odd last step.
inline bool use_pair(const lbch_handle* h) { return h->pair && pair_ok(h); }
inline bool use_sweep(const lbch_handle* h) { return !h->force_tile && !h->coupled; }
// sweep configurations built for the handle (those with Model III: the two unrolled ones)
inline int n_sweep_shapes(const lbch_handle* h) { return h->model3 ? kM3SweepShapes : kSweepShapes; }
inline int n_active(const lbch_handle* h)
{
    return h->coupled ? 1 : (use_pair(h) ? kPairShapes : (use_sweep(h) ? n_sweep_shapes(h) : n_shapes(h->prec)));
}
inline const lbch_handle::PerShape& active_ps(const lbch_handle* h)
{
    return use_pair(h) ? h->pr[h->pshape] : (use_sweep(h) ? h->sw[h->shape] : h->ps[h->shape]);
}
inline int active_grid(const lbch_handle* h)
{
    return !use_pair(h) && use_sweep(h) && sweep_gen(h) ? h->sw[h->shape].grid_gen : active_ps(h).grid;
}
inline Shape active_tile(const lbch_handle* h)
{
    return h->coupled ? Shape{0, 0}
         : use_pair(h) ? pair_shape(h->prec, h->pshape) : (use_sweep(h) ? sweep_tile(h->shape) : shape_of(h->prec, h->shape));
}
inline void drop_graphs(lbch_handle* h)  // graphs captured earlier launch another kernel or shape
{
    for (int k = 0; k < 2; k++) {
        for (int z = 0; z < 2; z++)
            if (h->graph[z][k]) { cudaGraphExecDestroy(h->graph[z][k]); h->graph[z][k] = nullptr; }
        if (h->tgraph[k].exec) { cudaGraphExecDestroy(h->tgraph[k].exec); h->tgraph[k] = lbch_handle::TapeGraph(); }
    }
}

cudaError_t launch_sweep(lbch_handle* h, int parity)
{
    if (h->model3) {
        switch (h->prec) {
        case LBCH_F64: return lbch_launch_sweep_f64_m3(h, parity);
        case LBCH_F32: return lbch_launch_sweep_f32_m3(h, parity);
        default: return lbch_launch_sweep_f16s_m3(h, parity);
        }
    }
    switch (h->prec) {
    case LBCH_F64: return lbch_launch_sweep_f64(h, parity);
    case LBCH_F32: return lbch_launch_sweep_f32(h, parity);
    default: return lbch_launch_sweep_f16s(h, parity);
    }
}

cudaError_t prepare_sweep(lbch_handle* h, int k)
{
    if (h->model3 && k < kM3SweepShapes) {
        switch (h->prec) {
        case LBCH_F64: return lbch_prepare_sweep_f64_m3(h, k);
        case LBCH_F32: return lbch_prepare_sweep_f32_m3(h, k);
        default: return lbch_prepare_sweep_f16s_m3(h, k);
        }
    }
    switch (h->prec) {
    case LBCH_F64: return lbch_prepare_sweep_f64(h, k);
    case LBCH_F32: return lbch_prepare_sweep_f32(h, k);
    default: return lbch_prepare_sweep_f16s(h, k);
    }
}

// Dynamic shared memory of the step kernel, and the persistent grid that fits the device, for shape k.
template <typename C, typename S, typename P, int TX, int TY, int NTT = NT>
cudaError_t prepare_step_t(lbch_handle* h, int k)
{
    using L = StepShape<C, S, P, TX, TY>;
    const void* kern = reinterpret_cast<const void*>(ch_step_kernel<C, S, P, TX, TY, NTT, false>);
    cudaError_t e = lbch_kernel_smem(kern, h->device, L::BYTES);
    if (e != cudaSuccess) return e;
    e = lbch_kernel_smem(reinterpret_cast<const void*>(ch_step_kernel<C, S, P, TX, TY, NTT, true>), h->device, L::BYTES);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = lbch_kernel_fit(kern, h->device, NTT, L::BYTES, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    h->ps[k].grid = std::max(1, std::min(h->ps[k].total_tiles, per_sm * sms));
    return cudaSuccess;
}

cudaError_t prepare_step(lbch_handle* h, int k)
{
    switch (h->prec) {
    case LBCH_F64:
        return k == 0 ? prepare_step_t<double, double, double, 32, 8>(h, k)
             : k == 1 ? prepare_step_t<double, double, double, 16, 8>(h, k)
             : k == 2 ? prepare_step_t<double, double, double, 32, 8, 512>(h, k)
             : k == 3 ? prepare_step_t<double, double, double, 32, 16, 736>(h, k)
                      : prepare_step_t<double, double, double, 32, 14, 672>(h, k);
    case LBCH_F32:
        return k == 0 ? prepare_step_t<float, float, float, 32, 16>(h, k)
             : k == 1 ? prepare_step_t<float, float, float, 32, 8>(h, k)
             : k == 2 ? prepare_step_t<float, float, float, 16, 8>(h, k) : prepare_step_t<float, float, float, 32, 16, 768>(h, k);
    default:
        return k == 0 ? prepare_step_t<float, __half, float, 32, 16>(h, k)
             : k == 1 ? prepare_step_t<float, __half, float, 32, 8>(h, k)
             : k == 2 ? prepare_step_t<float, __half, float, 16, 8>(h, k) : prepare_step_t<float, __half, float, 32, 16, 768>(h, k);
    }
}

template <typename C> const ns::NsConsts<C>& ns_consts(const lbch_handle* h);
template <> const ns::NsConsts<double>& ns_consts<double>(const lbch_handle* h) { return h->nsd; }
template <> const ns::NsConsts<float>& ns_consts<float>(const lbch_handle* h) { return h->nsf; }
template <typename C> const Consts<C>& ch_consts(const InstDev& I);
template <> const Consts<double>& ch_consts<double>(const InstDev& I) { return I.cd; }
template <> const Consts<float>& ch_consts<float>(const InstDev& I) { return I.cf; }

template <typename C>
ns::NsArgs<C> ns_args(lbch_handle* h, int parity)
{
    const InstDev& I = h->inst[0];
    const size_t N = (size_t)I.nx * I.ny;
    ns::NsArgs<C> a;
    a.nx = I.nx; a.ny = I.ny; a.walls = I.walls; a.model = I.model; a.pitch = h->pitch; a.row0 = I.row0;
    a.k = ch_consts<C>(I);
    a.n = ns_consts<C>(h);
    C* p = static_cast<C*>(h->ns);
    C* f[2] = {p, p + 9 * N};
    C* g[2] = {p + 18 * N, p + 27 * N};
    a.f_in = f[parity]; a.f_out = f[parity ^ 1];
    a.g_in = g[parity]; a.g_out = g[parity ^ 1];
    C* w = p + 36 * N;
    a.ux = w; a.uy = w + N; a.pr = w + 2 * N; a.mu = w + 3 * N;
    a.phi_in = static_cast<C*>(h->phi[parity]);
    a.phi_out = static_cast<C*>(h->phi[parity ^ 1]);
    return a;
}

// One coupled step: phi = sum g of the current state with the flow's u and p; both collisions with push
// streaming.  phi of the new state is formed by the next step (or by coupled_phi before an observation).
template <typename C>
cudaError_t launch_ns_t(lbch_handle* h, int parity)
{
    ns::NsArgs<C> a = ns_args<C>(h, parity);
    const int tiles = ns::tiles_of(a.nx, a.ny);
    ns::fields_kernel<C><<<tiles, ns::NT, 0, h->stream>>>(a);
    ns::collide_kernel<C><<<tiles, ns::NTC, 0, h->stream>>>(a);
    return cudaGetLastError();
}

// phi of the current state of a coupled handle into its phi array (the steps leave it to the next step).
template <typename C>
cudaError_t coupled_phi_t(lbch_handle* h)
{
    ns::NsArgs<C> a = ns_args<C>(h, cur_buf(h));
    const int nb = (int)(((long long)a.nx * a.ny + 255) / 256);
    ns::phi_kernel<C><<<nb, 256, 0, h->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t coupled_phi(lbch_handle* h)
{
    if (!h->coupled) return cudaSuccess;
    return h->prec == LBCH_F64 ? coupled_phi_t<double>(h) : coupled_phi_t<float>(h);
}

// The flow's u and p of the current state (for observation).
template <typename C>
cudaError_t ns_fields_t(lbch_handle* h, int parity)
{
    ns::NsArgs<C> a = ns_args<C>(h, parity);
    ns::fields_kernel<C><<<ns::tiles_of(a.nx, a.ny), ns::NT, 0, h->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_step(lbch_handle* h, int parity)
{
    if (h->coupled) return h->prec == LBCH_F64 ? launch_ns_t<double>(h, parity) : launch_ns_t<float>(h, parity);
    if (use_sweep(h)) return launch_sweep(h, parity);
    const int k = h->shape;
    switch (h->prec) {
    case LBCH_F64:
        return k == 0 ? launch_step_t<double, double, double, 32, 8>(h, parity)
             : k == 1 ? launch_step_t<double, double, double, 16, 8>(h, parity)
             : k == 2 ? launch_step_t<double, double, double, 32, 8, 512>(h, parity)
             : k == 3 ? launch_step_t<double, double, double, 32, 16, 736>(h, parity)
                      : launch_step_t<double, double, double, 32, 14, 672>(h, parity);
    case LBCH_F32:
        return k == 0 ? launch_step_t<float, float, float, 32, 16>(h, parity)
             : k == 1 ? launch_step_t<float, float, float, 32, 8>(h, parity)
             : k == 2 ? launch_step_t<float, float, float, 16, 8>(h, parity) : launch_step_t<float, float, float, 32, 16, 768>(h, parity);
    default:
        return k == 0 ? launch_step_t<float, __half, float, 32, 16>(h, parity)
             : k == 1 ? launch_step_t<float, __half, float, 32, 8>(h, parity)
             : k == 2 ? launch_step_t<float, __half, float, 16, 8>(h, parity) : launch_step_t<float, __half, float, 32, 16, 768>(h, parity);
    }
}

// Two steps by one launch of the two-step kernel, outside a graph (the launch advances the counter by
// two); phi(n + 2) lands in the other buffer, so the buffer of the current step flips.
cudaError_t launch_pair_now(lbch_handle* h)
{
    h->t_adv = 2;
    cudaError_t e = lbch_launch_pair(h, cur_buf(h));
    h->t_adv = 1;
    if (e == cudaSuccess) {
        h->n += 2;
        h->flip ^= 1;
    }
    return e;
}

lbch_status check_params(const lbch_params& p, int k)
{
    if (p.nx < 4 || p.ny < 4 || p.nx > (1 << 20) || p.ny > (1 << 20))
        return fail(LBCH_EINVAL, "instance %d: nx, ny must be in [4, 2^20] (got %d x %d)", k, p.nx, p.ny);
    if (!(p.tau > 0.5)) return fail(LBCH_EINVAL, "instance %d: tau must exceed 1/2", k);
    if (p.model < 1 || p.model > 3) return fail(LBCH_EINVAL, "instance %d: model must be 1, 2 or 3", k);
    if (p.model == 3 && p.vel == LBCH_VEL_COUPLED)
        return fail(LBCH_EINVAL, "instance %d: the coupled flow takes Model I or II", k);
    if (p.vel < 0 || p.vel > 6) return fail(LBCH_EINVAL, "instance %d: unknown velocity field %d", k, p.vel);
    if (p.vel == LBCH_VEL_COUPLED && !(p.nu > 0.0)) return fail(LBCH_EINVAL, "instance %d: coupled flow needs nu > 0", k);
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
    Consts<double>& c = d.cd;
    c.beta = 12.0 * p.sigma / (p.W * dphi * dphi * dphi * dphi);      // Eq. betakappa
    c.kappa = 3.0 * p.sigma * p.W / (2.0 * dphi * dphi);
    double M = p.M > 0.0 ? p.M
                         : p.Ustar * p.W / (p.Pe * c.beta * (p.phiA - p.phiB) * (p.phiA - p.phiB));  // Pe, Sec. III.A
    c.eta = M / (cs2 * (p.tau - 0.5));                                  // M = c_s^2 eta (tau - 1/2)
    c.a = (p.rhoA - p.rhoB) / (p.phiA - p.phiB);                        // Eq. rho
    c.b = (p.rhoB * p.phiA - p.phiB * p.rhoA) / (p.phiA - p.phiB);
    c.K = (p.tau - 1.0 / 6.0 - p.tau * p.tau) / (p.tau - 0.5);          // Eq. F2-1
    c.itau = 1.0 / p.tau;
    c.omt = 1.0 - 1.0 / p.tau;
    c.src = 1.0 - 1.0 / (2.0 * p.tau);
    c.phiA = p.phiA; c.phiB = p.phiB;
    c.cF1 = 2.0 * p.tau - 1.0 + 3.0 * c.K;                               // Eq. F2-1: coefficient of d_t F1
    c.cmu = 3.0 * cs2 * c.eta * c.K;                                     // and of d_t grad mu
    Consts<float>& f = d.cf;
    f.beta = (float)c.beta; f.kappa = (float)c.kappa; f.eta = (float)c.eta; f.a = (float)c.a; f.b = (float)c.b;
    f.K = (float)c.K; f.phiA = (float)c.phiA; f.phiB = (float)c.phiB;
    f.itau = (float)c.itau; f.omt = (float)c.omt; f.src = (float)c.src;
    f.cF1 = (float)c.cF1; f.cmu = (float)c.cmu;
    // the collision's per-class coefficients, each one product rounded in the kernel's arithmetic type
    // (the same rounding as forming them at a node would give)
    auto coll = [](auto& k) {
        using T = decltype(k.itau);
        const T w1 = T(1) / T(9), w5 = T(1) / T(36);
        k.k1a = w1 * k.itau;
        k.k1d = w5 * k.itau;
        k.k2a = T(3) * k.k1a;
        k.k2d = T(3) * k.k1d;
        k.k3a = (T(3) * w1) * k.src;
        k.k3d = (T(3) * w5) * k.src;
    };
    coll(c);
    coll(f);
    d.Tper = p.Tper;
    d.walls = p.walls; d.model = p.model; d.vel = p.vel;
}

// The prescribed flows are separable: ux = X1(x) Y1(y) T(t), uy = X2(x) Y2(y) T(t).  The tables are
// indexed like the stored arrays: X1, X2 by stored column (domain x = column - GC, periodic images in
// the ghost columns), Y1, Y2 by row of the instance's stored band (domain y = row - GR; periodic or
// mirror images in the ghost rows, matching the stored phi), then Y1, Y2 at the walls y = -1/2, ny - 1/2.
// A slab of a larger periodic grid (lb_ch_init_slab): the handle holds global rows y0 .. y0 + ny - 1.
struct SlabSpec {
    int y0;   // first global row of the slab
    int ny;   // rows of the slab
};

void velocity_tables(const lbch_params& p, int pitch, int ylen, std::vector<double>& t, const SlabSpec* slab = nullptr)
{
    const double pi = 3.14159265358979323846;
    const double Lx = (double)p.nx, Ly = (double)p.ny;
    auto X = [&](double x, double& X1, double& X2) {
        switch (p.vel) {
        case LBCH_VEL_COUPLED: X1 = 0.0; X2 = 0.0; break;  // the flow is solved, not prescribed
        case LBCH_VEL_UNIFORM: X1 = 1.0; X2 = 1.0; break;
        case LBCH_VEL_ROTATION: X1 = 1.0; X2 = p.U0 * pi * (x - p.xc) / p.half; break;
        case LBCH_VEL_VORTEX: { double s = std::sin(pi * x / Lx); X1 = -p.U0 * s * s; X2 = p.U0 * std::sin(2.0 * pi * x / Lx); break; }
        case LBCH_VEL_SHEAR: X1 = 1.0; X2 = 0.0; break;
        case LBCH_VEL_REV_SHEAR: X1 = -p.U0 * pi * std::cos(pi * (x / Lx - 0.5)); X2 = p.U0 * pi * std::sin(pi * (x / Lx - 0.5)); break;
        default: { double k = (double)p.nvort * pi; X1 = -p.U0 * std::sin(k * (x / Lx + 0.5)); X2 = -p.U0 * std::cos(k * (x / Lx + 0.5)); }
        }
    };
    auto Y = [&](double y, double& Y1, double& Y2) {
        switch (p.vel) {
        case LBCH_VEL_COUPLED: Y1 = 0.0; Y2 = 0.0; break;
        case LBCH_VEL_UNIFORM: Y1 = p.ux0; Y2 = p.uy0; break;
        case LBCH_VEL_ROTATION: Y1 = -p.U0 * pi * (y - p.yc) / p.half; Y2 = 1.0; break;
        case LBCH_VEL_VORTEX: { double s = std::sin(pi * y / Ly); Y1 = std::sin(2.0 * pi * y / Ly); Y2 = s * s; break; }
        case LBCH_VEL_SHEAR: Y1 = p.shear * (y - 0.5 * (double)(p.ny - 1)); Y2 = 0.0; break;
        case LBCH_VEL_REV_SHEAR: Y1 = std::sin(pi * (y / Lx - 0.5)); Y2 = std::cos(pi * (y / Lx - 0.5)); break;
        default: { double k = (double)p.nvort * pi; Y1 = std::sin(k * (y / Lx + 0.5)); Y2 = std::cos(k * (y / Lx + 0.5)); }
        }
    };
    size_t b = t.size();
    t.resize(b + 2 * (size_t)pitch + 2 * (size_t)ylen + 4, 0.0);
    double* X1 = &t[b];
    double* X2 = X1 + pitch;
    double* Y1 = X2 + pitch;
    double* Y2 = Y1 + ylen;
    double* W = Y2 + ylen;
    for (int col = 0; col < pitch; col++) {
        int x = col - GC;
        if (x < -GC || x >= p.nx + GC) continue;
        X((double)(((x % p.nx) + p.nx) % p.nx), X1[col], X2[col]);
    }
    const int ny_rows = slab ? slab->ny : p.ny;  // rows of the stored band (p.ny is the global grid's)
    for (int k = 0; k < ylen; k++) {
        int y = k - GR;
        if (y < -GR || y >= ny_rows + GR) continue;
        int yy;
        if (slab) yy = (((slab->y0 + y) % p.ny) + p.ny) % p.ny;  // the global row a slab's row stands for
        else yy = p.walls ? (y < 0 ? -1 - y : (y >= p.ny ? 2 * p.ny - 1 - y : y)) : ((y % p.ny) + p.ny) % p.ny;
        Y((double)yy, Y1[k], Y2[k]);
    }
    Y(-0.5, W[0], W[2]);
    Y((double)p.ny - 0.5, W[1], W[3]);
}

// ---------------------------------------------------------------------------------------- handle memory
// A handle's device buffers come from one stream-ordered memory pool per device, allocated and freed on the
// handle's stream; the pool keeps up to kPoolKeep bytes of freed memory for the next handle.  Where a handle
// is made and freed per problem, set-up and release then cost microseconds per buffer instead of a
// cudaMalloc and a device-synchronising cudaFree each (measured: init 1.25 ms and free 0.87 ms for one
// 256^2 handle before).  The pinned host staging buffers are kept between handles likewise, up to
// kStageKeep of them and kStageKeepBytes in all (pinning host memory costs far more than a copy through it).
constexpr unsigned long long kPoolKeep = 2ull << 30;
constexpr size_t kStageKeep = 4, kStageKeepBytes = size_t(256) << 20;

cudaError_t device_pool(int device, cudaMemPool_t* out)
{
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(device);
    if (it != pools.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = kPoolKeep;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
    }
    pools[device] = pool;
    *out = pool;
    return cudaSuccess;
}

// bytes of device memory for the handle, ordered on its stream; 256-byte aligned (the tensor maps need 16)
template <typename T>
cudaError_t dalloc(lbch_handle* h, T** p, size_t bytes)
{
    void* v = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&v, bytes, h->pool, h->stream);
    if (e != cudaSuccess) return e;
    if (reinterpret_cast<uintptr_t>(v) % 256 != 0) {
        cudaFreeAsync(v, h->stream);
        return cudaErrorMisalignedAddress;
    }
    *p = static_cast<T*>(v);
    return cudaSuccess;
}

template <typename T>
void dfree(lbch_handle* h, T*& p)
{
    if (p) cudaFreeAsync(p, h->stream);
    p = nullptr;
}

struct StageCache {
    std::mutex mu;
    std::vector<std::pair<void*, size_t>> kept;
};
StageCache& stage_cache()
{
    static StageCache c;
    return c;
}

// a kept pinned buffer of at least `bytes` (the smallest such), else a new one
cudaError_t stage_take(size_t bytes, double** p, size_t* got)
{
    {
        StageCache& c = stage_cache();
        std::lock_guard<std::mutex> lock(c.mu);
        int best = -1;
        for (int i = 0; i < (int)c.kept.size(); i++)
            if (c.kept[i].second >= bytes && (best < 0 || c.kept[i].second < c.kept[best].second)) best = i;
        if (best >= 0) {
            *p = static_cast<double*>(c.kept[best].first);
            *got = c.kept[best].second;
            c.kept.erase(c.kept.begin() + best);
            return cudaSuccess;
        }
    }
    void* v = nullptr;
    cudaError_t e = cudaMallocHost(&v, bytes);
    if (e != cudaSuccess) return e;
    *p = static_cast<double*>(v);
    *got = bytes;
    return cudaSuccess;
}

// back to the cache, or freed when the cache is full (the smallest kept buffer makes room for a larger one)
void stage_give(double* p, size_t bytes)
{
    if (!p) return;
    if (bytes <= kStageKeepBytes) {
        StageCache& c = stage_cache();
        std::lock_guard<std::mutex> lock(c.mu);
        size_t total = bytes;
        for (auto& k : c.kept) total += k.second;
        if (c.kept.size() < kStageKeep && total <= kStageKeepBytes) {
            c.kept.push_back({p, bytes});
            return;
        }
    }
    cudaFreeHost(p);
}

void release(lbch_handle* h)
{
    for (int k = 0; k < 2; k++) {
        for (int z = 0; z < 2; z++)
            if (h->graph[z][k]) cudaGraphExecDestroy(h->graph[z][k]);
        if (h->tgraph[k].exec) cudaGraphExecDestroy(h->tgraph[k].exec);
        dfree(h, h->g[k]);
        dfree(h, h->phi[k]);
        dfree(h, h->lo[k]);
        dfree(h, h->H[k]);
    }
    dfree(h, h->d_inst);
    dfree(h, h->d_tabs_f);
    for (int k = 0; k < kMaxShapes; k++) dfree(h, h->ps[k].d_tile_begin);
    for (int k = 0; k < kSweepShapes; k++) {
        dfree(h, h->sw[k].d_tile_begin);
        dfree(h, h->sw[k].d_tiles);
    }
    for (int k = 0; k < kPairShapes; k++) {
        dfree(h, h->pr[k].d_tile_begin);
        dfree(h, h->pr[k].d_ttabs);
    }
    dfree(h, h->d_node_begin);
    dfree(h, h->d_tabs);
    dfree(h, h->phi0);
    dfree(h, h->ctl);
    dfree(h, h->partials);
    dfree(h, h->result);
    dfree(h, h->ns);
    stage_give(h->h_stage, h->h_stage_bytes);
    h->h_stage = nullptr;
    h->h_stage_bytes = 0;
    if (h->adj) cudaFree(h->adj);  // the adjoint's workspace is a plain allocation (lb_ch_adjoint_begin)
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

lbch_status stage(lbch_handle* h, size_t bytes)
{
    if (h->h_stage_bytes >= bytes) return LBCH_OK;
    stage_give(h->h_stage, h->h_stage_bytes);
    h->h_stage = nullptr;
    h->h_stage_bytes = 0;
    CK(stage_take(bytes, &h->h_stage, &h->h_stage_bytes));
    return LBCH_OK;
}

lbch_status encode_maps(lbch_handle* h, int sk)
{
    const Shape sh = shape_of(h->prec, sk);
    lbch_handle::PerShape& ps = h->ps[sk];
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(LBCH_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    CUtensorMapDataType gt = h->prec == LBCH_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : (h->prec == LBCH_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    CUtensorMapDataType pt = h->phi_elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    for (int k = 0; k < 2; k++) {
        cuuint64_t gdim[3] = {(cuuint64_t)h->pitch, (cuuint64_t)h->nq, (cuuint64_t)h->rows};
        cuuint64_t gstr[2] = {(cuuint64_t)h->pitch * h->g_elem, (cuuint64_t)h->pitch * h->g_elem * h->nq};
        cuuint32_t gbox[3] = {(cuuint32_t)(sh.tx + 8), (cuuint32_t)h->nq, (cuuint32_t)(sh.ty + 2)};
        cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&ps.tm_g[k], gt, 3, h->g[k], gdim, gstr, gbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(LBCH_ECUDA, "tensor map of the populations: CUresult %d", (int)r);
        cuuint64_t pdim[2] = {(cuuint64_t)h->pitch, (cuuint64_t)h->rows};
        cuuint64_t pstr[1] = {(cuuint64_t)h->pitch * h->phi_elem};
        cuuint32_t pbox[2] = {(cuuint32_t)(sh.tx + 8), (cuuint32_t)(sh.ty + 6)};
        r = enc(&ps.tm_phi[k], pt, 2, h->phi[k], pdim, pstr, pbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(LBCH_ECUDA, "tensor map of phi: CUresult %d", (int)r);
        if (h->lo[k]) {
            cuuint32_t lbox[2] = {(cuuint32_t)sh.tx, (cuuint32_t)sh.ty};
            cuuint64_t lstr[1] = {(cuuint64_t)h->pitch * 4};
            r = enc(&ps.tm_lo[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->lo[k], pdim, lstr, lbox, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(LBCH_ECUDA, "tensor map of phi (low part): CUresult %d", (int)r);
        } else {
            ps.tm_lo[k] = ps.tm_phi[k];  // unused by the kernels without a low part
        }
    }
    return LBCH_OK;
}

// The row-sweep kernel's boxes: phi over 64 columns and the tile's rows plus three halo rows on each
// side; the low part of phi over the output rows.
lbch_status encode_sweep_maps(lbch_handle* h, int sk)
{
    const Shape sh = sweep_tile(sk);
    lbch_handle::PerShape& ps = h->sw[sk];
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(LBCH_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    CUtensorMapDataType pt = h->phi_elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint32_t es[2] = {1, 1};
    cuuint64_t pdim[2] = {(cuuint64_t)h->pitch, (cuuint64_t)h->rows};
    for (int k = 0; k < 2; k++) {
        cuuint64_t pstr[1] = {(cuuint64_t)h->pitch * h->phi_elem};
        cuuint32_t pbox[2] = {64u, (cuuint32_t)(sh.ty + 6)};
        CUresult r = enc(&ps.tm_phi[k], pt, 2, h->phi[k], pdim, pstr, pbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(LBCH_ECUDA, "tensor map of phi (row sweep): CUresult %d", (int)r);
        if (h->lo[k]) {
            cuuint64_t lstr[1] = {(cuuint64_t)h->pitch * 4};
            cuuint32_t lbox[2] = {64u, (cuuint32_t)sh.ty};
            r = enc(&ps.tm_lo[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->lo[k], pdim, lstr, lbox, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(LBCH_ECUDA, "tensor map of phi, low part (row sweep): CUresult %d", (int)r);
        } else {
            ps.tm_lo[k] = ps.tm_phi[k];  // unused without a low part
        }
        ps.tm_g[k] = ps.tm_phi[k];
    }
    return LBCH_OK;
}

// The row sweep's ring fills: one row of the population planes (64 columns x nq planes), and one row of
// the low part of phi.
lbch_status encode_row_maps(lbch_handle* h)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(LBCH_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    CUtensorMapDataType gt = h->prec == LBCH_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : (h->prec == LBCH_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    for (int k = 0; k < 2; k++) {
        cuuint64_t gdim[3] = {(cuuint64_t)h->pitch, (cuuint64_t)h->nq, (cuuint64_t)h->rows};
        cuuint64_t gstr[2] = {(cuuint64_t)h->pitch * h->g_elem, (cuuint64_t)h->pitch * h->g_elem * h->nq};
        cuuint32_t gbox[3] = {64u, (cuuint32_t)h->nq, 1u};
        cuuint32_t es[3] = {1, 1, 1};
        CUresult r = enc(&h->tm_grow[k], gt, 3, h->g[k], gdim, gstr, gbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(LBCH_ECUDA, "tensor map of a population row: CUresult %d", (int)r);
        if (h->lo[k]) {
            cuuint64_t ldim[2] = {(cuuint64_t)h->pitch, (cuuint64_t)h->rows};
            cuuint64_t lstr[1] = {(cuuint64_t)h->pitch * 4};
            cuuint32_t lbox[2] = {64u, 1u};
            r = enc(&h->tm_lorow[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->lo[k], ldim, lstr, lbox, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(LBCH_ECUDA, "tensor map of a row of phi's low part: CUresult %d", (int)r);
        } else {
            h->tm_lorow[k] = h->tm_grow[k];  // unused without a low part
        }
    }
    return LBCH_OK;
}

lbch_status check_err(lbch_handle* h)
{
    unsigned int err = 0;
    CK(cudaMemcpyAsync(&err, &h->ctl->err, sizeof err, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (err) return fail(LBCH_ETIMEOUT, "a bounded wait for a TMA copy in the step kernel ran out (flags %u)", err);
    return LBCH_OK;
}

lbch_status run_reduce(lbch_handle* h)
{
    int parity = cur_buf(h);
    dim3 grid(h->chunks, h->n_inst);
    if (h->phi_elem == 8)
        reduce_partials_kernel<double><<<grid, RED_NT, 0, h->stream>>>(h->d_inst, (const double*)h->phi[parity], nullptr, h->phi0,
                                                                       h->pitch, h->partials, h->chunks);
    else
        reduce_partials_kernel<float><<<grid, RED_NT, 0, h->stream>>>(h->d_inst, (const float*)h->phi[parity], h->lo[parity], h->phi0,
                                                                      h->pitch, h->partials, h->chunks);
    CK(cudaGetLastError());
    reduce_final_kernel<<<h->n_inst, RED_NT, 0, h->stream>>>(h->partials, h->chunks, h->result);
    CK(cudaGetLastError());
    return LBCH_OK;
}

// ----------------------------------------------------------------------------- state and adjoint helpers

size_t state_bytes(const lbch_handle* h)
{
    const size_t cells = (size_t)h->rows * h->pitch;
    size_t b = 256;  // header (StateHeader)
    b += (cells * h->nq * h->g_elem + 255) / 256 * 256;
    b += (cells * h->phi_elem + 255) / 256 * 256;
    if (h->lo[0]) b += (cells * 4 + 255) / 256 * 256;
    if (h->model3) b += (2 * cells * h->c_elem() + 255) / 256 * 256;
    return b;
}

// The first 256 bytes of a saved state: the step index and what the rest of the buffer was laid out for.
// lb_ch_state_load compares every field with the loading handle before it copies anything, so a buffer
// saved by a handle of another size, precision or model (or one that holds no saved state) is refused
// instead of being read past its end.
struct StateHeader {
    long long n;                 // step index of the saved state
    unsigned long long magic;    // kStateMagic
    long long bytes;             // state_bytes() of the saving handle
    int prec, nq, rows, pitch, n_inst, model3, lo;
    int pad_;
    unsigned long long layout;   // layout_hash() of the saving handle
};
static_assert(sizeof(StateHeader) <= 256, "the header fits the 256 bytes reserved for it");
constexpr unsigned long long kStateMagic = 0x4c4243485354415aull;  // "LBCHSTAZ"

// FNV-1a over each instance's size, origin row and boundary: equal for handles of the same layout.
unsigned long long layout_hash(const lbch_handle* h)
{
    unsigned long long x = 1469598103934665603ull;
    auto mix = [&](long long v) {
        for (int b = 0; b < 8; b++) {
            x ^= (unsigned long long)((v >> (8 * b)) & 0xff);
            x *= 1099511628211ull;
        }
    };
    for (const InstDev& d : h->inst) {
        mix(d.nx); mix(d.ny); mix(d.row0); mix(d.walls); mix(d.model);
    }
    return x;
}

StateHeader state_header(const lbch_handle* h, long long n)
{
    StateHeader hd;
    std::memset(&hd, 0, sizeof hd);
    hd.n = n;
    hd.magic = kStateMagic;
    hd.bytes = (long long)state_bytes(h);
    hd.prec = h->prec;
    hd.nq = h->nq;
    hd.rows = h->rows;
    hd.pitch = h->pitch;
    hd.n_inst = h->n_inst;
    hd.model3 = h->model3 ? 1 : 0;
    hd.lo = h->lo[0] ? 1 : 0;
    hd.layout = layout_hash(h);
    return hd;
}

// A slab's halo on one side, as lb_ch_halo_export writes it: GR rows of phi (the high part on the float
// path), GR rows of phi's low part (LBCH_F32), then one row of the stored populations (nq planes), each
// row `pitch` elements wide with its ghost columns.
size_t halo_bytes(const lbch_handle* h)
{
    size_t b = (size_t)GR * h->pitch * h->phi_elem;
    if (h->lo[0]) b += (size_t)GR * h->pitch * sizeof(float);
    b += (size_t)h->nq * h->pitch * h->g_elem;
    return b;
}

// Copy a halo between the buffer `buf` and the current state: phi and its low part on the GR stored rows
// from `phi_row`, the populations of stored row `g_row`; out = true copies state -> buf.  Stream-ordered.
lbch_status halo_copy(lbch_handle* h, void* buf, int phi_row, int g_row, bool out)
{
    const int par = cur_buf(h);
    char* b = static_cast<char*>(buf);
    auto cp = [&](void* state, size_t off, size_t n) {
        char* sp = static_cast<char*>(state) + off;
        return out ? cudaMemcpyAsync(b, sp, n, cudaMemcpyDeviceToDevice, h->stream)
                   : cudaMemcpyAsync(sp, b, n, cudaMemcpyDeviceToDevice, h->stream);
    };
    const size_t np = (size_t)GR * h->pitch * h->phi_elem;
    CK(cp(h->phi[par], (size_t)phi_row * h->pitch * h->phi_elem, np));
    b += np;
    if (h->lo[par]) {
        const size_t nl = (size_t)GR * h->pitch * sizeof(float);
        CK(cp(h->lo[par], (size_t)phi_row * h->pitch * sizeof(float), nl));
        b += nl;
    }
    const size_t ng = (size_t)h->nq * h->pitch * h->g_elem;
    CK(cp(h->g[par], (size_t)g_row * h->nq * h->pitch * h->g_elem, ng));
    return LBCH_OK;
}

struct AdjView {  // pointers into the adjoint workspace
    void* lam[2];
    void *mu, *gmb, *Fb, *phib, *mub, *Db, *ub;
    double* ds;
    double* dLds;
};

// planes of each lambda buffer: 9, or 1 at tau_g = 1 (the nine are equal there; lbch_adjoint.cuh, ONE)
inline int adj_planes(const lbch_handle* h) { return h->tau1 ? 1 : 9; }

AdjView adj_view(lbch_handle* h)
{
    const size_t N = (size_t)h->inst[0].nx * h->inst[0].ny, e = h->adj_elem;
    char* p = static_cast<char*>(h->adj);
    AdjView v;
    auto take = [&](size_t n) { void* r = p; p += (n * e + 255) / 256 * 256; return r; };
    v.lam[0] = take(adj_planes(h) * N);
    v.lam[1] = take(adj_planes(h) * N);
    v.mu = take(N);
    v.gmb = take(2 * N);
    v.Fb = take(2 * N);
    v.phib = take(N);
    v.mub = take(N);
    v.Db = take(N);
    v.ub = take(2 * N);
    v.ds = reinterpret_cast<double*>(p);
    p += (N * 8 + 255) / 256 * 256;
    v.dLds = reinterpret_cast<double*>(p);
    return v;
}

size_t adj_bytes(const lbch_handle* h)
{
    const size_t N = (size_t)h->inst[0].nx * h->inst[0].ny, e = h->adj_elem;
    auto r = [](size_t b) { return (b + 255) / 256 * 256; };
    return 2 * r(adj_planes(h) * N * e) + r(N * e) + 2 * r(2 * N * e) + 3 * r(N * e) + r(2 * N * e) + r(N * 8) + 256;
}

adj::AdjArgs adj_args(const lbch_handle* h, long long n)
{
    adj::AdjArgs a;
    a.nx = h->inst[0].nx;
    a.ny = h->inst[0].ny;
    a.model = h->inst[0].model;
    a.pitch = h->pitch;
    a.ylen = h->inst[0].ylen;
    a.n = n;
    return a;
}

// phi of the state in buffer `par` into a plain array of the tape type (see lb_ch_tape_phi).
cudaError_t tape_launch(lbch_handle* h, int par, void* dst)
{
    const long long N = (long long)h->inst[0].nx * h->inst[0].ny;
    const int nb = (int)((N + 255) / 256);
    if (h->prec == LBCH_F64)
        adj::tape_kernel<double, double><<<nb, 256, 0, h->stream>>>(h->d_inst, h->pitch, (const double*)h->phi[par],
                                                                    nullptr, (double*)dst);
    else
        adj::tape_kernel<float, float><<<nb, 256, 0, h->stream>>>(h->d_inst, h->pitch, (const float*)h->phi[par],
                                                                  h->lo[par], (float*)dst);
    return cudaGetLastError();
}

// One adjoint step.  The forward quantities are formed in the tape's type (CF = TP: float for the float
// path, as its forward step formed them, with the float velocity tables), everything carrying lambda in C.
template <typename C, typename TP>
cudaError_t adjoint_step_t(lbch_handle* h, const TP* phi_n, long long n)
{
    using CF = TP;
    AdjView v = adj_view(h);
    adj::AdjArgs a = adj_args(h, n);
    const long long N = (long long)a.nx * a.ny;
    const int nb = (int)((N + 255) / 256);
    const CF T = (CF)vel_t(h->inst[0].vel, h->inst[0].Tper, n);
    const CF* tabs = tables<CF>(h);
    const C* lam_next = static_cast<const C*>(v.lam[h->adj_par]);
    C* lam = static_cast<C*>(v.lam[h->adj_par ^ 1]);
    adj::fwd_mu_kernel<CF, TP><<<nb, 256, 0, h->stream>>>(h->d_inst, a, phi_n, (CF*)v.mu);
    const bool one = adj_planes(h) == 1;
    (one ? adj::local_kernel<C, CF, TP, true> : adj::local_kernel<C, CF, TP, false>)<<<nb, 256, 0, h->stream>>>(
        h->d_inst, tabs, a, T, phi_n, (const CF*)v.mu, lam_next, lam, (C*)v.gmb, (C*)v.Fb, (C*)v.phib, (C*)v.mub,
        (C*)v.ub);
    adj::transpose1_kernel<C><<<nb, 256, 0, h->stream>>>(h->d_inst, a, (const C*)v.gmb, (const C*)v.Fb, (C*)v.mub,
                                                         (C*)v.Db);
    (one ? adj::transpose2_kernel<C, CF, TP, true> : adj::transpose2_kernel<C, CF, TP, false>)<<<nb, 256, 0, h->stream>>>(
        h->d_inst, tabs, a, T, phi_n, (const C*)v.phib, (const C*)v.mub, (const C*)v.Db, (const C*)v.ub, lam_next,
        lam, v.ds);
    h->adj_par ^= 1;
    return cudaGetLastError();
}

template <typename C>
cudaError_t adjoint_end_t(lbch_handle* h, C* dphi0)
{
    AdjView v = adj_view(h);
    adj::AdjArgs a = adj_args(h, 0);
    const long long N = (long long)a.nx * a.ny;
    const int nb = (int)((N + 255) / 256);
    const double T = vel_t(h->inst[0].vel, h->inst[0].Tper, 0);
    const C* lam = static_cast<const C*>(v.lam[h->adj_par]);
    (adj_planes(h) == 1 ? adj::init_local_kernel<C, true> : adj::init_local_kernel<C, false>)<<<nb, 256, 0, h->stream>>>(
        h->d_inst, h->d_tabs, a, T, h->phi0, h->pitch, lam, (C*)v.mub, dphi0, v.ds);
    adj::init_transpose_kernel<C><<<nb, 256, 0, h->stream>>>(h->d_inst, a, h->phi0, h->pitch, (const C*)v.mub, dphi0);
    adj::sum_into_kernel<<<1, 256, 0, h->stream>>>(v.ds, N, v.dLds);
    return cudaGetLastError();
}

// lb_ch_init and lb_ch_init_slab.  With a slab, params is the one instance of the slab (the global problem
// with ny = slab->ny), gparams the global problem (for the velocity tables), and phi0 holds slab->ny + 2 GR
// rows: the slab's rows with GR rows of each neighbour (global rows y0 - GR .. y0 + ny + GR - 1, wrapped).
lbch_status init_impl(const lbch_params* params, int n_inst, const double* phi0, int prec, void* stream,
                      lbch_handle** out, const SlabSpec* slab, const lbch_params* gparams)
{
    if (!out) return fail(LBCH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || !phi0 || n_inst < 1) return fail(LBCH_EINVAL, "params/phi0 NULL or n_inst < 1");
    if (prec != LBCH_F64 && prec != LBCH_F32 && prec != LBCH_F16S) return fail(LBCH_EINVAL, "unknown precision %d", prec);
    for (int k = 0; k < n_inst; k++) {
        lbch_status s = check_params(params[k], k);
        if (s != LBCH_OK) return s;
    }
    bool coupled = false;
    for (int k = 0; k < n_inst; k++) coupled = coupled || params[k].vel == LBCH_VEL_COUPLED;
    if (coupled && (n_inst != 1 || prec == LBCH_F16S))
        return fail(LBCH_EINVAL, "the coupled flow needs a single instance in LBCH_F64 or LBCH_F32");
    if (coupled && (long long)params[0].nx * params[0].ny >= (1LL << 31))
        return fail(LBCH_EINVAL, "the coupled flow supports grids of fewer than 2^31 nodes");
    lbch_handle* h = new (std::nothrow) lbch_handle();
    if (!h) return fail(LBCH_ENOMEM, "host allocation failed");
    h->prec = prec;
    h->slab = slab != nullptr;
    h->coupled = coupled;
    h->tau1 = !coupled;
    for (int k = 0; k < n_inst; k++) h->tau1 = h->tau1 && params[k].tau == 1.0;
    h->n_inst = n_inst;
    for (int k = 0; k < n_inst; k++) h->model3 = h->model3 || params[k].model == 3;
    for (int k = 0; k < n_inst; k++) h->walls = h->walls || params[k].walls != 0;
    for (int k = 0; k < n_inst; k++)  // the flows with a time factor (vel_t), and Model III's first step
        h->need_time = h->need_time || params[k].model == 3 || params[k].vel == LBCH_VEL_VORTEX ||
                       params[k].vel == LBCH_VEL_DEFORM || params[k].vel == LBCH_VEL_REV_SHEAR;
    h->g_elem = prec == LBCH_F64 ? 8 : (prec == LBCH_F32 ? 4 : 2);
    h->phi_elem = prec == LBCH_F64 ? 8 : 4;  // the float path adds a float low part
    h->nq = prec == LBCH_F16S ? 8 : 9;

    // layout: uniform pitch; instance k takes ny_k + 2 GR stored rows
    h->inst.resize(n_inst);
    h->node_begin.resize(n_inst + 1);
    std::vector<double> tabs;
    int row = 0, max_w = 0;
    for (int k = 0; k < n_inst; k++) {
        const lbch_params& p = params[k];
        InstDev& d = h->inst[k];
        std::memset(&d, 0, sizeof d);
        derive(p, d);
        d.nx = p.nx;
        d.ny = p.ny;
        d.slab = slab ? 1 : 0;
        d.row0 = row + GR;
        // the Y slice of a tile spans TY + 8 rows from its first halo row; the last tile of a shape whose TY does
        // not divide 16 (FP64 32 x 14) reaches up to 15 rows past ny rounded up to 16, so 16 more entries
        d.ylen = (p.ny + 15) / 16 * 16 + 8 + 16;
        row += p.ny + 2 * GR;
        max_w = std::max(max_w, (p.nx + 31) / 32 * 32);
        h->node_begin[k] = h->nodes;
        h->nodes += (long long)p.nx * p.ny;
    }
    h->node_begin[n_inst] = h->nodes;
    h->rows = row;
    h->pitch = (max_w + 8 + 7) / 8 * 8;  // boxes reach 4 columns past the last tile; 16-byte rows for half
    std::vector<int> tile_begin[kMaxShapes];
    for (int sk = 0; sk < n_shapes(prec); sk++) {
        const Shape sh = shape_of(prec, sk);
        int t = 0;
        for (int k = 0; k < n_inst; k++) {
            tile_begin[sk].push_back(t);
            t += ((params[k].nx + sh.tx - 1) / sh.tx) * ((params[k].ny + sh.ty - 1) / sh.ty);
        }
        tile_begin[sk].push_back(t);
        h->ps[sk].total_tiles = t;
    }
    std::vector<int> sweep_begin[kSweepShapes];
    for (int sk = 0; sk < kSweepShapes; sk++) {
        const Shape sh = sweep_tile(sk);
        int t = 0;
        for (int k = 0; k < n_inst; k++) {
            sweep_begin[sk].push_back(t);
            t += ((params[k].nx + sh.tx - 1) / sh.tx) * ((params[k].ny + sh.ty - 1) / sh.ty);
        }
        sweep_begin[sk].push_back(t);
        h->sw[sk].total_tiles = t;
    }
    std::vector<int> pair_begin[kPairShapes];
    for (int sk = 0; sk < kPairShapes; sk++) {
        const Shape sh = pair_shape(prec, sk);
        int t = 0;
        for (int k = 0; k < n_inst; k++) {
            pair_begin[sk].push_back(t);
            t += ((params[k].nx + sh.tx - 1) / sh.tx) * ((params[k].ny + sh.ty - 1) / sh.ty);
        }
        pair_begin[sk].push_back(t);
        h->pr[sk].total_tiles = t;
    }
    for (int k = 0; k < n_inst; k++) {
        h->inst[k].tab = (int)tabs.size();
        if (slab) velocity_tables(*gparams, h->pitch, h->inst[k].ylen, tabs, slab);
        else velocity_tables(params[k], h->pitch, h->inst[k].ylen, tabs);
    }
    std::vector<float> tabs_f(tabs.begin(), tabs.end());

    auto bail = [&](lbch_status s) { release(h); delete h; return s; };
    cudaError_t e;
#define CKI(call)                                                    \
    do {                                                             \
        e = (call);                                                  \
        if (e != cudaSuccess) return bail(cuda_fail(e, #call));      \
    } while (0)
    CKI(cudaGetDevice(&h->device));
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        CKI(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    CKI(device_pool(h->device, &h->pool));
    // (every buffer below is allocated and filled in the order of the handle's stream; the uploads from
    // pageable host memory return once the driver has taken the data, so the host vectors may go)
    for (int sk = 0; sk < n_shapes(prec); sk++) {
        CKI(prepare_step(h, sk));
        CKI(dalloc(h, &h->ps[sk].d_tile_begin, sizeof(int) * (n_inst + 1)));
        CKI(cudaMemcpyAsync(h->ps[sk].d_tile_begin, tile_begin[sk].data(), sizeof(int) * (n_inst + 1),
                            cudaMemcpyHostToDevice, h->stream));
    }
    if (!coupled) {
        for (int sk = 0; sk < kSweepShapes; sk++) {
            CKI(prepare_sweep(h, sk));
            CKI(dalloc(h, &h->sw[sk].d_tile_begin, sizeof(int) * (n_inst + 1)));
            CKI(cudaMemcpyAsync(h->sw[sk].d_tile_begin, sweep_begin[sk].data(), sizeof(int) * (n_inst + 1),
                                cudaMemcpyHostToDevice, h->stream));
            // the tiles of every instance, those that need the wall body (their collision rows or the rows
            // their stencils read come within two rows of a wall) after all the others
            const Shape sh = sweep_tile(sk);
            std::vector<int4> inner, edge;
            for (int k = 0; k < n_inst; k++) {
                const lbch_params& p = params[k];
                const int tiles_x = (p.nx + sh.tx - 1) / sh.tx, tiles_y = (p.ny + sh.ty - 1) / sh.ty;
                for (int l = 0; l < tiles_x * tiles_y; l++) {
                    const int x0 = (l % tiles_x) * sh.tx, y0 = (l / tiles_x) * sh.ty;
                    const bool w = p.walls && (y0 < 2 || y0 + sh.ty + 1 > p.ny - 1);
                    (w ? edge : inner).push_back(make_int4(k, x0, y0, w ? 1 : 0));
                }
            }
            inner.insert(inner.end(), edge.begin(), edge.end());
            CKI(dalloc(h, &h->sw[sk].d_tiles, sizeof(int4) * inner.size()));
            CKI(cudaMemcpyAsync(h->sw[sk].d_tiles, inner.data(), sizeof(int4) * inner.size(), cudaMemcpyHostToDevice,
                                h->stream));
        }
        for (int sk = 0; sk < kPairShapes && prec != LBCH_F16S; sk++) {
            CKI(lbch_prepare_pair(h, sk));
            CKI(dalloc(h, &h->pr[sk].d_tile_begin, sizeof(int) * (n_inst + 1)));
            CKI(cudaMemcpyAsync(h->pr[sk].d_tile_begin, pair_begin[sk].data(), sizeof(int) * (n_inst + 1),
                                cudaMemcpyHostToDevice, h->stream));
            // each tile's velocity tables over the tile + 6 (periodically wrapped), contiguous per tile so that
            // one bulk copy brings them (the layout of PairShape: X1, X2 by column, Y1, Y2 by row, 16-byte
            // padded)
            const Shape sh = pair_shape(prec, sk);
            const int W6 = sh.tx + 12, H6 = sh.ty + 12;
            const size_t esz = prec == LBCH_F64 ? 8 : 4;
            const size_t stride = ((size_t)(2 * (W6 + H6)) * esz + 15) / 16 * 16 / esz;
            std::vector<double> tt((size_t)h->pr[sk].total_tiles * stride, 0.0);
            for (int k = 0; k < n_inst; k++) {
                const InstDev& d = h->inst[k];
                const double* X1 = &tabs[d.tab];
                const double* X2 = X1 + h->pitch;
                const double* Y1 = X2 + h->pitch;
                const double* Y2 = Y1 + d.ylen;
                const int tiles_x = (d.nx + sh.tx - 1) / sh.tx, tiles_y = (d.ny + sh.ty - 1) / sh.ty;
                for (int l = 0; l < tiles_x * tiles_y; l++) {
                    const int x0 = (l % tiles_x) * sh.tx, y0 = (l / tiles_x) * sh.ty;
                    double* o = &tt[(size_t)(pair_begin[sk][k] + l) * stride];
                    for (int c = 0; c < W6; c++) {
                        const int x = ((x0 - 6 + c) % d.nx + d.nx) % d.nx;
                        o[c] = X1[GC + x];
                        o[W6 + c] = X2[GC + x];
                    }
                    for (int r = 0; r < H6; r++) {
                        const int y = ((y0 - 6 + r) % d.ny + d.ny) % d.ny;
                        o[2 * W6 + r] = Y1[GR + y];
                        o[2 * W6 + H6 + r] = Y2[GR + y];
                    }
                }
            }
            CKI(dalloc(h, &h->pr[sk].d_ttabs, tt.size() * esz));
            if (prec == LBCH_F64) {
                CKI(cudaMemcpyAsync(h->pr[sk].d_ttabs, tt.data(), tt.size() * esz, cudaMemcpyHostToDevice, h->stream));
            } else {
                std::vector<float> tf(tt.begin(), tt.end());  // rounded as the float tables are
                CKI(cudaMemcpyAsync(h->pr[sk].d_ttabs, tf.data(), tf.size() * esz, cudaMemcpyHostToDevice, h->stream));
            }
        }
    }
    const size_t cells = (size_t)h->rows * h->pitch;
    const size_t gbytes = cells * h->nq * h->g_elem;
    const size_t pbytes = cells * h->phi_elem;
    for (int k = 0; k < 2; k++) {
        CKI(dalloc(h, &h->g[k], gbytes));
        CKI(dalloc(h, &h->phi[k], pbytes));
        if (prec == LBCH_F32) CKI(dalloc(h, &h->lo[k], cells * sizeof(float)));
        if (h->model3) CKI(dalloc(h, &h->H[k], 2 * cells * h->c_elem()));
    }
    CKI(dalloc(h, &h->phi0, cells * sizeof(double)));
    CKI(dalloc(h, &h->d_inst, sizeof(InstDev) * n_inst));
    CKI(dalloc(h, &h->d_node_begin, sizeof(long long) * (n_inst + 1)));
    CKI(dalloc(h, &h->d_tabs, sizeof(double) * tabs.size()));
    CKI(dalloc(h, &h->d_tabs_f, sizeof(float) * tabs_f.size()));
    CKI(dalloc(h, &h->ctl, sizeof(Ctl)));
    long long max_nodes = 0;
    for (auto& d : h->inst) max_nodes = std::max(max_nodes, (long long)d.nx * d.ny);
    h->chunks = (int)std::min<long long>(1024, (max_nodes + RED_NT * 8 - 1) / (RED_NT * 8));
    if (h->chunks < 1) h->chunks = 1;
    CKI(dalloc(h, &h->partials, sizeof(double) * RED_NV * (size_t)h->chunks * n_inst));
    CKI(dalloc(h, &h->result, sizeof(double) * RED_NV * (size_t)n_inst));
    lbch_status st = LBCH_OK;
    for (int sk = 0; sk < n_shapes(prec) && st == LBCH_OK; sk++) st = encode_maps(h, sk);
    for (int sk = 0; !coupled && sk < kSweepShapes && st == LBCH_OK; sk++) st = encode_sweep_maps(h, sk);
    if (!coupled && st == LBCH_OK) st = encode_row_maps(h);
    if (st != LBCH_OK) return bail(st);

    // the initial field in the padded layout, ghost frame included, through pinned staging
    st = stage(h, cells * sizeof(double));
    if (st != LBCH_OK) return bail(st);
    std::memset(h->h_stage, 0, cells * sizeof(double));
    const double* src = phi0;
    for (int k = 0; k < n_inst; k++) {
        const InstDev& d = h->inst[k];
        for (int y = -GR; y < d.ny + GR; y++) {
            int yy;
            const double* srow;
            if (slab) {
                srow = src + (size_t)(y + GR) * d.nx;  // the slab's field comes with its neighbours' rows
            } else {
                if (d.walls) yy = y < 0 ? -1 - y : (y >= d.ny ? 2 * d.ny - 1 - y : y);
                else yy = ((y % d.ny) + d.ny) % d.ny;
                yy = std::min(std::max(yy, 0), d.ny - 1);
                srow = src + (size_t)yy * d.nx;
            }
            double* rowp = h->h_stage + (size_t)(d.row0 + y) * h->pitch + GC;
            for (int x = -GC; x < d.nx + GC; x++) rowp[x] = srow[((x % d.nx) + d.nx) % d.nx];
        }
        src += (size_t)d.nx * d.ny;
    }
    CKI(cudaMemcpyAsync(h->phi0, h->h_stage, cells * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CKI(cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(InstDev) * n_inst, cudaMemcpyHostToDevice, h->stream));
    CKI(cudaMemcpyAsync(h->d_node_begin, h->node_begin.data(), sizeof(long long) * (n_inst + 1), cudaMemcpyHostToDevice, h->stream));
    CKI(cudaMemcpyAsync(h->d_tabs, tabs.data(), sizeof(double) * tabs.size(), cudaMemcpyHostToDevice, h->stream));
    CKI(cudaMemcpyAsync(h->d_tabs_f, tabs_f.data(), sizeof(float) * tabs_f.size(), cudaMemcpyHostToDevice, h->stream));
    CKI(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
    for (int k = 0; k < 2; k++) {
        CKI(cudaMemsetAsync(h->g[k], 0, gbytes, h->stream));
        CKI(cudaMemsetAsync(h->phi[k], 0, pbytes, h->stream));
        if (h->lo[k]) CKI(cudaMemsetAsync(h->lo[k], 0, cells * sizeof(float), h->stream));
    }
    int nb = (int)((h->nodes + 255) / 256);
    switch (prec) {
    case LBCH_F64:
        init_kernel<double, double, double><<<nb, 256, 0, h->stream>>>(h->d_inst, n_inst, h->d_tabs, h->phi0, h->pitch,
            (double*)h->g[0], (double*)h->phi[0], nullptr, h->nodes, h->d_node_begin);
        break;
    case LBCH_F32:
        init_kernel<float, float, float><<<nb, 256, 0, h->stream>>>(h->d_inst, n_inst, h->d_tabs, h->phi0, h->pitch,
            (float*)h->g[0], (float*)h->phi[0], h->lo[0], h->nodes, h->d_node_begin);
        break;
    default:
        init_kernel<float, __half, float><<<nb, 256, 0, h->stream>>>(h->d_inst, n_inst, h->d_tabs, h->phi0, h->pitch,
            (__half*)h->g[0], (float*)h->phi[0], nullptr, h->nodes, h->d_node_begin);
    }
    CKI(cudaGetLastError());
    if (coupled) {
        const lbch_params& p = params[0];
        const InstDev& d = h->inst[0];
        double dphi = std::fabs(p.phiA - p.phiB);
        double beta = 12.0 * p.sigma / (p.W * dphi * dphi * dphi * dphi);
        double M = p.M > 0.0 ? p.M : p.Ustar * p.W / (p.Pe * beta * (p.phiA - p.phiB) * (p.phiA - p.phiB));
        h->nsd.tauf = 3.0 * p.nu + 0.5;     // nu = c_s^2 (tau_f - 1/2)
        h->nsd.gx = p.gx; h->nsd.gy = p.gy; h->nsd.M = M; h->nsd.rbar = 0.5 * (p.rhoA + p.rhoB);
        h->nsf.tauf = (float)h->nsd.tauf; h->nsf.gx = (float)p.gx; h->nsf.gy = (float)p.gy;
        h->nsf.M = (float)M; h->nsf.rbar = (float)h->nsd.rbar;
        h->nsd.itauf = 1.0 / h->nsd.tauf; h->nsd.omtf = 1.0 - h->nsd.itauf; h->nsd.srcf = 1.0 - 0.5 / h->nsd.tauf;
        h->nsf.itauf = (float)h->nsd.itauf; h->nsf.omtf = (float)h->nsd.omtf; h->nsf.srcf = (float)h->nsd.srcf;
        const size_t N = (size_t)d.nx * d.ny, esz = prec == LBCH_F64 ? 8 : 4;
        CKI(dalloc(h, &h->ns, 40 * N * esz));  // f, g (two buffers each), u, p, mu
        CKI(cudaMemsetAsync(h->ns, 0, 40 * N * esz, h->stream));
        const int nbn = (int)((N + 255) / 256);
        if (prec == LBCH_F64) {
            ns::NsArgs<double> a = ns_args<double>(h, 1);  // writes the parity-0 buffers
            ns::init_kernel<double><<<nbn, 256, 0, h->stream>>>(a, h->phi0);
        } else {
            ns::NsArgs<float> a = ns_args<float>(h, 1);
            ns::init_kernel<float><<<nbn, 256, 0, h->stream>>>(a, h->phi0);
        }
        CKI(cudaGetLastError());
    }
    CKI(cudaStreamSynchronize(h->stream));  // the pinned staging buffer and the tables are reused after this
#undef CKI
    // Kernel before any tuning: the two-step kernel where it applies and its tiles fit the device in one
    // wave (a step of such a grid is bound by latency, and one launch per two steps halves the launches);
    // otherwise the row sweep.  lb_ch_tune measures instead.
    const int k2 = prec == LBCH_F64 ? 3 : 1;  // 32 x 14 tiles in either precision
    if (pair_ok(h) && h->pr[k2].d_tile_begin && h->pr[k2].grid == h->pr[k2].total_tiles) {
        h->pair = true;
        h->pshape = k2;
    }
    *out = h;
    return LBCH_OK;
}

}  // namespace

extern "C" {

lbch_status lb_ch_init(const lbch_params* params, int n_inst, const double* phi0, int prec, void* stream,
                       lbch_handle** out)
{
    NvtxRange nvtx_("lb_ch_init");
    return init_impl(params, n_inst, phi0, prec, stream, out, nullptr, nullptr);
}

lbch_status lb_ch_init_slab(const lbch_params* global, int y0, int ny_local, const double* phi0_halo, int prec,
                            void* stream, lbch_handle** out)
{
    NvtxRange nvtx_("lb_ch_init_slab");
    if (!out) return fail(LBCH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!global || !phi0_halo) return fail(LBCH_EINVAL, "global params or phi0 NULL");
    lbch_status st = check_params(*global, 0);
    if (st != LBCH_OK) return st;
    if (global->walls != 0) return fail(LBCH_EINVAL, "slabs split grids that are periodic in y (walls = 0)");
    if (global->vel == LBCH_VEL_COUPLED) return fail(LBCH_EINVAL, "slabs take prescribed flows");
    if (global->model == 3) return fail(LBCH_EINVAL, "slabs take Models I and II");
    if (y0 < 0 || ny_local < 4 || y0 >= global->ny || ny_local > global->ny - y0)
        return fail(LBCH_EINVAL, "slab rows [%d, %d) must lie in [0, %d) and number at least 4", y0, y0 + ny_local,
                    global->ny);
    lbch_params local = *global;
    local.ny = ny_local;
    const SlabSpec spec{y0, ny_local};
    return init_impl(&local, 1, phi0_halo, prec, stream, out, &spec, global);
}

lbch_status lb_ch_step(lbch_handle* h, long nsteps)
{
    NvtxRange nvtx_("lb_ch_step");
    if (!h || nsteps < 0) return fail(LBCH_EINVAL, "NULL handle or negative step count");
    if (h->slab && nsteps > 1 && !h->tuning)
        return fail(LBCH_EINVAL, "a slab handle advances one step per call: import its halos before every step");
    static const bool no_graph = std::getenv("LBCH_NO_GRAPH") != nullptr;
    const bool two = use_pair(h);
    while (nsteps > 0) {
        int parity = cur_buf(h);
        if (!no_graph && !h->debug_skip && nsteps >= kGraphChunk) {
            const int z = nsteps >= kGraphBig ? 1 : 0, chunk = z ? kGraphBig : kGraphChunk;
            cudaGraphExec_t& gx = h->graph[z][parity];
            if (!gx) {
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = cudaSuccess;
                // step k of the graph is the counter + k; only the last launch advances the counter.  With
                // the two-step kernel, launch s takes steps 2s and 2s + 1; the chunk's launch count is even,
                // so the graph ends in the buffer it starts from, as the one-step graph does.
                const int per = two ? 2 : 1, launches = chunk / per;
                for (int s = 0; s < launches && e == cudaSuccess; s++) {
                    h->t_off = s * per;
                    h->t_adv = s == launches - 1 ? chunk : 0;
                    e = two ? lbch_launch_pair(h, parity ^ (s & 1)) : launch_step(h, parity ^ (s & 1));
                }
                h->t_off = 0;
                h->t_adv = 1;
                cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
                if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "step launch during capture"); }
                if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&gx, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) { gx = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
            }
            CK(cudaGraphLaunch(gx, h->stream));
            h->n += chunk;
            nsteps -= chunk;
        } else if (two && nsteps >= 2) {
            CK(launch_pair_now(h));
            nsteps -= 2;
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
    NvtxRange nvtx_("lb_ch_observe");
    if (!h || !out) return fail(LBCH_EINVAL, "NULL handle or output");
    if (inst < 0 || inst >= h->n_inst) return fail(LBCH_EINVAL, "instance %d out of range", inst);
    if (what == LBCH_OBS_STEP) {
        *out = (double)h->n;
        return LBCH_OK;
    }
    CK(coupled_phi(h));
    if (what == LBCH_OBS_PHI) {
        const InstDev& d = h->inst[inst];
        int parity = cur_buf(h);
        lbch_status s = stage(h, (size_t)d.nx * d.ny * sizeof(double));
        if (s != LBCH_OK) return s;
        const size_t off = (size_t)d.row0 * h->pitch + GC;
        const char* base = static_cast<const char*>(h->phi[parity]) + off * h->phi_elem;
        CK(cudaMemcpy2DAsync(h->h_stage, (size_t)d.nx * h->phi_elem, base, (size_t)h->pitch * h->phi_elem,
                             (size_t)d.nx * h->phi_elem, d.ny, cudaMemcpyDeviceToHost, h->stream));
        float* lo_host = nullptr;
        if (h->lo[parity]) {  // the low part goes to the upper half of the staging buffer
            lo_host = reinterpret_cast<float*>(h->h_stage) + (size_t)d.nx * d.ny;
            CK(cudaMemcpy2DAsync(lo_host, (size_t)d.nx * 4, h->lo[parity] + off, (size_t)h->pitch * 4,
                                 (size_t)d.nx * 4, d.ny, cudaMemcpyDeviceToHost, h->stream));
        }
        s = check_err(h);  // synchronises the stream
        if (s != LBCH_OK) return s;
        long long N = (long long)d.nx * d.ny;
        bool finite = true;
        if (h->phi_elem == 8) {
            std::memcpy(out, h->h_stage, sizeof(double) * N);
        } else {
            const float* f = reinterpret_cast<const float*>(h->h_stage);
            for (long long k = 0; k < N; k++) out[k] = (double)f[k] + (lo_host ? (double)lo_host[k] : 0.0);
        }
        for (long long k = 0; k < N; k++) finite = finite && std::isfinite(out[k]);
        return finite ? LBCH_OK : fail(LBCH_ENONFINITE, "phi holds non-finite values");
    }
    if (what == LBCH_OBS_U || what == LBCH_OBS_P) {
        if (!h->coupled) return fail(LBCH_EINVAL, "velocity and pressure are observable on coupled handles only");
        const int parity = cur_buf(h);
        CK(h->prec == LBCH_F64 ? ns_fields_t<double>(h, parity) : ns_fields_t<float>(h, parity));
        const size_t N = (size_t)h->inst[0].nx * h->inst[0].ny, e = h->prec == LBCH_F64 ? 8 : 4;
        lbch_status s = stage(h, 2 * N * sizeof(double));
        if (s != LBCH_OK) return s;
        const char* w = static_cast<const char*>(h->ns) + 36 * N * e;  // ux, uy, pr, mu
        if (what == LBCH_OBS_U) CK(cudaMemcpyAsync(h->h_stage, w, 2 * N * e, cudaMemcpyDeviceToHost, h->stream));
        else CK(cudaMemcpyAsync(h->h_stage, w + 2 * N * e, N * e, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        const size_t cnt = what == LBCH_OBS_U ? 2 * N : N;
        if (e == 8) std::memcpy(out, h->h_stage, cnt * 8);
        else for (size_t k = 0; k < cnt; k++) out[k] = (double)reinterpret_cast<const float*>(h->h_stage)[k];
        return LBCH_OK;
    }
    if (what < LBCH_OBS_MASS || what > LBCH_OBS_MIN) return fail(LBCH_EINVAL, "unknown observable %d", what);
    lbch_status s = run_reduce(h);
    if (s != LBCH_OK) return s;
    double r[RED_NV];
    CK(cudaMemcpyAsync(r, h->result + (size_t)inst * RED_NV, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    s = check_err(h);
    if (s != LBCH_OK) return s;
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
    CK(coupled_phi(h));
    lbch_status s = run_reduce(h);
    if (s != LBCH_OK) return s;
    std::vector<double> r((size_t)RED_NV * h->n_inst);
    CK(cudaMemcpyAsync(r.data(), h->result, sizeof(double) * r.size(), cudaMemcpyDeviceToHost, h->stream));
    s = check_err(h);
    if (s != LBCH_OK) return s;
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
    double bytes = 2.0 * (h->nq * (double)h->g_elem + (double)h->phi_elem + (h->lo[0] ? 4.0 : 0.0));
    if (h->tau1 && !h->force_general)  // only phi is read and written (either kernel form)
        bytes = 2.0 * ((double)h->phi_elem + (h->lo[0] ? 4.0 : 0.0));
    if (use_pair(h)) bytes *= 0.5;     // the two-step kernel reads and writes phi once per two updates
    if (h->model3) bytes += 2.0 * 2.0 * (double)h->c_elem();  // H of Model III, read and written
    if (h->coupled) {  // f and g read and written, phi read and written, u and p written and read
        const double e = h->prec == LBCH_F64 ? 8.0 : 4.0;
        bytes = 2.0 * (18.0 * e + e) + 2.0 * 3.0 * e;
    }
    out[0] = (double)h->nodes;
    out[1] = bytes;
    out[2] = (double)active_grid(h);
    out[3] = (double)h->n;
    return LBCH_OK;
}

lbch_status lb_ch_kernel_info(lbch_handle* h, int* out)
{
    if (!h || !out) return fail(LBCH_EINVAL, "NULL handle or output");
    const Shape sh = active_tile(h);
    const bool sw = use_sweep(h);
    const bool pr = use_pair(h);
    out[0] = h->coupled ? 3 : pr ? 5 : (!sw ? (sweep_gen(h) ? 0 : 4) : (sweep_gen(h) ? 2 : 1));
    out[1] = pr ? h->pshape : h->shape;
    out[2] = sh.tx;
    out[3] = sh.ty;
    out[4] = sw && !pr ? kSweep[h->shape].ty : 0;
    out[5] = h->coupled ? 256 : sh.nt;
    return LBCH_OK;
}

void* lb_ch_stream(lbch_handle* h) { return h ? (void*)h->stream : nullptr; }

lbch_status lb_ch_state_bytes(lbch_handle* h, long long* bytes)
{
    if (!h || !bytes) return fail(LBCH_EINVAL, "NULL handle or output");
    *bytes = (long long)state_bytes(h);
    return LBCH_OK;
}

lbch_status lb_ch_state_save(lbch_handle* h, void* dst)
{
    if (!h || !dst) return fail(LBCH_EINVAL, "NULL handle or buffer");
    if (h->coupled) return fail(LBCH_EINVAL, "checkpoints are for prescribed-flow handles");
    const int par = cur_buf(h);
    const size_t cells = (size_t)h->rows * h->pitch;
    char* p = static_cast<char*>(dst);
    const StateHeader hd = state_header(h, h->n);
    CK(cudaMemcpyAsync(p, &hd, sizeof hd, cudaMemcpyHostToDevice, h->stream));
    p += 256;
    size_t gb = cells * h->nq * h->g_elem, pb = cells * h->phi_elem;
    CK(cudaMemcpyAsync(p, h->g[par], gb, cudaMemcpyDeviceToDevice, h->stream));
    p += (gb + 255) / 256 * 256;
    CK(cudaMemcpyAsync(p, h->phi[par], pb, cudaMemcpyDeviceToDevice, h->stream));
    p += (pb + 255) / 256 * 256;
    if (h->lo[par]) CK(cudaMemcpyAsync(p, h->lo[par], cells * 4, cudaMemcpyDeviceToDevice, h->stream));
    if (h->lo[par]) p += (cells * 4 + 255) / 256 * 256;
    if (h->model3) CK(cudaMemcpyAsync(p, h->H[par], 2 * cells * h->c_elem(), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));  // the header was copied from a host variable
    return LBCH_OK;
}

lbch_status lb_ch_state_load(lbch_handle* h, const void* src)
{
    if (!h || !src) return fail(LBCH_EINVAL, "NULL handle or buffer");
    if (h->coupled) return fail(LBCH_EINVAL, "checkpoints are for prescribed-flow handles");
    const char* p = static_cast<const char*>(src);
    StateHeader hd;
    CK(cudaMemcpyAsync(&hd, p, sizeof hd, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (hd.magic != kStateMagic) return fail(LBCH_EINVAL, "buffer does not hold a saved state");
    const StateHeader mine = state_header(h, hd.n);
    if (hd.bytes != mine.bytes || hd.prec != mine.prec || hd.nq != mine.nq || hd.rows != mine.rows ||
        hd.pitch != mine.pitch || hd.n_inst != mine.n_inst || hd.model3 != mine.model3 || hd.lo != mine.lo ||
        hd.layout != mine.layout)
        return fail(LBCH_EINVAL,
                    "saved state does not fit this handle (saved: %lld bytes, precision %d, %d instance(s), %d x %d "
                    "stored cells; this handle: %lld bytes, precision %d, %d instance(s), %d x %d)",
                    hd.bytes, hd.prec, hd.n_inst, hd.rows, hd.pitch, mine.bytes, mine.prec, mine.n_inst, mine.rows,
                    mine.pitch);
    const long long n = hd.n;
    if (n < 0) return fail(LBCH_EINVAL, "buffer does not hold a saved state");
    const int par = (int)(n & 1);
    const size_t cells = (size_t)h->rows * h->pitch;
    p += 256;
    size_t gb = cells * h->nq * h->g_elem, pb = cells * h->phi_elem;
    CK(cudaMemcpyAsync(h->g[par], p, gb, cudaMemcpyDeviceToDevice, h->stream));
    p += (gb + 255) / 256 * 256;
    CK(cudaMemcpyAsync(h->phi[par], p, pb, cudaMemcpyDeviceToDevice, h->stream));
    p += (pb + 255) / 256 * 256;
    if (h->lo[par]) CK(cudaMemcpyAsync(h->lo[par], p, cells * 4, cudaMemcpyDeviceToDevice, h->stream));
    if (h->lo[par]) p += (cells * 4 + 255) / 256 * 256;
    if (h->model3) CK(cudaMemcpyAsync(h->H[par], p, 2 * cells * h->c_elem(), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(&h->ctl->time, &n, sizeof n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->n = n;
    h->flip = 0;  // the state was written into the buffers of step n
    return LBCH_OK;
}

lbch_status lb_ch_halo_bytes(lbch_handle* h, long long* bytes)
{
    if (!h || !bytes) return fail(LBCH_EINVAL, "NULL handle or output");
    if (!h->slab) return fail(LBCH_EINVAL, "halos belong to slab handles (lb_ch_init_slab)");
    *bytes = (long long)halo_bytes(h);
    return LBCH_OK;
}

lbch_status lb_ch_halo_export(lbch_handle* h, int side, void* dst)
{
    if (!h || !dst || (side != 0 && side != 1)) return fail(LBCH_EINVAL, "NULL handle or buffer, or side not 0/1");
    if (!h->slab) return fail(LBCH_EINVAL, "halos belong to slab handles (lb_ch_init_slab)");
    const InstDev& d = h->inst[0];
    // side 0: domain rows 0..GR-1 and the populations of row 0; side 1: rows ny-GR..ny-1 and row ny-1
    return halo_copy(h, dst, d.row0 + (side == 0 ? 0 : d.ny - GR), d.row0 + (side == 0 ? 0 : d.ny - 1), true);
}

lbch_status lb_ch_halo_import(lbch_handle* h, int side, const void* src)
{
    if (!h || !src || (side != 0 && side != 1)) return fail(LBCH_EINVAL, "NULL handle or buffer, or side not 0/1");
    if (!h->slab) return fail(LBCH_EINVAL, "halos belong to slab handles (lb_ch_init_slab)");
    const InstDev& d = h->inst[0];
    // side 0: ghost rows -GR..-1 and the populations of row -1; side 1: rows ny..ny+GR-1 and row ny
    return halo_copy(h, const_cast<void*>(src), d.row0 + (side == 0 ? -GR : d.ny), d.row0 + (side == 0 ? -1 : d.ny),
                     false);
}

lbch_status lb_ch_step_taped(lbch_handle* h, long nsteps, void* tape)
{
    NvtxRange nvtx_("lb_ch_step_taped");
    if (!h || !tape || nsteps < 0) return fail(LBCH_EINVAL, "NULL handle or tape, or negative step count");
    if (h->n_inst != 1 || h->coupled || h->slab)
        return fail(LBCH_EINVAL, "taped steps are for single-instance prescribed-flow handles of a whole grid");
    const long long N = (long long)h->inst[0].nx * h->inst[0].ny;
    if (N >= (1LL << 31)) return fail(LBCH_EINVAL, "the adjoint supports grids of fewer than 2^31 nodes");
    const size_t stride = (size_t)N * (h->prec == LBCH_F64 ? 8 : 4);
    char* t = static_cast<char*>(tape);
    static const bool no_graph = std::getenv("LBCH_NO_GRAPH") != nullptr;
    // Long replays go through a captured graph (one per parity, kept while the tape and length repeat, as
    // the segments of a reverse sweep do); step k of it runs step counter + k, and only its last launch
    // advances the counter.
    if (!no_graph && !h->debug_skip && nsteps >= 8) {
        const int parity = cur_buf(h);
        lbch_handle::TapeGraph& tg = h->tgraph[parity];
        if (!tg.exec || tg.tape != tape || tg.nsteps != nsteps) {
            if (tg.exec) cudaGraphExecDestroy(tg.exec);
            tg.exec = nullptr;
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (long k = 0; k < nsteps && e == cudaSuccess; k++) {
                e = tape_launch(h, parity ^ (int)(k & 1), t + (size_t)k * stride);
                h->t_off = (int)k;
                h->t_adv = k == nsteps - 1 ? (int)nsteps : 0;
                if (e == cudaSuccess) e = launch_step(h, parity ^ (int)(k & 1));
            }
            h->t_off = 0;
            h->t_adv = 1;
            cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
            if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(e, "taped step launch during capture"); }
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&tg.exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { tg.exec = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
            tg.tape = tape;
            tg.nsteps = nsteps;
        }
        CK(cudaGraphLaunch(tg.exec, h->stream));
        h->n += nsteps;
        return LBCH_OK;
    }
    for (long k = 0; k < nsteps; k++) {
        CK(tape_launch(h, cur_buf(h), t + (size_t)k * stride));
        CK(launch_step(h, cur_buf(h)));  // a one-step launch (the two-step kernel would skip a tape entry)
        h->n += 1;
    }
    return LBCH_OK;
}

lbch_status lb_ch_adjoint_sweep(lbch_handle* h, const void* tape, long n0, long nsteps)
{
    NvtxRange nvtx_("lb_ch_adjoint_sweep");
    if (!h || !tape || n0 < 0 || nsteps < 0) return fail(LBCH_EINVAL, "NULL handle or tape, or negative step");
    if (!h->adj) return fail(LBCH_EINVAL, "lb_ch_adjoint_begin was not called");
    const long long N = (long long)h->inst[0].nx * h->inst[0].ny;
    const size_t stride = (size_t)N * (h->prec == LBCH_F64 ? 8 : 4);
    const char* t = static_cast<const char*>(tape);
    for (long k = nsteps - 1; k >= 0; k--) {
        cudaError_t e = h->prec == LBCH_F64
                            ? adjoint_step_t<double, double>(h, (const double*)(t + (size_t)k * stride), n0 + k)
                            : adjoint_step_t<double, float>(h, (const float*)(t + (size_t)k * stride), n0 + k);
        CK(e);
    }
    return LBCH_OK;
}

lbch_status lb_ch_tape_phi(lbch_handle* h, void* dst)
{
    if (!h || !dst) return fail(LBCH_EINVAL, "NULL handle or buffer");
    if (h->n_inst != 1) return fail(LBCH_EINVAL, "the adjoint supports single-instance handles");
    const long long N = (long long)h->inst[0].nx * h->inst[0].ny;
    if (N >= (1LL << 31)) return fail(LBCH_EINVAL, "the adjoint supports grids of fewer than 2^31 nodes");
    CK(tape_launch(h, cur_buf(h), dst));
    return LBCH_OK;
}

lbch_status lb_ch_adjoint_begin(lbch_handle* h, const void* dL_dphiT)
{
    if (!h || !dL_dphiT) return fail(LBCH_EINVAL, "NULL handle or gradient");
    if (h->n_inst != 1) return fail(LBCH_EINVAL, "the adjoint supports single-instance handles");
    if (h->inst[0].walls) return fail(LBCH_EINVAL, "the adjoint supports periodic domains only");
    if (h->coupled) return fail(LBCH_EINVAL, "the adjoint supports prescribed flows only");
    if (h->model3) return fail(LBCH_EINVAL, "the adjoint supports Models I and II");
    if (h->slab) return fail(LBCH_EINVAL, "the adjoint supports whole grids, not slabs");
    if ((long long)h->inst[0].nx * h->inst[0].ny >= (1LL << 31))
        return fail(LBCH_EINVAL, "the adjoint supports grids of fewer than 2^31 nodes");
    h->adj_elem = 8;  // the adjoint is carried in double for every storage precision
    if (!h->adj) CK(cudaMalloc(&h->adj, adj_bytes(h)));
    AdjView v = adj_view(h);
    const long long N = (long long)h->inst[0].nx * h->inst[0].ny;
    const int nb = (int)((N + 255) / 256);
    h->adj_par = 0;
    adj::adj_begin_kernel<double><<<nb, 256, 0, h->stream>>>(N, adj_planes(h), (const double*)dL_dphiT,
                                                            (double*)v.lam[0]);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(v.dLds, 0, sizeof(double), h->stream));
    CK(cudaMemsetAsync(v.ds, 0, (size_t)N * sizeof(double), h->stream));  // per-node dL/ds, summed at the end
    return LBCH_OK;
}

lbch_status lb_ch_adjoint_step(lbch_handle* h, const void* phi_n, long n)
{
    if (!h || !phi_n || n < 0) return fail(LBCH_EINVAL, "NULL handle, NULL phi or negative step");
    if (!h->adj) return fail(LBCH_EINVAL, "lb_ch_adjoint_begin was not called");
    cudaError_t e = h->prec == LBCH_F64 ? adjoint_step_t<double, double>(h, (const double*)phi_n, n)
                                        : adjoint_step_t<double, float>(h, (const float*)phi_n, n);
    CK(e);
    return LBCH_OK;
}

lbch_status lb_ch_adjoint_end(lbch_handle* h, void* dL_dphi0, double* dL_ds)
{
    if (!h || !dL_dphi0 || !dL_ds) return fail(LBCH_EINVAL, "NULL handle or output");
    if (!h->adj) return fail(LBCH_EINVAL, "lb_ch_adjoint_begin was not called");
    cudaError_t e = adjoint_end_t<double>(h, (double*)dL_dphi0);
    CK(e);
    CK(cudaMemcpyAsync(dL_ds, adj_view(h).dLds, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBCH_OK;
}

lbch_status lb_ch_tune(lbch_handle* h, int steps, int* tile_x, int* tile_y)
{
    if (!h || steps < 1) return fail(LBCH_EINVAL, "NULL handle or steps < 1");
    // Candidates: every row-sweep configuration and every tile kernel shape.  The two forms give the same
    // bits except on the half-storage path at tau_g = 1, where the tile kernel streams populations rounded
    // to half and the sweep keeps only phi; there the sweep alone is a candidate.
    // Where it applies, the two-step kernel is a candidate too (it then takes the steps two at a time; an odd
    // last step goes to the fastest one-step candidate).
    struct Cand { bool tile, pair; int shape; };
    std::vector<Cand> cands;
    if (!h->coupled) {
        for (int k = 0; k < n_sweep_shapes(h); k++) cands.push_back({false, false, k});
        if (!(h->prec == LBCH_F16S && h->tau1 && !h->force_general))
            for (int k = 0; k < n_shapes(h->prec); k++) cands.push_back({true, false, k});
        for (int k = 0; k < kPairShapes && pair_ok(h); k++) cands.push_back({false, true, k});
    }
    const int ns = (int)cands.size();
    struct Tuning {  // a slab handle may take several steps per lb_ch_step call while it is timed
        lbch_handle* h;
        explicit Tuning(lbch_handle* hh) : h(hh) { h->tuning = true; }
        ~Tuning() { h->tuning = false; }
    } tuning_(h);
    if (ns > 1) {
        long long bytes = 0;
        lb_ch_state_bytes(h, &bytes);
        void* backup = nullptr;
        CK(cudaMalloc(&backup, (size_t)bytes));
        lbch_status s = lb_ch_state_save(h, backup);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        float best_ms = 0.0f, best1_ms = 0.0f;  // per step: over all candidates; over the one-step ones
        Cand best = {h->force_tile, use_pair(h), use_pair(h) ? h->pshape : h->shape};
        Cand best1 = {h->force_tile, false, h->shape};
        // every candidate steps through lb_ch_step, as a caller's run does (CUDA graphs of kGraphChunk steps):
        // one graph of warm-up, which captures it, then the faster of two timed runs of `steps` steps rounded
        // up to whole graphs.  Fewer than kGraphChunk steps (large grids, where launches cost little) are
        // timed as they are, after two steps of warm-up.
        const long timed = steps < kGraphChunk ? steps : (long)((steps + kGraphChunk - 1) / kGraphChunk) * kGraphChunk;
        const long warm = steps < kGraphChunk ? 2 : kGraphChunk;
        if (s == LBCH_OK && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
            for (int k = 0; k < ns && s == LBCH_OK; k++) {
                const Cand c = cands[k];
                h->pair = c.pair;
                if (c.pair) h->pshape = c.shape;
                else { h->force_tile = c.tile; h->shape = c.shape; }
                drop_graphs(h);
                lbch_status r = lb_ch_step(h, warm);
                float ms = -1.0f;
                for (int rep = 0; rep < 2 && r == LBCH_OK; rep++) {
                    cudaError_t e = cudaEventRecord(e0, h->stream);
                    if (e == cudaSuccess) r = lb_ch_step(h, timed);
                    if (e == cudaSuccess && r == LBCH_OK) e = cudaEventRecord(e1, h->stream);
                    if (e == cudaSuccess && r == LBCH_OK) e = cudaEventSynchronize(e1);
                    float t = 0.0f;
                    if (e == cudaSuccess && r == LBCH_OK) e = cudaEventElapsedTime(&t, e0, e1);
                    if (e != cudaSuccess) r = cuda_fail(e, "timing a kernel candidate");
                    else if (r == LBCH_OK && (ms < 0.0f || t < ms)) ms = t;
                }
                if (r != LBCH_OK) s = r;
                else {
                    ms /= (float)timed;
                    if (k == 0 || ms < best_ms) { best_ms = ms; best = c; }
                    if (!c.pair && (k == 0 || ms < best1_ms)) { best1_ms = ms; best1 = c; }
                }
                r = lb_ch_state_load(h, backup);  // every candidate starts from the same state
                if (s == LBCH_OK) s = r;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(backup);
        h->force_tile = best1.tile;
        h->shape = best1.shape;
        h->pair = best.pair;
        if (best.pair) h->pshape = best.shape;
        if (s != LBCH_OK) return s;
        drop_graphs(h);  // graphs captured earlier launch the previous shape's kernel
    }
    const Shape sh = active_tile(h);
    if (tile_x) *tile_x = sh.tx;
    if (tile_y) *tile_y = sh.ty;
    return LBCH_OK;
}

lbch_status lb_ch_test_hook(lbch_handle* h, int hook, long value)
{
    if (!h) return fail(LBCH_EINVAL, "NULL handle");
    if (hook == LBCH_HOOK_SKIP_FIRST_LOAD) {
        h->debug_skip = value ? 1 : 0;
        return LBCH_OK;
    }
    if (hook == LBCH_HOOK_NO_PDL) {
        h->no_pdl = value != 0;
        drop_graphs(h);
        return LBCH_OK;
    }
    if (hook == LBCH_HOOK_TWO_STEP) {
        if (value && !pair_ok(h))
            return fail(LBCH_EINVAL, "the two-step kernel needs periodic instances with tau_g = 1 in f32 or f64");
        h->pair = value != 0;
        h->pshape = 0;
        drop_graphs(h);
        return LBCH_OK;
    }
    if (hook == LBCH_HOOK_TILE_KERNEL) {
        if (h->coupled) return fail(LBCH_EINVAL, "the coupled flow has no tile kernel");
        if (h->force_tile != (value != 0)) h->shape = 0;  // the shape index names the other kernel's list
        h->force_tile = value != 0;
        h->pair = false;  // either way a one-step kernel takes every step
        drop_graphs(h);
        return LBCH_OK;
    }
    if (hook == LBCH_HOOK_GENERAL_PATH) {
        h->force_general = value != 0;
        drop_graphs(h);
        return LBCH_OK;
    }
    if (hook == LBCH_HOOK_POISON) {  // every buffer of the next state filled with NaN (all bits set)
        const int nxt = cur_buf(h) ^ 1;
        if (h->coupled) {
            const InstDev& d = h->inst[0];
            const size_t N = (size_t)d.nx * d.ny, e = h->prec == LBCH_F64 ? 8 : 4;
            char* p = static_cast<char*>(h->ns);
            CK(cudaMemsetAsync(p + (size_t)nxt * 9 * N * e, 0xFF, 9 * N * e, h->stream));         // f
            CK(cudaMemsetAsync(p + (18 + (size_t)nxt * 9) * N * e, 0xFF, 9 * N * e, h->stream));  // g
            CK(cudaMemsetAsync(p + 36 * N * e, 0xFF, 4 * N * e, h->stream));                      // u, p, mu
            // phi of the current state: the next step forms it from the populations before reading it
            CK(cudaMemsetAsync(h->phi[nxt ^ 1], 0xFF, (size_t)h->rows * h->pitch * h->phi_elem, h->stream));
        } else {
            const size_t cells = (size_t)h->rows * h->pitch;
            CK(cudaMemsetAsync(h->g[nxt], 0xFF, cells * h->nq * h->g_elem, h->stream));
            if (h->lo[nxt]) CK(cudaMemsetAsync(h->lo[nxt], 0xFF, cells * sizeof(float), h->stream));
            if (h->H[nxt]) CK(cudaMemsetAsync(h->H[nxt], 0xFF, 2 * cells * h->c_elem(), h->stream));
        }
        CK(cudaMemsetAsync(h->phi[nxt], 0xFF, (size_t)h->rows * h->pitch * h->phi_elem, h->stream));
        return LBCH_OK;
    }
    if (hook == LBCH_HOOK_TILE_SHAPE) {
        if (h->coupled || value < 0 || value >= n_active(h)) return fail(LBCH_EINVAL, "no tile shape %ld", value);
        (use_pair(h) ? h->pshape : h->shape) = (int)value;
        drop_graphs(h);
        return LBCH_OK;
    }
    return fail(LBCH_EINVAL, "unknown hook %d", hook);
}

}  // extern "C"
