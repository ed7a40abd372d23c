// lbch_internal.h -- the handle of the C ABI and what the translation units of the library share.
#pragma once
#include <algorithm>
#include <vector>

#include "lbch.h"
#include "lbch_kernels.cuh"
#include "lbch_ns.cuh"

constexpr int kMaxShapes = 5;
struct Shape { int tx, ty, nt; };  // output nodes of a tile, threads per block

// Configurations of the row-sweep kernel (tau_g = 1): TY output rows per warp, NW warps per CTA; a tile
// is 56 columns by NW TY rows.  lb_ch_tune picks among them as among the tile shapes.
struct SweepCfg { int ty, nw; bool compact; };
constexpr SweepCfg kSweep[4] = {{12, 4, false}, {6, 4, false}, {6, 2, true}, {3, 4, true}};
constexpr int kSweepShapes = 4;
constexpr int kM3SweepShapes = 2;  // configurations built for handles with a Model III instance
constexpr int kSweepW = 56;
inline Shape sweep_tile(int k) { return Shape{kSweepW, kSweep[k].ty * kSweep[k].nw, 32 * kSweep[k].nw}; }

// Tile shapes of the two-step kernel (periodic instances, tau_g = 1; f32 and f64 only).
constexpr int kPairShapes = 4;
constexpr Shape kPairF[kPairShapes] = {{32, 16, 768}, {32, 14, 1024}, {32, 16, 1024}, {32, 8, 512}};
constexpr Shape kPair64[kPairShapes] = {{32, 8, 512}, {16, 8, 256}, {16, 16, 512}, {32, 14, 1024}};
inline Shape pair_shape(int prec, int k) { return prec == LBCH_F64 ? kPair64[k] : kPairF[k]; }

struct lbch_handle {
    int device = 0;
    int prec = LBCH_F64;
    int n_inst = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;  // the device's pool the handle's buffers come from (stream-ordered, on `stream`)
    std::vector<lbch::InstDev> inst;
    std::vector<long long> node_begin;  // first linear node index of each instance (+ total)
    lbch::InstDev* d_inst = nullptr;
    long long* d_node_begin = nullptr;
    double* d_tabs = nullptr;   // velocity tables in double (init kernel, FP64 step)
    float* d_tabs_f = nullptr;  // the same tables in float (float step kernels)
    int pitch = 0;              // elements per stored row
    int rows = 0;               // stored rows of all instances
    int nq = 9;                 // stored population planes
    size_t g_elem = 8, phi_elem = 8;
    long long nodes = 0;        // lattice nodes (all instances)
    int shape = 0;              // tile shape in use (index into the precision's shape list)
    bool tau1 = false;          // every instance has tau_g = 1: the populations drop out of the step
    bool force_general = false; // test hook: keep the populations even when tau1 holds
    bool force_tile = false;    // test hook: step with the tile kernel instead of the row sweep
    bool pair = false;          // step two at a time with the two-step kernel (when pair_ok holds); odd
    int pshape = 0;             // steps take the one-step kernel above; pshape indexes pair_shape()
    bool walls = false;         // an instance has walls
    bool slab = false;          // a slab of a larger periodic grid (lb_ch_init_slab): halos imported between steps
    bool tuning = false;        // lb_ch_tune is stepping the handle (a slab may then take several steps per call)
    bool model3 = false;        // an instance uses Model III (the row sweep's Model III build, or the tile kernel)
    bool need_time = false;     // an instance's step depends on the step index (time factor, Model III)
    void* H[2] = {nullptr, nullptr};  // Model III: H of Eq. F2-1's time derivatives, 2 planes, arithmetic type
    size_t c_elem() const { return prec == LBCH_F64 ? 8 : 4; }
    bool no_pdl = false;        // test hook: plain stream-ordered step launches
    struct PerShape {           // what depends on the tile shape
        int total_tiles = 0;
        int grid = 0;           // persistent CTAs per step launch
        int grid_gen = 0;       // row sweep with the populations (the tile kernel uses grid)
        int* d_tile_begin = nullptr;
        int4* d_tiles = nullptr;  // row-sweep configurations: each tile's (instance, x0, y0, wall body needed),
                                  // interior tiles first (see lbch_sweep.cuh)
        void* d_ttabs = nullptr;  // two-step shapes: each tile's velocity tables, contiguous (see lbch_pair.cuh)
        CUtensorMap tm_g[2], tm_phi[2], tm_lo[2];
    } ps[kMaxShapes], sw[kSweepShapes], pr[kPairShapes];  // tile kernel shapes; row-sweep configurations
                                                          // (tm_g unused); two-step shapes (no maps)
    CUtensorMap tm_grow[2], tm_lorow[2];  // one row of the populations / of phi's low part (row sweep)
    void* g[2] = {nullptr, nullptr};
    void* phi[2] = {nullptr, nullptr};
    float* lo[2] = {nullptr, nullptr};  // low part of phi (float path)
    double* phi0 = nullptr;     // initial field, double, padded layout
    lbch::Ctl* ctl = nullptr;
    double* partials = nullptr; // reduction scratch: n_inst * chunks * RED_NV doubles
    double* result = nullptr;   // n_inst * RED_NV doubles
    int chunks = 0;
    long long n = 0;            // host mirror of the step index
    int flip = 0;               // the state of step n is in buffer (n & 1) ^ flip (two-step launches toggle it)
    int t_off = 0, t_adv = 1;   // the next launch's step offset and counter advance (see Ctl)
    int debug_skip = 0;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [chunk size][starting parity]
    struct TapeGraph {          // a captured taped replay (lb_ch_step_taped) for one starting parity
        cudaGraphExec_t exec = nullptr;
        void* tape = nullptr;
        long nsteps = 0;
    } tgraph[2];
    double* h_stage = nullptr;  // pinned host staging
    size_t h_stage_bytes = 0;
    // adjoint workspace (instance 0), allocated by the first lb_ch_adjoint_begin
    void* adj = nullptr;        // one block: lambda[2] (9N each), mu, grad_mu_bar (2N), F_bar (2N), phi_bar,
                                // mu_bar, D_bar, u_bar (2N) in the adjoint type; then ds (N) and dL/ds, double
    size_t adj_elem = 8;
    int adj_par = 0;            // which lambda holds the current adjoint
    // coupled Navier-Stokes state (LBCH_VEL_COUPLED): f[2], g[2] ([9][N]) and u, p, mu ([N]), one block
    bool coupled = false;
    void* ns = nullptr;
    lbch::ns::NsConsts<double> nsd;
    lbch::ns::NsConsts<float> nsf;
};

// The velocity tables in the arithmetic type of a step kernel.
template <typename C> inline const C* tables(lbch_handle* h);
template <> inline const double* tables<double>(lbch_handle* h) { return h->d_tabs; }
template <> inline const float* tables<float>(lbch_handle* h) { return h->d_tabs_f; }

// The buffer (0 or 1 of each ping-pong pair) holding the state of the current step.
inline int cur_buf(const lbch_handle* h) { return (int)(h->n & 1) ^ h->flip; }

// The row sweep keeps the populations unless every instance has tau_g = 1 (and no test asks for them).
inline bool sweep_gen(const lbch_handle* h) { return !h->tau1 || h->force_general; }

// The two-step kernel serves handles whose instances are all periodic with tau_g = 1, in f32 or f64 (the
// half-storage path is left to the row sweep).
inline bool pair_ok(const lbch_handle* h)
{
    return h->tau1 && !h->force_general && !h->coupled && !h->model3 && !h->walls && !h->slab && h->prec != LBCH_F16S;
}

// Row-sweep launches and set-up, one translation unit per precision (lbch_sweep_*.cu).
#define LBCH_INTERNAL __attribute__((visibility("hidden")))
LBCH_INTERNAL cudaError_t lbch_launch_sweep_f64(lbch_handle* h, int parity);
LBCH_INTERNAL cudaError_t lbch_launch_sweep_f32(lbch_handle* h, int parity);
LBCH_INTERNAL cudaError_t lbch_launch_sweep_f16s(lbch_handle* h, int parity);
LBCH_INTERNAL cudaError_t lbch_prepare_sweep_f64(lbch_handle* h, int k);
LBCH_INTERNAL cudaError_t lbch_prepare_sweep_f32(lbch_handle* h, int k);
LBCH_INTERNAL cudaError_t lbch_prepare_sweep_f16s(lbch_handle* h, int k);
// The same for handles with a Model III instance (lbch_sweep_*_m3.cu; configurations 0 and 1).
LBCH_INTERNAL cudaError_t lbch_launch_sweep_f64_m3(lbch_handle* h, int parity);
LBCH_INTERNAL cudaError_t lbch_launch_sweep_f32_m3(lbch_handle* h, int parity);
LBCH_INTERNAL cudaError_t lbch_launch_sweep_f16s_m3(lbch_handle* h, int parity);
LBCH_INTERNAL cudaError_t lbch_prepare_sweep_f64_m3(lbch_handle* h, int k);
LBCH_INTERNAL cudaError_t lbch_prepare_sweep_f32_m3(lbch_handle* h, int k);
LBCH_INTERNAL cudaError_t lbch_prepare_sweep_f16s_m3(lbch_handle* h, int k);
// Two-step launches and set-up (lbch_pair.cu); pshape names a pair_shape().
LBCH_INTERNAL cudaError_t lbch_launch_pair(lbch_handle* h, int parity);
LBCH_INTERNAL cudaError_t lbch_prepare_pair(lbch_handle* h, int k);
// Launch limits of a kernel on a device, set and queried once per process (they depend on nothing else) and
// served from a table afterwards, so that making a handle does not repeat them for every kernel it may run:
// lbch_kernel_smem lets `kern` use `smem` bytes of dynamic shared memory; lbch_kernel_fit gives how many CTAs
// of `threads` threads with `smem` bytes one SM holds, and the device's SM count (lbch_api.cu).
LBCH_INTERNAL cudaError_t lbch_kernel_smem(const void* kern, int device, size_t smem);
LBCH_INTERNAL cudaError_t lbch_kernel_fit(const void* kern, int device, int threads, size_t smem, int* per_sm, int* sms);
