// lbch_sweep.cuh -- the step kernel as row sweeps in registers, for instances with tau_g = 1.
//
// At tau_g = 1, Eq. LB reduces to g* = g_eq + S / 2: the populations are multiplied by 1 - 1/tau = 0, so
// the step maps phi(t) to phi(t+1) = sum_i g*_i(x - c_i) and nothing else is carried between steps.
// Every quantity of the step at a node (mu, D = div(phi u), the gradients, the force, g*) depends only on
// phi within three rows and three columns, so one warp can produce a strip of output rows by sweeping
// upwards through it, one row per iteration, with everything the stencils need held in registers:
//
//   * a warp owns 64 consecutive columns, two per lane (a = 2 lane, b = 2 lane + 1, from domain column
//     x0 - 4); its 56 middle columns (lanes 2..29) are output, the four on each side are halo;
//   * the left neighbour of a and the right neighbour of b come from the adjacent lanes by shuffles;
//   * the rows below stay in registers: iteration j loads phi of row yf = wy0 - 3 + j, computes mu and D
//     of row yf - 1, collides row yf - 2 and completes phi(t+1) of row yf - 3;
//   * streaming needs only three values from each side: the populations 1, 5, 8 that arrive from the
//     column to the left are summed at their source node and cross one lane boundary as one number, as do
//     3, 6, 7 from the right (the grouping of the sum is the one the tile kernel uses too).
//
// A CTA of NW warps stacks its warps vertically over a tile of 56 x (NW TY) output nodes and shares one
// TMA box of phi (the tile plus three halo rows and four halo columns on each side; on the float path a
// second box brings the low part of phi for the output rows).  Persistent CTAs walk the tiles with a
// two-stage TMA pipeline, as the tile kernel does.  The velocity tables of the warp's columns are read
// once per tile into registers; the Y tables of its rows arrive one row per lane and are broadcast by
// shuffles.
//
// GEN (any tau_g): the populations are read and written as well.  Each warp keeps a four-slot ring of
// the rows it will collide in shared memory: one TMA box per row (64 columns x the population planes,
// plus the low part of phi on the float-float path), issued by lane 0 three rows ahead on the slot's
// mbarrier.  After the collision the nine g* of a node reach their destinations individually -- 1, 5, 8
// from the lane to the left, 3, 6, 7 from the right, 2 and 4 from the rows below and above -- and
// g(t+1) is stored plane by plane.
#pragma once
#include <type_traits>

#include "lbch_kernels.cuh"

namespace lbch {

template <typename C, typename S, typename P>
struct SweepArgs {
    InstDev inst0;          // the record of instance 0, for single-instance handles (read from the parameters)
    const InstDev* inst;
    const int* tile_begin;  // first tile of each instance (n_inst + 1 entries)
    const int4* tiles;      // several instances: tile t's (instance, x0, y0, wall body needed), interior tiles
                            // of every instance first and the tiles next to walls last (see the tile loop)
    const C* tabs;          // velocity tables in the arithmetic type
    int n_inst;
    int total_tiles;
    int pitch;
    int debug_skip;         // test hook: CTA 0 never issues its first load (its wait runs out)
    P* phi_out;
    float* lo_out;          // low part of phi on the float-float path
    Ctl* ctl;
    int t_off;              // this launch's step is ctl->time + t_off
    int t_adv;              // when nonzero, the launch's last CTA advances ctl->time by t_adv
    int need_time;          // some instance needs the step index (a time-dependent flow)
    S* g_out;               // populations (GEN): g[(row * nq + plane) * pitch + column]
    int rows;               // stored rows of the population arrays
    const C* H_in;          // M3 (Model III): H(t - 1) of Eq. F2-1's time derivatives, two planes (x, y) of
    C* H_out;               // rows x pitch values; H(t) is written for the warp's own nodes and their images
    long long H_plane;      // values per plane of H
};

template <typename P, typename S, bool FF, int TY, int NW, bool GEN>
struct SweepShape {
    static constexpr int W = 56;                 // output columns of a tile
    static constexpr int BW = 64;                // box columns: x0 - 4 .. x0 + 59, two per lane
    static constexpr int TH = NW * TY;           // output rows of a tile
    static constexpr int PBH = TH + 6;           // phi box rows: y0 - 3 .. y0 + TH + 2
    static constexpr unsigned PBOX_BYTES = PBH * BW * sizeof(P);
    static constexpr unsigned LBOX_BYTES = (FF && !GEN) ? TH * BW * 4 : 0;  // GEN: the low part rides in the ring
    __host__ __device__ static constexpr size_t a128(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t OFF_L = a128(PBOX_BYTES);
    static constexpr size_t STAGE = OFF_L + a128(LBOX_BYTES);
    static constexpr int NQ = sizeof(S) == 2 ? 8 : 9;  // stored population planes
    static constexpr int RING = 4;                      // ring slots per warp (rows k .. k + 3)
    static constexpr int NPL = NQ + (FF ? 1 : 0);       // planes per ring row: the populations, the low part of phi
    static constexpr int CH = BW * (int)sizeof(S) / 16; // 16-byte chunks per plane row
    static constexpr size_t RING_BYTES = GEN ? (size_t)RING * NPL * BW * sizeof(S) : 0;  // per warp
    static constexpr unsigned ROW_BYTES = NQ * BW * sizeof(S) + (FF ? BW * 4 : 0);  // one ring fill
    static constexpr size_t OFF_RING = 2 * STAGE;
    static constexpr size_t OFF_MBAR = OFF_RING + NW * RING_BYTES;
    static constexpr size_t BYTES = OFF_MBAR + 256 + 128;  // mbarriers (2 for the stages, RING per warp), slack
};

template <typename P> struct Pair;
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<double> { using T = double2; };
template <> struct Pair<__half> { using T = __half2; };

template <typename C, typename S2> __device__ __forceinline__ void unpair(S2 v, C& x, C& y) { x = cvt<C>(v.x); y = cvt<C>(v.y); }
template <typename C> __device__ __forceinline__ void unpair(__half2 v, C& x, C& y)
{
    x = (C)__low2float(v);
    y = (C)__high2float(v);
}
template <typename S, typename C> __device__ __forceinline__ typename Pair<S>::T mkpair(C x, C y)
{
    typename Pair<S>::T v;
    v.x = (S)x;
    v.y = (S)y;
    return v;
}
template <> __device__ __forceinline__ __half2 mkpair<__half, float>(float x, float y) { return __floats2half2_rn(x, y); }


// A stage flag known at compile time (it converts to a constant bool on the device).
template <bool V> struct Flag {
    __host__ __device__ constexpr operator bool() const { return V; }
};

template <typename C> __device__ __forceinline__ C from_left(C v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename C> __device__ __forceinline__ C from_right(C v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// One row of the sweep.  A slot is reused every third row, so each field lives at most three rows.
template <typename C>
struct SwRow {
    C pL, pa, pb, pR;              // phi: left neighbour of a, a, b, right neighbour of b
    C mL, ma, mb, mR;              // mu, the same four columns
    C dL, da, db, dR;              // D = div(phi u)
    C y1, y2;                      // the Y velocity tables of the row
    C u5a, u5b, u2a, u2b, u6a, u6b;         // g*_5, g*_2, g*_6 of the row: they stream to the row above
    C Ra, Rb, Ca, Cb, La, Lb, v0a, v0b;     // partial sums of the populations arriving at the row
    C e4a, e4b, e7a, e7b, e8a, e8b;         // at a top wall row: g_4, g_7, g_8 by bounce-back
    C n0a, n0b, n1a, n1b, n2a, n2b, n3a, n3b, n4a, n4b, n5a, n5b, n6a, n6b, n7a, n7b, n8a, n8b;  // GEN: g(t+1) of the row
};

// Writes phi(t+1) of domain node (x, y) into the ghost cells that stand for it (periodic images in x;
// periodic or mirror images in y, three deep).
template <typename P>
__device__ __forceinline__ void store_images(P* phi_out, long long row0, int pitch, int nx, int ny, int walls, int x,
                                             int y, P v)
{
    if (x >= 3 && x < nx - 3 && y >= 3 && y < ny - 3) return;
    constexpr int NONE = -1000000;
    const int xa = x < 3 ? x + nx : NONE, xb = x >= nx - 3 ? x - nx : NONE;
    const int ya = y < 3 ? (walls ? -1 - y : y + ny) : NONE;
    const int yb = y >= ny - 3 ? (walls ? 2 * ny - 1 - y : y - ny) : NONE;
    for (int iy = 0; iy < 3; iy++) {
        const int yy = iy == 0 ? y : (iy == 1 ? ya : yb);
        if (yy == NONE) continue;
        for (int ix = 0; ix < 3; ix++) {
            const int xx = ix == 0 ? x : (ix == 1 ? xa : xb);
            if (xx == NONE || (ix == 0 && iy == 0)) continue;
            phi_out[(row0 + yy) * pitch + GC + xx] = v;
        }
    }
}

// Writes g(t+1) of domain node (x, y) into the ghost cells that stand for it, one deep: periodic images
// in x, and in y unless the instance has walls there.
template <typename S, typename C, int QOFF, bool WALLS>
__device__ __forceinline__ void store_g_images(S* g_out, long long row0, int pitch, int nx, int ny, int x, int y,
                                               const C* v)
{
    constexpr int NONE = -1000000;
    const int gxa = x == 0 ? nx : (x == nx - 1 ? -1 : NONE);
    const int gya = WALLS ? NONE : (y == 0 ? ny : (y == ny - 1 ? -1 : NONE));
    if (gxa == NONE && gya == NONE) return;
    constexpr int NQ = 9 - QOFF;
    for (int iy = 0; iy < 2; iy++) {
        const int yy = iy == 0 ? y : gya;
        if (yy == NONE) continue;
        for (int ix = 0; ix < 2; ix++) {
            const int xx = ix == 0 ? x : gxa;
            if (xx == NONE || (ix == 0 && iy == 0)) continue;
            S* o = g_out + ((row0 + yy) * NQ) * pitch + GC + xx;
#pragma unroll
            for (int q = QOFF; q < 9; q++) o[(long long)(q - QOFF) * pitch] = to_s<S>(v[q]);
        }
    }
}

// The instance record a kernel reads: with SINGLE (a handle of one instance) the one in the launch
// parameters, whose fields the arithmetic then takes as constant-bank operands; otherwise the copy in
// shared memory of the tile's instance.
template <bool SINGLE>
__device__ __forceinline__ const InstDev& pick_inst(const InstDev& param, const InstDev& shared)
{
    if constexpr (SINGLE) return param;
    else return shared;
}

// M3: some instance uses Model III (the complete diffusive-scale force of Eq. F2-1): at every collision the
// force takes the backward difference of H = (2 tau - 1 + 3K) F1 + 3 c_s^2 eta K grad mu over one step
// (reading R15), with H(t - 1) read at the collided node and H(t) stored for the warp's own nodes, as the
// tile kernel does.
template <typename C, typename S, typename P, bool FF, int TY, int NW, bool GEN, bool COMPACT, bool SINGLE,
          bool M3 = false>
__global__ void __launch_bounds__(NW * 32, (sizeof(C) == 8 ? 8 : 12) / NW)
    ch_sweep_kernel(const __grid_constant__ CUtensorMap tm_phi, const __grid_constant__ CUtensorMap tm_lo,
                    const __grid_constant__ CUtensorMap tm_grow, const __grid_constant__ CUtensorMap tm_lorow,
                    const __grid_constant__ SweepArgs<C, S, P> a)
{
    static_assert(COMPACT || TY % 3 == 0, "the sweep advances three rows per unrolled step");
    static_assert(TY + 6 <= 32, "the Y tables of a warp's rows are held one row per lane");
    using L = SweepShape<P, S, FF, TY, NW, GEN>;
    using P2 = typename Pair<P>::T;
    using S2 = typename Pair<S>::T;
    constexpr int BW = L::BW, TH = L::TH, NQ = L::NQ, RING = L::RING, NPL = L::NPL;
    constexpr bool kShift = sizeof(C) == 4;     // float arithmetic on g_0 - phi
    constexpr bool kHalf = sizeof(S) == 2;      // half storage: g_0 not stored (implied by phi)
    constexpr int QOFF = kHalf ? 1 : 0;         // stored plane of population q is q - QOFF

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_aligned128(smem_raw);
    auto stage = [&](int k) { return base + (size_t)k * L::STAGE; };
    uint64_t* mbar = reinterpret_cast<uint64_t*>(base + L::OFF_MBAR);

    __shared__ long long s_time;
    __shared__ int s_tile_inst;
    __shared__ C s_T;
    __shared__ InstDev s_I;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int stride = gridDim.x;

    // Where tile t lies, and this lane's velocity tables for it (constant data, so they are read before
    // the waits): X by stored column (clamped: the clamped columns feed halo lanes only), Y by row of the
    // instance's stored band, one row of the warp per lane.
    int k_t = 0, x0 = 0, y0 = 0;
    bool w_t = false;  // the tile needs the wall body
    C X1m, X1a, X1b, X1p, X2m, X2a, X2b, X2p, ly1, ly2;
    auto locate = [&](int t) {
        int tab_t, ylen;
        if constexpr (SINGLE) {
            const int tiles_x = (a.inst0.nx + L::W - 1) / L::W;
            x0 = (t % tiles_x) * L::W;
            y0 = (t / tiles_x) * TH;
            w_t = a.inst0.walls && (y0 < 2 || y0 + TH + 1 > a.inst0.ny - 1);
            tab_t = a.inst0.tab;
            ylen = a.inst0.ylen;
        } else {
            const int4 tt = a.tiles[t];
            k_t = tt.x;
            x0 = tt.y;
            y0 = tt.z;
            w_t = tt.w != 0;
            tab_t = a.inst[k_t].tab;
            ylen = a.inst[k_t].ylen;
        }
        const C* tX1 = a.tabs + tab_t;
        const C* tX2 = tX1 + a.pitch;
        const C* tY1 = tX2 + a.pitch;
        const int sa = x0 + 2 * lane;
        const int cm = max(sa - 1, 0), ca = min(sa, a.pitch - 1), cb = min(sa + 1, a.pitch - 1), cp = min(sa + 2, a.pitch - 1);
        X1m = tX1[cm]; X1a = tX1[ca]; X1b = tX1[cb]; X1p = tX1[cp];
        X2m = tX2[cm]; X2a = tX2[ca]; X2b = tX2[cb]; X2p = tX2[cp];
        const int yk = min(max(y0 + warp * TY - 3 + lane + GR, 0), ylen - 1);
        ly1 = tY1[yk];
        ly2 = tY1[ylen + yk];
    };

    if (tid == 0) {
        for (int b = 0; b < 2 + (GEN ? NW * RING : 0); b++) mbar_init(&mbar[b], 1);
        fence_mbar_init();
        s_tile_inst = -1;
        if ((int)blockIdx.x < a.total_tiles) {  // instance data are constant: read before the dependency wait
            const int k = SINGLE ? 0 : a.tiles[blockIdx.x].x;
            s_I = SINGLE ? a.inst0 : a.inst[k];
            s_tile_inst = k;
        }
    }
    if ((int)blockIdx.x < a.total_tiles) locate(blockIdx.x);

    // producer: thread 0 issues the boxes of tile t into stage s
    auto issue = [&](int t, int s) {
        int bx, by, row0;
        if constexpr (SINGLE) {
            const int tiles_x = (a.inst0.nx + L::W - 1) / L::W;
            bx = (t % tiles_x) * L::W;
            by = (t / tiles_x) * TH;
            row0 = a.inst0.row0;
        } else {
            const int4 tt = a.tiles[t];
            bx = tt.y;
            by = tt.z;
            row0 = a.inst[tt.x].row0;
        }
        fence_proxy_async();
        mbar_expect_tx(&mbar[s], L::PBOX_BYTES + L::LBOX_BYTES);
        // box column origin: domain bx - 4 is stored column bx (a multiple of 4: 16-byte aligned)
        tma_load_2d(stage(s), &tm_phi, bx, row0 + by - 3, &mbar[s]);
        if (FF && !GEN) tma_load_2d(stage(s) + L::OFF_L, &tm_lo, bx, row0 + by, &mbar[s]);
    };

    // Launched as a programmatic dependent of the previous step: nothing that step writes (phi, the step
    // counter) is read before this wait.  The first boxes are issued before the counter is read, so the
    // two latencies overlap.
    grid_dependency_wait();
    grid_launch_dependents();
    if (tid == 0) {
        for (int j = 0; j < 2; j++) {
            const int t = blockIdx.x + j * stride;
            if (t < a.total_tiles && !(a.debug_skip && blockIdx.x == 0 && j == 0)) issue(t, j);
        }
        // the counter is read only when a flow depends on time; otherwise nothing waits on that load
        s_time = a.need_time ? a.ctl->time : 0;
        if (s_tile_inst >= 0) s_T = (C)vel_t(s_I.vel, s_I.Tper, s_time + a.t_off);
    }
    __syncthreads();
    // (the step index stays in shared memory: s_time + a.t_off, read where an instance changes and at exit,
    // so that it holds no registers through the sweep)

    // GEN: this warp's ring.  Fill n goes to slot n % RING and completes phase n / RING of the slot's
    // mbarrier; the fills and their uses run in the same row order, tile after tile.
    uint64_t* rbar = mbar + 2 + warp * RING;
    int fills = 0, uses = 0;
    bool ring_ok = true;

    // The sweep of one warp over its TY output rows of the tile in stage s.  WALLS: the instance has walls
    // in y (bounce-back rows, mirror substitution) -- a separate body, so that periodic tiles carry none
    // of that code.
    auto sweep = [&](auto walls_t, int s) {
        constexpr bool WALLS = decltype(walls_t)::value;
        const InstDev& I = pick_inst<SINGLE>(a.inst0, s_I);
        const int nx = I.nx, ny = I.ny;
        const int wy0 = y0 + warp * TY;  // the warp's first output row
        if (wy0 >= ny) return;
        const Consts<C>& K0 = consts<C>(I);
        const C beta = K0.beta, kappa = K0.kappa, phiA = K0.phiA, phiB = K0.phiB;
        const C ra = K0.a, rb = K0.b, K = K0.K;
        const bool model2 = M3 ? I.model >= 2 : I.model == 2;  // D = div(phi u) is needed (Models II, III)
        [[maybe_unused]] const bool model3 = M3 && I.model == 3;
        [[maybe_unused]] const bool first = M3 && s_time + a.t_off == 0;  // no H(t - 1) at the first step
        const C T = s_T;
        const int pitch = a.pitch;
        // this lane's column pair in the box, from the warp's first row (box row warp TY = domain wy0 - 3)
        const P* box = reinterpret_cast<const P*>(stage(s)) + warp * TY * BW + 2 * lane;
        const float* lbox = reinterpret_cast<const float*>(stage(s) + L::OFF_L) + warp * TY * BW + 2 * lane;
        const int sa = x0 + 2 * lane;  // stored column of node a
        const int xa = sa - GC, xb = xa + 1;
        const bool va = lane >= 2 && lane < 30 && xa < nx, vb = lane >= 2 && lane < 30 && xb < nx;
        // whether an output node of the warp's strip has ghost images (three columns or rows from the domain's
        // edge, the widest reach of store_images): elsewhere the image stores and their tests are skipped
        // as a whole, by a test the warp takes together.  Not in the phi-only sweep over several instances,
        // where the extra test cost more than it saved (registers spilled; the ragged shear ensemble ran
        // 61.9 instead of 65.2 GLUPS), while the other bodies gained 1 to 8 %.
        const bool img = (GEN || SINGLE) ? (x0 < 3 || x0 + L::W > nx - 3 || wy0 < 3 || wy0 + TY > ny - 3) : true;
        const long long row0 = I.row0;
        const C* tW = a.tabs + I.tab + 2 * pitch + 2 * I.ylen;  // Y1, Y2 at the walls y = -1/2, ny - 1/2
        // GEN: the ring of rows ([slot][plane][64 columns]: the population planes, then the low part of
        // phi on the float-float path).  Collision row k of the warp is domain row wy0 - 1 + k; its slot is
        // filled three rows before its collision and refilled after its phi(t+1) is written.
        [[maybe_unused]] S* ring = reinterpret_cast<S*>(base + L::OFF_RING + warp * L::RING_BYTES);
        auto g_fetch = [&](int k) {
            if constexpr (GEN) {
                if (k <= TY + 1 && ring_ok) {  // after a lost copy nothing more is issued
                    if (lane == 0) {
                        const int slot = fills % RING, row = (int)row0 + wy0 - 1 + k;
                        S* dst = ring + slot * NPL * BW;
                        fence_proxy_async();  // the slot's previous contents were read through the generic proxy
                        mbar_expect_tx(&rbar[slot], L::ROW_BYTES);
                        tma_load_3d(dst, &tm_grow, x0, 0, row, &rbar[slot]);
                        if (FF) tma_load_2d(dst + NQ * BW, &tm_lorow, x0, row, &rbar[slot]);
                    }
                    fills++;
                }
            }
        };
        if constexpr (GEN) {
            g_fetch(0);
            g_fetch(1);
            g_fetch(2);
        }

        // One row: A is the slot of row yf (it held yf - 3), B of row yf - 1, Cs of row yf - 2.  MU: mu and D
        // of row yf - 1; COL: collide row yf - 2; OUT: complete phi(t+1) of row yf - 3.  The three flags
        // are false only while the pipeline fills.
        auto row_step = [&](auto mu_t, auto col_t, auto out_t, const int j, SwRow<C>& A, SwRow<C>& B, SwRow<C>& Cs) {
            // the flags are compile-time constants (Flag<true> / Flag<false>) in the peeled and unrolled
            // forms and warp-uniform runtime values in the compact form
            const bool MU = mu_t, COL = col_t, OUT = out_t;
            const int yf = wy0 - 3 + j;
            {
                const P2 v = *reinterpret_cast<const P2*>(box + j * BW);
                A.pa = cvt<C>(v.x);
                A.pb = cvt<C>(v.y);
                A.pL = from_left(A.pb);
                A.pR = from_right(A.pa);
                A.y1 = __shfl_sync(0xffffffffu, ly1, j);
                A.y2 = __shfl_sync(0xffffffffu, ly2, j);
            }
            if (MU) {
                B.ma = node_mu(B.pa, B.pb, B.pL, A.pa, Cs.pa, A.pb, A.pL, Cs.pb, Cs.pL, beta, kappa, phiA, phiB);
                B.mb = node_mu(B.pb, B.pR, B.pa, A.pb, Cs.pb, A.pR, A.pa, Cs.pR, Cs.pa, beta, kappa, phiA, phiB);
                B.mL = from_left(B.mb);
                B.mR = from_right(B.ma);
                if (model2) {
                    B.da = node_div(B.pb, B.pL, A.pa, Cs.pa, A.pb, A.pL, Cs.pb, Cs.pL, X1m, X1b, X2m, X2a, X2b,
                                    Cs.y1, B.y1, A.y1, Cs.y2, A.y2, T);
                    B.db = node_div(B.pR, B.pa, A.pb, Cs.pb, A.pR, A.pa, Cs.pR, Cs.pa, X1a, X1p, X2a, X2b, X2p,
                                    Cs.y1, B.y1, A.y1, Cs.y2, A.y2, T);
                    B.dL = from_left(B.db);
                    B.dR = from_right(B.da);
                }
            }
            const int yc = yf - 2;
            C p8a = C(0), p8b = C(0), p7a = C(0), p7b = C(0), p4a = C(0), p4b = C(0);
            if (COL) {
                // GEN: the populations g(t) of row yc (collision row k = j - 4 of the warp)
                C ga[9], gb[9];
                if constexpr (GEN) {
                    // row k = j - 4 has landed (bounded wait; a lost copy is reported, not waited for)
                    const int slot = uses % RING;
                    if (ring_ok) ring_ok = mbar_wait_bounded(&rbar[slot], (unsigned)((uses / RING) & 1), 1u << 22);
                    uses++;
                    const S* rg = ring + slot * NPL * BW + 2 * lane;
                    if constexpr (kHalf) {
                        C resta = C(0), restb = C(0);
#pragma unroll
                        for (int q = 1; q < 9; q++) {
                            unpair(*reinterpret_cast<const S2*>(rg + (q - 1) * BW), ga[q], gb[q]);
                            resta += ga[q];
                            restb += gb[q];
                        }
                        ga[0] = -resta;  // g_0 - phi
                        gb[0] = -restb;
                    } else {
#pragma unroll
                        for (int q = 0; q < 9; q++) unpair(*reinterpret_cast<const S2*>(rg + q * BW), ga[q], gb[q]);
                    }
                }
                // at a wall, the ghost rows are not collided (nothing is pulled from them)
                if (!WALLS || (yc >= 0 && yc < ny)) {
                    if constexpr (WALLS) {
                        // next to a wall, mu and D of the ghost row take the values of the mirror row (yc);
                        // the ghost row's own values are used by no other node
                        if (yc == 0) { A.mL = Cs.mL; A.ma = Cs.ma; A.mb = Cs.mb; A.mR = Cs.mR;
                                       A.dL = Cs.dL; A.da = Cs.da; A.db = Cs.db; A.dR = Cs.dR; }
                        if (yc == ny - 1) { B.mL = Cs.mL; B.ma = Cs.ma; B.mb = Cs.mb; B.mR = Cs.mR;
                                            B.dL = Cs.dL; B.da = Cs.da; B.db = Cs.db; B.dR = Cs.dR; }
                    }
                    C gmxa, gmya, gmxb, gmyb, gDxa = C(0), gDya = C(0), gDxb = C(0), gDyb = C(0);
                    grad9(Cs.mb, Cs.mL, B.ma, A.ma, B.mb, B.mL, A.mb, A.mL, gmxa, gmya);
                    grad9(Cs.mR, Cs.ma, B.mb, A.mb, B.mR, B.ma, A.mR, A.ma, gmxb, gmyb);
                    if (model2) {
                        grad9(Cs.db, Cs.dL, B.da, A.da, B.db, B.dL, A.db, A.dL, gDxa, gDya);
                        grad9(Cs.dR, Cs.da, B.db, A.db, B.dR, B.da, A.dR, A.da, gDxb, gDyb);
                    }
                    C Fxa, Fya, Fxb, Fyb;
                    if (M3 && model3) {
                        // H(t - 1) at the collided nodes: rows -1 .. ny hold it (images one deep); other rows
                        // and columns past the stored ones collide for no output and read nothing
                        const bool hrow = !first && yc >= -1 && yc <= ny;
                        const long long hn = (row0 + yc) * pitch + sa;
                        const C Hpxa = hrow && sa < pitch ? a.H_in[hn] : C(0);
                        const C Hpya = hrow && sa < pitch ? a.H_in[a.H_plane + hn] : C(0);
                        const C Hpxb = hrow && sa + 1 < pitch ? a.H_in[hn + 1] : C(0);
                        const C Hpyb = hrow && sa + 1 < pitch ? a.H_in[a.H_plane + hn + 1] : C(0);
                        C Hxa, Hya, Hxb, Hyb;
                        node_force_full(Cs.pa, gmxa, gmya, gDxa, gDya, Hpxa, Hpya, first, ra, rb, K, K0.cF1, K0.cmu,
                                        Fxa, Fya, Hxa, Hya);
                        node_force_full(Cs.pb, gmxb, gmyb, gDxb, gDyb, Hpxb, Hpyb, first, ra, rb, K, K0.cF1, K0.cmu,
                                        Fxb, Fyb, Hxb, Hyb);
                        if (yc >= wy0 && yc < wy0 + TY && yc < ny) {  // the warp's own nodes
                            if (va) store_h(a.H_out, a.H_plane, (int)row0, pitch, nx, ny, I.walls, xa, yc, Hxa, Hya);
                            if (vb) store_h(a.H_out, a.H_plane, (int)row0, pitch, nx, ny, I.walls, xb, yc, Hxb, Hyb);
                        }
                    } else {
                        node_force(Cs.pa, gmxa, gmya, gDxa, gDya, model2, ra, rb, K, Fxa, Fya);
                        node_force(Cs.pb, gmxb, gmyb, gDxb, gDyb, model2, ra, rb, K, Fxb, Fyb);
                    }
                    C pa_[9], pb_[9];
                    collide9<C, !GEN, kShift, !GEN>(Cs.pa, Cs.ma, Fxa, Fya, node_u(X1a, Cs.y1, T), node_u(X2a, Cs.y2, T), ga,
                                              K0, pa_);
                    collide9<C, !GEN, kShift, !GEN>(Cs.pb, Cs.mb, Fxb, Fyb, node_u(X1b, Cs.y1, T), node_u(X2b, Cs.y2, T), gb,
                                              K0, pb_);
                    if constexpr (GEN && kHalf) {
                        // the streamed populations are stored in half: they travel rounded.  g*_0 stays at the
                        // node, in float, and takes what the rounded ones leave of phi (g*_0 - phi = -sum of
                        // the rounded g*_q, q > 0), so that the rounding moves no phi between nodes: sum phi is
                        // kept exactly as in the other precisions (the same sum in the same order as the tile
                        // kernel forms)
                        C resta = C(0), restb = C(0);
#pragma unroll
                        for (int q = 1; q < 9; q++) {
                            pa_[q] = (C)__half2float(__float2half_rn((float)pa_[q]));
                            pb_[q] = (C)__half2float(__float2half_rn((float)pb_[q]));
                            resta += pa_[q];
                            restb += pb_[q];
                        }
                        pa_[0] = -resta;
                        pb_[0] = -restb;
                    }
                    if constexpr (GEN) {
                        // g*_q reaches node x + c_q: the row above takes 2, 5, 6; this row 0, 1, 3; the row
                        // below 4, 7, 8 (1, 5, 8 from the lane to the left, 3, 6, 7 from the right)
                        B.n2a = pa_[2]; B.n2b = pb_[2];
                        B.n5a = from_left(pb_[5]); B.n5b = pa_[5];
                        B.n6a = pb_[6]; B.n6b = from_right(pa_[6]);
                        Cs.n0a = pa_[0]; Cs.n0b = pb_[0];
                        Cs.n1a = from_left(pb_[1]); Cs.n1b = pa_[1];
                        Cs.n3a = pb_[3]; Cs.n3b = from_right(pa_[3]);
                        A.n4a = pa_[4]; A.n4b = pb_[4];
                        A.n7a = pb_[7]; A.n7b = from_right(pa_[7]);
                        A.n8a = from_left(pb_[8]); A.n8b = pa_[8];
                        if constexpr (WALLS) {
                            if (yc == 0) {  // bottom wall: 2, 5, 6 of this row bounce back at the node
                                const C uxa = node_u(X1a, tW[0], T), uya = node_u(X2a, tW[2], T);
                                const C uxb = node_u(X1b, tW[0], T), uyb = node_u(X2b, tW[2], T);
                                Cs.n2a = bounce<C, 2>(pa_[4], Cs.pa, uxa, uya); Cs.n2b = bounce<C, 2>(pb_[4], Cs.pb, uxb, uyb);
                                Cs.n5a = bounce<C, 5>(pa_[7], Cs.pa, uxa, uya); Cs.n5b = bounce<C, 5>(pb_[7], Cs.pb, uxb, uyb);
                                Cs.n6a = bounce<C, 6>(pa_[8], Cs.pa, uxa, uya); Cs.n6b = bounce<C, 6>(pb_[8], Cs.pb, uxb, uyb);
                            }
                            if (yc == ny - 1) {  // top wall: 4, 7, 8 of this row
                                const C uxa = node_u(X1a, tW[1], T), uya = node_u(X2a, tW[3], T);
                                const C uxb = node_u(X1b, tW[1], T), uyb = node_u(X2b, tW[3], T);
                                Cs.n4a = bounce<C, 4>(pa_[2], Cs.pa, uxa, uya); Cs.n4b = bounce<C, 4>(pb_[2], Cs.pb, uxb, uyb);
                                Cs.n7a = bounce<C, 7>(pa_[5], Cs.pa, uxa, uya); Cs.n7b = bounce<C, 7>(pb_[5], Cs.pb, uxb, uyb);
                                Cs.n8a = bounce<C, 8>(pa_[6], Cs.pa, uxa, uya); Cs.n8b = bounce<C, 8>(pb_[6], Cs.pb, uxb, uyb);
                            }
                        }
                    } else {
                    Cs.u5a = pa_[5]; Cs.u5b = pb_[5];
                    Cs.u2a = pa_[2]; Cs.u2b = pb_[2];
                    Cs.u6a = pa_[6]; Cs.u6b = pb_[6];
                    // (g_1 + g_5) and (g_3 + g_6) at their source nodes; g_2 from the row below
                    Cs.Ra = pa_[1] + A.u5a; Cs.Rb = pb_[1] + A.u5b;
                    Cs.La = pa_[3] + A.u6a; Cs.Lb = pb_[3] + A.u6b;
                    Cs.Ca = A.u2a; Cs.Cb = A.u2b;
                    Cs.v0a = pa_[0];
                    Cs.v0b = pb_[0];
                    if constexpr (WALLS) {
                        if (yc == 0) {
                            // bottom wall row: 2, 5, 6 would come from the ghost row; they bounce back at the
                            // node, so the sums from the sides are formed here, at the destination
                            const C uxa = node_u(X1a, tW[0], T), uya = node_u(X2a, tW[2], T);
                            const C uxb = node_u(X1b, tW[0], T), uyb = node_u(X2b, tW[2], T);
                            Cs.Ra = from_left(pb_[1]) + bounce<C, 5>(pa_[7], Cs.pa, uxa, uya);
                            Cs.Rb = pa_[1] + bounce<C, 5>(pb_[7], Cs.pb, uxb, uyb);
                            Cs.La = pb_[3] + bounce<C, 6>(pa_[8], Cs.pa, uxa, uya);
                            Cs.Lb = from_right(pa_[3]) + bounce<C, 6>(pb_[8], Cs.pb, uxb, uyb);
                            Cs.Ca = bounce<C, 2>(pa_[4], Cs.pa, uxa, uya);
                            Cs.Cb = bounce<C, 2>(pb_[4], Cs.pb, uxb, uyb);
                        }
                        if (yc == ny - 1) {
                            // top wall row: 4, 7, 8 would come from the ghost row above
                            const C uxa = node_u(X1a, tW[1], T), uya = node_u(X2a, tW[3], T);
                            const C uxb = node_u(X1b, tW[1], T), uyb = node_u(X2b, tW[3], T);
                            Cs.e4a = bounce<C, 4>(pa_[2], Cs.pa, uxa, uya); Cs.e4b = bounce<C, 4>(pb_[2], Cs.pb, uxb, uyb);
                            Cs.e7a = bounce<C, 7>(pa_[5], Cs.pa, uxa, uya); Cs.e7b = bounce<C, 7>(pb_[5], Cs.pb, uxb, uyb);
                            Cs.e8a = bounce<C, 8>(pa_[6], Cs.pa, uxa, uya); Cs.e8b = bounce<C, 8>(pb_[6], Cs.pb, uxb, uyb);
                        }
                    }
                    p8a = pa_[8]; p8b = pb_[8];
                    p7a = pa_[7]; p7b = pb_[7];
                    p4a = pa_[4]; p4b = pb_[4];
                    }
                }
            }
            if (GEN && OUT) {
                // g(t+1) and phi(t+1) of row yo = yf - 3 (slot A): every population has arrived
                const int yo = yf - 3;
                const C suma = stream_sum(A.n1a, A.n2a, A.n3a, A.n4a, A.n5a, A.n6a, A.n7a, A.n8a);
                const C sumb = stream_sum(A.n1b, A.n2b, A.n3b, A.n4b, A.n5b, A.n6b, A.n7b, A.n8b);
                P hia, hib;
                float loa = 0.0f, lob = 0.0f;
                C g0a = A.n0a, g0b = A.n0b;  // the stored rest population
                if constexpr (FF) {
                    const P2 hv = *reinterpret_cast<const P2*>(box + (j - 3) * BW);
                    // the low part of row yo = the previous collision row, one slot back
                    const float2 lv = *reinterpret_cast<const float2*>(
                        reinterpret_cast<const float*>(ring) + ((uses - 2) % RING) * NPL * BW + NQ * BW + 2 * lane);
                    {
                        const float h = (float)hv.x, tt = lv.x + (float)(A.n0a + suma);
                        const float sm = h + tt, bb = sm - h;
                        loa = (h - (sm - bb)) + (tt - bb);
                        hia = (P)sm;
                    }
                    {
                        const float h = (float)hv.y, tt = lv.y + (float)(A.n0b + sumb);
                        const float sm = h + tt, bb = sm - h;
                        lob = (h - (sm - bb)) + (tt - bb);
                        hib = (P)sm;
                    }
                    g0a = -suma;  // g_0 - phi(t+1) = -sum_{q>0} g_q(t+1)
                    g0b = -sumb;
                } else if constexpr (kShift) {
                    const P2 hv = *reinterpret_cast<const P2*>(box + (j - 3) * BW);
                    hia = (P)((float)hv.x + (float)(A.n0a + suma));
                    hib = (P)((float)hv.y + (float)(A.n0b + sumb));
                } else {
                    hia = (P)(A.n0a + suma);
                    hib = (P)(A.n0b + sumb);
                }
                if (yo < ny) {
                    const long long node = (row0 + yo) * pitch + sa;
                    const C va_[9] = {g0a, A.n1a, A.n2a, A.n3a, A.n4a, A.n5a, A.n6a, A.n7a, A.n8a};
                    const C vb_[9] = {g0b, A.n1b, A.n2b, A.n3b, A.n4b, A.n5b, A.n6b, A.n7b, A.n8b};
                    S* go = a.g_out + ((row0 + yo) * NQ) * pitch + sa;
                    if (va && vb) {
                        P2 o;
                        o.x = hia;
                        o.y = hib;
                        *reinterpret_cast<P2*>(a.phi_out + node) = o;
                        if (FF) *reinterpret_cast<float2*>(a.lo_out + node) = make_float2(loa, lob);
#pragma unroll
                        for (int q = QOFF; q < 9; q++)
                            *reinterpret_cast<S2*>(go + (long long)(q - QOFF) * pitch) = mkpair<S>(va_[q], vb_[q]);
                    } else if (va) {
                        a.phi_out[node] = hia;
                        if (FF) a.lo_out[node] = loa;
#pragma unroll
                        for (int q = QOFF; q < 9; q++) go[(long long)(q - QOFF) * pitch] = to_s<S>(va_[q]);
                    }
                    if (img) {
                        if (va) {
                            store_images(a.phi_out, row0, pitch, nx, ny, I.walls, xa, yo, hia);
                            store_g_images<S, C, QOFF, WALLS>(a.g_out, row0, pitch, nx, ny, xa, yo, va_);
                        }
                        if (vb) {
                            store_images(a.phi_out, row0, pitch, nx, ny, I.walls, xb, yo, hib);
                            store_g_images<S, C, QOFF, WALLS>(a.g_out, row0, pitch, nx, ny, xb, yo, vb_);
                        }
                    }
                }
            }
            if (GEN && COL) {
                // the slot of collision row j - 5 (read by the collision before and the output just done)
                // takes row j - 1 = k + 3
                __syncwarp();
                g_fetch(j - 1);
            }
            if (!GEN && OUT) {
                // phi(t+1) of row yo = yf - 3 (slot A), with g*_4, g*_7, g*_8 of row yo + 1 just computed
                const int yo = yf - 3;
                C Ra, Rb, Ca, Cb, La, Lb;
                if (WALLS && yo == ny - 1) {
                    // top wall row (no collision above): the sums (g_1 + g_5), (g_3 + g_6) cross to their
                    // destinations, where the bounced-back 8, 7 and 4 complete them
                    Ra = from_left(A.Rb) + A.e8a; Rb = A.Ra + A.e8b;
                    La = A.Lb + A.e7a; Lb = from_right(A.La) + A.e7b;
                    Ca = A.Ca + A.e4a; Cb = A.Cb + A.e4b;
                } else if (WALLS && yo == 0) {
                    // bottom wall row: the sums are already at the destinations
                    Ra = A.Ra + from_left(p8b); Rb = A.Rb + p8a;
                    La = A.La + p7b; Lb = A.Lb + from_right(p7a);
                    Ca = A.Ca + p4a; Cb = A.Cb + p4b;
                } else {
                    const C Rsa = A.Ra + p8a, Rsb = A.Rb + p8b, Lsa = A.La + p7a, Lsb = A.Lb + p7b;
                    Ra = from_left(Rsb); Rb = Rsa;
                    La = Lsb; Lb = from_right(Lsa);
                    Ca = A.Ca + p4a; Cb = A.Cb + p4b;
                }
                const C suma = (Ra + Ca) + La, sumb = (Rb + Cb) + Lb;  // the grouping of stream_sum
                P hia, hib;
                float loa = 0.0f, lob = 0.0f;
                if constexpr (FF) {
                    // phi(t+1) = phi(t) + (g*_0 - phi(t)) + sum_{q>0}; hi + lo absorbs it exactly (TwoSum)
                    const P2 hv = *reinterpret_cast<const P2*>(box + (j - 3) * BW);
                    const float2 lv = *reinterpret_cast<const float2*>(lbox + (j - 6) * BW);
                    {
                        const float h = (float)hv.x, tt = lv.x + (float)(A.v0a + suma);
                        const float sm = h + tt, bb = sm - h;
                        loa = (h - (sm - bb)) + (tt - bb);
                        hia = (P)sm;
                    }
                    {
                        const float h = (float)hv.y, tt = lv.y + (float)(A.v0b + sumb);
                        const float sm = h + tt, bb = sm - h;
                        lob = (h - (sm - bb)) + (tt - bb);
                        hib = (P)sm;
                    }
                } else if constexpr (kShift) {
                    const P2 hv = *reinterpret_cast<const P2*>(box + (j - 3) * BW);
                    hia = (P)((float)hv.x + (float)(A.v0a + suma));
                    hib = (P)((float)hv.y + (float)(A.v0b + sumb));
                } else {
                    hia = (P)(A.v0a + suma);
                    hib = (P)(A.v0b + sumb);
                }
                if (yo < ny) {
                    const long long node = (row0 + yo) * pitch + sa;
                    if (va && vb) {
                        P2 o;
                        o.x = hia;
                        o.y = hib;
                        *reinterpret_cast<P2*>(a.phi_out + node) = o;
                        if (FF) *reinterpret_cast<float2*>(a.lo_out + node) = make_float2(loa, lob);
                    } else if (va) {
                        a.phi_out[node] = hia;
                        if (FF) a.lo_out[node] = loa;
                    }
                    if (img) {
                        if (va) store_images(a.phi_out, row0, pitch, nx, ny, I.walls, xa, yo, hia);
                        if (vb) store_images(a.phi_out, row0, pitch, nx, ny, I.walls, xb, yo, hib);
                    }
                }
            }
        };

        using F = Flag<false>;
        using Tr = Flag<true>;
        SwRow<C> r0 = {}, r1 = {}, r2 = {};
        if constexpr (COMPACT) {
            // One loop body for the whole sweep, the pipeline's stages switched on by row: the least code,
            // for grids too small to fill the GPU, where every launch fetches its instructions afresh.
#pragma unroll 1
            for (int j = 0; j < TY + 6; j++) {
                row_step(j >= 2, j >= 4, j >= 6, j, r0, r1, r2);
                SwRow<C> t_ = r0; r0 = r2; r2 = r1; r1 = t_;
            }
            return;
        }
        // the pipeline fills: rows wy0 - 3 .. wy0 + 2 enter; mu from the third, collisions from the fifth,
        // outputs from the seventh
        row_step(F(), F(), F(), 0, r0, r1, r2);
        row_step(F(), F(), F(), 1, r2, r0, r1);
        row_step(Tr(), F(), F(), 2, r1, r2, r0);
        row_step(Tr(), F(), F(), 3, r0, r1, r2);
        row_step(Tr(), Tr(), F(), 4, r2, r0, r1);
        row_step(Tr(), Tr(), F(), 5, r1, r2, r0);
        if constexpr (GEN) {
            // steady state, one row per iteration with the slots rotated by register moves: the body with
            // the populations is large enough that three copies of it (the unrolled rotation below) cost
            // more in instruction fetch than the moves do (measured: 54 against 49 GLUPS at 4096^2, FP32; again
            // on a build with 7 % fewer instructions per update, 56.8 against 52.8, and 40.0 against 36.0 GLUPS
            // on the ragged shear ensemble)
#pragma unroll 1
            for (int j = 6; j < TY + 6; j++) {
                row_step(Tr(), Tr(), Tr(), j, r0, r1, r2);
                SwRow<C> t_ = r0; r0 = r2; r2 = r1; r1 = t_;
            }
        } else {
            // steady state: one output row per row entering, three rows per iteration so that the slots
            // rotate by renaming (measured faster than one row with moves for this smaller body)
#pragma unroll 1
            for (int j = 6; j < TY + 6; j += 3) {
                row_step(Tr(), Tr(), Tr(), j, r0, r1, r2);
                row_step(Tr(), Tr(), Tr(), j + 1, r2, r0, r1);
                row_step(Tr(), Tr(), Tr(), j + 2, r1, r2, r0);
            }
        }
    };

    for (int it = 0;; it++) {
        const int t = blockIdx.x + it * stride;
        if (t >= a.total_tiles) break;
        const int s = it & 1;
        if (it > 0) locate(t);  // the table loads are in flight during the wait
        const bool ok = mbar_wait_bounded(&mbar[s], (unsigned)((it >> 1) & 1), 1u << 22);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&a.ctl->err, 1u);
                // let a copy already issued into the other stage land before the CTA exits (bounded)
                if (t + stride < a.total_tiles)
                    mbar_wait_bounded(&mbar[s ^ 1], (unsigned)(((it + 1) >> 1) & 1), 1u << 22);
            }
            break;
        }
        // (this barrier also keeps the warps of a CTA in step from tile to tile, which measured faster than
        // letting them drift: 324 against 334 us per step at 4096^2 with the populations)
        if (k_t != s_tile_inst) {  // (the same for every thread: k_t and s_tile_inst are block-uniform)
            // the tile's instance record, copied by the whole block (with one thread copying it word by word,
            // a serial stall at every change of instance -- every tile in the interior-first order -- the
            // ragged shear ensemble ran 60.7 instead of 65.2 GLUPS)
            const int* src = reinterpret_cast<const int*>(a.inst + k_t);
            int* dst = reinterpret_cast<int*>(&s_I);
            for (int w = tid; w < (int)(sizeof(InstDev) / 4); w += NW * 32) dst[w] = src[w];
            __syncthreads();
            if (tid == 0) {
                s_tile_inst = k_t;
                s_T = (C)vel_t(s_I.vel, s_I.Tper, s_time + a.t_off);
            }
        }
        __syncthreads();
        // The wall body (bounce-back rows, mu and D of the ghost rows taken from the mirror rows) is needed only
        // by a tile whose collision rows y0 - 1 .. y0 + TH, or the rows their stencils read, come within two rows
        // of a wall: elsewhere every operand is a domain value and the periodic body gives the same bits (the
        // ghost images it writes follow the instance's boundary).  The choice is per tile, so that the warps of
        // a block run one body; for several instances the tile order puts every interior tile first and the
        // wall tiles last, so that the blocks of an SM mostly run the same body (two bodies at once measured
        // slower than the wall body alone: their code does not stay in the instruction caches together).  A
        // single instance keeps one body for all its tiles: a per-tile choice there cost 6% on the step with
        // the populations (57.6 against 54.6 GLUPS at 4096^2, same box), through the code it generates.
        if (SINGLE ? (bool)a.inst0.walls : w_t) sweep(std::true_type(), s);
        else sweep(std::false_type(), s);
        if (GEN && !ring_ok && lane == 0) atomicOr(&a.ctl->err, 1u);
        __syncthreads();  // the stage is free again
        const int t2 = t + 2 * stride;
        if (t2 < a.total_tiles && tid == 0) issue(t2, s);
    }

    // GEN, after a ring wait gave up: the copies still in flight (at most one per slot) land before exit
    if (GEN && !ring_ok && lane == 0) {
        for (int b = 0; b < RING; b++) {
            const int nb = fills - 1 - ((fills - 1 - b) % RING + RING) % RING;  // the last fill into slot b
            if (nb >= 0) mbar_wait_bounded(&rbar[b], (unsigned)((nb / RING) & 1), 1u << 22);
        }
    }

    // the last CTA of a batch's last launch advances the step counter read by the next launch (no fence:
    // the counter orders no other data, and the next launch reads it only after this grid has completed)
    if (a.t_adv && tid == 0) {
        const unsigned int prev = atomicAdd(&a.ctl->done, 1u);
        if (prev == gridDim.x - 1) {
            a.ctl->done = 0u;
            a.ctl->time = (a.need_time ? s_time : a.ctl->time) + a.t_adv;
        }
    }
}

}  // namespace lbch
