// lbch_pair.cuh -- two consecutive steps of the Cahn-Hilliard lattice Boltzmann equation per launch.
//
// For handles whose instances all have tau_g = 1 and periodic boundaries.  At tau_g = 1, Eq. LB gives
// g* = g_eq + S/2, so the state is phi alone (the populations are multiplied by 1 - 1/tau = 0).  The output
// phi(t+1) of a node depends on phi(t) three nodes out: mu and D = div(phi u) one node out (Eq. mu,
// Eq. mark3), their gradients, the force and the collision one node further (Eqs. liangFi, geq), and the
// pull of the streamed populations one more.  Two steps therefore need phi(t) on the tile + 6.
//
// A CTA loads phi(t) (and the low part of the float path) on tile + 6 with the domain indices wrapped
// periodically -- the stored ghost frame, three deep, is not used -- runs step t on tile + 3 and step t+1
// on the tile, entirely in shared memory, and stores phi(t+2) with the ghost images a one-step launch
// reads.  Each node value is formed by the same per-node helpers in the same order as in the one-step
// kernels (a halo node is computed as the periodic image it stands for), so the result is bit for bit
// that of two one-step launches.  The neighbouring tiles recompute the halo; what this buys is one
// launch -- fixed latency, dependency wait, prologue, load round trip -- per two steps, on grids small
// enough for a step to be latency-bound.
#pragma once
#include "lbch_kernels.cuh"

namespace lbch {

template <typename C, typename P>
struct PairArgs {
    InstDev inst0;          // the record of instance 0, for single-instance handles (read from the parameters)
    const InstDev* inst;
    const int* tile_begin;  // first tile of each instance for this launch's tile shape
    const C* ttabs;         // each tile's velocity tables over tile + 6, PairShape::TAB_STRIDE values per tile
    int n_inst;
    int total_tiles;
    int pitch;
    const P* phi_in;        // phi(t): the high part on the float path
    const float* lo_in;     // low part of phi(t) (float path)
    P* phi_out;             // phi(t+2), with its ghost images
    float* lo_out;
    Ctl* ctl;
    int t_off;              // the launch's first step is ctl->time + t_off, its second one step later
    int t_adv;              // when nonzero, the launch's last CTA advances ctl->time by t_adv
    int need_time;          // some instance's flow depends on the step index
    int debug_skip;         // test hook: CTA 0 never issues its first table copy (its bounded wait runs out)
};

// Shared-memory regions, each centred on the tile: region k spans the tile plus k nodes on every side.
template <typename C, typename P, int TX, int TY>
struct PairShape {
    static constexpr bool FF = sizeof(C) == 4;  // float-float phi
    static constexpr int W6 = TX + 12, H6 = TY + 12, N6 = W6 * H6;  // phi(t), velocity tables
    static constexpr int W5 = TX + 10, H5 = TY + 10, N5 = W5 * H5;  // mu, D of step t
    static constexpr int W4 = TX + 8, H4 = TY + 8, N4 = W4 * H4;    // post-collision populations of step t
    static constexpr int W3 = TX + 6, H3 = TY + 6, N3 = W3 * H3;    // phi(t+1); low parts of phi(t), phi(t+1)
    static constexpr int W2 = TX + 4, H2 = TY + 4, N2 = W2 * H2;    // mu, D of step t+1
    static constexpr int W1 = TX + 2, H1 = TY + 2, N1 = W1 * H1;    // post-collision populations of step t+1
    __host__ __device__ static constexpr size_t a128(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t OFF_LO0 = a128(N6 * sizeof(P));
    static constexpr size_t OFF_HI1 = OFF_LO0 + (FF ? a128(N3 * 4) : 0);
    static constexpr size_t OFF_LO1 = OFF_HI1 + a128(N3 * sizeof(P));
    static constexpr size_t OFF_MU = OFF_LO1 + (FF ? a128(N3 * 4) : 0);
    static constexpr size_t OFF_D = OFF_MU + a128(N5 * sizeof(C));
    static constexpr size_t OFF_POST = OFF_D + a128(N5 * sizeof(C));
    static constexpr size_t OFF_TAB = OFF_POST + a128(9 * N4 * sizeof(C));
    // a tile's velocity tables: X1, X2 over the W6 columns, Y1, Y2 over the H6 rows, padded to 16 bytes
    static constexpr int TAB_N = 2 * W6 + 2 * H6;
    static constexpr unsigned TAB_BYTES = (TAB_N * sizeof(C) + 15) / 16 * 16;
    static constexpr int TAB_STRIDE = TAB_BYTES / sizeof(C);
    static constexpr size_t BYTES = OFF_TAB + a128(TAB_BYTES) + 128;  // + alignment slack
};

// i reduced into [0, n); i lies within a few periods of the domain
__device__ __forceinline__ int wrap_near(int i, int n)
{
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

// mu (Eq. mu) and D = div(phi u) on a region of width W, height H, from phi on the region one node wider
// (row stride PW); the velocity tables are indexed by the phi region's columns/rows shifted by `to`.
template <typename C, typename P, int W, int H, int PW, int NT>
__device__ __forceinline__ void pair_mu_div(const P* ph, const C* sX1, const C* sX2, const C* sY1, const C* sY2,
                                            int to, const Consts<C>& K0, bool model2, C T, C* s_mu, C* s_D)
{
    for_region<W, H, sizeof(C) == 4 ? PW : W, NT>([&](int e, int r, int c) {
        const P* q = ph + (r + 1) * PW + c + 1;
        const C ce = cvt<C>(q[0]);
        const C pE = cvt<C>(q[1]), pW = cvt<C>(q[-1]), pN = cvt<C>(q[PW]), pS = cvt<C>(q[-PW]);
        const C pNE = cvt<C>(q[PW + 1]), pNW = cvt<C>(q[PW - 1]), pSE = cvt<C>(q[-PW + 1]), pSW = cvt<C>(q[-PW - 1]);
        s_mu[e] = node_mu(ce, pE, pW, pN, pS, pNE, pNW, pSE, pSW, K0.beta, K0.kappa, K0.phiA, K0.phiB);
        if (model2) {
            const int tc = c + to, tr = r + to;  // the table index of the node's column/row minus one
            s_D[e] = node_div(pE, pW, pN, pS, pNE, pNW, pSE, pSW, sX1[tc], sX1[tc + 2], sX2[tc], sX2[tc + 1],
                              sX2[tc + 2], sY1[tr], sY1[tr + 1], sY1[tr + 2], sY2[tr], sY2[tr + 2], T);
        }
    });
}

// Force, equilibrium, source and collision at tau = 1 (Eqs. liangFi, mark3, geq, LB) on a region of width
// W, height H; mu and D come from the region one node wider (stride MW), phi from the region two nodes
// wider (stride PW), the velocity at table index (row, col) + tu.  The nine post-collision populations
// are stored as planes of W * H values.
template <typename C, typename P, int W, int H, int MW, int PW, int NT, bool kShift>
__device__ __forceinline__ void pair_collide(const P* ph_reg, const C* s_mu, const C* s_D, const C* sX1,
                                             const C* sX2, const C* sY1, const C* sY2, int tu, const Consts<C>& K0,
                                             bool model2, C T, C* s_post)
{
    for_region<W, H, sizeof(C) == 4 ? MW : W, NT>([&](int e, int r, int c) {
        const int m = (r + 1) * MW + (c + 1);
        C gmx, gmy, gDx = C(0), gDy = C(0);
        grad9(s_mu[m + 1], s_mu[m - 1], s_mu[m + MW], s_mu[m - MW], s_mu[m + MW + 1], s_mu[m + MW - 1],
              s_mu[m - MW + 1], s_mu[m - MW - 1], gmx, gmy);
        if (model2)
            grad9(s_D[m + 1], s_D[m - 1], s_D[m + MW], s_D[m - MW], s_D[m + MW + 1], s_D[m + MW - 1], s_D[m - MW + 1],
                  s_D[m - MW - 1], gDx, gDy);
        const C ph = cvt<C>(ph_reg[(r + 2) * PW + c + 2]);
        C Fx, Fy;
        node_force(ph, gmx, gmy, gDx, gDy, model2, K0.a, K0.b, K0.K, Fx, Fy);
        const C ux = node_u(sX1[c + tu], sY1[r + tu], T), uy = node_u(sX2[c + tu], sY2[r + tu], T);
        C g[9], post[9];
#pragma unroll
        for (int q = 0; q < 9; q++) g[q] = C(0);  // not read at tau = 1
        collide9<C, true, kShift>(ph, s_mu[m], Fx, Fy, ux, uy, g, K0, post);
#pragma unroll
        for (int q = 0; q < 9; q++) s_post[q * (W * H) + e] = post[q];
    });
}

// The streamed populations at node (r, c) of a region of width W, from the post-collision planes of the
// region one node wider (width W + 2, planes of NP values): g_q(x) = g*_q(x - c_q).  Returns g_0 and the
// sum of g_1..g_8 in the order of the one-step kernels.
template <typename C, int W, int NP>
__device__ __forceinline__ C pair_pull(const C* s_post, int r, int c, C& v0)
{
    constexpr int PW = W + 2;
    const int p = (r + 1) * PW + (c + 1);
    C v[9];
    v0 = s_post[p];
#pragma unroll
    for (int q = 1; q < 9; q++) v[q] = s_post[q * NP + p - cy(q) * PW - cx(q)];
    return stream_sum(v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8]);
}

// phi(t+1) = phi(t) + g_0 + sum_q g_q on the float path: hi + lo absorbs the increment exactly (TwoSum),
// as in the one-step kernels; on the double path phi(t+1) is the plain sum.
template <typename C, typename P, bool kFF>
__device__ __forceinline__ P pair_phi(P h_in, float lo_in, C v0, C sumq, float& lo_out)
{
    if (kFF) {
        const float h = (float)h_in;
        const float tt = lo_in + (float)(v0 + sumq);
        const float sm = h + tt;
        const float bb = sm - h;
        lo_out = (h - (sm - bb)) + (tt - bb);
        return (P)sm;
    }
    lo_out = 0.0f;
    return (P)(v0 + sumq);
}

// Shared-memory views of one CTA's regions.
template <typename C, typename P, int TX, int TY>
struct PairSmem {
    P* phi0;     // phi(t) on tile + 6
    float* lo0;  // its low part on tile + 3 (float path)
    P* hi1;      // phi(t+1) on tile + 3
    float* lo1;
    C *mu, *D;   // mu and D of the step in progress
    C* post;     // post-collision populations of the step in progress, nine planes
    C *X1, *X2, *Y1, *Y2;  // velocity tables over the columns / rows of tile + 6
    __device__ explicit PairSmem(unsigned char* raw)
    {
        using L = PairShape<C, P, TX, TY>;
        unsigned char* base = smem_aligned128(raw);
        phi0 = reinterpret_cast<P*>(base);
        lo0 = reinterpret_cast<float*>(base + L::OFF_LO0);
        hi1 = reinterpret_cast<P*>(base + L::OFF_HI1);
        lo1 = reinterpret_cast<float*>(base + L::OFF_LO1);
        mu = reinterpret_cast<C*>(base + L::OFF_MU);
        D = reinterpret_cast<C*>(base + L::OFF_D);
        post = reinterpret_cast<C*>(base + L::OFF_POST);
        X1 = reinterpret_cast<C*>(base + L::OFF_TAB);
        X2 = X1 + L::W6;
        Y1 = X2 + L::W6;
        Y2 = Y1 + L::H6;
    }
};

// A tile's velocity tables (columns and rows of tile + 6, periodically wrapped; laid out per tile at
// set-up) arrive by one bulk copy on an mbarrier, issued by thread 0 first thing, so that the copy's
// latency overlaps the dependency wait and the phi loads.  Thread 0 waits for it (bounded: a copy that never
// lands is reported through ctl->err) before the barrier that precedes the first phase.
template <typename C, typename P, int TX, int TY>
__device__ __forceinline__ void pair_fetch_tables(const PairSmem<C, P, TX, TY>& S, const C* ttabs, int t, uint64_t* bar)
{
    using L = PairShape<C, P, TX, TY>;
    fence_proxy_async();  // the table region was last read through the generic proxy
    mbar_expect_tx(bar, L::TAB_BYTES);
    bulk_load(S.X1, ttabs + (size_t)t * L::TAB_STRIDE, L::TAB_BYTES, bar);
}

// The values one thread loads for a tile: phi on tile + 6 and (float path) its low part on tile + 3, at
// periodically wrapped domain positions.  The offsets, from the instance's first domain node, are computed
// once per tile; -1 marks no value.
template <typename C, typename P, int TX, int TY, int NT>
struct PairLoad {
    using L = PairShape<C, P, TX, TY>;
    static constexpr int IT6 = (L::N6 + NT - 1) / NT, IT3 = (L::N3 + NT - 1) / NT;
    long long o6[IT6], o3[IT3];
    __device__ void init(int nx, int ny, int pitch, int x0, int y0)
    {
#pragma unroll
        for (int i = 0; i < IT6; i++) {
            const int e = threadIdx.x + i * NT, r = e / L::W6, c = e - r * L::W6;
            o6[i] = e < L::N6 ? (long long)wrap_near(y0 - 6 + r, ny) * pitch + wrap_near(x0 - 6 + c, nx) : -1;
        }
#pragma unroll
        for (int i = 0; i < IT3; i++) {
            const int e = threadIdx.x + i * NT, r = e / L::W3, c = e - r * L::W3;
            o3[i] = e < L::N3 && L::FF ? (long long)wrap_near(y0 - 3 + r, ny) * pitch + wrap_near(x0 - 3 + c, nx) : -1;
        }
    }
    // every load is in flight before the first store to shared memory; L2 only (another CTA wrote them)
    __device__ void load(const PairSmem<C, P, TX, TY>& S, const P* phi, const float* lo) const
    {
        P v[IT6];
        float w[IT3];
#pragma unroll
        for (int i = 0; i < IT6; i++)
            if (o6[i] >= 0) v[i] = __ldcg(phi + o6[i]);
#pragma unroll
        for (int i = 0; i < IT3; i++)
            if (o3[i] >= 0) w[i] = __ldcg(lo + o3[i]);
#pragma unroll
        for (int i = 0; i < IT6; i++)
            if (o6[i] >= 0) S.phi0[threadIdx.x + i * NT] = v[i];
#pragma unroll
        for (int i = 0; i < IT3; i++)
            if (o3[i] >= 0) S.lo0[threadIdx.x + i * NT] = w[i];
    }
};

// Steps t and t+1 of one tile from phi(t) and the tables in shared memory (loaded and synchronised by the
// caller): phi(t+2) of the tile's domain nodes and their ghost images into phi_out (rb: the instance's first
// domain node).  T0, T1: the flow's time factor at the two steps.  Ends without a barrier.
template <typename C, typename P, int TX, int TY, int NT>
__device__ __forceinline__ void pair_steps(const PairSmem<C, P, TX, TY>& S, const InstDev& I, C T0, C T1, int x0,
                                           int y0, int pitch, long long rb, P* phi_out, float* lo_out)
{
    using L = PairShape<C, P, TX, TY>;
    constexpr bool kFF = L::FF;
    constexpr bool kShift = sizeof(C) == 4;  // float arithmetic carries g_0 - phi
    constexpr int W6 = L::W6, W3 = L::W3;
    constexpr int NONE = -0x40000000;
    const Consts<C>& K0 = consts<C>(I);
    const bool model2 = I.model == 2;

    // step t: mu, D on tile + 5; collision on tile + 4; streaming to phi(t+1) on tile + 3
    pair_mu_div<C, P, L::W5, L::H5, W6, NT>(S.phi0, S.X1, S.X2, S.Y1, S.Y2, 0, K0, model2, T0, S.mu, S.D);
    __syncthreads();
    pair_collide<C, P, L::W4, L::H4, L::W5, W6, NT, kShift>(S.phi0, S.mu, S.D, S.X1, S.X2, S.Y1, S.Y2, 2, K0, model2, T0,
                                                           S.post);
    __syncthreads();
    for_region<W3, L::H3, sizeof(C) == 4 ? L::W4 : W3, NT>([&](int e, int r, int c) {
        C v0;
        const C sumq = pair_pull<C, W3, L::N4>(S.post, r, c, v0);
        float lo1;
        S.hi1[e] = pair_phi<C, P, kFF>(S.phi0[(r + 3) * W6 + c + 3], kFF ? S.lo0[e] : 0.0f, v0, sumq, lo1);
        if (kFF) S.lo1[e] = lo1;
    });
    __syncthreads();

    // step t+1: mu, D on tile + 2; collision on tile + 1; streaming to phi(t+2) on the tile
    pair_mu_div<C, P, L::W2, L::H2, W3, NT>(S.hi1, S.X1, S.X2, S.Y1, S.Y2, 3, K0, model2, T1, S.mu, S.D);
    __syncthreads();
    pair_collide<C, P, L::W1, L::H1, L::W2, W3, NT, kShift>(S.hi1, S.mu, S.D, S.X1, S.X2, S.Y1, S.Y2, 5, K0, model2, T1,
                                                           S.post);
    __syncthreads();
    const int nx = I.nx, ny = I.ny;
    for_region<TX, TY, sizeof(C) == 4 ? L::W1 : TX, NT>([&](int e, int r, int c) {
        const int gx = x0 + c, gy = y0 + r;
        if (gx >= nx || gy >= ny) return;
        C v0;
        const C sumq = pair_pull<C, TX, L::N1>(S.post, r, c, v0);
        const int h1 = (r + 3) * W3 + c + 3;
        float lo;
        const P hi = pair_phi<C, P, kFF>(S.hi1[h1], kFF ? S.lo1[h1] : 0.0f, v0, sumq, lo);
        const long long node = rb + (long long)gy * pitch + gx;
        phi_out[node] = hi;
        if (kFF) lo_out[node] = lo;
        if (gx < 3 || gx >= nx - 3 || gy < 3 || gy >= ny - 3) {
            // the node's periodic images in the ghost frame (three deep), read by one-step launches
            const int xa = gx < 3 ? gx + nx : NONE, xb = gx >= nx - 3 ? gx - nx : NONE;
            const int ya = gy < 3 ? gy + ny : NONE, yb = gy >= ny - 3 ? gy - ny : NONE;
            for (int iy = 0; iy < 3; iy++) {
                const int yy = iy == 0 ? gy : (iy == 1 ? ya : yb);
                if (yy == NONE) continue;
                for (int ix = 0; ix < 3; ix++) {
                    const int xx = ix == 0 ? gx : (ix == 1 ? xa : xb);
                    if (xx == NONE || (ix == 0 && iy == 0)) continue;
                    phi_out[rb + (long long)yy * pitch + xx] = hi;
                }
            }
        }
    });
}

// The instance and origin of tile t.
template <int TX, int TY>
__device__ __forceinline__ void pair_locate(const int* tile_begin, int n_inst, const InstDev* inst, int t, int& k,
                                            int& x0, int& y0)
{
    k = find_inst(tile_begin, n_inst, t);
    const int local = t - tile_begin[k];
    const int tiles_x = (inst[k].nx + TX - 1) / TX;
    x0 = (local % tiles_x) * TX;
    y0 = (local / tiles_x) * TY;
}

// One launch per two steps: a persistent CTA walks its tiles.  SINGLE (a handle of one instance): the
// instance record stays in the launch parameters, so the tile's origin, tables and load offsets need no
// memory round trip (the table loads start at once, the phi loads right after the dependency wait), and the
// per-node helpers take the instance's constants as constant-bank operands instead of loading them.
template <typename C, typename P, int TX, int TY, int NT, bool SINGLE>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 2) ch_pair_kernel(const __grid_constant__ PairArgs<C, P> a)
{
    extern __shared__ unsigned char smem_raw[];
    const PairSmem<C, P, TX, TY> S(smem_raw);
    __shared__ long long s_time;
    __shared__ int s_k, s_x0, s_y0;
    __shared__ C s_T[2];
    __shared__ InstDev s_I;
    __shared__ __align__(8) uint64_t s_tbar;  // completion of the table copy
    __shared__ int s_abort;                    // a table wait ran out: the CTA stops after it
    const int tid = threadIdx.x;
    const int stride = gridDim.x;
    const bool any = (int)blockIdx.x < a.total_tiles;
    PairLoad<C, P, TX, TY, NT> ld;
    long long n = 0;
    int tuse = 0;  // table copies waited for so far (the mbarrier's phase)
    // thread 0: wait (bounded) for the tile's table copy.  When the wait runs out the kernel records the
    // error, lets the copy land if it was issued (bounded again) so that no copy into this CTA's shared
    // memory outlives it, and tells the CTA to stop; the step counter is still kept consistent below.
    auto wait_tables = [&]() {
        if (!mbar_wait_bounded(&s_tbar, (unsigned)(tuse & 1), 1u << 22)) {
            atomicOr(&a.ctl->err, 1u);
            mbar_wait_bounded(&s_tbar, (unsigned)(tuse & 1), 1u << 22);
            s_abort = 1;
        }
        tuse++;
    };
    if (tid == 0) s_abort = 0;
    if (tid == 0 && any) {
        mbar_init(&s_tbar, 1);
        fence_mbar_init();
        if (!(a.debug_skip && blockIdx.x == 0)) pair_fetch_tables<C, P, TX, TY>(S, a.ttabs, blockIdx.x, &s_tbar);
    }

    if constexpr (SINGLE) {
        const InstDev& I = a.inst0;
        const int tiles_x = (I.nx + TX - 1) / TX;
        const long long rb = (long long)I.row0 * a.pitch + GC;
        int x0 = ((int)blockIdx.x % tiles_x) * TX, y0 = ((int)blockIdx.x / tiles_x) * TY;
        if (any) ld.init(I.nx, I.ny, a.pitch, x0, y0);  // constant data: before the dependency wait
        grid_dependency_wait();
        grid_launch_dependents();
        if (any) ld.load(S, a.phi_in + rb, a.lo_in + rb);
        if (tid == 0) {
            if (any) wait_tables();
            s_time = a.need_time ? a.ctl->time : 0;
            s_T[0] = (C)vel_t(I.vel, I.Tper, s_time + a.t_off);
            s_T[1] = (C)vel_t(I.vel, I.Tper, s_time + a.t_off + 1);
        }
        __syncthreads();
        n = s_time + a.t_off;
        for (int t = blockIdx.x; t < a.total_tiles && !s_abort; t += stride) {
            if (t != (int)blockIdx.x) {
                __syncthreads();  // the previous tile's shared data are read no more
                if (tid == 0) pair_fetch_tables<C, P, TX, TY>(S, a.ttabs, t, &s_tbar);
                x0 = (t % tiles_x) * TX;
                y0 = (t / tiles_x) * TY;
                ld.init(I.nx, I.ny, a.pitch, x0, y0);
                ld.load(S, a.phi_in + rb, a.lo_in + rb);
                if (tid == 0) wait_tables();
                __syncthreads();
                if (s_abort) break;
            }
            pair_steps<C, P, TX, TY, NT>(S, I, s_T[0], s_T[1], x0, y0, a.pitch, rb, a.phi_out, a.lo_out);
        }
    } else {
        // thread 0: tile t's instance (copied when it changes) and origin
        auto locate = [&](int t) {
            int k, x0, y0;
            pair_locate<TX, TY>(a.tile_begin, a.n_inst, a.inst, t, k, x0, y0);
            const bool changed = k != s_k;
            if (changed) s_I = a.inst[k];
            s_k = k;
            s_x0 = x0;
            s_y0 = y0;
            return changed;
        };
        // the first tile: instance, tables and load offsets are constant data, set up before the wait
        if (tid == 0) {
            s_k = -1;
            if (any) locate(blockIdx.x);
        }
        __syncthreads();
        if (any) ld.init(s_I.nx, s_I.ny, a.pitch, s_x0, s_y0);
        long long rb = (long long)s_I.row0 * a.pitch + GC;
        grid_dependency_wait();
        grid_launch_dependents();
        if (any) ld.load(S, a.phi_in + rb, a.lo_in + rb);
        if (tid == 0) {
            if (any) wait_tables();
            s_time = a.need_time ? a.ctl->time : 0;
            if (s_k >= 0) {
                s_T[0] = (C)vel_t(s_I.vel, s_I.Tper, s_time + a.t_off);
                s_T[1] = (C)vel_t(s_I.vel, s_I.Tper, s_time + a.t_off + 1);
            }
        }
        __syncthreads();
        n = s_time + a.t_off;
        for (int t = blockIdx.x; t < a.total_tiles && !s_abort; t += stride) {
            if (t != (int)blockIdx.x) {
                __syncthreads();  // the previous tile's shared data are read no more
                if (tid == 0) {
                    pair_fetch_tables<C, P, TX, TY>(S, a.ttabs, t, &s_tbar);
                    if (locate(t)) {
                        s_T[0] = (C)vel_t(s_I.vel, s_I.Tper, n);
                        s_T[1] = (C)vel_t(s_I.vel, s_I.Tper, n + 1);
                    }
                }
                __syncthreads();
                ld.init(s_I.nx, s_I.ny, a.pitch, s_x0, s_y0);
                rb = (long long)s_I.row0 * a.pitch + GC;
                ld.load(S, a.phi_in + rb, a.lo_in + rb);
                if (tid == 0) wait_tables();
                __syncthreads();
                if (s_abort) break;
            }
            pair_steps<C, P, TX, TY, NT>(S, s_I, s_T[0], s_T[1], s_x0, s_y0, a.pitch, rb, a.phi_out, a.lo_out);
        }
    }

    // the last CTA of a batch's last launch advances the step counter (as in the one-step kernels)
    if (a.t_adv && tid == 0) {
        unsigned int prev = atomicAdd(&a.ctl->done, 1u);
        if (prev == gridDim.x - 1) {
            a.ctl->done = 0u;
            a.ctl->time = (a.need_time ? n - a.t_off : a.ctl->time) + a.t_adv;
        }
    }
}

}  // namespace lbch
