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
    const InstDev* inst;
    const int* tile_begin;  // first tile of each instance for this launch's tile shape
    const C* tabs;          // velocity tables of all instances (constant after set-up)
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
    static constexpr size_t BYTES = OFF_TAB + a128((2 * W6 + 2 * H6) * sizeof(C)) + 128;  // + alignment slack
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
    for (int e = threadIdx.x; e < W * H; e += NT) {
        const int r = e / W, c = e - r * W;
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
    }
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
    for (int e = threadIdx.x; e < W * H; e += NT) {
        const int r = e / W, c = e - r * W;
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
    }
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

template <typename C, typename P, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 2) ch_pair_kernel(PairArgs<C, P> a)
{
    using L = PairShape<C, P, TX, TY>;
    constexpr bool kFF = L::FF;
    constexpr bool kShift = sizeof(C) == 4;  // float arithmetic carries g_0 - phi
    constexpr int W6 = L::W6, H6 = L::H6, W3 = L::W3;
    constexpr int NONE = -0x40000000;
    constexpr int IT6 = (L::N6 + NT - 1) / NT, IT3 = (L::N3 + NT - 1) / NT;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    P* s_phi0 = reinterpret_cast<P*>(base);
    float* s_lo0 = reinterpret_cast<float*>(base + L::OFF_LO0);
    P* s_hi1 = reinterpret_cast<P*>(base + L::OFF_HI1);
    float* s_lo1 = reinterpret_cast<float*>(base + L::OFF_LO1);
    C* s_mu = reinterpret_cast<C*>(base + L::OFF_MU);
    C* s_D = reinterpret_cast<C*>(base + L::OFF_D);
    C* s_post = reinterpret_cast<C*>(base + L::OFF_POST);
    C* sX1 = reinterpret_cast<C*>(base + L::OFF_TAB);  // X1, X2 over the columns of tile + 6
    C* sX2 = sX1 + W6;
    C* sY1 = sX2 + W6;                                 // Y1, Y2 over its rows
    C* sY2 = sY1 + H6;

    __shared__ long long s_time;
    __shared__ int s_k, s_x0, s_y0;
    __shared__ C s_T[2];
    __shared__ InstDev s_I;

    const int tid = threadIdx.x;
    const int stride = gridDim.x;

    // thread 0: the instance and origin of tile t (the instance record is copied when it changes)
    auto locate = [&](int t) {
        const int k = find_inst(a.tile_begin, a.n_inst, t);
        if (k != s_k) {
            s_I = a.inst[k];
            s_k = k;
        }
        const int local = t - a.tile_begin[k];
        const int tiles_x = (s_I.nx + TX - 1) / TX;
        s_x0 = (local % tiles_x) * TX;
        s_y0 = (local / tiles_x) * TY;
    };
    // the velocity tables of tile + 6, by wrapped stored column and row (constant after set-up)
    auto load_tables = [&]() {
        const C* tX1 = a.tabs + s_I.tab;
        const C* tY1 = tX1 + 2 * a.pitch;
        for (int e = tid; e < 2 * (W6 + H6); e += NT) {
            if (e < 2 * W6) {
                const int j = e >= W6, c = e - j * W6;
                sX1[e] = __ldg(tX1 + j * a.pitch + GC + wrap_near(s_x0 - 6 + c, s_I.nx));
            } else {
                const int j = (e - 2 * W6) >= H6, r = e - 2 * W6 - j * H6;
                sY1[e - 2 * W6] = __ldg(tY1 + j * s_I.ylen + GR + wrap_near(s_y0 - 6 + r, s_I.ny));
            }
        }
    };
    // phi(t) on tile + 6 and its low part on tile + 3, all loads in flight before the first store (L2
    // only: the previous launch wrote them)
    auto load_phi = [&]() {
        const int nx = s_I.nx, ny = s_I.ny, x0 = s_x0, y0 = s_y0;
        const long long rb = (long long)s_I.row0 * a.pitch + GC;
        P v[IT6];
        float w[IT3];
#pragma unroll
        for (int i = 0; i < IT6; i++) {
            const int e = tid + i * NT;
            if (e < L::N6) {
                const int r = e / W6, c = e - r * W6;
                v[i] = __ldcg(a.phi_in + rb + (long long)wrap_near(y0 - 6 + r, ny) * a.pitch + wrap_near(x0 - 6 + c, nx));
            }
        }
        if (kFF) {
#pragma unroll
            for (int i = 0; i < IT3; i++) {
                const int e = tid + i * NT;
                if (e < L::N3) {
                    const int r = e / W3, c = e - r * W3;
                    w[i] = __ldcg(a.lo_in + rb + (long long)wrap_near(y0 - 3 + r, ny) * a.pitch + wrap_near(x0 - 3 + c, nx));
                }
            }
        }
#pragma unroll
        for (int i = 0; i < IT6; i++)
            if (tid + i * NT < L::N6) s_phi0[tid + i * NT] = v[i];
        if (kFF) {
#pragma unroll
            for (int i = 0; i < IT3; i++)
                if (tid + i * NT < L::N3) s_lo0[tid + i * NT] = w[i];
        }
    };

    // the first tile's instance and tables are constant data: read before the dependency wait, so they
    // overlap the previous launch's tail
    if (tid == 0) {
        s_k = -1;
        if ((int)blockIdx.x < a.total_tiles) locate(blockIdx.x);
    }
    __syncthreads();
    if ((int)blockIdx.x < a.total_tiles) load_tables();
    grid_dependency_wait();
    grid_launch_dependents();
    if ((int)blockIdx.x < a.total_tiles) load_phi();
    if (tid == 0) {
        s_time = a.need_time ? a.ctl->time : 0;
        if (s_k >= 0) {
            s_T[0] = (C)vel_t(s_I.vel, s_I.Tper, s_time + a.t_off);
            s_T[1] = (C)vel_t(s_I.vel, s_I.Tper, s_time + a.t_off + 1);
        }
    }
    __syncthreads();
    const long long n = s_time + a.t_off;

    for (int t = blockIdx.x; t < a.total_tiles; t += stride) {
        if (t != (int)blockIdx.x) {
            __syncthreads();  // the previous tile's shared data are read no more
            if (tid == 0) {
                const int k0 = s_k;
                locate(t);
                if (s_k != k0) {
                    s_T[0] = (C)vel_t(s_I.vel, s_I.Tper, n);
                    s_T[1] = (C)vel_t(s_I.vel, s_I.Tper, n + 1);
                }
            }
            __syncthreads();
            load_tables();
            load_phi();
            __syncthreads();
        }
        const Consts<C>& K0 = consts<C>(s_I);
        const bool model2 = s_I.model == 2;

        // step t: mu, D on tile + 5; collision on tile + 4; streaming to phi(t+1) on tile + 3
        pair_mu_div<C, P, L::W5, L::H5, W6, NT>(s_phi0, sX1, sX2, sY1, sY2, 0, K0, model2, s_T[0], s_mu, s_D);
        __syncthreads();
        pair_collide<C, P, L::W4, L::H4, L::W5, W6, NT, kShift>(s_phi0, s_mu, s_D, sX1, sX2, sY1, sY2, 2, K0, model2,
                                                               s_T[0], s_post);
        __syncthreads();
        for (int e = tid; e < L::N3; e += NT) {
            const int r = e / W3, c = e - r * W3;
            C v0;
            const C sumq = pair_pull<C, W3, L::N4>(s_post, r, c, v0);
            float lo1;
            s_hi1[e] = pair_phi<C, P, kFF>(s_phi0[(r + 3) * W6 + c + 3], kFF ? s_lo0[e] : 0.0f, v0, sumq, lo1);
            if (kFF) s_lo1[e] = lo1;
        }
        __syncthreads();

        // step t+1: mu, D on tile + 2; collision on tile + 1; streaming to phi(t+2) on the tile
        pair_mu_div<C, P, L::W2, L::H2, W3, NT>(s_hi1, sX1, sX2, sY1, sY2, 3, K0, model2, s_T[1], s_mu, s_D);
        __syncthreads();
        pair_collide<C, P, L::W1, L::H1, L::W2, W3, NT, kShift>(s_hi1, s_mu, s_D, sX1, sX2, sY1, sY2, 5, K0, model2,
                                                               s_T[1], s_post);
        __syncthreads();
        const int nx = s_I.nx, ny = s_I.ny, x0 = s_x0, y0 = s_y0, pitch = a.pitch;
        const long long rb = (long long)s_I.row0 * pitch + GC;
        for (int e = tid; e < TX * TY; e += NT) {
            const int r = e / TX, c = e - r * TX;
            const int gx = x0 + c, gy = y0 + r;
            if (gx >= nx || gy >= ny) continue;
            C v0;
            const C sumq = pair_pull<C, TX, L::N1>(s_post, r, c, v0);
            const int h1 = (r + 3) * W3 + c + 3;
            float lo;
            const P hi = pair_phi<C, P, kFF>(s_hi1[h1], kFF ? s_lo1[h1] : 0.0f, v0, sumq, lo);
            const long long node = rb + (long long)gy * pitch + gx;
            a.phi_out[node] = hi;
            if (kFF) a.lo_out[node] = lo;
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
                        a.phi_out[rb + (long long)yy * pitch + xx] = hi;
                    }
                }
            }
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
