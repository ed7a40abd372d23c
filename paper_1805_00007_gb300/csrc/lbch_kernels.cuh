// lbch_kernels.cuh -- sm_103a device code of the Cahn-Hilliard lattice Boltzmann step.
//
// Method: Zhang, Guo & Liang, arXiv:1805.00007, Sec. II (Eqs. LB, geq, liangFi, macroscopicg, mu, bulk,
// betakappa, rho, t0-phiu, mark3).  The step is one fused, memory-bound tile kernel; no tensor cores.
//
// Per step and tile (TX x TY output nodes) the kernel
//   1. builds the wrapped/mirrored row and column maps and separable velocity tables for the tile + 3 halo,
//   2. loads phi(t) on tile + 3 into shared memory (phi is stored, so g is never re-summed for the halo),
//   3. computes mu = f'(phi) - kappa lap phi and D = div(phi u) on tile + 2,
//   4. on tile + 1 computes grad mu, grad D, the force F, g_eq and S, reads g(t) and collides,
//   5. pulls the post-collision populations g*_i(x - c_i) from shared memory for every tile node, applies
//      halfway bounce-back at walls, and writes g(t+1) and phi(t+1) = sum_i g_i(t+1).
// HBM traffic per lattice update is one read and one write of the 9 populations and of phi; the halo
// re-reads of neighbouring tiles are served by L2.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbch {

// ------------------------------------------------------------------------------------------ lattice
// D2Q9 (Sec. II.B): c0=(0,0), c1=-c3=(1,0), c2=-c4=(0,1), c5=-c7=(1,1), c6=-c8=(-1,1).
__host__ __device__ constexpr int cx(int q) { return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0); }
__host__ __device__ constexpr int cy(int q) { return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 5 + 2) % 4) + 5); }
// Weights w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36, as exact fractions of the compute type.
template <typename C> __host__ __device__ constexpr C wq(int q) { return q == 0 ? C(4) / C(9) : (q <= 4 ? C(1) / C(9) : C(1) / C(36)); }

enum Vel { VEL_UNIFORM = 0, VEL_ROTATION = 1, VEL_VORTEX = 2, VEL_SHEAR = 3, VEL_REV_SHEAR = 4, VEL_DEFORM = 5 };

// Per-instance parameters and derived constants, resident in device memory.
struct InstDev {
    long long off;          // element offset of node (0, 0) inside every population plane
    int nx, ny, pitch;      // lattice size and row pitch (elements)
    int walls, model, vel, nvort;
    int tiles_x, tiles_y, tile_begin;
    int pad_;
    double tau, beta, kappa, eta, a, b, K, phiA, phiB;
    double U0, ux0, uy0, xc, yc, half, Tper, shear;
};

// Step counter shared by the launches of one handle: the last block of each step advances `time`.
struct Ctl {
    long long time;
    unsigned int done;
    unsigned int err;
};

// ------------------------------------------------------------------------------------------ velocity
// Every prescribed flow is a sum-free separable product: ux = X1(x) Y1(y) T(t), uy = X2(x) Y2(y) T(t).
// The tables are evaluated in double and stored in the compute type.
__device__ inline void vel_x(const InstDev& I, double x, double& X1, double& X2)
{
    const double pi = 3.14159265358979323846;
    const double L = (double)I.nx;
    switch (I.vel) {
    case VEL_UNIFORM: X1 = 1.0; X2 = 1.0; break;
    case VEL_ROTATION: X1 = 1.0; X2 = I.U0 * pi * (x - I.xc) / I.half; break;
    case VEL_VORTEX: { double s = sin(pi * x / L); X1 = -I.U0 * s * s; X2 = I.U0 * sin(2.0 * pi * x / L); break; }
    case VEL_SHEAR: X1 = 1.0; X2 = 0.0; break;
    case VEL_REV_SHEAR: X1 = -I.U0 * pi * cos(pi * (x / L - 0.5)); X2 = I.U0 * pi * sin(pi * (x / L - 0.5)); break;
    case VEL_DEFORM: { double k = (double)I.nvort * pi; X1 = -I.U0 * sin(k * (x / L + 0.5)); X2 = -I.U0 * cos(k * (x / L + 0.5)); break; }
    default: X1 = 0.0; X2 = 0.0;
    }
}

__device__ inline void vel_y(const InstDev& I, double y, double& Y1, double& Y2)
{
    const double pi = 3.14159265358979323846;
    const double Lx = (double)I.nx, Ly = (double)I.ny;
    switch (I.vel) {
    case VEL_UNIFORM: Y1 = I.ux0; Y2 = I.uy0; break;
    case VEL_ROTATION: Y1 = -I.U0 * pi * (y - I.yc) / I.half; Y2 = 1.0; break;
    case VEL_VORTEX: { double s = sin(pi * y / Ly); Y1 = sin(2.0 * pi * y / Ly); Y2 = s * s; break; }
    case VEL_SHEAR: Y1 = I.shear * (y - 0.5 * (double)(I.ny - 1)); Y2 = 0.0; break;
    case VEL_REV_SHEAR: Y1 = sin(pi * (y / Lx - 0.5)); Y2 = cos(pi * (y / Lx - 0.5)); break;
    case VEL_DEFORM: { double k = (double)I.nvort * pi; Y1 = sin(k * (y / Lx + 0.5)); Y2 = cos(k * (y / Lx + 0.5)); break; }
    default: Y1 = 0.0; Y2 = 0.0;
    }
}

__device__ inline double vel_t(const InstDev& I, long long n)
{
    const double pi = 3.14159265358979323846;
    switch (I.vel) {
    case VEL_VORTEX:
    case VEL_DEFORM: return cos(pi * (double)n / I.Tper);
    case VEL_REV_SHEAR: return ((double)n < I.Tper) ? 1.0 : -1.0;
    default: return 1.0;
    }
}

// ------------------------------------------------------------------------------------------ storage
template <typename T> __device__ __forceinline__ float to_f(T v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <typename C, typename T> __device__ __forceinline__ C ld(const T* p) { return (C)to_f(*p); }
template <> __device__ __forceinline__ double ld<double, double>(const double* p) { return *p; }
template <typename T, typename C> __device__ __forceinline__ void st(T* p, C v) { *p = (T)v; }
template <> __device__ __forceinline__ void st<__half, float>(__half* p, float v) { *p = __float2half_rn(v); }

// Population plane q: shifted-half storage keeps only planes 1..8 (g0 is implied by phi).
template <typename S> __device__ __forceinline__ long long plane_of(int q, long long plane)
{
    return (sizeof(S) == 2) ? (long long)(q - 1) * plane : (long long)q * plane;
}

template <typename S, typename P>
struct StepArgs {
    const InstDev* inst;
    int n_inst;
    int total_tiles;
    long long plane;  // elements per population plane
    const S* g_in;
    S* g_out;
    const P* phi_in;
    P* phi_out;
    Ctl* ctl;
};

__device__ __forceinline__ int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }
__device__ __forceinline__ int mirror_clamp(int j, int n)
{
    if (j < 0) j = -1 - j;
    if (j >= n) j = 2 * n - 1 - j;
    return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

__device__ __forceinline__ int find_inst(const InstDev* inst, int n_inst, int tile)
{
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (inst[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename C> __device__ __forceinline__ C dfdphi(C phi, C beta, C phiA, C phiB)
{
    // d/dphi of beta (phi - phiA)^2 (phi - phiB)^2 (Eq. bulk)
    return C(2) * beta * (phi - phiA) * (phi - phiB) * (C(2) * phi - phiA - phiB);
}

template <int TX, int TY, typename C>
struct TileSmem {
    static constexpr int PW = TX + 6, PH = TY + 6, MW = TX + 4, MH = TY + 4, GW = TX + 2, GH = TY + 2;
    static constexpr int P = PW * PH, M = MW * MH, G = GW * GH;
    // layout in units of C: phi, jx, jy [P]; mu, D [M]; post [9 G]; X1 X2 [PW]; Y1 Y2 [PH]; then ints
    static constexpr int n_c = 3 * P + 2 * M + 9 * G + 2 * PW + 2 * PH;
    static constexpr size_t bytes = sizeof(C) * n_c + sizeof(int) * (PW + PH) + 16;
};

// ------------------------------------------------------------------------------------------ step
template <typename C, typename S, typename P, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) ch_step_kernel(StepArgs<S, P> a)
{
    using L = TileSmem<TX, TY, C>;
    constexpr int PW = L::PW, MW = L::MW, GW = L::GW, MH = L::MH, PH = L::PH;
    constexpr bool kHalf = sizeof(S) == 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s_phi = reinterpret_cast<C*>(smem_raw);
    C* s_jx = s_phi + L::P;
    C* s_jy = s_jx + L::P;
    C* s_mu = s_jy + L::P;
    C* s_D = s_mu + L::M;
    C* s_post = s_D + L::M;
    C* s_X1 = s_post + 9 * L::G;
    C* s_X2 = s_X1 + PW;
    C* s_Y1 = s_X2 + PW;
    C* s_Y2 = s_Y1 + PH;
    int* s_col = reinterpret_cast<int*>(s_Y2 + PH);
    int* s_row = s_col + PW;
    __shared__ int s_inst;
    __shared__ long long s_time;

    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    if (tid == 0) {
        s_inst = find_inst(a.inst, a.n_inst, tile);
        s_time = a.ctl->time;
    }
    __syncthreads();
    const InstDev& I = a.inst[s_inst];
    const int nx = I.nx, ny = I.ny, pitch = I.pitch, walls = I.walls, model = I.model;
    const long long off = I.off, plane = a.plane;
    const int local = tile - I.tile_begin;
    const int x0 = (local % I.tiles_x) * TX;
    const int y0 = (local / I.tiles_x) * TY;
    const long long n = s_time;
    const C T = (C)vel_t(I, n);

    // 1. row/column maps and separable velocity tables on tile + 3
    for (int e = tid; e < PW + PH; e += NT) {
        if (e < PW) {
            int xw = wrap(x0 - 3 + e, nx);
            double X1, X2;
            vel_x(I, (double)xw, X1, X2);
            s_col[e] = xw; s_X1[e] = (C)X1; s_X2[e] = (C)X2;
        } else {
            int r = e - PW;
            int gy = y0 - 3 + r;
            int yw = walls ? mirror_clamp(gy, ny) : wrap(gy, ny);
            double Y1, Y2;
            vel_y(I, (double)yw, Y1, Y2);
            s_row[r] = yw; s_Y1[r] = (C)Y1; s_Y2[r] = (C)Y2;
        }
    }
    __syncthreads();

    // 2. phi(t) and the flux phi u on tile + 3
    for (int e = tid; e < L::P; e += NT) {
        int r = e / PW, c = e - r * PW;
        long long gi = off + (long long)s_row[r] * pitch + s_col[c];
        C ph = ld<C>(a.phi_in + gi);
        s_phi[e] = ph;
        s_jx[e] = ph * (s_X1[c] * s_Y1[r] * T);
        s_jy[e] = ph * (s_X2[c] * s_Y2[r] * T);
    }
    __syncthreads();

    // 3. mu = f'(phi) - kappa lap phi (Eq. mu) and D = div(phi u) on tile + 2
    const C beta = (C)I.beta, kappa = (C)I.kappa, phiA = (C)I.phiA, phiB = (C)I.phiB;
    for (int e = tid; e < L::M; e += NT) {
        int r = e / MW, c = e - r * MW;
        int p = (r + 1) * PW + (c + 1);
        C ce = s_phi[p];
        C ax = s_phi[p + 1] + s_phi[p - 1] + s_phi[p + PW] + s_phi[p - PW];
        C dg = s_phi[p + PW + 1] + s_phi[p + PW - 1] + s_phi[p - PW + 1] + s_phi[p - PW - 1];
        // lap = sum_k 2 w_k (psi_k - psi_c) / c_s^2 (isotropic central Laplacian)
        C lap = (C(2) / C(3)) * (ax - C(4) * ce) + (C(1) / C(6)) * (dg - C(4) * ce);
        s_mu[e] = dfdphi(ce, beta, phiA, phiB) - kappa * lap;
        if (model == 2) {
            // div = sum_k w_k c_k . (phi u)(x + c_k) / c_s^2
            C ax1 = (s_jx[p + 1] - s_jx[p - 1]) + (s_jy[p + PW] - s_jy[p - PW]);
            C dg1 = (s_jx[p + PW + 1] + s_jy[p + PW + 1]) + (-s_jx[p + PW - 1] + s_jy[p + PW - 1])
                  + (-s_jx[p - PW - 1] - s_jy[p - PW - 1]) + (s_jx[p - PW + 1] - s_jy[p - PW + 1]);
            s_D[e] = (C(1) / C(3)) * ax1 + (C(1) / C(12)) * dg1;
        }
    }
    if (walls && (y0 < 2 || y0 + TY + 2 > ny)) {
        // every stencil operand takes at a ghost row the value at the mirror row: mu and D at rows
        // -2, -1, ny, ny+1 are copied from rows 1, 0, ny-1, ny-2 (all inside this region)
        __syncthreads();
        for (int e = tid; e < 4 * MW; e += NT) {
            int k = e / MW, c = e - k * MW;
            int gy = (k == 0) ? -2 : (k == 1) ? -1 : (k == 2) ? ny : ny + 1;
            int r = gy - (y0 - 2);
            int rm = (-1 - gy >= 0 ? -1 - gy : 2 * ny - 1 - gy) - (y0 - 2);
            C vmu = 0, vD = 0;
            bool ok = (r >= 0 && r < MH && rm >= 0 && rm < MH);
            // mirror rows are interior rows (ny >= 4), so reads and writes never touch the same row
            if (ok) { vmu = s_mu[rm * MW + c]; vD = s_D[rm * MW + c]; }
            if (ok) { s_mu[r * MW + c] = vmu; if (model == 2) s_D[r * MW + c] = vD; }
        }
    }
    __syncthreads();

    // 4. force, equilibrium, source and collision on tile + 1
    const C eta = (C)I.eta, ra = (C)I.a, rb = (C)I.b, K = (C)I.K;
    const C inv_tau = C(1) / (C)I.tau;
    const C src = C(1) - C(1) / (C(2) * (C)I.tau);
    for (int e = tid; e < L::G; e += NT) {
        int r = e / GW, c = e - r * GW;
        int gy = y0 - 1 + r;
        if (walls && (gy < 0 || gy >= ny)) {
#pragma unroll
            for (int q = 0; q < 9; q++) s_post[q * L::G + e] = C(0);
            continue;
        }
        int m = (r + 1) * MW + (c + 1);
        int p = (r + 2) * PW + (c + 2);
        // grad psi = sum_k w_k c_k psi(x + c_k) / c_s^2
        C gmx = (C(1) / C(3)) * (s_mu[m + 1] - s_mu[m - 1])
              + (C(1) / C(12)) * ((s_mu[m + MW + 1] - s_mu[m + MW - 1]) + (s_mu[m - MW + 1] - s_mu[m - MW - 1]));
        C gmy = (C(1) / C(3)) * (s_mu[m + MW] - s_mu[m - MW])
              + (C(1) / C(12)) * ((s_mu[m + MW + 1] + s_mu[m + MW - 1]) - (s_mu[m - MW + 1] + s_mu[m - MW - 1]));
        C ph = s_phi[p];
        C mu = s_mu[m];
        C rho = ra * ph + rb;                     // Eq. rho
        C fct = ph / rho;
        C Fx = fct * (-ph * gmx);                 // F1 = (phi/rho)(Fs - grad p), Fs = -phi grad mu, grad p = 0
        C Fy = fct * (-ph * gmy);
        if (model == 2) {                         // F2 = 3 c_s^2 K grad(div(phi u)), Eq. mark3
            C gDx = (C(1) / C(3)) * (s_D[m + 1] - s_D[m - 1])
                  + (C(1) / C(12)) * ((s_D[m + MW + 1] - s_D[m + MW - 1]) + (s_D[m - MW + 1] - s_D[m - MW - 1]));
            C gDy = (C(1) / C(3)) * (s_D[m + MW] - s_D[m - MW])
                  + (C(1) / C(12)) * ((s_D[m + MW + 1] + s_D[m + MW - 1]) - (s_D[m - MW + 1] + s_D[m - MW - 1]));
            Fx += K * gDx;
            Fy += K * gDy;
        }
        C ux = s_X1[c + 2] * s_Y1[r + 2] * T;
        C uy = s_X2[c + 2] * s_Y2[r + 2] * T;
        long long gi = off + (long long)s_row[r + 2] * pitch + s_col[c + 2];
        C g[9];
        if (kHalf) {
            C rest = C(0);
#pragma unroll
            for (int q = 1; q < 9; q++) { g[q] = ld<C>(a.g_in + plane_of<S>(q, plane) + gi); rest += g[q]; }
            g[0] = ph - rest;
        } else {
#pragma unroll
            for (int q = 0; q < 9; q++) g[q] = ld<C>(a.g_in + plane_of<S>(q, plane) + gi);
        }
        C uu = ux * ux + uy * uy;
        C emu = eta * mu;
#pragma unroll
        for (int q = 0; q < 9; q++) {
            C geq;
            if (q == 0) {
                geq = ph + (wq<C>(0) - C(1)) * emu - wq<C>(0) * ph * uu * C(1.5);   // Eq. geq, i = 0
            } else {
                C cu = (C)cx(q) * ux + (C)cy(q) * uy;
                geq = wq<C>(q) * emu + wq<C>(q) * ph * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
            }
            C Sq = C(3) * wq<C>(q) * ((C)cx(q) * Fx + (C)cy(q) * Fy);              // Eq. liangFi
            s_post[q * L::G + e] = g[q] - (g[q] - geq) * inv_tau + src * Sq;       // Eq. LB
        }
    }
    __syncthreads();

    // 5. pull streaming from shared memory, bounce-back at walls, write g(t+1), phi(t+1)
    for (int e = tid; e < TX * TY; e += NT) {
        int r = e / TX, c = e - r * TX;
        int gx = x0 + c, gy = y0 + r;
        if (gx >= nx || gy >= ny) continue;
        int b = (r + 1) * GW + (c + 1);
        long long gi = off + (long long)gy * pitch + gx;
        C phin = C(0);
        C v[9];
#pragma unroll
        for (int q = 0; q < 9; q++) {
            int sy = gy - cy(q);
            if (walls && (sy < 0 || sy >= ny)) {
                // halfway bounce-back: the population that left along -c_q returns along c_q, plus the
                // moving-wall term 2 w_q phi (c_q . u_w) / c_s^2
                double X1, X2, Y1, Y2;
                vel_x(I, (double)gx, X1, X2);
                vel_y(I, sy < 0 ? -0.5 : (double)ny - 0.5, Y1, Y2);
                C uwx = (C)X1 * (C)Y1 * T, uwy = (C)X2 * (C)Y2 * T;
                C ph = s_phi[(r + 3) * PW + (c + 3)];
                v[q] = s_post[opp(q) * L::G + b]
                     + C(2) * wq<C>(q) * ph * ((C)cx(q) * uwx + (C)cy(q) * uwy) * C(3);
            } else {
                v[q] = s_post[q * L::G + b - cy(q) * GW - cx(q)];
            }
            phin += v[q];
        }
#pragma unroll
        for (int q = (kHalf ? 1 : 0); q < 9; q++) st(a.g_out + plane_of<S>(q, plane) + gi, v[q]);
        st(a.phi_out + gi, phin);
    }

    // the last block of the launch advances the step counter read by the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned int prev = atomicAdd(&a.ctl->done, 1u);
        if (prev == gridDim.x - 1) {
            a.ctl->done = 0u;
            a.ctl->time = n + 1;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------------------------------------ init
// g_i(x, 0) = g_i^eq(phi0, mu(phi0), u(x, 0)); phi(0) = phi0.  One thread per node.
template <typename C, typename S, typename P>
__global__ void init_kernel(const InstDev* inst, int n_inst, const double* phi0, long long plane,
                            S* g, P* phi, long long total_nodes_padded)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total_nodes_padded) return;
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (inst[mid].off <= k) lo = mid; else hi = mid - 1;
    }
    const InstDev& I = inst[lo];
    long long loc = k - I.off;
    int j = (int)(loc / I.pitch), i = (int)(loc - (long long)j * I.pitch);
    if (j >= I.ny || i >= I.nx) return;
    auto at = [&](int di, int dj) -> double {
        int ii = wrap(i + di, I.nx);
        int jj = I.walls ? mirror_clamp(j + dj, I.ny) : wrap(j + dj, I.ny);
        return phi0[I.off + (long long)jj * I.pitch + ii];
    };
    double c0 = at(0, 0);
    double ax = at(1, 0) + at(-1, 0) + at(0, 1) + at(0, -1);
    double dg = at(1, 1) + at(-1, 1) + at(1, -1) + at(-1, -1);
    double lap = (2.0 / 3.0) * (ax - 4.0 * c0) + (1.0 / 6.0) * (dg - 4.0 * c0);
    C mu = (C)(dfdphi<double>(c0, I.beta, I.phiA, I.phiB) - I.kappa * lap);
    double X1, X2, Y1, Y2;
    vel_x(I, (double)i, X1, X2);
    vel_y(I, (double)j, Y1, Y2);
    double T = vel_t(I, 0);
    C ux = (C)(X1 * Y1 * T), uy = (C)(X2 * Y2 * T);
    C ph = (C)c0, eta = (C)I.eta;
    C uu = ux * ux + uy * uy;
#pragma unroll
    for (int q = 0; q < 9; q++) {
        C geq;
        if (q == 0) {
            geq = ph + (wq<C>(0) - C(1)) * eta * mu - wq<C>(0) * ph * uu * C(1.5);
        } else {
            C cu = (C)cx(q) * ux + (C)cy(q) * uy;
            geq = wq<C>(q) * eta * mu + wq<C>(q) * ph * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
        }
        if (sizeof(S) == 2 && q == 0) continue;
        st(g + plane_of<S>(q, plane) + k, geq);
    }
    st(phi + k, ph);
}

// ------------------------------------------------------------------------------------------ reductions
// Observables in double: [0] sum phi, [1] sum (phi - phi0)^2, [2] sum phi0^2, [3] max, [4] min,
// [5] count of non-finite values.  Pass 1: grid (chunks, n_inst) writes per-block partials in a fixed
// order; pass 2: one block per instance reduces them in a fixed order, so results are reproducible.
constexpr int RED_NT = 256;
constexpr int RED_NV = 6;

__device__ __forceinline__ void red_combine(double* a, const double* b)
{
    a[0] += b[0]; a[1] += b[1]; a[2] += b[2];
    a[3] = fmax(a[3], b[3]); a[4] = fmin(a[4], b[4]); a[5] += b[5];
}

__device__ inline void block_reduce(double* v, double (*sh)[RED_NV])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double t[RED_NV];
#pragma unroll
        for (int k = 0; k < RED_NV; k++) t[k] = __shfl_down_sync(0xffffffffu, v[k], o);
        red_combine(v, t);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < RED_NV; k++) sh[w][k] = v[k];
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        double t[RED_NV];
        if (lane < nw) {
#pragma unroll
            for (int k = 0; k < RED_NV; k++) t[k] = sh[lane][k];
        } else {
            t[0] = t[1] = t[2] = t[5] = 0.0; t[3] = -INFINITY; t[4] = INFINITY;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double u[RED_NV];
#pragma unroll
            for (int k = 0; k < RED_NV; k++) u[k] = __shfl_down_sync(0xffffffffu, t[k], o);
            red_combine(t, u);
        }
#pragma unroll
        for (int k = 0; k < RED_NV; k++) v[k] = t[k];
    }
}

template <typename P>
__global__ void __launch_bounds__(RED_NT) reduce_partials_kernel(const InstDev* inst, const P* phi,
                                                                 const double* phi0, double* partials,
                                                                 int chunks)
{
    __shared__ double sh[RED_NT / 32][RED_NV];
    const InstDev& I = inst[blockIdx.y];
    const long long N = (long long)I.nx * I.ny;
    double v[RED_NV] = {0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    for (long long k = (long long)blockIdx.x * RED_NT + threadIdx.x; k < N; k += (long long)chunks * RED_NT) {
        int j = (int)(k / I.nx), i = (int)(k - (long long)j * I.nx);
        long long gi = I.off + (long long)j * I.pitch + i;
        double p = (double)phi[gi], p0 = phi0[gi];
        if (!isfinite(p)) { v[5] += 1.0; continue; }
        v[0] += p; v[1] += (p - p0) * (p - p0); v[2] += p0 * p0;
        v[3] = fmax(v[3], p); v[4] = fmin(v[4], p);
    }
    block_reduce(v, sh);
    if (threadIdx.x == 0) {
        double* out = partials + ((long long)blockIdx.y * chunks + blockIdx.x) * RED_NV;
#pragma unroll
        for (int k = 0; k < RED_NV; k++) out[k] = v[k];
    }
}

__global__ void __launch_bounds__(RED_NT) reduce_final_kernel(const double* partials, int chunks, double* result)
{
    __shared__ double sh[RED_NT / 32][RED_NV];
    double v[RED_NV] = {0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    const double* base = partials + (long long)blockIdx.x * chunks * RED_NV;
    for (int c = threadIdx.x; c < chunks; c += RED_NT) red_combine(v, base + (long long)c * RED_NV);
    block_reduce(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < RED_NV; k++) result[blockIdx.x * RED_NV + k] = v[k];
    }
}

}  // namespace lbch
