// lbch_kernels.cuh -- sm_103a device code of the Cahn-Hilliard lattice Boltzmann step.
//
// Method: Zhang, Guo & Liang, arXiv:1805.00007, Sec. II (Eqs. LB, geq, liangFi, macroscopicg, mu, bulk,
// betakappa, rho, t0-phiu, mark3).  The step is one fused, memory-bound kernel; no tensor cores.
//
// Storage ("padded image layout").  Every stored row has the same pitch.  An instance occupies
// ny + 2*GR consecutive stored rows; domain node (x, y) sits at stored row row0 + y, column GC + x.  The
// ghost rows and columns around the domain hold copies of the nodes they stand for -- periodic images,
// or mirror images next to walls -- written by the step that produces those nodes, so that the halo of
// every tile is one contiguous box of the stored array.  The populations are interleaved by row:
// g[(row * nq + q) * pitch + col], so one 3-D TMA box (columns x planes x rows) brings a tile's planes.
// phi is a plain 2-D array phi[row * pitch + col].
//
// Per step a persistent CTA walks its tiles (TX x TY output nodes) with a two-stage TMA pipeline:
// while tile k is computed, the population box (tile + 1 halo) and the phi box (tile + 3 halo) of the
// next tile are in flight.  For each tile the CTA
//   1. forms phi and the flux phi u on tile + 3 (velocity from per-instance separable tables),
//   2. computes mu = f'(phi) - kappa lap phi and D = div(phi u) on tile + 2,
//   3. on tile + 1 computes grad mu, grad D, the force F, g_eq and S and collides, in place in the box,
//   4. pulls g*_i(x - c_i) from shared memory for every tile node (halfway bounce-back at walls) and
//      stores g(t+1) and phi(t+1), with the ghost images the next step's boxes need.
// HBM traffic per lattice update is one read and one write of the stored populations and of phi; the
// overlap of neighbouring tiles' boxes is served from L2.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbch {

constexpr int GC = 4;  // ghost columns on each side (keeps box starts 16-byte aligned)
constexpr int GR = 3;  // ghost rows on each side (phi halo of the stencil chain)

// ------------------------------------------------------------------------------------------ lattice
// D2Q9 (Sec. II.B): c0=(0,0), c1=-c3=(1,0), c2=-c4=(0,1), c5=-c7=(1,1), c6=-c8=(-1,1).
__host__ __device__ constexpr int cx(int q) { return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0); }
__host__ __device__ constexpr int cy(int q) { return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 5 + 2) % 4) + 5); }
// Weights w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36.
template <typename C> __host__ __device__ constexpr C wq(int q) { return q == 0 ? C(4) / C(9) : (q <= 4 ? C(1) / C(9) : C(1) / C(36)); }

enum Vel { VEL_UNIFORM = 0, VEL_ROTATION = 1, VEL_VORTEX = 2, VEL_SHEAR = 3, VEL_REV_SHEAR = 4, VEL_DEFORM = 5 };

// Derived constants of one instance in the arithmetic type of a kernel.
template <typename C>
struct Consts {
    C beta, kappa, eta, a, b, K, phiA, phiB;
    C itau, omt, src;  // 1/tau, 1 - 1/tau, 1 - 1/(2 tau)
    C cF1, cmu;        // Model III: 2 tau - 1 + 3K and 3 c_s^2 eta K, the coefficients of d_t F1 and d_t grad mu
    // the collision's coefficients per direction class (axis a, diagonal d), each one rounded product:
    // w/tau, 3 (w/tau), (3 w)(1 - 1/(2 tau)), formed once at set-up rather than at every node
    C k1a, k1d, k2a, k2d, k3a, k3d;
};

// Per-instance parameters, derived constants and layout, resident in device memory.
struct InstDev {
    int nx, ny;
    int row0;          // stored row of domain row 0 (the instance's first ghost row is row0 - GR)
    int walls, model, vel;
    int ylen;          // length of each Y velocity table: ny rounded up to 16, plus 24 (ghost rows and the
                       // reach of the last tile's slice)
    int tab;           // offset of the velocity tables: X1, X2 [pitch]; Y1, Y2 [ylen]; W[4]
    int slab;          // a slab of a larger periodic grid: its ghost rows hold the neighbouring slabs' rows
                       // (imported between steps), not images of its own rows
    double Tper;
    Consts<double> cd;  // the constants in double (FP64 path, initial state)
    Consts<float> cf;   // and rounded once to float (float paths)
};

template <typename C> __device__ __forceinline__ const Consts<C>& consts(const InstDev& I);
template <> __device__ __forceinline__ const Consts<double>& consts<double>(const InstDev& I) { return I.cd; }
template <> __device__ __forceinline__ const Consts<float>& consts<float>(const InstDev& I) { return I.cf; }

// Step counter shared by the launches of one handle.  A launch's step is time + its offset; the launch
// that ends a batch (a captured graph of steps, or a single step) advances `time` from its last CTA.
struct Ctl {
    long long time;
    unsigned int done;
    unsigned int err;   // bit 0: a TMA wait timed out
};

// Time factor of the prescribed flows: u(x, y, t) = (X1(x) Y1(y), X2(x) Y2(y)) T(t).
__host__ __device__ inline double vel_t(int vel, double Tper, long long n)
{
    const double pi = 3.14159265358979323846;
    switch (vel) {
    case VEL_VORTEX:
    case VEL_DEFORM: return cos(pi * (double)n / Tper);
    case VEL_REV_SHEAR: return ((double)n < Tper) ? 1.0 : -1.0;
    default: return 1.0;
    }
}

// ------------------------------------------------------------------------------------------ helpers
template <typename T> __device__ __forceinline__ float to_f(T v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <typename C, typename T> __device__ __forceinline__ C cvt(T v) { return (C)to_f(v); }
template <> __device__ __forceinline__ double cvt<double, double>(double v) { return v; }
template <typename T, typename C> __device__ __forceinline__ T to_s(C v) { return (T)v; }
template <> __device__ __forceinline__ __half to_s<__half, float>(float v) { return __float2half_rn(v); }

template <typename C> __device__ __forceinline__ C rcp(C v);
template <> __device__ __forceinline__ float rcp<float>(float v) { return __frcp_rn(v); }
// double reciprocal: a float seed refined by two Newton-Raphson steps r <- r (2 - v r); the error
// squares at each step (2^-23 -> 2^-46 -> below double rounding)
template <> __device__ __forceinline__ double rcp<double>(double v)
{
    double r = (double)__frcp_rn((float)v);
    r = r * fma(-v, r, 2.0);
    r = r * fma(-v, r, 2.0);
    return r;
}

template <typename C> __device__ __forceinline__ C dfdphi(C phi, C beta, C phiA, C phiB)
{
    // d/dphi of beta (phi - phiA)^2 (phi - phiB)^2 (Eq. bulk)
    return C(2) * beta * (phi - phiA) * (phi - phiB) * (C(2) * phi - phiA - phiB);
}

// The instance owning tile `tile`: tile_begin[k] is the first tile of instance k for the launch's shape.
__device__ __forceinline__ int find_inst(const int* tile_begin, int n_inst, int tile)
{
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_begin[mid] <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }
__device__ __forceinline__ int mirror(int j, int n)
{
    if (j < 0) j = -1 - j;
    if (j >= n) j = 2 * n - 1 - j;
    return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

// ------------------------------------------------------------------------------------------ per-node arithmetic
// Used by both forms of the step kernel (tiles in shared memory; row sweeps in registers), so that every
// quantity is evaluated by the same operations in both.  Every product is an explicit rounded multiply
// or an explicit fused multiply-add: the compiler's own contraction of a*b + c depends on how often a
// product is reused, which differs between the two forms, and would change the last bits.
__device__ __forceinline__ float op_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double op_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float op_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double op_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// d/dphi of beta (phi - phiA)^2 (phi - phiB)^2 (Eq. bulk)
template <typename C> __device__ __forceinline__ C node_dfdphi(C phi, C beta, C phiA, C phiB)
{
    const C s = op_fma(C(2), phi, -phiA) - phiB;
    return op_mul(op_mul(op_mul(op_mul(C(2), beta), phi - phiA), phi - phiB), s);
}

// Eq. mu: mu = f'(phi) - kappa lap phi, with the isotropic nine-point Laplacian
// lap psi = sum_k 2 w_k (psi(x + c_k) - psi(x)) / c_s^2.
template <typename C>
__device__ __forceinline__ C node_mu(C ce, C pE, C pW, C pN, C pS, C pNE, C pNW, C pSE, C pSW, C beta, C kappa,
                                     C phiA, C phiB)
{
    const C ax = (pE + pW) + (pN + pS);
    const C dg = (pNE + pNW) + (pSE + pSW);
    const C lap = op_fma(C(2) / C(3), op_fma(C(-4), ce, ax), op_mul(C(1) / C(6), op_fma(C(-4), ce, dg)));
    return op_fma(-kappa, lap, node_dfdphi(ce, beta, phiA, phiB));
}

// D = div(phi u) = sum_k w_k c_k . (phi u)(x + c_k) / c_s^2 for the separable flow u = (X1 Y1, X2 Y2) T:
// x*m / x*c / x*p are the X tables at column offsets -1 / 0 / +1, y*m / y*c / y*p the Y tables at row
// offsets -1 / 0 / +1.  D is linear in u, so the time factor T multiplies once at the end.
template <typename C>
__device__ __forceinline__ C node_div(C pE, C pW, C pN, C pS, C pNE, C pNW, C pSE, C pSW, C x1m, C x1p, C x2m, C x2c,
                                      C x2p, C y1m, C y1c, C y1p, C y2m, C y2p, C T)
{
    // axis neighbours: (phi ux)(E) - (phi ux)(W) + (phi uy)(N) - (phi uy)(S)
    const C ax1 = op_fma(pE, op_mul(x1p, y1c), -op_mul(pW, op_mul(x1m, y1c)))
                + op_fma(pN, op_mul(x2c, y2p), -op_mul(pS, op_mul(x2c, y2m)));
    // diagonal neighbours: c_k . (phi u)(x + c_k) for NE, NW, SW, SE
    const C bNE = op_fma(x1p, y1p, op_mul(x2p, y2p));
    const C bNW = op_fma(x2m, y2p, -op_mul(x1m, y1p));
    const C bSW = op_fma(x1m, y1m, op_mul(x2m, y2m));
    const C bSE = op_fma(x1p, y1m, -op_mul(x2p, y2m));
    const C dg1 = op_fma(pSE, bSE, op_fma(-pSW, bSW, op_fma(pNW, bNW, op_mul(pNE, bNE))));
    return op_mul(op_fma(C(1) / C(3), ax1, op_mul(C(1) / C(12), dg1)), T);
}

// Isotropic gradient grad psi = sum_k w_k c_k psi(x + c_k) / c_s^2.
template <typename C>
__device__ __forceinline__ void grad9(C E, C W, C N, C S, C NE, C NW, C SE, C SW, C& gx, C& gy)
{
    gx = op_fma(C(1) / C(3), E - W, op_mul(C(1) / C(12), (NE - NW) + (SE - SW)));
    gy = op_fma(C(1) / C(3), N - S, op_mul(C(1) / C(12), (NE + NW) - (SE + SW)));
}

// The force: F1 = (phi / rho)(-phi grad mu) with rho = a phi + b (Eq. liangFi, with grad p = 0), plus
// F2 = 3 c_s^2 K grad(div(phi u)) for Model II (Eq. mark3).
template <typename C>
__device__ __forceinline__ void node_force(C ph, C gmx, C gmy, C gDx, C gDy, bool model2, C ra, C rb, C K, C& Fx,
                                           C& Fy)
{
    const C fct = op_mul(op_mul(-ph, ph), rcp<C>(op_fma(ra, ph, rb)));
    Fx = op_mul(fct, gmx);
    Fy = op_mul(fct, gmy);
    if (model2) {
        Fx = op_fma(K, gDx, Fx);
        Fy = op_fma(K, gDy, Fy);
    }
}

// Model III: the complete diffusive-scale force of Eq. F2-1, with the time derivatives on the convective
// scale replaced by backward differences over one step (Remarks I, II).  H = cF1 F1 + cmu grad mu is the
// part under the time derivative; F = F1 + (H - Hprev) + 3 c_s^2 K grad D.  Hprev = H at the first step.
template <typename C>
__device__ __forceinline__ void node_force_full(C ph, C gmx, C gmy, C gDx, C gDy, C Hpx, C Hpy, bool first, C ra, C rb,
                                                C K, C cF1, C cmu, C& Fx, C& Fy, C& Hx, C& Hy)
{
    C F1x, F1y;
    node_force(ph, gmx, gmy, C(0), C(0), false, ra, rb, K, F1x, F1y);
    Hx = op_fma(cF1, F1x, op_mul(cmu, gmx));
    Hy = op_fma(cF1, F1y, op_mul(cmu, gmy));
    const C dHx = first ? C(0) : Hx - Hpx, dHy = first ? C(0) : Hy - Hpy;
    Fx = op_fma(K, gDx, F1x + dHx);
    Fy = op_fma(K, gDy, F1y + dHy);
}

// The prescribed velocity X(x) Y(y) T at a node.
template <typename C> __device__ __forceinline__ C node_u(C X, C Y, C T) { return op_mul(op_mul(X, Y), T); }

// Eq. LB as g* = (1 - 1/tau) g + g_eq / tau + (1 - 1/(2 tau)) S, with Eq. geq and the source
// S_i = w_i c_i . F / c_s^2 (Eq. liangFi), split into the parts even and odd in c_i.  With kShift the
// rest population is carried as g_0 - phi.  With TAU1 (tau = 1) the populations g are not read.  PRE:
// take the per-class coefficients precomputed in K0, else form them here (the same rounded products, so
// the same bits; which is faster depends on the kernel's register budget).
template <typename C, bool TAU1, bool kShift, bool PRE = true>
__device__ __forceinline__ void collide9(C ph, C mu, C Fx, C Fy, C ux, C uy, const C* g, const Consts<C>& K0, C* post)
{
    const C itau = K0.itau, omt = K0.omt;
    // per direction class (axis, diagonal): w/tau, 3 w/tau, 3 w (1 - 1/(2 tau))
    const C k1a = PRE ? K0.k1a : op_mul(wq<C>(1), itau), k1d = PRE ? K0.k1d : op_mul(wq<C>(5), itau);
    const C k2a = PRE ? K0.k2a : op_mul(C(3), k1a), k2d = PRE ? K0.k2d : op_mul(C(3), k1d);
    const C k3a = PRE ? K0.k3a : op_mul(C(3) * wq<C>(1), K0.src), k3d = PRE ? K0.k3d : op_mul(C(3) * wq<C>(5), K0.src);
    const C emu = op_mul(K0.eta, mu);
    const C phuu = op_mul(ph, op_fma(ux, ux, op_mul(uy, uy)));
    const C even = op_fma(C(-1.5), phuu, emu);
    const C ph45 = op_mul(C(4.5), ph);
    C g0eq = op_fma(wq<C>(0) - C(1), emu, op_mul(-wq<C>(0) * C(1.5), phuu));
    if (!kShift) g0eq = ph + g0eq;
    post[0] = TAU1 ? g0eq : op_fma(omt, g[0], op_mul(itau, g0eq));
    // pairs (q, opp q): (1,3) c=(1,0); (2,4) c=(0,1); (5,7) c=(1,1); (6,8) c=(-1,1)
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int q = (k == 0) ? 1 : (k == 1) ? 2 : (k == 2) ? 5 : 6;
        const int o = opp(q);
        const C cu = (k == 0) ? ux : (k == 1) ? uy : (k == 2) ? ux + uy : uy - ux;
        const C cF = (k == 0) ? Fx : (k == 1) ? Fy : (k == 2) ? Fx + Fy : Fy - Fx;
        const C k1 = (q < 5) ? k1a : k1d, k2 = (q < 5) ? k2a : k2d, k3 = (q < 5) ? k3a : k3d;
        const C A = op_mul(k1, op_fma(op_mul(ph45, cu), cu, even));
        const C B = op_fma(k2, op_mul(ph, cu), op_mul(k3, cF));
        post[q] = TAU1 ? A + B : op_fma(omt, g[q], A + B);
        post[o] = TAU1 ? A - B : op_fma(omt, g[o], A - B);
    }
}

// Halfway bounce-back at a wall node: g_q arriving from the ghost row is the node's own post-collision
// g_opp(q) plus the moving-wall term 2 w_q phi (c_q . u_w) / c_s^2.
template <typename C, int q>
__device__ __forceinline__ C bounce(C post_opp, C ph, C uwx, C uwy)
{
    const C cuw = cx(q) == 0 ? (cy(q) > 0 ? uwy : -uwy)
                : (cy(q) == 0 ? (cx(q) > 0 ? uwx : -uwx)
                : (cx(q) > 0 ? (cy(q) > 0 ? uwx + uwy : uwx - uwy) : (cy(q) > 0 ? uwy - uwx : -(uwx + uwy))));
    return op_fma(op_mul(C(6) * wq<C>(q), ph), cuw, post_opp);
}

// Sum of the streamed populations g_1..g_8(t+1) at a node, grouped by the column they come from: the
// three from x - 1 (1, 5, 8), the two from x (2, 4), the three from x + 1 (3, 6, 7).
template <typename C>
__device__ __forceinline__ C stream_sum(C v1, C v2, C v3, C v4, C v5, C v6, C v7, C v8)
{
    return (((v1 + v5) + v8) + (v2 + v4)) + ((v3 + v6) + v7);
}

// ------------------------------------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The dynamic shared memory of a kernel from its first 128-byte boundary.  The offset is added to the shared
// array itself (not formed by a round trip through an integer address), so the compiler still knows every
// pointer derived from it addresses shared memory and issues shared-memory loads and stores rather than
// generic ones.
__device__ __forceinline__ unsigned char* smem_aligned128(unsigned char* raw)
{
    return raw + ((128u - (unsigned)(reinterpret_cast<uintptr_t>(raw) & 127u)) & 127u);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls (each poll may suspend the thread for a short while).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit)
{
    for (unsigned k = 0; k < limit; k++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// programmatic dependent launch: wait for the prerequisite grid to complete with its writes visible (a
// no-op without a programmatic dependency), and allow the dependent grid to be scheduled
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)), "l"(tm), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// plain bulk copy (not tensor-mapped): 16-byte aligned source and destination, size a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)), "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Model III: H(t) of domain node (x, y) and its ghost images one deep (periodic in x; in y unless walls).
template <typename C>
__device__ __forceinline__ void store_h(C* H, long long plane, int row0, int pitch, int nx, int ny, int walls, int x,
                                        int y, C hx, C hy)
{
    const int xa = x == 0 ? nx : (x == nx - 1 ? -1 : x);
    const int ya = walls ? y : (y == 0 ? ny : (y == ny - 1 ? -1 : y));
    for (int iy = 0; iy < 2; iy++) {
        const int yy = iy == 0 ? y : ya;
        if (iy == 1 && yy == y) continue;
        for (int ix = 0; ix < 2; ix++) {
            const int xx = ix == 0 ? x : xa;
            if (ix == 1 && xx == x) continue;
            const long long k = (long long)(row0 + yy) * pitch + GC + xx;
            H[k] = hx;
            H[plane + k] = hy;
        }
    }
}

// The nodes of a W x H region that the CTA's NT threads take in one phase: f(e, r, c) for node e = r W + c.
// STRIDE = W: consecutive threads take consecutive nodes.  STRIDE = W + 2, the row width of the region the
// phase reads its stencil operands from: thread index i stands for row i / STRIDE and column i % STRIDE, and
// the two columns past W idle.  A warp's operand reads then cover consecutive words of the source region;
// with the compact order a warp that crosses a row boundary spans STRIDE + 2 words, so that two of its reads
// fall in one shared-memory bank.  The wider order is taken only where it needs no more passes of the NT
// threads than the compact one, and only where the step is bound by latency rather than a pipe: the FP64
// kernels are bound by the FP64 pipe, where a warp's idle lanes still take their pipe slots (the FP64 tile
// kernel ran 6 % slower with it).  The two-step kernel in float uses it.
template <int W, int H, int STRIDE, int NT, typename F>
__device__ __forceinline__ void for_region(F&& f)
{
    constexpr int SW = (H * STRIDE + NT - 1) / NT == (H * W + NT - 1) / NT ? STRIDE : W;
    for (int i = threadIdx.x; i < H * SW; i += NT) {
        const int r = i / SW, c = i - r * SW;
        if (SW != W && c >= W) continue;
        f(r * W + c, r, c);
    }
}

// ------------------------------------------------------------------------------------------ step
// Storage types: S populations, P phi (the high part on the float path), C arithmetic.  The float path
// (C = S = float) keeps phi as an unevaluated sum of two floats, phi = hi + lo: hi feeds the stencils,
// lo is carried only at the node, and phi(t+1) = phi(t) + increment is formed with an exact TwoSum.
template <typename C, typename S, typename P>
struct StepArgs {
    const InstDev* inst;
    const int* tile_begin;  // first tile of each instance for this launch's tile shape
    const C* tabs;       // velocity tables of all instances, indexed by stored column / instance row
    int n_inst;
    int total_tiles;
    int pitch;           // elements per stored row
    int debug_skip;      // test hook: when nonzero, CTA 0 never issues its first load (its wait runs out)
    S* g_out;
    P* phi_out;
    float* lo_out;       // low part of phi on the float path
    Ctl* ctl;
    const C* H_in;       // Model III: H(t - 1), two planes (x, y) of rows x pitch values; nullptr otherwise
    C* H_out;            // H(t), written for the tile's own nodes and their ghost images
    long long H_plane;   // values per plane of H
    int t_off;           // this launch's step is ctl->time + t_off
    int t_adv;           // when nonzero, the launch's last CTA advances ctl->time by t_adv
    int need_time;       // some instance needs the step index (a time-dependent flow or Model III)
};

template <typename C, typename S, typename P, int TX, int TY>
struct StepShape {
    static constexpr bool FF = sizeof(C) == 4 && sizeof(S) == 4;  // float-float phi
    static constexpr int NQ = (sizeof(S) == 2) ? 8 : 9;        // stored planes
    static constexpr int BW = TX + 8;                          // box width (x0-4 .. x0+TX+3)
    static constexpr int GBH = TY + 2, PBH = TY + 6;           // box heights
    static constexpr int PW = TX + 6, PH = TY + 6;             // tile + 3
    static constexpr int MW = TX + 4, MH = TY + 4;             // tile + 2
    static constexpr int GW = TX + 2, GH = TY + 2;             // tile + 1
    static constexpr int NP = PW * PH, NM = MW * MH, NG = GW * GH;  // region sizes
    static constexpr unsigned GBOX_BYTES = GBH * NQ * BW * sizeof(S);
    static constexpr unsigned PBOX_BYTES = PBH * BW * sizeof(P);
    static constexpr unsigned LBOX_BYTES = FF ? TX * TY * 4 : 0;
    // velocity-table slices of the tile: X1, X2 over the box columns, Y1, Y2 over TY + 8 rows
    static constexpr int YT = TY + 8;
    static constexpr unsigned XT_BYTES = BW * sizeof(C), YT_BYTES = YT * sizeof(C);
    static constexpr unsigned TAB_BYTES = 2 * XT_BYTES + 2 * YT_BYTES;
    __host__ __device__ static constexpr size_t a128(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t OFF_P = a128(GBOX_BYTES), OFF_L = OFF_P + a128(PBOX_BYTES);
    static constexpr size_t OFF_T = OFF_L + a128(LBOX_BYTES);
    static constexpr size_t STAGE = OFF_T + a128(TAB_BYTES);
    static constexpr size_t WORK1 = a128(sizeof(C) * (2 * NM));
    static constexpr size_t WORK = WORK1 + (sizeof(S) == 2 ? a128(sizeof(C) * NG) : 0);  // + h*_0 (half path)
    static constexpr size_t BYTES = 2 * STAGE + WORK + 128 + 128;  // mbarriers, alignment slack
};

// TAU1: the kernel for instances that all have tau_g = 1.  Then Eq. LB gives g* = g_eq + S/2: the
// populations are multiplied by 1 - 1/tau = 0, so they are neither loaded nor stored -- the state is phi
// alone, and the result is bit for bit the general kernel's (which multiplies them by exactly zero).
template <typename C, typename S, typename P, int TX, int TY, int NT, bool TAU1 = false>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : (sizeof(C) == 8 ? 2 : 3)) ch_step_kernel(const __grid_constant__ CUtensorMap tm_g,
                                                     const __grid_constant__ CUtensorMap tm_phi,
                                                     const __grid_constant__ CUtensorMap tm_lo,
                                                     StepArgs<C, S, P> a)
{
    using L = StepShape<C, S, P, TX, TY>;
    constexpr int NQ = L::NQ, BW = L::BW, MW = L::MW, MH = L::MH, GW = L::GW;
    constexpr bool kHalf = sizeof(S) == 2;    // g_0 not stored: implied by phi
    constexpr bool kShift = sizeof(C) == 4;   // float arithmetic on g_0 - phi instead of g_0
    constexpr bool kFF = L::FF;
    constexpr int QOFF = kHalf ? 1 : 0;       // stored plane of population q is q - QOFF
    constexpr int NONE = -0x40000000;

    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_aligned128(smem_raw);
    auto stage = [&](int k) { return base + (size_t)k * L::STAGE; };
    C* s_mu = reinterpret_cast<C*>(base + 2 * L::STAGE);
    C* s_D = s_mu + L::NM;
    C* s_h0 = reinterpret_cast<C*>(base + 2 * L::STAGE + L::WORK1);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(base + 2 * L::STAGE + L::WORK);

    __shared__ long long s_time;
    __shared__ int s_tile_inst;
    __shared__ int3 s_info[2];  // (instance, x0, y0) of the tile in each stage, written when it is issued
    __shared__ C s_T;
    __shared__ InstDev s_I;  // the current tile's instance, copied when the instance changes

    const int tid = threadIdx.x;
    const int stride = gridDim.x;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
        s_tile_inst = -1;
        if ((int)blockIdx.x < a.total_tiles) {  // instance data are constant: read before the dependency wait
            const int k = find_inst(a.tile_begin, a.n_inst, blockIdx.x);
            s_I = a.inst[k];
            s_tile_inst = k;
        }
    }

    // producer: thread 0 issues the boxes of tile t into stage s
    auto issue = [&](int t, int s) {
        int k = find_inst(a.tile_begin, a.n_inst, t);
        const InstDev& I = a.inst[k];
        int local = t - a.tile_begin[k];
        int tiles_x = (I.nx + TX - 1) / TX;
        int x0 = (local % tiles_x) * TX, y0 = (local / tiles_x) * TY;
        s_info[s] = make_int3(k, x0, y0);
        fence_proxy_async();
        mbar_expect_tx(&mbar[s], (TAU1 ? 0u : L::GBOX_BYTES) + L::PBOX_BYTES + L::LBOX_BYTES + L::TAB_BYTES);
        // box column origin: domain x0 - 4 is stored column x0 - 4 + GC = x0
        if (!TAU1) tma_load_3d(stage(s), &tm_g, x0, 0, I.row0 + y0 - 1, &mbar[s]);
        tma_load_2d(stage(s) + L::OFF_P, &tm_phi, x0, I.row0 + y0 - 3, &mbar[s]);
        if (kFF) tma_load_2d(stage(s) + L::OFF_L, &tm_lo, x0 + GC, I.row0 + y0, &mbar[s]);
        // the velocity tables of the box's columns and rows (the Y tables start at the box's first row)
        const C* tX1 = a.tabs + I.tab;
        const C* tY1 = tX1 + 2 * a.pitch;
        unsigned char* tb = stage(s) + L::OFF_T;
        bulk_load(tb, tX1 + x0, L::XT_BYTES, &mbar[s]);
        bulk_load(tb + L::XT_BYTES, tX1 + a.pitch + x0, L::XT_BYTES, &mbar[s]);
        bulk_load(tb + 2 * L::XT_BYTES, tY1 + y0, L::YT_BYTES, &mbar[s]);
        bulk_load(tb + 2 * L::XT_BYTES + L::YT_BYTES, tY1 + I.ylen + y0, L::YT_BYTES, &mbar[s]);
    };

    // Launched as a programmatic dependent of the previous step: everything above overlaps its tail;
    // nothing it writes (phi, g, the step counter) is touched before this wait.  The first boxes are
    // issued before the counter is read, so the two latencies overlap.
    grid_dependency_wait();
    grid_launch_dependents();
    if (tid == 0) {
        for (int j = 0; j < 2; j++) {
            int t = blockIdx.x + j * stride;
            if (t < a.total_tiles && !(a.debug_skip && blockIdx.x == 0 && j == 0)) issue(t, j);
        }
        // the counter is read only when a flow depends on time (or Model III needs the step index);
        // otherwise nothing waits on that load
        s_time = a.need_time ? a.ctl->time : 0;
        if (s_tile_inst >= 0) s_T = (C)vel_t(s_I.vel, s_I.Tper, s_time + a.t_off);
    }
    __syncthreads();
    const long long n = s_time + a.t_off;
    int cur_inst = s_tile_inst;  // the instance in s_I (a register copy, so that no thread races thread 0)

    for (int it = 0;; it++) {
        const int t = blockIdx.x + it * stride;
        if (t >= a.total_tiles) break;
        const int s = it & 1;
        // every thread observes the completion of the stage's copies itself (bounded wait)
        bool ok = mbar_wait_bounded(&mbar[s], (unsigned)((it >> 1) & 1), 1u << 22);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(&a.ctl->err, 1u);
                // let a copy already issued into the other stage land before the CTA exits (bounded)
                if (t + stride < a.total_tiles)
                    mbar_wait_bounded(&mbar[s ^ 1], (unsigned)(((it + 1) >> 1) & 1), 1u << 22);
            }
            break;  // skip the remaining tiles; the step counter below is still kept consistent
        }
        if (s_info[s].x != cur_inst) {  // uniform: a tile of another instance (never the first tile)
            cur_inst = s_info[s].x;
            if (tid == 0) {
                s_I = a.inst[cur_inst];
                s_tile_inst = cur_inst;
                s_T = (C)vel_t(s_I.vel, s_I.Tper, n);  // time factor of the flow, once per instance
            }
            __syncthreads();
        }
        const InstDev& I = s_I;
        const Consts<C>& K0 = consts<C>(I);
        const int nx = I.nx, ny = I.ny, walls = I.walls, model = I.model;
        const int x0 = s_info[s].y, y0 = s_info[s].z;
        const C T = s_T;
        S* gb = reinterpret_cast<S*>(stage(s));
        const P* pb = reinterpret_cast<const P*>(stage(s) + L::OFF_P);  // phi on tile + 3 at box column c + 1
        // velocity tables: X by stored column, Y by row of the instance's stored band
        const C* tX1 = a.tabs + I.tab;
        const C* tX2 = tX1 + a.pitch;
        const C* tY1 = tX2 + a.pitch;
        const C* tY2 = tY1 + I.ylen;
        const C* tW = tY2 + I.ylen;

        // the velocity-table slices arrived with the boxes: X by box column, Y by box row; the prescribed
        // velocity at box (row, col) is (X1[col] Y1[row], X2[col] Y2[row]) T
        const C* sX1 = reinterpret_cast<const C*>(stage(s) + L::OFF_T);
        const C* sX2 = sX1 + BW;
        const C* sY1 = sX2 + BW;
        const C* sY2 = sY1 + L::YT;

        // 2. mu (Eq. mu) and D = div(phi u) on tile + 2
        const C beta = K0.beta, kappa = K0.kappa, phiA = K0.phiA, phiB = K0.phiB;
        // (the compact order in every phase: the strided order of for_region measured no faster here, 4.56
        // against 4.55 us per step for 256^2 at tau_g = 0.8 in FP32, 4.30 against 4.23 with half storage)
        for_region<MW, L::MH, MW, NT>([&](int e, int r, int c) {
            const P* q = pb + (r + 1) * BW + c + 2;
            C ce = cvt<C>(q[0]);
            C pE = cvt<C>(q[1]), pW = cvt<C>(q[-1]), pN = cvt<C>(q[BW]), pS = cvt<C>(q[-BW]);
            C pNE = cvt<C>(q[BW + 1]), pNW = cvt<C>(q[BW - 1]), pSE = cvt<C>(q[-BW + 1]), pSW = cvt<C>(q[-BW - 1]);
            s_mu[e] = node_mu(ce, pE, pW, pN, pS, pNE, pNW, pSE, pSW, beta, kappa, phiA, phiB);
            if (model >= 2)  // the tables at box columns c+1..c+3 and box rows r..r+2
                s_D[e] = node_div(pE, pW, pN, pS, pNE, pNW, pSE, pSW, sX1[c + 1], sX1[c + 3], sX2[c + 1], sX2[c + 2],
                                  sX2[c + 3], sY1[r], sY1[r + 1], sY1[r + 2], sY2[r], sY2[r + 2], T);
        });
        if (walls && (y0 < 2 || y0 + TY + 2 > ny)) {
            // every stencil operand takes at a ghost row the value at the mirror row: mu and D at rows
            // -2, -1, ny, ny+1 are copied from rows 1, 0, ny-1, ny-2 (interior rows, as ny >= 4)
            __syncthreads();
            for (int e = tid; e < 4 * MW; e += NT) {
                int k = e / MW, c = e - k * MW;
                int gy = (k == 0) ? -2 : (k == 1) ? -1 : (k == 2) ? ny : ny + 1;
                int r = gy - (y0 - 2);
                int rm = (gy < 0 ? -1 - gy : 2 * ny - 1 - gy) - (y0 - 2);
                if (r >= 0 && r < MH && rm >= 0 && rm < MH) {
                    C vmu = s_mu[rm * MW + c], vD = s_D[rm * MW + c];
                    s_mu[r * MW + c] = vmu;
                    if (model >= 2) s_D[r * MW + c] = vD;
                }
            }
        }
        __syncthreads();

        // 3. force, equilibrium, source and collision on tile + 1, written back into the box
        const C ra = K0.a, rb = K0.b, K = K0.K;
        for_region<GW, L::GH, GW, NT>([&](int e, int r, int c) {
            int gy = y0 - 1 + r;
            if (walls && (gy < 0 || gy >= ny)) return;  // ghost rows: never pulled (bounce-back)
            int m = (r + 1) * MW + (c + 1);
            C gmx, gmy, gDx = C(0), gDy = C(0);
            grad9(s_mu[m + 1], s_mu[m - 1], s_mu[m + MW], s_mu[m - MW], s_mu[m + MW + 1], s_mu[m + MW - 1],
                  s_mu[m - MW + 1], s_mu[m - MW - 1], gmx, gmy);
            if (model >= 2)
                grad9(s_D[m + 1], s_D[m - 1], s_D[m + MW], s_D[m - MW], s_D[m + MW + 1], s_D[m + MW - 1],
                      s_D[m - MW + 1], s_D[m - MW - 1], gDx, gDy);
            C ph = cvt<C>(pb[(r + 2) * BW + c + 3]);
            C mu = s_mu[m];
            C Fx, Fy;
            if (model == 3) {
                // H(t - 1) at this node (halo nodes included: its images are stored one deep); H(t) is
                // stored for the tile's own nodes only
                const int gx = x0 - 1 + c;
                const long long hn = (long long)(I.row0 + gy) * a.pitch + GC + gx;
                const bool first = n == 0;
                const C Hpx = first ? C(0) : a.H_in[hn], Hpy = first ? C(0) : a.H_in[a.H_plane + hn];
                C Hx, Hy;
                node_force_full(ph, gmx, gmy, gDx, gDy, Hpx, Hpy, first, ra, rb, K, K0.cF1, K0.cmu, Fx, Fy, Hx, Hy);
                if (r >= 1 && r <= TY && c >= 1 && c <= TX && gx < nx && gy < ny)
                    store_h(a.H_out, a.H_plane, I.row0, a.pitch, nx, ny, walls, gx, gy, Hx, Hy);
            } else {
                node_force(ph, gmx, gmy, gDx, gDy, model == 2, ra, rb, K, Fx, Fy);
            }
            const C ux = node_u(sX1[c + 3], sY1[r + 2], T), uy = node_u(sX2[c + 3], sY2[r + 2], T);  // box row r+2, col c+3
            // the node's populations in the box: row r, plane q - QOFF, column c + 3
            S* gp = gb + (r * NQ) * BW + c + 3;
            C g[9];
            if (TAU1) {
#pragma unroll
                for (int q = 0; q < 9; q++) g[q] = C(0);   // multiplied by 1 - 1/tau = 0 below
            } else if (kHalf) {
                C rest = C(0);
#pragma unroll
                for (int q = 1; q < 9; q++) { g[q] = cvt<C>(gp[(q - QOFF) * BW]); rest += g[q]; }
                g[0] = -rest;  // g_0 - phi
            } else {
#pragma unroll
                for (int q = 0; q < 9; q++) g[q] = cvt<C>(gp[q * BW]);
            }
            C post[9];
            collide9<C, TAU1, kShift>(ph, mu, Fx, Fy, ux, uy, g, K0, post);
            if (kHalf) {
                // the rest population takes what the half-rounded moving ones leave of phi (see the row sweep)
                C rest = C(0);
#pragma unroll
                for (int q = 1; q < 9; q++) rest += cvt<C>(to_s<S>(post[q]));
                s_h0[e] = -rest;
            }
#pragma unroll
            for (int q = QOFF; q < 9; q++) gp[(q - QOFF) * BW] = to_s<S>(post[q]);
        });
        __syncthreads();

        // 4. pull streaming from the box, bounce-back at walls; store g(t+1), phi(t+1) and ghost images.
        //    Interior nodes (no wall neighbour, no ghost image) take a straight path without the checks.
        const int pitch = a.pitch;
        const float* lb = reinterpret_cast<const float*>(stage(s) + L::OFF_L);
        for_region<TX, TY, TX, NT>([&](int e, int r, int c) {
            int gx = x0 + c, gy = y0 + r;
            if (gx >= nx || gy >= ny) return;
            const bool wallrow = walls && (gy == 0 || gy == ny - 1);
            const bool edge = gx < 3 || gx >= nx - 3 || gy < 3 || gy >= ny - 3;
            const S* src = gb + ((r + 1) * NQ) * BW + c + 4;   // this node's box position, plane 0
            C v[9];
            v[0] = kHalf ? s_h0[(r + 1) * GW + (c + 1)] : cvt<C>(src[0]);
#pragma unroll
            for (int q = 1; q < 9; q++) v[q] = cvt<C>(src[(-cy(q) * NQ + q - QOFF) * BW - cx(q)]);
            if (wallrow) {
                // populations that would come from a ghost row are bounced back at the node
                const C ph = cvt<C>(pb[(r + 3) * BW + c + 4]);
                if (gy == 0) {
                    const C uwx = node_u(tX1[gx + GC], tW[0], T), uwy = node_u(tX2[gx + GC], tW[2], T);
                    v[2] = bounce<C, 2>(cvt<C>(src[(4 - QOFF) * BW]), ph, uwx, uwy);
                    v[5] = bounce<C, 5>(cvt<C>(src[(7 - QOFF) * BW]), ph, uwx, uwy);
                    v[6] = bounce<C, 6>(cvt<C>(src[(8 - QOFF) * BW]), ph, uwx, uwy);
                }
                if (gy == ny - 1) {
                    const C uwx = node_u(tX1[gx + GC], tW[1], T), uwy = node_u(tX2[gx + GC], tW[3], T);
                    v[4] = bounce<C, 4>(cvt<C>(src[(2 - QOFF) * BW]), ph, uwx, uwy);
                    v[7] = bounce<C, 7>(cvt<C>(src[(5 - QOFF) * BW]), ph, uwx, uwy);
                    v[8] = bounce<C, 8>(cvt<C>(src[(6 - QOFF) * BW]), ph, uwx, uwy);
                }
            }
            const C sumq = stream_sum(v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8]);
            P hi;
            float lo = 0.0f;
            if (kFF) {
                // g_0(t+1) = phi(t) + v_0 stays at the node: phi(t+1) = phi(t) + (v_0 + sum_{q>0} g_q(t+1));
                // hi + lo absorbs the increment exactly (TwoSum); g_0 - phi is stored as -sum_{q>0} g_q
                float h = (float)pb[(r + 3) * BW + c + 4];
                float tt = lb[r * TX + c] + (float)(v[0] + sumq);
                float sm = h + tt;
                float bb = sm - h;
                lo = (h - (sm - bb)) + (tt - bb);
                hi = (P)sm;
                v[0] = -sumq;
            } else if (kShift) {
                // half path: phi(t+1) = phi(t) + v_0 + sum_{q>0} g_q(t+1) in float; g_0 stays implied
                hi = (P)((float)pb[(r + 3) * BW + c + 4] + (float)(v[0] + sumq));
            } else {
                hi = (P)(v[0] + sumq);
            }
            const long long node = (long long)(I.row0 + gy) * pitch + GC + gx;
            a.phi_out[node] = hi;
            if (kFF) a.lo_out[node] = lo;
            if (!TAU1) {
                S* o = a.g_out + ((long long)(I.row0 + gy) * NQ) * pitch + GC + gx;
#pragma unroll
                for (int q = QOFF; q < 9; q++) o[(q - QOFF) * pitch] = to_s<S>(v[q]);
            }
            if (edge) {
                // the node's images in the ghost columns/rows (phi three deep, the populations one deep;
                // in y only for periodic y, mirror images next to walls)
                const int xa = gx < 3 ? gx + nx : NONE, xb = gx >= nx - 3 ? gx - nx : NONE;
                const int ya = gy < 3 ? (walls ? -1 - gy : gy + ny) : NONE;
                const int yb = gy >= ny - 3 ? (walls ? 2 * ny - 1 - gy : gy - ny) : NONE;
                for (int iy = 0; iy < 3; iy++) {
                    const int yy = iy == 0 ? gy : (iy == 1 ? ya : yb);
                    if (yy == NONE) continue;
                    for (int ix = 0; ix < 3; ix++) {
                        const int xx = ix == 0 ? gx : (ix == 1 ? xa : xb);
                        if (xx == NONE || (ix == 0 && iy == 0)) continue;
                        a.phi_out[(long long)(I.row0 + yy) * pitch + GC + xx] = hi;
                    }
                }
                const int gxa = gx == 0 ? nx : (gx == nx - 1 ? -1 : NONE);
                const int gya = walls ? NONE : (gy == 0 ? ny : (gy == ny - 1 ? -1 : NONE));
                for (int iy = 0; iy < (TAU1 ? 0 : 2); iy++) {
                    const int yy = iy == 0 ? gy : gya;
                    if (yy == NONE) continue;
                    for (int ix = 0; ix < 2; ix++) {
                        const int xx = ix == 0 ? gx : gxa;
                        if (xx == NONE || (ix == 0 && iy == 0)) continue;
                        S* oi = a.g_out + ((long long)(I.row0 + yy) * NQ) * pitch + GC + xx;
                        for (int q = QOFF; q < 9; q++) oi[(q - QOFF) * pitch] = to_s<S>(v[q]);
                    }
                }
            }
        });
        // the stage takes the tile after next once every thread is done with it (the next iteration's
        // wait is a barrier too, so without a tile to issue nothing needs to wait here)
        const int t2 = t + 2 * stride;
        if (t2 < a.total_tiles) {
            __syncthreads();
            if (tid == 0) issue(t2, s);
        }
    }

    // the last CTA of a batch's last launch advances the step counter read by the next launch.  No
    // fence: the counter orders no other data, every CTA read the time before its increment, and the next
    // launch reads it only after this grid has completed (kernel boundary or the dependency wait).
    if (a.t_adv && tid == 0) {
        unsigned int prev = atomicAdd(&a.ctl->done, 1u);
        if (prev == gridDim.x - 1) {
            a.ctl->done = 0u;
            a.ctl->time = (a.need_time ? n - a.t_off : a.ctl->time) + a.t_adv;
        }
    }
}

// ------------------------------------------------------------------------------------------ init
// g_i(x, 0) = g_i^eq(phi0, mu(phi0), u(x, 0)); phi(0) = phi0 (hi + lo on the float path); the ghost
// images are written too.  phi0 arrives in the padded layout with its ghost frame filled; the
// velocity tables are the double ones, indexed like the step kernel's.
template <typename C, typename S, typename P>
__global__ void init_kernel(const InstDev* inst, int n_inst, const double* tabs, const double* phi0, int pitch,
                            S* g, P* phi, float* lo, long long nodes_total, const long long* node_begin)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nodes_total) return;
    int lo_i = 0, hi_i = n_inst - 1;
    while (lo_i < hi_i) {
        int mid = (lo_i + hi_i + 1) >> 1;
        if (node_begin[mid] <= k) lo_i = mid; else hi_i = mid - 1;
    }
    const InstDev& I = inst[lo_i];
    const int NQ = (sizeof(S) == 2) ? 8 : 9, QOFF = (sizeof(S) == 2) ? 1 : 0;
    long long loc = k - node_begin[lo_i];
    int y = (int)(loc / I.nx), x = (int)(loc - (long long)y * I.nx);
    auto at = [&](int dx, int dy) -> double {
        int xx = wrap(x + dx, I.nx);
        int yy = I.slab ? y + dy : (I.walls ? mirror(y + dy, I.ny) : wrap(y + dy, I.ny));
        return phi0[(long long)(I.row0 + yy) * pitch + GC + xx];
    };
    double c0 = at(0, 0);
    double ax = at(1, 0) + at(-1, 0) + at(0, 1) + at(0, -1);
    double dg = at(1, 1) + at(-1, 1) + at(1, -1) + at(-1, -1);
    double lap = (2.0 / 3.0) * (ax - 4.0 * c0) + (1.0 / 6.0) * (dg - 4.0 * c0);
    C mu = (C)(dfdphi<double>(c0, I.cd.beta, I.cd.phiA, I.cd.phiB) - I.cd.kappa * lap);
    const double* tX1 = tabs + I.tab;
    const double* tX2 = tX1 + pitch;
    const double* tY1 = tX2 + pitch;
    const double* tY2 = tY1 + I.ylen;
    double T = vel_t(I.vel, I.Tper, 0);
    C ux = (C)(tX1[x + GC] * tY1[y + GR] * T), uy = (C)(tX2[x + GC] * tY2[y + GR] * T);
    C ph = (C)c0, eta = (C)I.cd.eta;
    C uu = ux * ux + uy * uy;
    C v[9];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        if (q == 0) {
            // the float paths store g_0 - phi
            v[q] = (sizeof(C) == 4 ? C(0) : ph) + (wq<C>(0) - C(1)) * eta * mu - wq<C>(0) * C(1.5) * ph * uu;
        } else {
            C cu = (C)cx(q) * ux + (C)cy(q) * uy;
            v[q] = wq<C>(q) * eta * mu + wq<C>(q) * ph * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
        }
    }
    const P hi = (P)c0;
    if (lo) lo[(long long)(I.row0 + y) * pitch + GC + x] = (float)(c0 - (double)hi);
    const int NONE = -0x40000000;
    const int xa = x < 3 ? x + I.nx : NONE, xb = x >= I.nx - 3 ? x - I.nx : NONE;
    // a slab's ghost rows are the neighbouring slabs' rows, imported before its first step
    const int ya = y < 3 && !I.slab ? (I.walls ? -1 - y : y + I.ny) : NONE;
    const int yb = y >= I.ny - 3 && !I.slab ? (I.walls ? 2 * I.ny - 1 - y : y - I.ny) : NONE;
    for (int iy = 0; iy < 3; iy++) {
        const int yy = iy == 0 ? y : (iy == 1 ? ya : yb);
        if (yy == NONE) continue;
        for (int ix = 0; ix < 3; ix++) {
            const int xx = ix == 0 ? x : (ix == 1 ? xa : xb);
            if (xx == NONE) continue;
            long long row = I.row0 + yy;
            phi[row * pitch + GC + xx] = hi;
            S* o = g + (row * NQ) * pitch + GC + xx;
            for (int q = QOFF; q < 9; q++) o[(q - QOFF) * pitch] = to_s<S>(v[q]);
        }
    }
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
__global__ void __launch_bounds__(RED_NT) reduce_partials_kernel(const InstDev* inst, const P* phi, const float* lo,
                                                                 const double* phi0, int pitch,
                                                                 double* partials, int chunks)
{
    __shared__ double sh[RED_NT / 32][RED_NV];
    const InstDev& I = inst[blockIdx.y];
    const long long N = (long long)I.nx * I.ny;
    double v[RED_NV] = {0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    for (long long k = (long long)blockIdx.x * RED_NT + threadIdx.x; k < N; k += (long long)chunks * RED_NT) {
        int y = (int)(k / I.nx), x = (int)(k - (long long)y * I.nx);
        long long gi = (long long)(I.row0 + y) * pitch + GC + x;
        double p = (double)phi[gi] + (lo ? (double)lo[gi] : 0.0), p0 = phi0[gi];
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

static __global__ void __launch_bounds__(RED_NT) reduce_final_kernel(const double* partials, int chunks, double* result)
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
