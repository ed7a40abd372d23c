// lbch_ns.cuh -- the coupled Cahn-Hilliard / Navier-Stokes step (flows that are not prescribed).
//
// For the Rayleigh-Taylor problem (Sec. III.E) the velocity is not prescribed but solved by a second
// D2Q9 lattice Boltzmann equation for Eq. NS.  The paper calls that equation standard without writing
// it out; the library takes the incompressible, pressure-based single-relaxation-time form with forcing:
//   f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq)/tau_f + (1 - 1/(2 tau_f)) G_i,   tau_f = nu/c_s^2 + 1/2,
//   f_0^eq = (w_0 - 1) p/c_s^2 + rho s_0(u),  f_i^eq = w_i p/c_s^2 + rho s_i(u),
//   s_i(u) = w_i [c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u^2/(2 c_s^2)],  Gamma_i = w_i + s_i(u),
//   G_i = (c_i - u) . [Gamma_i F + s_i(u) c_s^2 grad rho] / c_s^2,
//   rho u = sum_i c_i f_i + F/2,   p = c_s^2/(1 - w_0) [sum_{i>0} f_i + (1/2) u.grad rho + rho s_0(u)],
// with rho = a phi + b (Eq. rho) and F = -phi grad mu - (rho - (rhoA + rhoB)/2) g + (d rho/d phi) M lap(mu) u
// (Eq. NS, form c).  The Cahn-Hilliard lattice uses this u and F1 = (phi/rho)(-phi grad mu - grad p)
// (Eq. t0-phiu) plus the Eq. mark3 term.  Walls: halfway bounce-back for both lattices at rest; stencil
// operands at ghost rows take the mirror values.
//
// One step is two kernels on 32 x 8 tiles of nodes, with the stencil operands staged in shared memory: one
// node per thread in the fields kernel, two in the collision kernel.  fields_kernel sums phi = sum_q g_q on tile + 2 (storing it for the tile's nodes),
// forms mu on tile + 1 and gives mu, u and p at the tile's nodes.  collide_kernel stages phi (and phi u)
// on tile + 2 and mu and p on tile + 1, forms D = div(phi u) on tile + 1 for Model II (kept there rather
// than stored), collides both lattices and pushes them to the neighbours (bounce-back at walls).  phi of
// the state a step leaves is therefore formed by the next step's fields kernel; phi_kernel forms it on
// demand before an observation.  A stencil operand
// at a ghost row beyond a wall takes the value of the mirror node: a staged operand is read at that node,
// and a derived one is formed at the mirror row of the tile's region.
#pragma once
#include "lbch_kernels.cuh"

namespace lbch {
namespace ns {

template <typename C>
struct NsConsts {
    C tauf, gx, gy, M, rbar;
    C itauf, omtf, srcf;  // 1/tau_f, 1 - 1/tau_f and 1 - 1/(2 tau_f), formed once on the host
};

template <typename C>
struct NsArgs {
    int nx, ny, walls, model, pitch, row0;
    Consts<C> k;      // the Cahn-Hilliard constants
    NsConsts<C> n;    // the flow's constants
    C* f_in; C* f_out; C* g_in; C* g_out;   // [9][N]
    C* phi_in; C* phi_out;                  // padded phi of the handle
    C *ux, *uy, *pr, *mu;                   // [N], written by fields_kernel
};

// tiles and the regions staged around them; the collision kernel takes two nodes per thread (rows ty and
// ty + TY/2), so that each thread has two independent chains of loads, arithmetic and stores to overlap
// (measured: 16.3 against 17.7 us per step for the 256 x 1024 Rayleigh-Taylor grid, FP32; two nodes per
// thread in the fields kernel as well gained nothing)
constexpr int TX = 32, TY = 8, NT = TX * TY, NTC = NT / 2;
constexpr int W2 = TX + 4, H2 = TY + 4, N2 = W2 * H2;  // tile + 2
constexpr int W1 = TX + 2, H1 = TY + 2, N1 = W1 * H1;  // tile + 1

__host__ __device__ inline int tiles_of(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }

__device__ __forceinline__ int wrap_any(int v, int n)
{
    if (v < 0 || v >= n) {
        v %= n;
        if (v < 0) v += n;
    }
    return v;
}

// The node whose value a stencil operand at coordinate (x, y) takes: periodic in x; periodic in y or
// mirrored at walls.  (Coordinates more than one row beyond a wall occur only in the region of a ragged
// tile, where no node reads them; they are clamped into the domain.)
__device__ __forceinline__ int2 node_at(int nx, int ny, int walls, int x, int y)
{
    x = wrap_any(x, nx);
    if (walls) {
        y = y < 0 ? -1 - y : (y >= ny ? 2 * ny - 1 - y : y);
        y = min(max(y, 0), ny - 1);
    } else {
        y = wrap_any(y, ny);
    }
    return make_int2(x, y);
}

// The row of region tile + 1 (origin row y0 - 1) at which a derived field is formed for its row j: j
// itself, or the mirror row of a ghost row beyond a wall.
__device__ __forceinline__ int r1_row(int walls, int ny, int y0, int j)
{
    if (!walls) return j;
    const int y = y0 - 1 + j;
    const int m = (y < 0 ? -1 - y : (y >= ny ? 2 * ny - 1 - y : y)) - (y0 - 1);
    return (m >= 0 && m < H1) ? m : j;
}

// phi at node (x, y) in the handle's padded array
template <typename C> __device__ __forceinline__ C phi_xy(const NsArgs<C>& a, int x, int y)
{
    return a.phi_in[(long long)(a.row0 + y) * a.pitch + GC + x];
}

// The isotropic stencils on a staged region of row width W around flat index c (x to the east, y to the
// north): grad psi = sum_k w_k c_k psi(x + c_k) / c_s^2 and lap psi = sum_k 2 w_k (psi(x + c_k) - psi) / c_s^2.
template <typename C, int W> __device__ __forceinline__ C sgx(const C* s, int c)
{
    return op_fma(C(1) / C(3), s[c + 1] - s[c - 1],
                  op_mul(C(1) / C(12), (s[c + W + 1] - s[c + W - 1]) + (s[c - W + 1] - s[c - W - 1])));
}
template <typename C, int W> __device__ __forceinline__ C sgy(const C* s, int c)
{
    return op_fma(C(1) / C(3), s[c + W] - s[c - W],
                  op_mul(C(1) / C(12), (s[c + W + 1] + s[c + W - 1]) - (s[c - W + 1] + s[c - W - 1])));
}
template <typename C, int W> __device__ __forceinline__ C slap(const C* s, int c)
{
    const C ce = s[c];
    const C ax = (s[c + 1] + s[c - 1]) + (s[c + W] + s[c - W]);
    const C dg = (s[c + W + 1] + s[c + W - 1]) + (s[c - W + 1] + s[c - W - 1]);
    return op_fma(C(2) / C(3), op_fma(C(-4), ce, ax), op_mul(C(1) / C(6), op_fma(C(-4), ce, dg)));
}

// The tile of this block: origin (x0, y0)
__device__ __forceinline__ void tile_origin(int nx, int& x0, int& y0)
{
    const int tiles_x = (nx + TX - 1) / TX;
    x0 = ((int)blockIdx.x % tiles_x) * TX;
    y0 = ((int)blockIdx.x / tiles_x) * TY;
}

// phi = sum_q g_q (Eq. macroscopicg) at node k of the [q][node] populations g, summed in the order of q
template <typename C> __device__ __forceinline__ C sum_g(const C* g, long long N, long long k)
{
    C s = C(0);
#pragma unroll
    for (int q = 0; q < 9; q++) s += g[q * N + k];
    return s;
}

// phi on tile + 2 into s2 (and, with jx, the components of phi u there).  FROM_G: phi is summed from the
// populations of the current state instead of read from the phi array (the fields kernel, which then
// stores it for the tile's own nodes).
template <typename C, bool FROM_G = false, int NTH = NT>
__device__ __forceinline__ void stage_phi(const NsArgs<C>& a, int x0, int y0, C* s2, C* jx, C* jy)
{
    for (int e = threadIdx.x; e < N2; e += NTH) {
        const int j = e / W2, i = e - j * W2;
        const int2 v = node_at(a.nx, a.ny, a.walls, x0 - 2 + i, y0 - 2 + j);
        const C ph = FROM_G ? sum_g(a.g_in, (long long)a.nx * a.ny, (long long)v.y * a.nx + v.x) : phi_xy(a, v.x, v.y);
        s2[e] = ph;
        if (jx) {
            const int k = v.y * a.nx + v.x;
            jx[e] = ph * a.ux[k];
            jy[e] = ph * a.uy[k];
        }
    }
}

// mu (Eq. mu) on tile + 1 from phi on tile + 2
template <typename C, int NTH = NT>
__device__ __forceinline__ void form_mu(const NsArgs<C>& a, int y0, const C* s2, C* mu1)
{
    for (int e = threadIdx.x; e < N1; e += NTH) {
        const int j = e / W1, i = e - j * W1;
        const int c = (r1_row(a.walls, a.ny, y0, j) + 1) * W2 + i + 1;
        mu1[e] = op_fma(-a.k.kappa, slap<C, W2>(s2, c), node_dfdphi(s2[c], a.k.beta, a.k.phiA, a.k.phiB));
    }
}

// phi = sum_q g_q of the current state, then mu and the flow's velocity and pressure at every node; phi is
// stored into the current state's phi array for the collision kernel that follows and for observation (so a
// step is two kernels: the sum of the populations streamed by the previous step is formed here, where its
// neighbourhood is staged anyway)
template <typename C>
__global__ void __launch_bounds__(NT) fields_kernel(NsArgs<C> a)
{
    __shared__ C s2[N2], mu1[N1];
    int x0, y0;
    tile_origin(a.nx, x0, y0);
    stage_phi<C, true>(a, x0, y0, s2, nullptr, nullptr);
    __syncthreads();
    form_mu(a, y0, s2, mu1);
    __syncthreads();
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX, x = x0 + tx, y = y0 + ty;
    if (x >= a.nx || y >= a.ny) return;
    const int c1 = (ty + 1) * W1 + tx + 1, c2 = (ty + 2) * W2 + tx + 2;
    a.phi_in[(long long)(a.row0 + y) * a.pitch + GC + x] = s2[c2];
    const long long N = (long long)a.nx * a.ny;  // plane size of the [q][node] arrays
    const int k = y * a.nx + x;
    const C gmx = sgx<C, W1>(mu1, c1), gmy = sgy<C, W1>(mu1, c1), lap = slap<C, W1>(mu1, c1);
    const C phi = s2[c2], rho = op_fma(a.k.a, phi, a.k.b);
    const C grx = op_mul(a.k.a, sgx<C, W2>(s2, c2)), gry = op_mul(a.k.a, sgy<C, W2>(s2, c2));  // grad rho
    const C db = rho - a.n.rbar;
    const C F0x = -op_fma(phi, gmx, op_mul(db, a.n.gx)), F0y = -op_fma(phi, gmy, op_mul(db, a.n.gy));
    C f[9];
#pragma unroll
    for (int q = 0; q < 9; q++) f[q] = a.f_in[q * N + k];
    const C mx = ((f[1] - f[3]) + (f[5] - f[7])) + (f[8] - f[6]);
    const C my = ((f[2] - f[4]) + (f[5] - f[7])) + (f[6] - f[8]);
    const C s1 = ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8]));
    // rho u = m + F/2 with F = F0 + a M lap(mu) u, solved for u
    const C r = rcp<C>(op_fma(C(-0.5) * a.k.a, op_mul(a.n.M, lap), rho));
    const C ux = op_mul(op_fma(C(0.5), F0x, mx), r), uy = op_mul(op_fma(C(0.5), F0y, my), r);
    const C uu = op_fma(ux, ux, op_mul(uy, uy));
    // p = c_s^2/(1 - w_0) [sum_{q>0} f_q + u.grad rho / 2 + rho s_0(u)],  s_0 = -(3/2) w_0 u^2
    const C t = op_fma(C(0.5), op_fma(ux, grx, op_mul(uy, gry)), s1);
    a.ux[k] = ux;
    a.uy[k] = uy;
    a.mu[k] = mu1[c1];
    a.pr[k] = op_mul(C(3) / C(5), op_fma(-C(1.5) * wq<C>(0), op_mul(rho, uu), t));
}

// both lattices: collide at x, push to x + c_q (bounce-back at walls)
template <typename C>
__global__ void __launch_bounds__(NTC, sizeof(C) == 4 ? 8 : 6) collide_kernel(NsArgs<C> a)
{
    __shared__ C s2[N2], jx2[N2], jy2[N2], mu1[N1], p1[N1], D1[N1];
    int x0, y0;
    tile_origin(a.nx, x0, y0);
    const bool model2 = a.model == 2;
    stage_phi<C, false, NTC>(a, x0, y0, s2, model2 ? jx2 : nullptr, jy2);
    for (int e = threadIdx.x; e < N1; e += NTC) {  // p on tile + 1
        const int j = e / W1, i = e - j * W1;
        const int2 v = node_at(a.nx, a.ny, a.walls, x0 - 1 + i, y0 - 1 + j);
        p1[e] = a.pr[v.y * a.nx + v.x];
        mu1[e] = a.mu[v.y * a.nx + v.x];
    }
    __syncthreads();
    if (model2) {  // D = div(phi u) on tile + 1
        for (int e = threadIdx.x; e < N1; e += NTC) {
            const int j = e / W1, i = e - j * W1;
            const int c = (r1_row(a.walls, a.ny, y0, j) + 1) * W2 + i + 1;
            D1[e] = sgx<C, W2>(jx2, c) + sgy<C, W2>(jy2, c);
        }
    }
    __syncthreads();
    // the populations are read from the current state and written to the other one: the two never overlap,
    // so the second node's loads may be issued ahead of the first node's stores
    const C* __restrict__ f_in = a.f_in;
    const C* __restrict__ g_in = a.g_in;
    C* __restrict__ f_out = a.f_out;
    C* __restrict__ g_out = a.g_out;
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int tx = threadIdx.x % TX, ty = threadIdx.x / TX + r * (TY / 2), x = x0 + tx, y = y0 + ty;
        if (x >= a.nx || y >= a.ny) continue;
        const int c1 = (ty + 1) * W1 + tx + 1, c2 = (ty + 2) * W2 + tx + 2;
        const long long N = (long long)a.nx * a.ny;  // plane size of the [q][node] arrays
        const int k = y * a.nx + x;

        // the node's fields
        const C phi = s2[c2], mu = mu1[c1], pr = p1[c1], ux = a.ux[k], uy = a.uy[k];
        const C rho = op_fma(a.k.a, phi, a.k.b);
        const C gmx = sgx<C, W1>(mu1, c1), gmy = sgy<C, W1>(mu1, c1), lap = slap<C, W1>(mu1, c1);
        const C gpx = sgx<C, W1>(p1, c1), gpy = sgy<C, W1>(p1, c1);
        const C gr3x = op_mul(a.k.a * (C(1) / C(3)), sgx<C, W2>(s2, c2));  // c_s^2 grad rho
        const C gr3y = op_mul(a.k.a * (C(1) / C(3)), sgy<C, W2>(s2, c2));
        // Cahn-Hilliard force with the flow's pressure (Eq. t0-phiu), plus Eq. mark3 for Model II
        const C por = op_mul(phi, rcp<C>(rho));
        C Fx = op_mul(por, -op_fma(phi, gmx, gpx)), Fy = op_mul(por, -op_fma(phi, gmy, gpy));
        if (model2) {
            Fx = op_fma(a.k.K, sgx<C, W1>(D1, c1), Fx);
            Fy = op_fma(a.k.K, sgy<C, W1>(D1, c1), Fy);
        }
        // the flow's force F = -phi grad mu - (rho - rbar) g + a M lap(mu) u
        const C db = rho - a.n.rbar, aml = op_mul(a.k.a, op_mul(a.n.M, lap));
        const C FFx = op_fma(aml, ux, -op_fma(phi, gmx, op_mul(db, a.n.gx)));
        const C FFy = op_fma(aml, uy, -op_fma(phi, gmy, op_mul(db, a.n.gy)));

        // The collision (Eq. LB for g with Eq. geq and the source of Eq. liangFi; the flow's lattice with
        // f_eq and G as above) in pairs of opposite directions: with cu = c.u, s_q = e + o and
        // s_opp = e - o, e = w (9/2 cu^2 - 3/2 u^2), o = 3 w cu; and G = 3 (c - u).(A + o B) for q and
        // 3 (-c - u).(A - o B) for opp, A = (w + e) F + e c_s^2 grad rho, B = F + c_s^2 grad rho.
        const C itau = a.k.itau, omt = a.k.omt, itauf = a.n.itauf, omtf = a.n.omtf;
        const C src3 = C(3) * a.k.src, srcf3 = C(3) * a.n.srcf;
        const C uu = op_fma(ux, ux, op_mul(uy, uy));
        const C P1 = op_mul(itau, phi), Pf = op_mul(itauf, rho);
        const C ietamu = op_mul(itau, op_mul(a.k.eta, mu)), itfp3 = op_mul(C(3) * itauf, pr);
        const C Bx = FFx + gr3x, By = FFy + gr3y;
        const C uB = op_fma(ux, Bx, op_mul(uy, By));
        const C uF = op_fma(ux, FFx, op_mul(uy, FFy)), ug = op_fma(ux, gr3x, op_mul(uy, gr3y));

        C pg[9], pf[9];
        {   // q = 0: s_0 = -(3/2) w_0 u^2, S_0 = 0, G_0 = -3 (Gamma_0 u.F + s_0 u.c_s^2 grad rho)
            const C s0 = op_mul(C(-1.5) * wq<C>(0), uu);
            const C geq = op_fma(phi, s0, op_fma(wq<C>(0) - C(1), op_mul(a.k.eta, mu), phi));
            pg[0] = op_fma(omt, g_in[k], op_mul(itau, geq));
            const C feq = op_fma(rho, s0, op_mul(C(3) * (wq<C>(0) - C(1)), pr));
            const C G = op_mul(C(-3), op_fma(wq<C>(0) + s0, uF, op_mul(s0, ug)));
            pf[0] = op_fma(omtf, f_in[k], op_fma(itauf, feq, op_mul(a.n.srcf, G)));
        }
    #pragma unroll
        for (int m = 0; m < 4; m++) {
            // pairs (q, opp q): (1, 3) c = (1, 0); (2, 4) c = (0, 1); (5, 7) c = (1, 1); (6, 8) c = (-1, 1)
            const int q = (m == 0) ? 1 : (m == 1) ? 2 : (m == 2) ? 5 : 6, o_ = opp(q);
            const C w = wq<C>(q);
            const C cu = (m == 0) ? ux : (m == 1) ? uy : (m == 2) ? ux + uy : uy - ux;
            const C cF = (m == 0) ? Fx : (m == 1) ? Fy : (m == 2) ? Fx + Fy : Fy - Fx;
            const C cB = (m == 0) ? Bx : (m == 1) ? By : (m == 2) ? Bx + By : By - Bx;
            const C e = op_fma(op_mul(C(4.5) * w, cu), cu, op_mul(C(-1.5) * w, uu));
            const C o = op_mul(C(3) * w, cu);
            // Cahn-Hilliard lattice: post = (1 - 1/tau) g + g_eq/tau + (1 - 1/(2 tau)) S
            const C Ge = op_fma(P1, e, op_mul(w, ietamu));
            const C Go = op_fma(P1, o, op_mul(w * src3, cF));
            pg[q] = op_fma(omt, g_in[q * N + k], Ge + Go);
            pg[o_] = op_fma(omt, g_in[o_ * N + k], Ge - Go);
            // the flow's lattice
            const C we = w + e;
            const C Ax = op_fma(we, FFx, op_mul(e, gr3x)), Ay = op_fma(we, FFy, op_mul(e, gr3y));
            const C cA = (m == 0) ? Ax : (m == 1) ? Ay : (m == 2) ? Ax + Ay : Ay - Ax;
            const C uA = op_fma(ux, Ax, op_mul(uy, Ay));
            const C Fe = op_fma(srcf3, op_fma(o, cB, -uA), op_fma(Pf, e, op_mul(w, itfp3)));
            const C Fo = op_fma(Pf, o, op_mul(srcf3, op_fma(-o, uB, cA)));
            pf[q] = op_fma(omtf, f_in[q * N + k], Fe + Fo);
            pf[o_] = op_fma(omtf, f_in[o_ * N + k], Fe - Fo);
        }
    #pragma unroll
        for (int q = 0; q < 9; q++) {
            const int yy = y + cy(q);
            if (a.walls && (yy < 0 || yy >= a.ny)) {
                g_out[opp(q) * N + k] = pg[q];  // halfway bounce-back at a wall at rest
                f_out[opp(q) * N + k] = pf[q];
            } else {
                int xx = x + cx(q);
                xx = xx < 0 ? xx + a.nx : (xx >= a.nx ? xx - a.nx : xx);
                const int y2 = yy < 0 ? yy + a.ny : (yy >= a.ny ? yy - a.ny : yy);
                const int j = y2 * a.nx + xx;
                g_out[q * N + j] = pg[q];
                f_out[q * N + j] = pf[q];
            }
        }
    }
}

// phi = sum_q g_q of the current state into its padded phi array (before an observation); one thread per node
template <typename C>
__global__ void phi_kernel(NsArgs<C> a)
{
    const long long N = (long long)a.nx * a.ny;  // plane size of the [q][node] arrays
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int y = k / a.nx, x = k - y * a.nx;
    a.phi_in[(long long)(a.row0 + y) * a.pitch + GC + x] = sum_g(a.g_in, N, k);
}

// initial state: g = g_eq(phi0, mu0, 0), f = f_eq(0, rho(phi0), 0) = 0; phi = phi0
template <typename C>
__global__ void init_kernel(NsArgs<C> a, const double* phi0)
{
    const long long N = (long long)a.nx * a.ny;  // plane size of the [q][node] arrays
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int y = k / a.nx, x = k - y * a.nx;
    auto at = [&](int dx, int dy) -> double {
        const int2 v = node_at(a.nx, a.ny, a.walls, x + dx, y + dy);
        return phi0[(long long)(a.row0 + v.y) * a.pitch + GC + v.x];
    };
    double c0 = at(0, 0), s = 0.0;
    for (int q = 1; q < 9; q++) s += 2.0 * wq<double>(q) * (at(cx(q), cy(q)) - c0);
    double mu = dfdphi<double>(c0, (double)a.k.beta, (double)a.k.phiA, (double)a.k.phiB) - (double)a.k.kappa * 3.0 * s;
    for (int q = 0; q < 9; q++) {
        double geq = (q == 0) ? c0 + (wq<double>(0) - 1.0) * (double)a.k.eta * mu : wq<double>(q) * (double)a.k.eta * mu;
        a.g_out[q * N + k] = (C)geq;
        a.f_out[q * N + k] = C(0);
    }
    a.phi_out[(long long)(a.row0 + y) * a.pitch + GC + x] = (C)c0;
}

}  // namespace ns
}  // namespace lbch
