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
// One step is five one-thread-per-node kernels over plain [q][node] population arrays: mu from phi;
// the flow's moments (u, p) and forces; D = div(phi u); the coupled collide-and-push-stream of both
// lattices; phi(t+1) = sum_q g_q into the handle's padded phi array (which observations read).
#pragma once
#include "lbch_kernels.cuh"

namespace lbch {
namespace ns {

template <typename C>
struct NsConsts {
    C tauf, gx, gy, M, rbar;
    C itauf, srcf;  // 1/tau_f and 1 - 1/(2 tau_f), formed once on the host (no divisions in the kernels)
};

template <typename C>
struct NsArgs {
    int nx, ny, walls, model, pitch, row0;
    Consts<C> k;      // the Cahn-Hilliard constants
    NsConsts<C> n;    // the flow's constants
    C* f_in; C* f_out; C* g_in; C* g_out;   // [9][N]
    C* phi_in; C* phi_out;                  // padded phi of the handle
    C *mu, *ux, *uy, *pr, *Fx, *Fy, *grx, *gry, *gmx, *gmy, *D;  // [N]
};

// The coordinates of neighbour (x + dx, y + dy): periodic in x; periodic in y or mirrored at walls.
__device__ __forceinline__ int2 nbxy(int nx, int ny, int walls, int x, int y, int dx, int dy)
{
    int xx = x + dx, yy = y + dy;
    xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
    if (walls) yy = yy < 0 ? -1 - yy : (yy >= ny ? 2 * ny - 1 - yy : yy);
    else yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
    return make_int2(xx, yy);
}
// its index in the [node] arrays
__device__ __forceinline__ int nb(int nx, int ny, int walls, int x, int y, int dx, int dy)
{
    const int2 v = nbxy(nx, ny, walls, x, y, dx, dy);
    return v.y * nx + v.x;
}

// phi at node (x, y) in the handle's padded array
template <typename C> __device__ __forceinline__ C phi_xy(const NsArgs<C>& a, int x, int y)
{
    return a.phi_in[(long long)(a.row0 + y) * a.pitch + GC + x];
}
template <typename C> __device__ __forceinline__ C phi_nb(const NsArgs<C>& a, int x, int y, int dx, int dy)
{
    const int2 v = nbxy(a.nx, a.ny, a.walls, x, y, dx, dy);
    return phi_xy(a, v.x, v.y);
}

// The node of this thread: index k, coordinates (x, y) (a coupled handle has fewer than 2^31 nodes, which
// lb_ch_init checks; the coordinates take one 32-bit division).
__device__ __forceinline__ bool node_of(int nx, int ny, int& k, int& x, int& y)
{
    k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx * ny) return false;
    y = k / nx;
    x = k - y * nx;
    return true;
}

template <typename C>
__global__ void mu_kernel(NsArgs<C> a)
{
    int k, x, y;
    if (!node_of(a.nx, a.ny, k, x, y)) return;
    C c = phi_xy(a, x, y), s = C(0);
#pragma unroll
    for (int q = 1; q < 9; q++) s += C(2) * wq<C>(q) * (phi_nb(a, x, y, cx(q), cy(q)) - c);
    a.mu[k] = dfdphi(c, a.k.beta, a.k.phiA, a.k.phiB) - a.k.kappa * C(3) * s;
}

// the flow's moments and forces at every node
template <typename C>
__global__ void fields_kernel(NsArgs<C> a)
{
    const long long N = (long long)a.nx * a.ny;  // plane size of the [q][node] arrays
    int k, x, y;
    if (!node_of(a.nx, a.ny, k, x, y)) return;
    C gmx = C(0), gmy = C(0), gpx = C(0), gpy = C(0), lap = C(0);
    C m0 = a.mu[k];
#pragma unroll
    for (int q = 1; q < 9; q++) {
        const int2 v = nbxy(a.nx, a.ny, a.walls, x, y, cx(q), cy(q));
        C m = a.mu[v.y * a.nx + v.x], ph = phi_xy(a, v.x, v.y);
        // (unrolled: terms with a zero lattice component are left out, not multiplied by zero)
        if (cx(q) != 0) {
            gmx += wq<C>(q) * (C)cx(q) * m;
            gpx += wq<C>(q) * (C)cx(q) * ph;
        }
        if (cy(q) != 0) {
            gmy += wq<C>(q) * (C)cy(q) * m;
            gpy += wq<C>(q) * (C)cy(q) * ph;
        }
        lap += C(2) * wq<C>(q) * (m - m0);
    }
    gmx *= C(3); gmy *= C(3); lap *= C(3);
    C phi = phi_xy(a, x, y), rho = a.k.a * phi + a.k.b;
    C grx = a.k.a * C(3) * gpx, gry = a.k.a * C(3) * gpy;   // grad rho = a grad phi
    C F0x = -phi * gmx - (rho - a.n.rbar) * a.n.gx;
    C F0y = -phi * gmy - (rho - a.n.rbar) * a.n.gy;
    C mx = C(0), my = C(0), s1 = C(0);
#pragma unroll
    for (int q = 0; q < 9; q++) {
        C fq = a.f_in[q * N + k];
        if (cx(q) != 0) mx += (C)cx(q) * fq;
        if (cy(q) != 0) my += (C)cy(q) * fq;
        if (q > 0) s1 += fq;
    }
    C den = rho - C(0.5) * a.k.a * a.n.M * lap;   // rho u = m + F/2 with F = F0 + a M lap(mu) u
    C ux = (mx + C(0.5) * F0x) / den, uy = (my + C(0.5) * F0y) / den;
    C uu = ux * ux + uy * uy;
    C s0 = -wq<C>(0) * C(1.5) * uu;
    a.ux[k] = ux; a.uy[k] = uy;
    a.Fx[k] = F0x + a.k.a * a.n.M * lap * ux;
    a.Fy[k] = F0y + a.k.a * a.n.M * lap * uy;
    a.pr[k] = (C(1) / C(3)) / (C(1) - wq<C>(0)) * (s1 + C(0.5) * (ux * grx + uy * gry) + rho * s0);
    a.grx[k] = grx; a.gry[k] = gry; a.gmx[k] = gmx; a.gmy[k] = gmy;
}

// D = div(phi u) (Model II)
template <typename C>
__global__ void div_kernel(NsArgs<C> a)
{
    int k, x, y;
    if (!node_of(a.nx, a.ny, k, x, y)) return;
    C s = C(0);
#pragma unroll
    for (int q = 1; q < 9; q++) {
        const int2 v = nbxy(a.nx, a.ny, a.walls, x, y, cx(q), cy(q));
        const int j = v.y * a.nx + v.x;
        C ph = phi_xy(a, v.x, v.y);
        const C t = cx(q) == 0 ? (C)cy(q) * ph * a.uy[j]
                  : (cy(q) == 0 ? (C)cx(q) * ph * a.ux[j] : (C)cx(q) * ph * a.ux[j] + (C)cy(q) * ph * a.uy[j]);
        s += wq<C>(q) * t;
    }
    a.D[k] = C(3) * s;
}

// both lattices: collide at x, push to x + c_q (bounce-back at walls)
template <typename C>
__global__ void collide_kernel(NsArgs<C> a)
{
    const long long N = (long long)a.nx * a.ny;  // plane size of the [q][node] arrays
    int k, x, y;
    if (!node_of(a.nx, a.ny, k, x, y)) return;
    C gpx = C(0), gpy = C(0), gdx = C(0), gdy = C(0);
#pragma unroll
    for (int q = 1; q < 9; q++) {
        const int j = nb(a.nx, a.ny, a.walls, x, y, cx(q), cy(q));
        if (cx(q) != 0) gpx += wq<C>(q) * (C)cx(q) * a.pr[j];
        if (cy(q) != 0) gpy += wq<C>(q) * (C)cy(q) * a.pr[j];
        if (a.model == 2) {
            if (cx(q) != 0) gdx += wq<C>(q) * (C)cx(q) * a.D[j];
            if (cy(q) != 0) gdy += wq<C>(q) * (C)cy(q) * a.D[j];
        }
    }
    gpx *= C(3); gpy *= C(3); gdx *= C(3); gdy *= C(3);
    C phi = phi_xy(a, x, y), rho = a.k.a * phi + a.k.b;
    C ux = a.ux[k], uy = a.uy[k], mu = a.mu[k];
    // Cahn-Hilliard force with the flow's pressure (Eq. t0-phiu) and Eq. mark3
    C Fx = phi / rho * (-phi * a.gmx[k] - gpx) + a.k.K * gdx;
    C Fy = phi / rho * (-phi * a.gmy[k] - gpy) + a.k.K * gdy;
    C FFx = a.Fx[k], FFy = a.Fy[k], pr = a.pr[k];
    const C grx3 = a.grx[k] / C(3), gry3 = a.gry[k] / C(3);  // c_s^2 grad rho
    C uu = ux * ux + uy * uy;
    const C itauf = a.n.itauf, srcf = a.n.srcf;
#pragma unroll
    for (int q = 0; q < 9; q++) {
        const C cu = cx(q) == 0 ? (C)cy(q) * uy : (cy(q) == 0 ? (C)cx(q) * ux : (C)cx(q) * ux + (C)cy(q) * uy);
        C s = wq<C>(q) * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
        // Cahn-Hilliard lattice: Eq. geq, Eq. liangFi, Eq. LB
        C geq = (q == 0) ? phi + (wq<C>(0) - C(1)) * a.k.eta * mu - wq<C>(0) * C(1.5) * phi * uu
                         : wq<C>(q) * a.k.eta * mu + phi * s;
        const C cF = cx(q) == 0 ? (C)cy(q) * Fy : (cy(q) == 0 ? (C)cx(q) * Fx : (C)cx(q) * Fx + (C)cy(q) * Fy);
        C Sq = C(3) * wq<C>(q) * cF;
        C gq = a.g_in[q * N + k];
        C pg = gq - (gq - geq) * a.k.itau + a.k.src * Sq;
        // flow lattice
        C feq = (q == 0 ? (wq<C>(0) - C(1)) : wq<C>(q)) * C(3) * pr + rho * s;
        C Gam = wq<C>(q) + s;
        C G = C(3) * (((C)cx(q) - ux) * (Gam * FFx + s * grx3) + ((C)cy(q) - uy) * (Gam * FFy + s * gry3));
        C fq = a.f_in[q * N + k];
        C pf = fq - (fq - feq) * itauf + srcf * G;
        int yy = y + cy(q);
        if (a.walls && (yy < 0 || yy >= a.ny)) {
            a.g_out[opp(q) * N + k] = pg;  // halfway bounce-back at a wall at rest
            a.f_out[opp(q) * N + k] = pf;
        } else {
            const int j = nb(a.nx, a.ny, 0, x, y, cx(q), cy(q));
            a.g_out[q * N + j] = pg;
            a.f_out[q * N + j] = pf;
        }
    }
}

// phi(t+1) = sum_q g_q into the padded phi array
template <typename C>
__global__ void phi_kernel(NsArgs<C> a)
{
    const long long N = (long long)a.nx * a.ny;  // plane size of the [q][node] arrays
    int k, x, y;
    if (!node_of(a.nx, a.ny, k, x, y)) return;
    C s = C(0);
#pragma unroll
    for (int q = 0; q < 9; q++) s += a.g_out[q * N + k];
    a.phi_out[(long long)(a.row0 + y) * a.pitch + GC + x] = s;
}

// initial state: g = g_eq(phi0, mu0, 0), f = f_eq(0, rho(phi0), 0) = 0; phi = phi0
template <typename C>
__global__ void init_kernel(NsArgs<C> a, const double* phi0)
{
    const long long N = (long long)a.nx * a.ny;  // plane size of the [q][node] arrays
    int k, x, y;
    if (!node_of(a.nx, a.ny, k, x, y)) return;
    auto at = [&](int dx, int dy) -> double {
        const int2 v = nbxy(a.nx, a.ny, a.walls, x, y, dx, dy);
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
