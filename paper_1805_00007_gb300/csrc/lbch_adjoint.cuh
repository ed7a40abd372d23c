// lbch_adjoint.cuh -- reverse-mode adjoint of the step kernel (one instance, periodic domain).
//
// For a loss L of phi(T), lambda_q(x) = dL/dg_q(x).  One forward step (Eq. LB with Eqs. geq, liangFi,
// mu, t0-phiu, mark3) is
//   phi = sum_q g_q;  mu = f'(phi) - kappa lap phi;  F = -(phi^2/rho) grad mu [+ K grad div(phi u)];
//   post_q = (1 - 1/tau) g_q + g_eq_q(phi, mu, u)/tau + (1 - 1/(2 tau)) S_q(F);  g'_q(x + c_q) = post_q(x).
// Its Jacobian depends on the populations only through phi, so the backward sweep needs the forward phi
// of each step (a tape) and nothing else.  The transpose of every linear map is applied explicitly:
// streaming becomes a gather from x + c_q, the gradient stencil G becomes (G^T v)(x) = sum_k w_k c_k
// v(x - c_k)/c_s^2, the Laplacian L becomes (L^T v)(x) = sum_k 2 w_k (v(x - c_k) - v(x))/c_s^2.  The velocity
// is u = s u_ref and dL/ds (at s = 1) is accumulated in double.
//
// Layout: plain arrays over the instance, node index y*nx + x; lambda is [9][N].  The adjoint is carried
// in double for every storage precision (at tau = 1 all nine lambda_q are equal and dL/du is formed from
// differences of neighbouring lambda, which float storage would round away); the tape keeps the
// forward phi in the precision of the forward path, so the gradient is that of the path actually run.
// Four one-thread-per-node kernels per adjoint step (forward mu; local adjoints; mu_bar and D_bar; phi_bar
// and the new lambda), and one deterministic sum of dL/ds at the end of the sweep.
//
// CF: the type the forward quantities are formed in (mu, its gradient, the velocity, rho and the force's
// coefficient, f''(phi)) -- float for a float tape, as the float forward step formed them, double for a double
// tape.  Everything that carries lambda is double in either case.
//
// ONE (tau_g = 1): lambda_q = (1 - 1/tau) lambda'_q(x + c_q) + phi_bar(x) is phi_bar(x) for every q, since
// 1 - 1/tau is exactly 0, so lambda is kept as one plane instead of nine.  The kernels read that plane where
// they would read plane q and write it once; the values are those of the nine-plane form bit for bit (for
// finite lambda, 0 * lambda' + phi_bar is phi_bar).

#pragma once
#include "lbch_kernels.cuh"

namespace lbch {
namespace adj {

struct AdjArgs {
    int nx, ny, model;
    int pitch;                 // of the velocity tables' X part
    int ylen;                  // length of each Y table
    long long n;               // forward step index of this adjoint step
};

__device__ __forceinline__ int wp(int i, int n) { return i >= n ? i - n : (i < 0 ? i + n : i); }

// the prescribed velocity at node (x, y) from the velocity tables of type CF (the forward step's), as the
// forward step forms it: X Y T, two rounded products
template <typename CF>
__device__ __forceinline__ void vel_at(const InstDev& I, const CF* tabs, const AdjArgs& a, int x, int y, CF T, CF& ux,
                                       CF& uy)
{
    const CF* tX1 = tabs + I.tab;
    const CF* tX2 = tX1 + a.pitch;
    const CF* tY1 = tX2 + a.pitch;
    const CF* tY2 = tY1 + a.ylen;
    ux = node_u(tX1[x + GC], tY1[y + GR], T);
    uy = node_u(tX2[x + GC], tY2[y + GR], T);
}

template <typename C> __device__ __forceinline__ C d2f(C phi, C beta, C phiA, C phiB)
{
    // f''(phi) of f = beta (phi - phiA)^2 (phi - phiB)^2 (Eq. bulk)
    return C(2) * beta * ((phi - phiB) * (C(2) * phi - phiA - phiB) + (phi - phiA) * (C(2) * phi - phiA - phiB)
                          + C(2) * (phi - phiA) * (phi - phiB));
}

// The contractions sum_q l_q d g_eq_q / d(phi, mu, u) at one node (Eq. geq), for the adjoint l of the
// equilibria.  g_eq_q is quadratic in c_q . u, so they depend on l only through l_0 and its moments
// m0 = sum_q w_q l_q, m1 = sum_q w_q l_q c_q and m2 = sum_q w_q l_q c_q c_q, formed from the sums and
// differences of opposite directions.  m1 is returned too (the source term S_q is linear in c_q).
template <typename C>
__device__ __forceinline__ void geq_contract(const C* l, C phi, C ux, C uy, C eta, C& pl, C& ml, C& bx, C& by,
                                             C& m1x, C& m1y)
{
    // opposite pairs (1, 3) c = (1, 0); (2, 4) c = (0, 1); (5, 7) c = (1, 1); (6, 8) c = (-1, 1)
    const C E1 = l[1] + l[3], O1 = l[1] - l[3], E2 = l[2] + l[4], O2 = l[2] - l[4];
    const C E5 = l[5] + l[7], O5 = l[5] - l[7], E6 = l[6] + l[8], O6 = l[6] - l[8];
    const C wa = wq<C>(1), wd = wq<C>(5);
    const C Ed = wd * (E5 + E6);
    const C m2xx = wa * E1 + Ed, m2yy = wa * E2 + Ed, m2xy = wd * (E5 - E6);
    const C m0 = wq<C>(0) * l[0] + (wa * (E1 + E2) + Ed);
    m1x = wa * O1 + wd * (O5 - O6);
    m1y = wa * O2 + wd * (O5 + O6);
    const C vx = ux * m2xx + uy * m2xy, vy = ux * m2xy + uy * m2yy;  // sum_q w_q l_q (c_q . u) c_q
    const C uu = ux * ux + uy * uy;
    // d g_eq_0/d phi = 1 - (3/2) w_0 u^2;  d g_eq_q/d phi = w_q (3 c_q.u + (9/2)(c_q.u)^2 - (3/2) u^2)
    pl = l[0] + C(3) * (ux * m1x + uy * m1y) + C(4.5) * (ux * vx + uy * vy) - C(1.5) * uu * m0;
    // d g_eq_0/d mu = (w_0 - 1) eta;  d g_eq_q/d mu = w_q eta
    ml = eta * (m0 - l[0]);
    // d g_eq_q/d u = w_q phi (3 c_q + 9 (c_q.u) c_q - 3 u), q = 0 included
    bx = phi * (C(3) * m1x + C(9) * vx - C(3) * ux * m0);
    by = phi * (C(3) * m1y + C(9) * vy - C(3) * uy * m0);
}

// The isotropic stencils on the periodic lattice, grouped by axis and diagonal neighbours:
// (G v)(x) = sum_k w_k c_k v(x + c_k)/c_s^2 and (L v)(x) = sum_k 2 w_k (v(x + c_k) - v(x))/c_s^2.  Their
// transposes follow by substituting c_k -> -c_k: G^T = -G and L^T = L.
template <typename C, typename V>
__device__ __forceinline__ C at_nb(const V* v, int nx, int ny, int x, int y, int dx, int dy)
{
    return (C)v[(long long)wp(y + dy, ny) * nx + wp(x + dx, nx)];
}
template <typename C, typename V>
__device__ __forceinline__ C grad_c(const V* v, int nx, int ny, int x, int y, int comp)
{
    auto at = [&](int dx, int dy) { return at_nb<C>(v, nx, ny, x, y, dx, dy); };
    if (comp == 0)
        return C(1) / C(3) * (at(1, 0) - at(-1, 0)) + C(1) / C(12) * ((at(1, 1) - at(-1, 1)) + (at(1, -1) - at(-1, -1)));
    return C(1) / C(3) * (at(0, 1) - at(0, -1)) + C(1) / C(12) * ((at(1, 1) + at(-1, 1)) - (at(1, -1) + at(-1, -1)));
}
template <typename C, typename V>
__device__ __forceinline__ C lap_c(const V* v, int nx, int ny, int x, int y)
{
    auto at = [&](int dx, int dy) { return at_nb<C>(v, nx, ny, x, y, dx, dy); };
    const C c = at(0, 0);
    const C ax = (at(1, 0) + at(-1, 0)) + (at(0, 1) + at(0, -1));
    const C dg = (at(1, 1) + at(-1, 1)) + (at(1, -1) + at(-1, -1));
    return C(2) / C(3) * (ax - C(4) * c) + C(1) / C(6) * (dg - C(4) * c);
}
// (G^T v)(x), component comp
template <typename C>
__device__ __forceinline__ C gradT(const C* v, int nx, int ny, int x, int y, int comp)
{
    return -grad_c<C>(v, nx, ny, x, y, comp);
}
// (L^T v)(x)
template <typename C>
__device__ __forceinline__ C lapT(const C* v, int nx, int ny, int x, int y)
{
    return lap_c<C>(v, nx, ny, x, y);
}

// forward mu = f'(phi) - kappa lap phi at step n (phi from the tape, of type TP), in the forward type CF
template <typename CF, typename TP>
__global__ void fwd_mu_kernel(const InstDev* inst, AdjArgs a, const TP* phi, CF* mu)
{
    const InstDev& I = inst[0];
    const Consts<CF>& K0 = consts<CF>(I);
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)a.nx * a.ny) return;
    int y = (int)k / a.nx, x = (int)k - y * a.nx;  // fewer than 2^31 nodes (lb_ch_adjoint_begin checks)
    mu[k] = dfdphi((CF)phi[k], K0.beta, K0.phiA, K0.phiB) - K0.kappa * lap_c<CF>(phi, a.nx, a.ny, x, y);
}

// local adjoints of collision, g_eq, S and F1 (lambda itself is written by transpose2_kernel)
template <typename C, typename CF, typename TP, bool ONE>
__global__ void local_kernel(const InstDev* inst, const CF* tabs, AdjArgs a, CF T, const TP* phi, const CF* mu,
                             const C* lam_next, C* lam, C* gmb, C* Fb, C* phib, C* mub, C* ub)
{
    const InstDev& I = inst[0];
    const Consts<C>& K0 = consts<C>(I);
    const Consts<CF>& KF = consts<CF>(I);
    const long long N = (long long)a.nx * a.ny;
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    int y = (int)k / a.nx, x = (int)k - y * a.nx;  // fewer than 2^31 nodes (lb_ch_adjoint_begin checks)
    // the forward quantities at the node, in CF
    const CF phf = (CF)phi[k];
    CF uxf, uyf;
    vel_at(I, tabs, a, x, y, T, uxf, uyf);
    const CF gxf = grad_c<CF>(mu, a.nx, a.ny, x, y, 0), gyf = grad_c<CF>(mu, a.nx, a.ny, x, y, 1);  // grad mu
    const CF rhof = KF.a * phf + KF.b, rf = rcp<CF>(rhof);
    const CF coeff = phf * phf * rf;                                    // F1 = -coef grad mu
    const CF dcoeff = phf * (KF.a * phf + CF(2) * KF.b) * (rf * rf);   // d coef / d phi
    const C ph = (C)phf, ux = (C)uxf, uy = (C)uyf, gx = (C)gxf, gy = (C)gyf, coef = (C)coeff, dcoef = (C)dcoeff;
    C pb[9];
#pragma unroll
    for (int q = 0; q < 9; q++) {
        // reverse streaming: post_q(x) was sent to x + c_q
        pb[q] = lam_next[(ONE ? 0 : q * N) + (long long)wp(y + cy(q), a.ny) * a.nx + wp(x + cx(q), a.nx)];
    }
    // post_q takes g_eq_q / tau and (1 - 1/(2 tau)) S_q, S_q = w_q c_q . F / c_s^2
    C pl, ml, bx, by, m1x, m1y;
    geq_contract(pb, ph, ux, uy, K0.eta, pl, ml, bx, by, m1x, m1y);
    pl *= K0.itau;
    ml *= K0.itau;
    bx *= K0.itau;
    by *= K0.itau;
    const C fbx = C(3) * K0.src * m1x, fby = C(3) * K0.src * m1y;
    gmb[k] = -coef * fbx;
    gmb[N + k] = -coef * fby;
    Fb[k] = fbx;
    Fb[N + k] = fby;
    phib[k] = pl - dcoef * (fbx * gx + fby * gy);
    mub[k] = ml;
    ub[k] = bx;
    ub[N + k] = by;
}

// mu_bar += G^T grad_mu_bar;  D_bar = 3 c_s^2 K G^T F_bar
template <typename C>
__global__ void transpose1_kernel(const InstDev* inst, AdjArgs a, const C* gmb, const C* Fb, C* mub, C* Db)
{
    const InstDev& I = inst[0];
    const Consts<C>& K0 = consts<C>(I);
    const long long N = (long long)a.nx * a.ny;
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    int y = (int)k / a.nx, x = (int)k - y * a.nx;  // fewer than 2^31 nodes (lb_ch_adjoint_begin checks)
    mub[k] += gradT(gmb, a.nx, a.ny, x, y, 0) + gradT(gmb + N, a.nx, a.ny, x, y, 1);
    Db[k] = (a.model == 2) ? K0.K * (gradT(Fb, a.nx, a.ny, x, y, 0) + gradT(Fb + N, a.nx, a.ny, x, y, 1)) : C(0);
}

// phi_bar = local + f''(phi) mu_bar - kappa L^T mu_bar + u . G^T D_bar;
// lambda_q(x) = (1 - 1/tau) lambda_next_q(x + c_q) + phi_bar(x); dL/ds per node
template <typename C, typename CF, typename TP, bool ONE>
__global__ void transpose2_kernel(const InstDev* inst, const CF* tabs, AdjArgs a, CF T, const TP* phi,
                                  const C* phib, const C* mub, const C* Db, const C* ub, const C* lam_next, C* lam,
                                  double* ds)
{
    const InstDev& I = inst[0];
    const Consts<C>& K0 = consts<C>(I);
    const Consts<CF>& KF = consts<CF>(I);
    const long long N = (long long)a.nx * a.ny;
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    int y = (int)k / a.nx, x = (int)k - y * a.nx;  // fewer than 2^31 nodes (lb_ch_adjoint_begin checks)
    // the forward quantities at the node, in CF
    const CF phf = (CF)phi[k];
    CF uxf, uyf;
    vel_at(I, tabs, a, x, y, T, uxf, uyf);
    const C ph = (C)phf, ux = (C)uxf, uy = (C)uyf;
    const C f2 = (C)d2f(phf, KF.beta, KF.phiA, KF.phiB);
    C pb = phib[k] + f2 * mub[k] - K0.kappa * lapT(mub, a.nx, a.ny, x, y);
    C bx = ub[k], by = ub[N + k];
    if (a.model == 2) {
        C jbx = gradT(Db, a.nx, a.ny, x, y, 0), jby = gradT(Db, a.nx, a.ny, x, y, 1);
        pb += ux * jbx + uy * jby;
        bx += ph * jbx;
        by += ph * jby;
    }
    // u = s u_ref: du/ds = u.  Accumulated per node over the adjoint steps and summed once at the end.
    ds[k] += (double)bx * (double)ux + (double)by * (double)uy;
    if constexpr (ONE) {
        lam[k] = pb;  // (1 - 1/tau) = 0: the reverse streaming and collision leave phi_bar alone
    } else {
#pragma unroll
        for (int q = 0; q < 9; q++)  // reverse streaming and collision, plus phi = sum_q g_q
            lam[q * N + k] = K0.omt * lam_next[q * N + (long long)wp(y + cy(q), a.ny) * a.nx + wp(x + cx(q), a.nx)] + pb;
    }
}

// adjoint of the initial equilibria: dL/dphi0 (two kernels: local, then the mu transpose)
template <typename C, bool ONE>
__global__ void init_local_kernel(const InstDev* inst, const double* tabs, AdjArgs a, double T, const double* phi0,
                                  int pitch0, const C* lam, C* mub, C* dphi0, double* ds)
{
    const InstDev& I = inst[0];
    const Consts<C>& K0 = consts<C>(I);
    const long long N = (long long)a.nx * a.ny;
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    int y = (int)k / a.nx, x = (int)k - y * a.nx;  // fewer than 2^31 nodes (lb_ch_adjoint_begin checks)
    C ph = (C)phi0[(long long)(I.row0 + y) * pitch0 + GC + x];
    C ux, uy;
    vel_at<C>(I, tabs, a, x, y, (C)T, ux, uy);
    C l[9];
#pragma unroll
    for (int q = 0; q < 9; q++) l[q] = lam[(ONE ? 0 : q * N) + k];
    C pl, ml, bx, by, m1x, m1y;
    geq_contract(l, ph, ux, uy, K0.eta, pl, ml, bx, by, m1x, m1y);
    dphi0[k] = pl;
    mub[k] = ml;
    ds[k] += (double)bx * (double)ux + (double)by * (double)uy;
}

template <typename C>
__global__ void init_transpose_kernel(const InstDev* inst, AdjArgs a, const double* phi0, int pitch0, const C* mub,
                                      C* dphi0)
{
    const InstDev& I = inst[0];
    const Consts<C>& K0 = consts<C>(I);
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)a.nx * a.ny) return;
    int y = (int)k / a.nx, x = (int)k - y * a.nx;  // fewer than 2^31 nodes (lb_ch_adjoint_begin checks)
    C ph = (C)phi0[(long long)(I.row0 + y) * pitch0 + GC + x];
    dphi0[k] += d2f(ph, K0.beta, K0.phiA, K0.phiB) * mub[k] - K0.kappa * lapT(mub, a.nx, a.ny, x, y);
}

// deterministic sum of ds[0..N) into *acc (one block, fixed order), executed once, at the end of the adjoint
// sweep (ds holds each node's contributions from every step)
__global__ void __launch_bounds__(256) sum_into_kernel(const double* ds, long long N, double* acc)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (long long k = threadIdx.x; k < N; k += 256) s += ds[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += sh[0];
}

// phi of the instance (padded storage, plus the low part on the float path) into a plain array
template <typename P, typename C>
__global__ void tape_kernel(const InstDev* inst, int pitch, const P* phi, const float* lo, C* out)
{
    const InstDev& I = inst[0];
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)I.nx * I.ny) return;
    int y = (int)k / I.nx, x = (int)k - y * I.nx;  // fewer than 2^31 nodes (lb_ch_tape_phi checks)
    long long gi = (long long)(I.row0 + y) * pitch + GC + x;
    out[k] = (C)((double)phi[gi] + (lo ? (double)lo[gi] : 0.0));
}

// lambda_T: dL/dg_q = dL/dphi(T) for every q (nq planes: 9, or 1 with ONE)
template <typename C>
__global__ void adj_begin_kernel(long long N, int nq, const C* dphiT, C* lam)
{
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    C v = dphiT[k];
    for (int q = 0; q < nq; q++) lam[q * N + k] = v;
}

}  // namespace adj
}  // namespace lbch
