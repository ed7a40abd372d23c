/*
 * lbch_oracle.c -- plain, slow FP64 CPU oracle of the D2Q9 single-relaxation-time lattice Boltzmann
 * model for the Cahn-Hilliard equation with the high-order source term of Zhang, Guo & Liang,
 * "A high-order lattice Boltzmann model for the Cahn-Hilliard equation" (arXiv:1805.00007).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is compared against.  It shares no
 * code, header, table or helper with the product library; only tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It is written for a reader who checks it against the
 * paper by eye: one loop per field, in the order the paper introduces the quantities, double precision
 * throughout, no blocking, no fusion.  Build with -O2 -fno-fast-math -ffp-contract=off.  The optional
 * OpenMP pragmas parallelise loops whose iterations are independent, so results do not depend on the
 * thread count.
 *
 * Lattice units: dx = dt = c = 1, so c_s^2 = 1/3 and 3 c_s^2 = 1.  Node (i, j) sits at x = i, y = j and is
 * stored at index j*nx + i.  Distributions are stored structure-of-arrays: g[q*N + node], N = nx*ny.
 *
 * Where the paper is silent the oracle takes these readings (each is restated where it is used):
 *   R1  no pressure field for prescribed velocities: grad p = 0, so F1 = -(phi^2/rho) grad mu   (Eq. t0-phiu)
 *   R2  initial distributions are the equilibria of phi0, mu0 = mu(phi0), u(t=0)                 (Eq. geq)
 *   R3  Model II uses the diffusive-scale force of Eq. mark3 with the general K(tau), for any tau
 *   R4  the isotropic central stencils are the D2Q9-weighted forms (Sec. III cites them only)
 *   R5  grad(div(phi u)) is the gradient stencil applied to the divergence stencil (5x5 footprint)
 *   R6  the step n -> n+1 uses u(x, t = n)
 *   R7  walls (when enabled) sit half-way below row 0 and above row ny-1: halfway bounce-back of the
 *       distributions with the moving-wall term 2 w_i phi (c_i . u_w)/c_s^2, and every stencil operand
 *       (phi, mu, phi*u, div(phi u)) takes at a ghost row the value of that operand at the mirror row
 *   R8  the order of a step is phi -> mu -> grad mu -> u -> F -> g_eq, S -> collide -> stream
 *   R15 Model III (model = 3) is Model II with the complete diffusive-scale force of Eq. F2-1: the time
 *       derivatives on the convective scale are replaced by the whole time derivative (as Remarks I and
 *       II allow), taken as the backward difference over one step; at the first step (no previous step)
 *       they are zero
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

/* D2Q9 velocity set (Sec. II.B): c0=(0,0), c1=-c3=(1,0), c2=-c4=(0,1), c5=-c7=(1,1), c6=-c8=(-1,1). */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Weights w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36 (Sec. II.B, after Eq. geq). */
static const double WQ[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* Index of the opposite direction -c_i. */
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0;

enum { VEL_UNIFORM = 0, VEL_ROTATION = 1, VEL_VORTEX = 2, VEL_SHEAR = 3, VEL_REV_SHEAR = 4, VEL_DEFORM = 5,
       VEL_COUPLED = 6 };

/* Problem parameters, in the paper's notation.  Plain numbers; the derived constants are computed here. */
typedef struct {
    int nx, ny;
    int walls;          /* 0: periodic in x and y; 1: periodic in x, walls at y = -1/2 and y = ny - 1/2 */
    int model;          /* 1: Model I (F = F1); 2: Model II (F = F1 + F2 of Eq. mark3); 3: F2 of Eq. F2-1 */
    int vel;            /* velocity field, VEL_* */
    int nvort;          /* vortex count n of the deformation field (Eq. deformation) */
    double phiA, phiB;  /* bulk values of the order parameter */
    double sigma, W;    /* surface tension and interface width (Eq. betakappa) */
    double M;           /* mobility; when <= 0 it is derived from Pe (Sec. III.A) */
    double Pe, Ustar;   /* Peclet number and characteristic velocity, used when M <= 0 */
    double tau;         /* tau_g */
    double rhoA, rhoB;  /* bulk densities (Eq. rho) */
    double U0, ux0, uy0;/* velocity amplitude; uniform velocity components */
    double xc, yc, half;/* rotation centre and half-length of the rotation field */
    double Tper;        /* period / reversal time of the time-dependent fields, in steps */
    double shear;       /* shear rate of the wall-driven shear flow */
    double nu;          /* kinematic viscosity of the coupled flow (VEL_COUPLED) */
    double gx, gy;      /* gravity of the coupled flow; buoyancy force -(rho - (rhoA + rhoB)/2) g */
} ora_params;

/* Constants the model derives from the parameters. */
typedef struct {
    double beta, kappa;  /* Eq. betakappa */
    double M, eta;       /* mobility M = c_s^2 eta (tau - 1/2), after Eq. phit3 */
    double a, b;         /* rho = a phi + b, Eq. rho */
    double K;            /* K = (tau - 1/6 - tau^2)/(tau - 1/2), after Eq. F2-1 */
} ora_consts;

/* ---------------------------------------------------------------- parameters */

void ora_derive(const ora_params* p, ora_consts* c)
{
    double dphi = fabs(p->phiA - p->phiB);
    /* Eq. betakappa */
    c->beta = 12.0 * p->sigma / (p->W * dphi * dphi * dphi * dphi);
    c->kappa = 3.0 * p->sigma * p->W / (2.0 * dphi * dphi);
    /* Pe = U* W / (M beta (phiA - phiB)^2), Sec. III.A, solved for M when M is not given */
    if (p->M > 0.0)
        c->M = p->M;
    else
        c->M = p->Ustar * p->W / (p->Pe * c->beta * (p->phiA - p->phiB) * (p->phiA - p->phiB));
    /* M = c_s^2 eta (tau_g - 0.5), stated after Eq. phit3 */
    c->eta = c->M / (CS2 * (p->tau - 0.5));
    /* Eq. rho */
    c->a = (p->rhoA - p->rhoB) / (p->phiA - p->phiB);
    c->b = (p->rhoB * p->phiA - p->phiB * p->rhoA) / (p->phiA - p->phiB);
    /* K of Eq. F2-1 */
    c->K = (p->tau - 1.0 / 6.0 - p->tau * p->tau) / (p->tau - 0.5);
}

/* ---------------------------------------------------------------- prescribed velocity */

/* u(x, y, t) of the benchmark flows, evaluated at a point (x, y) and time step n (reading R6). */
void ora_velocity(const ora_params* p, double x, double y, long n, double* ux, double* uy)
{
    const double pi = 3.14159265358979323846;
    double L = (double)p->nx;
    switch (p->vel) {
    case VEL_UNIFORM: /* diagonal translation, u = (U0, U0) in Sec. III.A; here any constant vector */
        *ux = p->ux0;
        *uy = p->uy0;
        break;
    case VEL_ROTATION: /* solid-body rotation of Zalesak's disk (Sec. III.B) about (xc, yc) */
        *ux = -p->U0 * pi * (y - p->yc) / p->half;
        *uy = p->U0 * pi * (x - p->xc) / p->half;
        break;
    case VEL_VORTEX: { /* single vortex, reversed by cos(pi t / T) */
        double Ly = (double)p->ny;
        double sx = sin(pi * x / L), sy = sin(pi * y / Ly);
        double ct = cos(pi * (double)n / p->Tper);
        *ux = -p->U0 * sx * sx * sin(2.0 * pi * y / Ly) * ct;
        *uy = p->U0 * sin(2.0 * pi * x / L) * sy * sy * ct;
        break;
    }
    case VEL_SHEAR: /* wall-driven shear, zero at mid-channel; walls at y = -1/2 and ny - 1/2 */
        *ux = p->shear * (y - 0.5 * (double)(p->ny - 1));
        *uy = 0.0;
        break;
    case VEL_REV_SHEAR: { /* Eq. shear; the field changes sign at t = T (Sec. III.C) */
        double s = ((double)n < p->Tper) ? 1.0 : -1.0;
        *ux = -s * p->U0 * pi * cos(pi * (x / L - 0.5)) * sin(pi * (y / L - 0.5));
        *uy = s * p->U0 * pi * sin(pi * (x / L - 0.5)) * cos(pi * (y / L - 0.5));
        break;
    }
    case VEL_DEFORM: { /* Eq. deformation with n vortices and period T0 = Tper */
        double k = (double)p->nvort * pi;
        double ct = cos(pi * (double)n / p->Tper);
        *ux = -p->U0 * sin(k * (x / L + 0.5)) * sin(k * (y / L + 0.5)) * ct;
        *uy = -p->U0 * cos(k * (x / L + 0.5)) * cos(k * (y / L + 0.5)) * ct;
        break;
    }
    default:
        *ux = 0.0;
        *uy = 0.0;
    }
}

/* ---------------------------------------------------------------- single-node pieces */

/* Equilibrium distribution, Eq. geq. */
void ora_geq(double phi, double mu, double ux, double uy, double eta, double* geq)
{
    double uu = ux * ux + uy * uy;
    geq[0] = phi + (WQ[0] - 1.0) * eta * mu - WQ[0] * phi * uu / (2.0 * CS2);
    for (int i = 1; i < Q; i++) {
        double cu = CX[i] * ux + CY[i] * uy;
        geq[i] = WQ[i] * eta * mu
               + WQ[i] * phi * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Source distribution S_i = w_i c_i . F / c_s^2, Eq. liangFi. */
void ora_source(double Fx, double Fy, double* S)
{
    for (int i = 0; i < Q; i++)
        S[i] = WQ[i] * (CX[i] * Fx + CY[i] * Fy) / CS2;
}

/* Bulk part of the chemical potential, d f / d phi for f = beta (phi - phiA)^2 (phi - phiB)^2 (Eq. bulk). */
double ora_dfdphi(double phi, double beta, double phiA, double phiB)
{
    return 2.0 * beta * (phi - phiA) * (phi - phiB) * (phi - phiB)
         + 2.0 * beta * (phi - phiA) * (phi - phiA) * (phi - phiB);
}

/* ---------------------------------------------------------------- stencils */

/* Neighbour index of node (i, j) in direction (dx, dy): periodic in x; periodic or mirrored in y (R7). */
static long nbr(int nx, int ny, int walls, int i, int j, int dx, int dy)
{
    int ii = i + dx, jj = j + dy;
    ii = ((ii % nx) + nx) % nx;
    if (walls) {
        if (jj < 0) jj = -1 - jj;
        if (jj >= ny) jj = 2 * ny - 1 - jj;
    } else {
        jj = ((jj % ny) + ny) % ny;
    }
    return (long)jj * nx + ii;
}

/* Isotropic central gradient (R4): grad psi(x) = sum_k w_k c_k psi(x + c_k) / c_s^2. */
void ora_grad(int nx, int ny, int walls, const double* psi, double* gx, double* gy)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double sx = 0.0, sy = 0.0;
            for (int k = 1; k < Q; k++) {
                double v = psi[nbr(nx, ny, walls, i, j, CX[k], CY[k])];
                sx += WQ[k] * CX[k] * v;
                sy += WQ[k] * CY[k] * v;
            }
            gx[(long)j * nx + i] = sx / CS2;
            gy[(long)j * nx + i] = sy / CS2;
        }
}

/* Isotropic central Laplacian (R4): lap psi(x) = sum_k 2 w_k (psi(x + c_k) - psi(x)) / c_s^2. */
void ora_lap(int nx, int ny, int walls, const double* psi, double* lap)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double c = psi[(long)j * nx + i];
            double s = 0.0;
            for (int k = 1; k < Q; k++)
                s += 2.0 * WQ[k] * (psi[nbr(nx, ny, walls, i, j, CX[k], CY[k])] - c);
            lap[(long)j * nx + i] = s / CS2;
        }
}

/* Divergence of a vector field with the isotropic gradient stencil. */
void ora_div(int nx, int ny, int walls, const double* vx, const double* vy, double* div)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double s = 0.0;
            for (int k = 1; k < Q; k++) {
                long m = nbr(nx, ny, walls, i, j, CX[k], CY[k]);
                s += WQ[k] * (CX[k] * vx[m] + CY[k] * vy[m]);
            }
            div[(long)j * nx + i] = s / CS2;
        }
}

/* ---------------------------------------------------------------- macroscopic fields */

/* phi = sum_i g_i, Eq. macroscopicg. */
void ora_phi(int nx, int ny, const double* g, double* phi)
{
    long N = (long)nx * ny;
    for (long n = 0; n < N; n++) {
        double s = 0.0;
        for (int i = 0; i < Q; i++) s += g[i * N + n];
        phi[n] = s;
    }
}

/* Chemical potential mu = df/dphi - kappa lap phi, Eq. mu. */
void ora_mu(const ora_params* p, const ora_consts* c, const double* phi, double* mu)
{
    long N = (long)p->nx * p->ny;
    double* lap = (double*)malloc(sizeof(double) * N);
    ora_lap(p->nx, p->ny, p->walls, phi, lap);
    for (long n = 0; n < N; n++)
        mu[n] = ora_dfdphi(phi[n], c->beta, p->phiA, p->phiB) - c->kappa * lap[n];
    free(lap);
}

/* Velocity field at every node at step n. */
void ora_velocity_field(const ora_params* p, long n, double* ux, double* uy)
{
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++)
            ora_velocity(p, (double)i, (double)j, n, &ux[(long)j * p->nx + i], &uy[(long)j * p->nx + i]);
}

/* The force F of Eq. reFi at every node, as the paper runs it (Remark III):
 *   F1 = (phi/rho)(Fs - grad p), Fs = -phi grad mu, grad p = 0 for prescribed flows (R1)  -- Eq. t0-phiu
 *   F2 = 3 c_s^2 K grad(div(phi u))                                                   -- Eq. mark3 (R3, R5)
 * Model I keeps F1 only; Model II adds F2. */
void ora_force(const ora_params* p, const ora_consts* c, const double* phi, const double* mu,
               const double* ux, const double* uy, double* Fx, double* Fy)
{
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double* gmx = (double*)malloc(sizeof(double) * N);
    double* gmy = (double*)malloc(sizeof(double) * N);
    ora_grad(nx, ny, p->walls, mu, gmx, gmy);
    for (long n = 0; n < N; n++) {
        double rho = c->a * phi[n] + c->b;           /* Eq. rho */
        double Fsx = -phi[n] * gmx[n], Fsy = -phi[n] * gmy[n];  /* surface tension force after Eq. NS */
        Fx[n] = phi[n] / rho * Fsx;
        Fy[n] = phi[n] / rho * Fsy;
    }
    if (p->model == 2) {
        double* jx = (double*)malloc(sizeof(double) * N);
        double* jy = (double*)malloc(sizeof(double) * N);
        double* D = (double*)malloc(sizeof(double) * N);
        double* gDx = (double*)malloc(sizeof(double) * N);
        double* gDy = (double*)malloc(sizeof(double) * N);
        for (long n = 0; n < N; n++) {
            jx[n] = phi[n] * ux[n];
            jy[n] = phi[n] * uy[n];
        }
        ora_div(nx, ny, p->walls, jx, jy, D);
        ora_grad(nx, ny, p->walls, D, gDx, gDy);
        for (long n = 0; n < N; n++) {
            Fx[n] += 3.0 * CS2 * c->K * gDx[n];
            Fy[n] += 3.0 * CS2 * c->K * gDy[n];
        }
        free(jx); free(jy); free(D); free(gDx); free(gDy);
    }
    free(gmx);
    free(gmy);
}

/* ---------------------------------------------------------------- initial state and one step */

/* Initial distributions g_i(x, 0) = g_i^eq(phi0, mu0, u(x, 0)) (reading R2). */
void ora_init(const ora_params* p, const double* phi0, double* g)
{
    ora_consts c;
    ora_derive(p, &c);
    long N = (long)p->nx * p->ny;
    double* mu = (double*)malloc(sizeof(double) * N);
    ora_mu(p, &c, phi0, mu);
    for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) {
            long n = (long)j * p->nx + i;
            double ux, uy, geq[Q];
            ora_velocity(p, (double)i, (double)j, 0, &ux, &uy);
            ora_geq(phi0[n], mu[n], ux, uy, c.eta, geq);
            for (int q = 0; q < Q; q++) g[q * N + n] = geq[q];
        }
    free(mu);
}

/* One step n -> n+1 of Eq. LB: g_i(x + c_i, t + 1) = g_i - (g_i - g_i^eq)/tau + (1 - 1/(2 tau)) S_i.
 * gin and gout are distinct arrays of 9*N values. */
void ora_step(const ora_params* p, const double* gin, double* gout, long n)
{
    ora_consts c;
    ora_derive(p, &c);
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double* phi = (double*)malloc(sizeof(double) * N);
    double* mu = (double*)malloc(sizeof(double) * N);
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* Fx = (double*)malloc(sizeof(double) * N);
    double* Fy = (double*)malloc(sizeof(double) * N);

    ora_phi(nx, ny, gin, phi);                 /* Eq. macroscopicg */
    ora_mu(p, &c, phi, mu);                    /* Eq. mu */
    ora_velocity_field(p, n, ux, uy);          /* prescribed u at t = n (R6) */
    ora_force(p, &c, phi, mu, ux, uy, Fx, Fy); /* Eqs. t0-phiu, mark3 */

#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long x = (long)j * nx + i;
            double geq[Q], S[Q];
            ora_geq(phi[x], mu[x], ux[x], uy[x], c.eta, geq);  /* Eq. geq */
            ora_source(Fx[x], Fy[x], S);                       /* Eq. liangFi */
            for (int q = 0; q < Q; q++) {
                /* collision, Eq. LB right-hand side */
                double post = gin[q * N + x] - (gin[q * N + x] - geq[q]) / p->tau
                            + (1.0 - 1.0 / (2.0 * p->tau)) * S[q];
                /* streaming to x + c_q */
                int ii = ((i + CX[q]) % nx + nx) % nx;
                int jj = j + CY[q];
                if (!p->walls) {
                    jj = ((jj % ny) + ny) % ny;
                } else if (jj < 0 || jj >= ny) {
                    /* halfway bounce-back from the wall with its velocity u_w (R7): the population that
                     * leaves along c_q returns along c_opp with 2 w_opp phi (c_opp . u_w)/c_s^2 added */
                    double uwx, uwy;
                    ora_velocity(p, (double)i, jj < 0 ? -0.5 : (double)ny - 0.5, n, &uwx, &uwy);
                    int o = OPP[q];
                    gout[o * N + x] = post + 2.0 * WQ[o] * phi[x] * (CX[o] * uwx + CY[o] * uwy) / CS2;
                    continue;
                }
                gout[q * N + (long)jj * nx + ii] = post;
            }
        }
    free(phi); free(mu); free(ux); free(uy); free(Fx); free(Fy);
}

/* nsteps steps starting at step index n0; g holds the state on entry and on return. */
/* Threads of the parallel loops from now on (n > 0; 1 gives the single-threaded oracle); returns the count
 * in effect.  Results do not depend on it: every parallel loop writes disjoint nodes. */
int ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int ora_run(const ora_params* p, double* g, long n0, long nsteps)
{
    long N = (long)p->nx * p->ny;
    double* tmp = (double*)malloc(sizeof(double) * Q * N);
    if (!tmp) return -1;
    for (long s = 0; s < nsteps; s++) {
        ora_step(p, g, tmp, n0 + s);
        memcpy(g, tmp, sizeof(double) * Q * N);
    }
    free(tmp);
    return 0;
}

/* ---------------------------------------------------------------- Model III: the complete F2 of Eq. F2-1 */

/* F = F1 + F2 with the complete diffusive-scale force of Eq. F2-1 (reading R15):
 *   F2 = (2 tau - 1 + 3K) d_t F1 + 3 c_s^2 eta K d_t grad mu + 3 c_s^2 K grad(div(phi u)).
 * The two time derivatives share one backward difference: with
 *   H(t) = (2 tau - 1 + 3K) F1(t) + 3 c_s^2 eta K grad mu(t),
 * F2 = H(t) - H(t - 1) + 3 c_s^2 K grad(div(phi u)).  Hprev (two arrays of N) holds H(t - 1), or is NULL at the
 * first step (the derivatives are then zero); Hout receives H(t). */
void ora_force_full(const ora_params* p, const ora_consts* c, const double* phi, const double* mu, const double* ux,
                    const double* uy, const double* Hprevx, const double* Hprevy, double* Fx, double* Fy,
                    double* Houtx, double* Houty)
{
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double* gmx = (double*)malloc(sizeof(double) * N);
    double* gmy = (double*)malloc(sizeof(double) * N);
    double* jx = (double*)malloc(sizeof(double) * N);
    double* jy = (double*)malloc(sizeof(double) * N);
    double* D = (double*)malloc(sizeof(double) * N);
    double* gDx = (double*)malloc(sizeof(double) * N);
    double* gDy = (double*)malloc(sizeof(double) * N);
    ora_grad(nx, ny, p->walls, mu, gmx, gmy);
    for (long n = 0; n < N; n++) {
        jx[n] = phi[n] * ux[n];
        jy[n] = phi[n] * uy[n];
    }
    ora_div(nx, ny, p->walls, jx, jy, D);
    ora_grad(nx, ny, p->walls, D, gDx, gDy);
    double cF1 = 2.0 * p->tau - 1.0 + 3.0 * c->K;  /* coefficient of d_t F1 */
    double cmu = 3.0 * CS2 * c->eta * c->K;       /* coefficient of d_t grad mu */
    for (long n = 0; n < N; n++) {
        double rho = c->a * phi[n] + c->b;                       /* Eq. rho */
        double F1x = phi[n] / rho * (-phi[n] * gmx[n]);          /* Eq. t0-phiu with grad p = 0 (R1) */
        double F1y = phi[n] / rho * (-phi[n] * gmy[n]);
        double Hx = cF1 * F1x + cmu * gmx[n];
        double Hy = cF1 * F1y + cmu * gmy[n];
        double dHx = Hprevx ? Hx - Hprevx[n] : 0.0;              /* backward difference over one step */
        double dHy = Hprevy ? Hy - Hprevy[n] : 0.0;
        Fx[n] = F1x + dHx + 3.0 * CS2 * c->K * gDx[n];
        Fy[n] = F1y + dHy + 3.0 * CS2 * c->K * gDy[n];
        Houtx[n] = Hx;
        Houty[n] = Hy;
    }
    free(gmx); free(gmy); free(jx); free(jy); free(D); free(gDx); free(gDy);
}

/* One step of Model III: as ora_step, with F from ora_force_full.  H holds 2 N values (x components, then
 * y): H(t - 1) on entry (ignored when first != 0) and H(t) on return. */
void ora_step_full(const ora_params* p, const double* gin, double* gout, double* H, int first, long n)
{
    ora_consts c;
    ora_derive(p, &c);
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double* phi = (double*)malloc(sizeof(double) * N);
    double* mu = (double*)malloc(sizeof(double) * N);
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* Fx = (double*)malloc(sizeof(double) * N);
    double* Fy = (double*)malloc(sizeof(double) * N);
    double* Hn = (double*)malloc(sizeof(double) * 2 * N);

    ora_phi(nx, ny, gin, phi);                 /* Eq. macroscopicg */
    ora_mu(p, &c, phi, mu);                    /* Eq. mu */
    ora_velocity_field(p, n, ux, uy);          /* prescribed u at t = n (R6) */
    ora_force_full(p, &c, phi, mu, ux, uy, first ? NULL : H, first ? NULL : H + N, Fx, Fy, Hn, Hn + N);
    memcpy(H, Hn, sizeof(double) * 2 * N);

#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long x = (long)j * nx + i;
            double geq[Q], S[Q];
            ora_geq(phi[x], mu[x], ux[x], uy[x], c.eta, geq);  /* Eq. geq */
            ora_source(Fx[x], Fy[x], S);                       /* Eq. liangFi */
            for (int q = 0; q < Q; q++) {
                double post = gin[q * N + x] - (gin[q * N + x] - geq[q]) / p->tau
                            + (1.0 - 1.0 / (2.0 * p->tau)) * S[q];
                int ii = ((i + CX[q]) % nx + nx) % nx;
                int jj = j + CY[q];
                if (!p->walls) {
                    jj = ((jj % ny) + ny) % ny;
                } else if (jj < 0 || jj >= ny) {
                    double uwx, uwy;
                    ora_velocity(p, (double)i, jj < 0 ? -0.5 : (double)ny - 0.5, n, &uwx, &uwy);
                    int o = OPP[q];
                    gout[o * N + x] = post + 2.0 * WQ[o] * phi[x] * (CX[o] * uwx + CY[o] * uwy) / CS2;
                    continue;
                }
                gout[q * N + (long)jj * nx + ii] = post;
            }
        }
    free(phi); free(mu); free(ux); free(uy); free(Fx); free(Fy); free(Hn);
}

/* nsteps steps of Model III from step index n0; g and H (2 N) hold the state on entry and on return (H is
 * ignored on entry when n0 = 0). */
int ora_run_full(const ora_params* p, double* g, double* H, long n0, long nsteps)
{
    long N = (long)p->nx * p->ny;
    double* tmp = (double*)malloc(sizeof(double) * Q * N);
    if (!tmp) return -1;
    for (long s = 0; s < nsteps; s++) {
        ora_step_full(p, g, tmp, H, n0 + s == 0, n0 + s);
        memcpy(g, tmp, sizeof(double) * Q * N);
    }
    free(tmp);
    return 0;
}

/* ---------------------------------------------------------------- observables */

/* out[0] = sum phi (mass), out[1] = ||E_phi||_2 against phi0 (Eq. err), out[2] = max phi, out[3] = min phi,
 * out[4] = sum (phi - phi0)^2, out[5] = sum phi0^2. */
void ora_observe(int nx, int ny, const double* phi, const double* phi0, double* out)
{
    long N = (long)nx * ny;
    double m = 0.0, e = 0.0, r = 0.0, mx = phi[0], mn = phi[0];
    for (long n = 0; n < N; n++) {
        m += phi[n];
        e += (phi[n] - phi0[n]) * (phi[n] - phi0[n]);
        r += phi0[n] * phi0[n];
        if (phi[n] > mx) mx = phi[n];
        if (phi[n] < mn) mn = phi[n];
    }
    out[0] = m;
    out[1] = sqrt(e / r);
    out[2] = mx;
    out[3] = mn;
    out[4] = e;
    out[5] = r;
}

/* ---------------------------------------------------------------- adjoint (reverse mode) of the step
 *
 * For a loss L of the final state, lambda_q(x) = dL/dg_q(x).  The step of Eq. LB is
 *   phi = sum_q g_q;  mu = f'(phi) - kappa lap phi;  F = -(phi^2/rho) grad mu [+ K grad div(phi u)];
 *   post_q = (1 - 1/tau) g_q + g_eq_q(phi, mu, u)/tau + (1 - 1/(2 tau)) S_q(F);  g'_q(x + c_q) = post_q(x),
 * and its adjoint runs these operations backwards with every linear map transposed.  The transposed
 * stencils are written out as (A^T v)(x) = sum_k A_k v(x - c_k).  The velocity field enters as u = s u_ref;
 * dLds accumulates dL/ds at s = 1.  Periodic domains only (returns -2 when walls are set).
 */

/* f''(phi) for the double well of Eq. bulk. */
double ora_d2fdphi2(double phi, double beta, double phiA, double phiB)
{
    return 2.0 * beta * ((phi - phiB) * (2.0 * phi - phiA - phiB) + (phi - phiA) * (2.0 * phi - phiA - phiB)
                         + 2.0 * (phi - phiA) * (phi - phiB));
}

/* Partial derivatives of Eq. geq at one node: dphi[q], dmu[q], dux[q], duy[q]. */
static void geq_partials(double phi, double ux, double uy, double eta, double* dphi, double* dmu, double* dux,
                         double* duy)
{
    double uu = ux * ux + uy * uy;
    dphi[0] = 1.0 - WQ[0] * uu / (2.0 * CS2);
    dmu[0] = (WQ[0] - 1.0) * eta;
    dux[0] = -WQ[0] * phi * ux / CS2;
    duy[0] = -WQ[0] * phi * uy / CS2;
    for (int q = 1; q < Q; q++) {
        double cu = CX[q] * ux + CY[q] * uy;
        dphi[q] = WQ[q] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
        dmu[q] = WQ[q] * eta;
        dux[q] = WQ[q] * phi * (CX[q] / CS2 + cu * CX[q] / (CS2 * CS2) - ux / CS2);
        duy[q] = WQ[q] * phi * (CY[q] / CS2 + cu * CY[q] / (CS2 * CS2) - uy / CS2);
    }
}

/* (G^T v)(x) for the isotropic gradient G: sum_k w_k c_k v(x - c_k) / c_s^2, one component. */
static double gradT(int nx, int ny, const double* v, int i, int j, int comp)
{
    double s = 0.0;
    for (int k = 1; k < Q; k++) {
        long m = nbr(nx, ny, 0, i, j, -CX[k], -CY[k]);
        s += WQ[k] * (comp == 0 ? CX[k] : CY[k]) * v[m];
    }
    return s / CS2;
}

/* (L^T v)(x) for the isotropic Laplacian L: sum_k 2 w_k (v(x - c_k) - v(x)) / c_s^2. */
static double lapT(int nx, int ny, const double* v, int i, int j)
{
    double c = v[(long)j * nx + i], s = 0.0;
    for (int k = 1; k < Q; k++) s += 2.0 * WQ[k] * (v[nbr(nx, ny, 0, i, j, -CX[k], -CY[k])] - c);
    return s / CS2;
}

/* lambda_n from lambda_{n+1} for the step n -> n+1 taken from state gin (the forward g at step n). */
int ora_adjoint_step(const ora_params* p, const double* gin, const double* lam_next, double* lam, long n,
                     double* dLds)
{
    if (p->walls) return -2;
    ora_consts c;
    ora_derive(p, &c);
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double* phi = (double*)malloc(sizeof(double) * N);
    double* mu = (double*)malloc(sizeof(double) * N);
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* gmx = (double*)malloc(sizeof(double) * N);
    double* gmy = (double*)malloc(sizeof(double) * N);
    double* gmubx = (double*)malloc(sizeof(double) * N);   /* adjoint of grad mu */
    double* gmuby = (double*)malloc(sizeof(double) * N);
    double* Fbx = (double*)malloc(sizeof(double) * N);     /* adjoint of F */
    double* Fby = (double*)malloc(sizeof(double) * N);
    double* phib = (double*)malloc(sizeof(double) * N);    /* adjoint of phi */
    double* mub = (double*)malloc(sizeof(double) * N);     /* adjoint of mu */
    double* Db = (double*)malloc(sizeof(double) * N);      /* adjoint of D = div(phi u) */
    double* ubx = (double*)malloc(sizeof(double) * N);     /* adjoint of u */
    double* uby = (double*)malloc(sizeof(double) * N);

    /* forward quantities at step n */
    ora_phi(nx, ny, gin, phi);
    ora_mu(p, &c, phi, mu);
    ora_velocity_field(p, n, ux, uy);
    ora_grad(nx, ny, 0, mu, gmx, gmy);

    /* streaming reversed, collision, g_eq, S and F1 (local) */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long x = (long)j * nx + i;
            double pb[Q], dphi[Q], dmu[Q], dux[Q], duy[Q];
            for (int q = 0; q < Q; q++) pb[q] = lam_next[q * N + nbr(nx, ny, 0, i, j, CX[q], CY[q])];
            geq_partials(phi[x], ux[x], uy[x], c.eta, dphi, dmu, dux, duy);
            double fbx = 0.0, fby = 0.0, pl = 0.0, ml = 0.0, bx = 0.0, by = 0.0;
            for (int q = 0; q < Q; q++) {
                lam[q * N + x] = (1.0 - 1.0 / p->tau) * pb[q];
                double geqb = pb[q] / p->tau;
                double Sb = (1.0 - 1.0 / (2.0 * p->tau)) * pb[q];
                fbx += Sb * WQ[q] * CX[q] / CS2;      /* S_q = w_q c_q . F / c_s^2 */
                fby += Sb * WQ[q] * CY[q] / CS2;
                pl += geqb * dphi[q];
                ml += geqb * dmu[q];
                bx += geqb * dux[q];
                by += geqb * duy[q];
            }
            double rho = c.a * phi[x] + c.b;
            double coef = phi[x] * phi[x] / rho;                         /* F1 = -coef grad mu */
            double dcoef = phi[x] * (c.a * phi[x] + 2.0 * c.b) / (rho * rho);
            gmubx[x] = -coef * fbx;
            gmuby[x] = -coef * fby;
            pl += -dcoef * (fbx * gmx[x] + fby * gmy[x]);
            Fbx[x] = fbx; Fby[x] = fby;
            phib[x] = pl; mub[x] = ml; ubx[x] = bx; uby[x] = by;
        }
    /* grad mu = G mu  ->  mu_bar += G^T grad_mu_bar;  F2 = K G D  ->  D_bar = K G^T F_bar */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long x = (long)j * nx + i;
            mub[x] += gradT(nx, ny, gmubx, i, j, 0) + gradT(nx, ny, gmuby, i, j, 1);
            Db[x] = (p->model == 2) ? 3.0 * CS2 * c.K * (gradT(nx, ny, Fbx, i, j, 0) + gradT(nx, ny, Fby, i, j, 1)) : 0.0;
        }
    /* mu = f'(phi) - kappa L phi;  D = G . (phi u)  ->  j_bar = G^T D_bar */
    double acc = 0.0;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long x = (long)j * nx + i;
            double pb = phib[x] + ora_d2fdphi2(phi[x], c.beta, p->phiA, p->phiB) * mub[x] - c.kappa * lapT(nx, ny, mub, i, j);
            if (p->model == 2) {
                double jbx = gradT(nx, ny, Db, i, j, 0), jby = gradT(nx, ny, Db, i, j, 1);
                pb += ux[x] * jbx + uy[x] * jby;
                ubx[x] += phi[x] * jbx;
                uby[x] += phi[x] * jby;
            }
            acc += ubx[x] * ux[x] + uby[x] * uy[x];   /* u = s u_ref: du/ds = u */
            for (int q = 0; q < Q; q++) lam[q * N + x] += pb;  /* phi = sum_q g_q */
        }
    *dLds += acc;
    free(phi); free(mu); free(ux); free(uy); free(gmx); free(gmy); free(gmubx); free(gmuby); free(Fbx); free(Fby);
    free(phib); free(mub); free(Db); free(ubx); free(uby);
    return 0;
}

/* Adjoint of the initial state g_q(x, 0) = g_eq_q(phi0, mu(phi0), u(x, 0)): dL/dphi0 from lambda_0. */
int ora_adjoint_init(const ora_params* p, const double* phi0, const double* lam0, double* dphi0, double* dLds)
{
    if (p->walls) return -2;
    ora_consts c;
    ora_derive(p, &c);
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* mub = (double*)malloc(sizeof(double) * N);
    ora_velocity_field(p, 0, ux, uy);
    double acc = 0.0;
    for (long x = 0; x < N; x++) {
        double dphi[Q], dmu[Q], dux[Q], duy[Q];
        geq_partials(phi0[x], ux[x], uy[x], c.eta, dphi, dmu, dux, duy);
        double pl = 0.0, ml = 0.0, bx = 0.0, by = 0.0;
        for (int q = 0; q < Q; q++) {
            pl += lam0[q * N + x] * dphi[q];
            ml += lam0[q * N + x] * dmu[q];
            bx += lam0[q * N + x] * dux[q];
            by += lam0[q * N + x] * duy[q];
        }
        dphi0[x] = pl;
        mub[x] = ml;
        acc += bx * ux[x] + by * uy[x];
    }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long x = (long)j * nx + i;
            dphi0[x] += ora_d2fdphi2(phi0[x], c.beta, p->phiA, p->phiB) * mub[x] - c.kappa * lapT(nx, ny, mub, i, j);
        }
    *dLds += acc;
    free(ux); free(uy); free(mub);
    return 0;
}


/* ---------------------------------------------------------------- coupled Navier-Stokes step
 *
 * For flows that are not prescribed (Sec. III.E, Rayleigh-Taylor) the velocity comes from a second
 * D2Q9 lattice Boltzmann equation for the Navier-Stokes equations (Eq. NS).  The paper calls that
 * equation standard without writing it out; the oracle takes (reading R14) the incompressible,
 * pressure-based single-relaxation-time form with the forcing of the phase-field literature it cites:
 *   f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq)/tau_f + (1 - 1/(2 tau_f)) G_i,   tau_f = nu/c_s^2 + 1/2,
 *   f_0^eq = (w_0 - 1) p/c_s^2 + rho s_0(u),  f_i^eq = w_i p/c_s^2 + rho s_i(u)  (i > 0),
 *   s_i(u) = w_i [c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u^2/(2 c_s^2)],  Gamma_i = w_i + s_i(u),
 *   G_i = (c_i - u) . [Gamma_i F + (Gamma_i - w_i) c_s^2 grad rho] / c_s^2,
 *   rho u = sum_i c_i f_i + F/2,   p = c_s^2/(1 - w_0) [sum_{i>0} f_i + (1/2) u . grad rho + rho s_0(u)],
 * with rho = a phi + b (Eq. rho) and the total force
 *   F = -phi grad mu - (rho - (rhoA + rhoB)/2) g + (d rho/d phi) M lap(mu) u        (Eq. NS, form c).
 * The Cahn-Hilliard step then uses this u and F1 = (phi/rho)(-phi grad mu - grad p) (Eq. t0-phiu).
 * Walls: both lattices bounce back halfway (no slip, u_w = 0); stencil operands at ghost rows take the
 * mirror values (R7), p and the components of phi u included.
 */

/* equilibrium and forcing of the Navier-Stokes lattice at one node */
static void ns_feq(double pr, double rho, double ux, double uy, double* feq)
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < Q; i++) {
        double cu = CX[i] * ux + CY[i] * uy;
        double s = WQ[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
        feq[i] = (i == 0 ? (WQ[0] - 1.0) : WQ[i]) * pr / CS2 + rho * s;
    }
}

static void ns_forcing(double ux, double uy, double Fx, double Fy, double grx, double gry, double* G)
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < Q; i++) {
        double cu = CX[i] * ux + CY[i] * uy;
        double s = WQ[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
        double Gam = WQ[i] + s;
        double ex = CX[i] - ux, ey = CY[i] - uy;
        G[i] = (ex * (Gam * Fx + s * CS2 * grx) + ey * (Gam * Fy + s * CS2 * gry)) / CS2;
    }
}

/* Macroscopic fields of the coupled state: phi, mu, grad mu, grad rho, lap mu, force F, u, p. */
typedef struct {
    double *phi, *mu, *gmx, *gmy, *grx, *gry, *lmu, *Fx, *Fy, *ux, *uy, *pr;
} ns_fields;

static void ns_alloc(ns_fields* w, long N)
{
    double** a[] = {&w->phi, &w->mu, &w->gmx, &w->gmy, &w->grx, &w->gry, &w->lmu, &w->Fx, &w->Fy, &w->ux, &w->uy, &w->pr};
    for (int k = 0; k < 12; k++) *a[k] = (double*)malloc(sizeof(double) * N);
}

static void ns_free(ns_fields* w)
{
    double* a[] = {w->phi, w->mu, w->gmx, w->gmy, w->grx, w->gry, w->lmu, w->Fx, w->Fy, w->ux, w->uy, w->pr};
    for (int k = 0; k < 12; k++) free(a[k]);
}

static void ns_compute_fields(const ora_params* p, const ora_consts* c, const double* f, const double* g, ns_fields* w)
{
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double rbar = 0.5 * (p->rhoA + p->rhoB);
    ora_phi(nx, ny, g, w->phi);                          /* Eq. macroscopicg */
    ora_mu(p, c, w->phi, w->mu);                         /* Eq. mu */
    ora_grad(nx, ny, p->walls, w->mu, w->gmx, w->gmy);
    ora_grad(nx, ny, p->walls, w->phi, w->grx, w->gry);  /* grad rho = a grad phi (Eq. rho) */
    ora_lap(nx, ny, p->walls, w->mu, w->lmu);
    for (long x = 0; x < N; x++) {
        double phi = w->phi[x], rho = c->a * phi + c->b;
        w->grx[x] *= c->a;
        w->gry[x] *= c->a;
        double F0x = -phi * w->gmx[x] - (rho - rbar) * p->gx;
        double F0y = -phi * w->gmy[x] - (rho - rbar) * p->gy;
        double mx = 0.0, my = 0.0, sum1 = 0.0;
        for (int i = 0; i < Q; i++) {
            mx += CX[i] * f[i * N + x];
            my += CY[i] * f[i * N + x];
            if (i > 0) sum1 += f[i * N + x];
        }
        /* rho u = m + F/2 with F = F0 + a M lap(mu) u, solved for u */
        double den = rho - 0.5 * c->a * c->M * w->lmu[x];
        double ux = (mx + 0.5 * F0x) / den, uy = (my + 0.5 * F0y) / den;
        w->ux[x] = ux;
        w->uy[x] = uy;
        w->Fx[x] = F0x + c->a * c->M * w->lmu[x] * ux;
        w->Fy[x] = F0y + c->a * c->M * w->lmu[x] * uy;
        double uu = ux * ux + uy * uy;
        double s0 = WQ[0] * (-uu / (2.0 * CS2));
        w->pr[x] = CS2 / (1.0 - WQ[0]) * (sum1 + 0.5 * (ux * w->grx[x] + uy * w->gry[x]) + rho * s0);
    }
}

/* Macroscopic velocity and pressure of a coupled state (ux, uy, p), for observation. */
void ora_ns_fields(const ora_params* p, const double* f, const double* g, double* ux, double* uy, double* pr)
{
    ora_consts c;
    ora_derive(p, &c);
    long N = (long)p->nx * p->ny;
    ns_fields w;
    ns_alloc(&w, N);
    ns_compute_fields(p, &c, f, g, &w);
    memcpy(ux, w.ux, sizeof(double) * N);
    memcpy(uy, w.uy, sizeof(double) * N);
    memcpy(pr, w.pr, sizeof(double) * N);
    ns_free(&w);
}

/* Initial coupled state: g = g_eq(phi0, mu0, u0), f = f_eq(p = 0, rho(phi0), u0), u0 given per node. */
void ora_ns_init(const ora_params* p, const double* phi0, const double* ux0, const double* uy0, double* f, double* g)
{
    ora_consts c;
    ora_derive(p, &c);
    long N = (long)p->nx * p->ny;
    double* mu = (double*)malloc(sizeof(double) * N);
    ora_mu(p, &c, phi0, mu);
    for (long x = 0; x < N; x++) {
        double geq[Q], feq[Q];
        ora_geq(phi0[x], mu[x], ux0[x], uy0[x], c.eta, geq);
        ns_feq(0.0, c.a * phi0[x] + c.b, ux0[x], uy0[x], feq);
        for (int q = 0; q < Q; q++) {
            g[q * N + x] = geq[q];
            f[q * N + x] = feq[q];
        }
    }
    free(mu);
}

/* One coupled step n -> n+1: the Cahn-Hilliard lattice g and the Navier-Stokes lattice f. */
void ora_ns_step(const ora_params* p, const double* fin, const double* gin, double* fout, double* gout, long n)
{
    (void)n;
    ora_consts c;
    ora_derive(p, &c);
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double tauf = p->nu / CS2 + 0.5;
    ns_fields w;
    ns_alloc(&w, N);
    ns_compute_fields(p, &c, fin, gin, &w);
    double* gpx = (double*)malloc(sizeof(double) * N);
    double* gpy = (double*)malloc(sizeof(double) * N);
    double* Fx = (double*)malloc(sizeof(double) * N);
    double* Fy = (double*)malloc(sizeof(double) * N);
    ora_grad(nx, ny, p->walls, w.pr, gpx, gpy);
    /* the Cahn-Hilliard force with the flow's pressure, Eqs. t0-phiu and mark3 */
    for (long x = 0; x < N; x++) {
        double phi = w.phi[x], rho = c.a * phi + c.b;
        Fx[x] = phi / rho * (-phi * w.gmx[x] - gpx[x]);
        Fy[x] = phi / rho * (-phi * w.gmy[x] - gpy[x]);
    }
    if (p->model == 2) {
        double* jx = (double*)malloc(sizeof(double) * N);
        double* jy = (double*)malloc(sizeof(double) * N);
        double* D = (double*)malloc(sizeof(double) * N);
        double* gDx = (double*)malloc(sizeof(double) * N);
        double* gDy = (double*)malloc(sizeof(double) * N);
        for (long x = 0; x < N; x++) {
            jx[x] = w.phi[x] * w.ux[x];
            jy[x] = w.phi[x] * w.uy[x];
        }
        ora_div(nx, ny, p->walls, jx, jy, D);
        ora_grad(nx, ny, p->walls, D, gDx, gDy);
        for (long x = 0; x < N; x++) {
            Fx[x] += 3.0 * CS2 * c.K * gDx[x];
            Fy[x] += 3.0 * CS2 * c.K * gDy[x];
        }
        free(jx); free(jy); free(D); free(gDx); free(gDy);
    }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long x = (long)j * nx + i;
            double geq[Q], S[Q], feq[Q], G[Q];
            double rho = c.a * w.phi[x] + c.b;
            ora_geq(w.phi[x], w.mu[x], w.ux[x], w.uy[x], c.eta, geq);
            ora_source(Fx[x], Fy[x], S);
            ns_feq(w.pr[x], rho, w.ux[x], w.uy[x], feq);
            ns_forcing(w.ux[x], w.uy[x], w.Fx[x], w.Fy[x], w.grx[x], w.gry[x], G);
            for (int q = 0; q < Q; q++) {
                double pg = gin[q * N + x] - (gin[q * N + x] - geq[q]) / p->tau + (1.0 - 1.0 / (2.0 * p->tau)) * S[q];
                double pf = fin[q * N + x] - (fin[q * N + x] - feq[q]) / tauf + (1.0 - 1.0 / (2.0 * tauf)) * G[q];
                int ii = ((i + CX[q]) % nx + nx) % nx;
                int jj = j + CY[q];
                if (!p->walls) {
                    jj = ((jj % ny) + ny) % ny;
                } else if (jj < 0 || jj >= ny) {
                    /* halfway bounce-back at a wall at rest */
                    gout[OPP[q] * N + x] = pg;
                    fout[OPP[q] * N + x] = pf;
                    continue;
                }
                gout[q * N + (long)jj * nx + ii] = pg;
                fout[q * N + (long)jj * nx + ii] = pf;
            }
        }
    free(gpx); free(gpy); free(Fx); free(Fy);
    ns_free(&w);
}
