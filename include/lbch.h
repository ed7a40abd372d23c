/*
 * lbch.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for the Cahn-Hilliard equation.
 *
 * Method: Zhang, Guo & Liang, "A high-order lattice Boltzmann model for the Cahn-Hilliard equation"
 * (arXiv:1805.00007).  One step advances the D2Q9 distributions g_i of the order parameter phi by the
 * single-relaxation-time equation of Eq. LB, with the equilibrium of Eq. geq, the source of Eq. liangFi
 * and the force of Eq. reFi as the paper runs it (Remark III): F = (phi/rho)(-phi grad mu) for Model I,
 * plus 3 c_s^2 K grad(div(phi u)) (Eq. mark3) for Model II.  The chemical potential is Eq. mu with the
 * double well of Eq. bulk and the constants of Eq. betakappa; phi = sum_i g_i (Eq. macroscopicg).
 *
 * Conventions.  Lattice units (dx = dt = 1).  Node (i, j) sits at x = i, y = j; host fields are row-major
 * double arrays of ny*nx values (index j*nx + i).  The domain is periodic in x; in y it is periodic, or
 * (walls = 1) bounded by halfway bounce-back walls at y = -1/2 and y = ny - 1/2 that move with the
 * prescribed velocity evaluated there.  The velocity field is prescribed (lbch_vel); it is evaluated at
 * t = n for the step n -> n+1.
 *
 * Ownership.  The caller owns every host buffer it passes; the library copies what it needs before the
 * call returns (lb_ch_init) or writes into it (lb_ch_observe).  The library owns all device memory of a
 * handle and releases it in lb_ch_free.  A handle is bound to the CUDA device current at lb_ch_init and
 * to one CUDA stream; calls on one handle must not run concurrently from several host threads.
 *
 * Errors.  Every entry point returns an lbch_status; nothing aborts.  LBCH_EINVAL for bad arguments
 * (nothing is changed), LBCH_ENOMEM when device memory runs out, LBCH_ECUDA for any other CUDA error
 * (the handle should then be freed), LBCH_ENONFINITE from lb_ch_observe when phi holds a NaN or Inf.
 * lb_ch_last_error() gives a message for the most recent failure on the calling thread.
 */
#ifndef LBCH_H
#define LBCH_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBCH_OK = 0,
    LBCH_EINVAL = 1,
    LBCH_ENOMEM = 2,
    LBCH_ECUDA = 3,
    LBCH_ETIMEOUT = 4,
    LBCH_ENONFINITE = 5
} lbch_status;

/* Storage and arithmetic precision of the lattice state.
 *   LBCH_F64  : g and phi stored in double, double arithmetic.
 *   LBCH_F32  : shifted float storage -- g_1..g_8 and g_0 - phi stored in float; phi carried as a pair
 *               of floats (a high part that feeds the stencils and a low part kept at the node), float
 *               arithmetic on these small quantities, and phi(t+1) = phi(t) + (float increment) formed
 *               exactly by a TwoSum of the pair (velocity tables built in double and rounded once to
 *               float).  88 bytes per lattice update (16 when every tau_g = 1, phi alone).
 *   LBCH_F16S : shifted half storage -- phi kept in float, g_1..g_8 stored in half, g_0 not stored but
 *               recovered as phi - sum_{i>0} g_i, so sum_i g_i = phi holds exactly; float arithmetic.
 *               40 bytes per lattice update. */
typedef enum { LBCH_F64 = 0, LBCH_F32 = 1, LBCH_F16S = 2 } lbch_prec;

/* Prescribed velocity fields u(x, y, t) of the benchmark problems (paper Sec. III).
 *   UNIFORM  : u = (ux0, uy0)                                          (diagonal translation, Sec. III.A)
 *   ROTATION : u = (-U0 pi (y - yc)/half, U0 pi (x - xc)/half)          (Zalesak's disk, Sec. III.B)
 *   VORTEX   : u = U0 (-sin^2(pi x/nx) sin(2 pi y/ny), sin(2 pi x/nx) sin^2(pi y/ny)) cos(pi t/Tper)
 *   SHEAR    : u = (shear (y - (ny-1)/2), 0), used with walls = 1      (wall-driven shear flow)
 *   REV_SHEAR: Eq. shear with L0 = nx, sign reversed for t >= Tper     (Sec. III.C)
 *   DEFORM   : Eq. deformation with L0 = nx, n = nvort, T0 = Tper      (Sec. III.D)
 *   COUPLED  : not prescribed -- solved by a second D2Q9 lattice for Eq. NS (the Rayleigh-Taylor
 *              problem of Sec. III.E): the incompressible pressure-based single-relaxation-time form
 *              with forcing, total force -phi grad mu - (rho - (rhoA+rhoB)/2)(gx, gy) + (d rho/d phi) M
 *              lap(mu) u, and F1 = (phi/rho)(-phi grad mu - grad p) in the Cahn-Hilliard source.
 *              Single-instance handles, LBCH_F64 or LBCH_F32 (plain float storage). */
typedef enum {
    LBCH_VEL_UNIFORM = 0,
    LBCH_VEL_ROTATION = 1,
    LBCH_VEL_VORTEX = 2,
    LBCH_VEL_SHEAR = 3,
    LBCH_VEL_REV_SHEAR = 4,
    LBCH_VEL_DEFORM = 5,
    LBCH_VEL_COUPLED = 6
} lbch_vel;

/* Quantities lb_ch_observe returns.  Sums are accumulated in double on the GPU in a fixed order, so
 * repeated calls on the same state give identical results.
 *   MASS    : sum_x phi                                                  (1 value)
 *   ERR_L2  : ||E_phi||_2 = sqrt(sum (phi - phi0)^2 / sum phi0^2), Eq. err (1 value)
 *   MAX/MIN : extreme values of phi (Sec. III.A prints them)              (1 value)
 *   PHI     : the field phi as ny*nx doubles, row-major                   (nx*ny values)
 *   STEP    : the step index n of the current state                       (1 value)
 *   U, P    : coupled handles only: the flow's velocity (ux field then uy field, 2*nx*ny values) and
 *             pressure (nx*ny values) of the current state */
typedef enum {
    LBCH_OBS_MASS = 0,
    LBCH_OBS_ERR_L2 = 1,
    LBCH_OBS_MAX = 2,
    LBCH_OBS_MIN = 3,
    LBCH_OBS_PHI = 4,
    LBCH_OBS_STEP = 5,
    LBCH_OBS_U = 6,
    LBCH_OBS_P = 7
} lbch_obs;

/* Parameters of one problem instance, in the paper's notation.  The derived constants are computed by
 * the library: beta, kappa (Eq. betakappa); eta from M = c_s^2 eta (tau - 1/2); a, b (Eq. rho);
 * K = (tau - 1/6 - tau^2)/(tau - 1/2) (Eq. F2-1); and, when M <= 0, M = Ustar W / (Pe beta (phiA-phiB)^2)
 * from the Peclet number of Sec. III.A. */
typedef struct {
    int nx, ny;          /* lattice size, each >= 4 */
    int walls;           /* 0: periodic in y; 1: moving bounce-back walls at y = -1/2 and ny - 1/2 */
    int model;           /* 1: Model I; 2: Model II (Eq. mark3 force added); 3: Model II with the complete
                            diffusive-scale force of Eq. F2-1, whose time derivatives are backward
                            differences over one step (zero at step 0); steps with the row sweep's
                            Model III build (its two unrolled configurations) or the tile kernel, not
                            with the adjoint, the coupled flow or slabs */
    int vel;             /* lbch_vel */
    int nvort;           /* vortex count of the deformation field */
    double phiA, phiB;   /* bulk values of phi */
    double sigma, W;     /* surface tension, interface width */
    double M;            /* mobility (if <= 0, derived from Pe and Ustar) */
    double Pe, Ustar;    /* Peclet number and characteristic speed */
    double tau;          /* relaxation time tau_g, > 1/2 */
    double rhoA, rhoB;   /* bulk densities */
    double U0, ux0, uy0; /* velocity amplitude; uniform velocity */
    double xc, yc, half; /* rotation centre and half-length */
    double Tper;         /* period or reversal time of time-dependent flows, in steps */
    double shear;        /* shear rate */
    double nu;           /* LBCH_VEL_COUPLED: kinematic viscosity (tau_f = 3 nu + 1/2) */
    double gx, gy;       /* LBCH_VEL_COUPLED: buoyancy force -(rho - (rhoA + rhoB)/2) (gx, gy) */
} lbch_params;

typedef struct lbch_handle lbch_handle;

/* Create a simulation of n_inst independent instances (an ensemble when n_inst > 1; instances may have
 * different sizes and parameters but share the precision).  params: n_inst structs (host).  phi0: the
 * initial order parameter of every instance, concatenated in instance order, each ny*nx row-major
 * doubles (host).  The initial distributions are the equilibria of phi0, mu(phi0) and u(t = 0).
 * stream: a cudaStream_t, or NULL for a stream the library creates; a caller's stream must outlive the
 * handle (the handle's device memory is allocated and released in its order, from a pool per device that
 * keeps freed memory for the next handle).  On success *out receives the handle and the state is at
 * step 0. */
lbch_status lb_ch_init(const lbch_params* params, int n_inst, const double* phi0, int prec,
                       void* stream, lbch_handle** out);

/* ---- domain decomposition: one periodic grid split into slabs of rows over several handles ----
 *
 * Eq. LB is explicit and local: phi(t+1) at a node depends on the state at time t only within three nodes
 * (mu and D = div(phi u) one node out, their gradients and the collision one further, the pull of the
 * streaming one more; Eqs. mu, mark3, LB with the isotropic stencils of Sec. III).  A grid that is
 * periodic in y can therefore be split into slabs of consecutive rows, each stepped by its own handle (on
 * its own GPU, or several on one), if before every step each slab receives from its two neighbours the
 * three rows of phi next to it and the one row of populations that streams across the cut.  The result is
 * the whole-grid result, bit for bit.
 *
 * lb_ch_init_slab: a handle for global rows y0 .. y0 + ny_local - 1 of the problem `global` (walls = 0,
 * a prescribed flow, Model I or II; ny_local >= 4).  phi0_halo (host) holds ny_local + 6 rows of global->nx
 * doubles: global rows y0 - 3 .. y0 + ny_local + 2, taken periodically, so that the initial equilibria at
 * the slab's edge rows see their true neighbours.  The velocity field is evaluated at global coordinates.
 * A slab handle steps with the row sweep or the tile kernel (not the two-step kernel), advances at most one
 * step per lb_ch_step call (LBCH_EINVAL otherwise), and must receive both halos before every step,
 * including the first.  Observables are the slab's own (sum them over the slabs for global ones).
 * lb_ch_halo_bytes: size of one side's halo (the same for every slab of a grid in one precision).
 * lb_ch_halo_export: the slab's own edge rows into dst (device, lb_ch_halo_bytes bytes): side 0 = its
 *   lowest rows (for the slab below), side 1 = its highest rows (for the slab above).
 * lb_ch_halo_import: the neighbour's export into the slab's ghost rows: side 0 = the rows below it (the
 *   lower neighbour's side-1 export), side 1 = the rows above it (the upper neighbour's side-0 export).
 * Both are stream-ordered on the handle's stream and apply to the current state; the caller moves the
 * buffers between slabs (a device-to-device copy, a peer copy or an NCCL send/recv into each GPU's own
 * memory) and orders the streams.  Halo layout: 3 rows of phi (the high part in LBCH_F32), 3 rows of phi's
 * low part (LBCH_F32 only), one row of the stored populations; each row is one stored row of the handle,
 * ghost columns included, so slabs of one grid must share nx and the precision. */
lbch_status lb_ch_init_slab(const lbch_params* global, int y0, int ny_local, const double* phi0_halo, int prec,
                            void* stream, lbch_handle** out);
lbch_status lb_ch_halo_bytes(lbch_handle* h, long long* bytes);
lbch_status lb_ch_halo_export(lbch_handle* h, int side, void* dst);
lbch_status lb_ch_halo_import(lbch_handle* h, int side, const void* src);

/* Advance every instance by nsteps >= 0 steps of Eq. LB.  Asynchronous on the handle's stream: the work
 * is enqueued (in CUDA graphs of 64 steps when possible) and the call returns.  When every instance has
 * tau_g = 1 (the paper's default), Eq. LB reduces to g* = g_eq + S/2 and the populations drop out of the
 * step: the library then reads and writes phi only (the stored populations are left unchanged and are
 * not part of the state), with the same results bit for bit.  Until lb_ch_tune chooses otherwise, a
 * handle whose instances are all periodic with tau_g = 1 (LBCH_F32 or LBCH_F64) and whose grid fits the
 * device in one wave of two-step tiles (up to about 68 K nodes) steps two steps per launch
 * with the two-step kernel; every other handle steps with the row sweep. */
lbch_status lb_ch_step(lbch_handle* h, long nsteps);

/* Read an observable of instance inst into out (host, sized as lbch_obs states).  Synchronises the
 * handle's stream.  Returns LBCH_ENONFINITE (with out filled) when phi holds a NaN or Inf. */
lbch_status lb_ch_observe(lbch_handle* h, int inst, int what, double* out);

/* One scalar observable (MASS, ERR_L2, MAX or MIN) for every instance: out receives n_inst values. */
lbch_status lb_ch_observe_all(lbch_handle* h, int what, double* out);

/* Release every resource of the handle (safe on NULL): waits for the handle's stream, then returns the
 * device memory to the device's pool in that stream's order (up to 2 GB of it stays reserved for later
 * handles) and the pinned staging buffer to a small cache of the library's. */
lbch_status lb_ch_free(lbch_handle* h);

/* Human-readable name of a status, and the message of the last failure on this thread. */
const char* lb_ch_strerror(lbch_status s);
const char* lb_ch_last_error(void);

/* Sizes for a caller who times the step kernel itself: out[0] = total lattice nodes, out[1] = algorithmic
 * HBM bytes per lattice update of the step kernel (one read and one write of the stored populations and
 * of phi; of phi alone when every tau_g = 1; half that with the two-step kernel, which reads and writes
 * phi once per two updates), out[2] = persistent thread blocks of one step launch, out[3] = current step
 * index. */
lbch_status lb_ch_info(lbch_handle* h, double* out);

/* Which step kernel advances the handle, for a caller who reports on it: out[0] = its form (0 = tile
 * kernel, 1 = row sweep without the populations -- every instance has tau_g = 1 --, 2 = row sweep with
 * the populations, 3 = the coupled Navier-Stokes kernels, 4 = tile kernel without the populations, 5 = the
 * two-step kernel: two steps per launch, periodic instances with tau_g = 1),
 * out[1] = the shape index in use (see
 * lb_ch_tune), out[2] x out[3] = output nodes of one tile, out[4] = output rows per warp of the row
 * sweep (0 otherwise), out[5] = threads per thread block.  out must hold 6 ints. */
lbch_status lb_ch_kernel_info(lbch_handle* h, int* out);

/* The CUDA stream the handle enqueues on (a cudaStream_t). */
void* lb_ch_stream(lbch_handle* h);

/* Kernel and tile-shape autotuner.  The step has three kernel forms, each built for several shapes: the
 * row sweep (warps sweeping 56-column strips; tiles of 56 x 48, 56 x 24 and twice 56 x 12 output nodes),
 * the tile kernel (each tile's stencil fields staged in shared memory; 32x16, 32x8 and 16x8 with 256
 * threads and 32x16 with 768 on the float paths; 32x8 and 16x8 with 256 and 32x8 with 512 for LBCH_F64)
 * and, for handles whose instances are all periodic with tau_g = 1 in LBCH_F32 or LBCH_F64, the two-step
 * kernel (two steps per launch from phi on the tile + 6; 32x16 with 768 threads, 32x14 and 32x16 with
 * 1024 and 32x8 with 512 in LBCH_F32; 32x8 with 512, 16x8 with 256, 16x16 with 512 and 32x14 with 1024
 * in LBCH_F64; an odd last step of lb_ch_step then runs the fastest one-step candidate).  lb_ch_tune
 * times every candidate on the handle's own problem through lb_ch_step (as a run steps: CUDA graphs of 64
 * steps) -- one graph of warm-up, then the faster of two runs of `steps` steps rounded up to whole graphs
 * (below 64 steps: two steps of warm-up and two runs of `steps` steps) --, restores the state after each,
 * keeps the fastest, and reports its tile size in
 * *tile_x, *tile_y (either may be NULL).  The result of the simulation does not depend on the choice (on
 * the half-storage path with every tau_g = 1 only the row sweep is a candidate, as the tile kernel would
 * round the streamed populations to half).  Allocates a temporary state copy; synchronises. */
lbch_status lb_ch_tune(lbch_handle* h, int steps, int* tile_x, int* tile_y);

/* ---- checkpoints and the differentiable adjoint (single-instance, periodic handles) ----
 *
 * The step's Jacobian depends on the populations only through phi (Eq. LB with Eqs. geq, liangFi,
 * mu, t0-phiu, mark3 are linear in g except through phi = sum g), so reverse mode needs, for every
 * forward step n, the forward phi(n) (a tape entry) and nothing else.  The tape type is the forward
 * path's: double for LBCH_F64 handles, float otherwise.  Gradients (dL_dphiT, dL_dphi0) are double for
 * every precision, and the adjoint itself is carried in double.  Every array below is a device pointer
 * the caller owns.
 *
 * lb_ch_state_bytes / lb_ch_state_save / lb_ch_state_load: the full state (populations, phi, step
 * index) to and from a caller buffer of lb_ch_state_bytes() bytes -- the checkpoints of a segmented
 * reverse sweep.  Loading also restores the step index.  The buffer starts with a 256-byte header that
 * records the layout it was saved for (sizes, precision, instances, model); lb_ch_state_load reads that
 * header first and returns LBCH_EINVAL, copying nothing, for a buffer that holds no saved state or was
 * saved by a handle of another layout, precision or model.
 * lb_ch_tape_phi: phi of the current state into dst (nx*ny values, row-major, tape type).
 * lb_ch_adjoint_begin: lambda = dL/dg_q(T) = dL/dphi(T) for every q (dL_dphiT: nx*ny values).
 * lb_ch_adjoint_step: one step backwards: lambda_n from lambda_{n+1}, given phi_n (the forward phi at
 *   step n) and n; accumulates dL/ds, where the prescribed velocity is s times the configured one.
 * lb_ch_adjoint_end: the adjoint of the initial equilibria: dL/dphi0 into dL_dphi0 (nx*ny values)
 *   and dL/ds (at s = 1) into *dL_ds (host).  Synchronises the stream.
 * lb_ch_step_taped: nsteps forward steps, writing phi of each step's starting state into the tape:
 *   entry k (nx*ny values of the tape type, at tape + k * nx*ny) holds phi(n + k), n the step index on
 *   entry -- the replay of a checkpointed segment in one call (one-step launches, captured in a CUDA graph
 *   that is kept while the tape and length repeat).
 * lb_ch_adjoint_sweep: lb_ch_adjoint_step for n = n0 + nsteps - 1 down to n0, with phi_n the tape entry
 *   n - n0 (a tape lb_ch_step_taped wrote from step n0).
 * Walls and ensembles are rejected with LBCH_EINVAL. */
lbch_status lb_ch_state_bytes(lbch_handle* h, long long* bytes);
lbch_status lb_ch_state_save(lbch_handle* h, void* dst);
lbch_status lb_ch_state_load(lbch_handle* h, const void* src);
lbch_status lb_ch_tape_phi(lbch_handle* h, void* dst);
lbch_status lb_ch_adjoint_begin(lbch_handle* h, const void* dL_dphiT);
lbch_status lb_ch_adjoint_step(lbch_handle* h, const void* phi_n, long n);
lbch_status lb_ch_adjoint_end(lbch_handle* h, void* dL_dphi0, double* dL_ds);
lbch_status lb_ch_step_taped(lbch_handle* h, long nsteps, void* tape);
lbch_status lb_ch_adjoint_sweep(lbch_handle* h, const void* tape, long n0, long nsteps);

/* Test hook for the failure path of the step kernel's bounded waits.  With hook
 * LBCH_HOOK_SKIP_FIRST_LOAD and value != 0, the next step launches run without CUDA graphs and their
 * first thread block never issues its first tile copy, so its bounded wait runs out (after about a
 * second); the kernel then returns cleanly and the next lb_ch_observe reports LBCH_ETIMEOUT.  The
 * handle's state is not advanced correctly afterwards and should be freed.  With hook
 * LBCH_HOOK_TILE_SHAPE, value selects the tile shape by its index in the list lb_ch_tune describes
 * (for tests that compare shapes).  With hook LBCH_HOOK_GENERAL_PATH and value != 0, handles whose
 * instances all have tau_g = 1 keep and stream the populations instead of dropping them (see
 * lb_ch_step); the two give the same bits.  With hook LBCH_HOOK_TILE_KERNEL and value != 0, the steps
 * run the tile kernel (each tile's stencil fields staged in shared memory) instead of the row sweep, with
 * the populations; the tile shape hook then indexes its own list of shapes, and the results are the same
 * bits again; with value 0, the row sweep (either value turns the two-step kernel off).  With hook LBCH_HOOK_TWO_STEP and value != 0 (periodic instances with tau_g = 1 in
 * LBCH_F32 or LBCH_F64, else LBCH_EINVAL), lb_ch_step takes the steps two at a time with the two-step
 * kernel (the tile shape hook then indexes its list), the same bits once more; value 0 returns to the
 * one-step kernel.  With hook LBCH_HOOK_NO_PDL and value != 0,
 * step launches are ordinary stream-ordered launches instead of programmatic dependents of the previous
 * step (whose launch and prologue overlap that step's tail); the results are the same bits.  With hook
 * LBCH_HOOK_POISON (value ignored), every device buffer the next step writes -- phi, its low part, the
 * populations and Model III's H of the next state, or on coupled handles f, g, u, p, mu and phi of the
 * current state (which a coupled step forms from the populations) -- is filled
 * with all bits set (NaN in every storage type), stream-ordered before the next step; a step that reads
 * a cell it did not write first carries NaN into phi.  Not for production use. */
enum {
    LBCH_HOOK_SKIP_FIRST_LOAD = 1,
    LBCH_HOOK_TILE_SHAPE = 2,
    LBCH_HOOK_GENERAL_PATH = 3,
    LBCH_HOOK_NO_PDL = 4,
    LBCH_HOOK_TILE_KERNEL = 5,
    LBCH_HOOK_TWO_STEP = 6,
    LBCH_HOOK_POISON = 7
};
lbch_status lb_ch_test_hook(lbch_handle* h, int hook, long value);

/* Statistics of a caller-owned field without allocating anything (the paper has no counterpart; this
 * serves callers that may not allocate device memory, e.g. code running inside another framework's
 * memory pool or a plugin restricted to the buffers it is handed).
 *
 * phi, phi0: device pointers to ny rows of nx doubles, row r starting at element r * pitch.
 * out: device pointer to 6 doubles, written asynchronously on `stream` (a cudaStream_t, NULL = legacy
 * default stream): out[0] = sum phi, out[1] = sum (phi - phi0)^2, out[2] = sum phi0^2 (so the relative
 * L2 difference of phi from phi0 is sqrt(out[1] / out[2])), out[3] = max phi, out[4] = min phi, out[5] =
 * number of non-finite phi values (left out of the other five).  The values equal those lb_ch_observe reports
 * for the same field up to the order of the floating-point sums.
 *
 * The per-block partial sums go to a file-scope device array of LBCH_NOALLOC_MAX_BLOCKS x 6 doubles
 * (48 KiB), which every GPU that loads this library holds until the process exits.  The first call in a
 * CUDA context looks up that array's device address (with the context's device current) and caches it
 * for that context (thread-safe); make that first call before any stream capture.  Calls share the array: each overwrites what it uses, but calls that
 * overlap on the GPU race.  Fields of more than LBCH_NOALLOC_MAX_NODES nodes are rejected with
 * LBCH_EINVAL; no cudaMalloc, cudaFree or allocating library routine is ever called. */
#define LBCH_NOALLOC_MAX_BLOCKS 1024
#define LBCH_NOALLOC_MAX_NODES (1LL << 31)
lbch_status lb_ch_field_stats_noalloc(const double* phi, const double* phi0, int nx, int ny, int pitch,
                                      double* out, void* stream);

/* Fused multiply-add throughput of the current device in prec (LBCH_F32 or LBCH_F64, else LBCH_EINVAL), for
 * the arithmetic rooflines reported beside the step (the paper has no counterpart).  One kernel fills every
 * SM with threads that each run eight independent chains of FMAs; a short run sizes the measured one to
 * about 20 ms and the fastest of three counts (2 flop per FMA).  *flop_per_s receives flop/s (host).
 * Allocates one element of device memory; synchronises `stream` (a cudaStream_t, NULL = legacy default). */
lbch_status lb_ch_alu_peak(int prec, void* stream, double* flop_per_s);

#ifdef __cplusplus
}
#endif
#endif /* LBCH_H */
