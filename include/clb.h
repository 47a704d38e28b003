/*
 * clb.h -- C ABI of the GB300 (sm_103a) REV-scale cascaded lattice Boltzmann
 * library for convection heat transfer in porous media.
 *
 * Method: Feng, Liu & He, "Numerical simulations of convection heat transfer
 * in porous media using a cascaded lattice Boltzmann method",
 * arXiv:2110.05943.  One time step is the coupled update of
 *   - the D2Q9 porous cascaded flow solver of Sec. 2.1 (Eqs. 4-23: shift to
 *     porosity-aware central moments by N of Eq. 14, cascaded relaxation of
 *     Eq. 11, implicit Brinkman-Forchheimer velocity of Eqs. 22-23, force of
 *     Eq. 4 with the Ergun coefficient of Eq. 5, streaming of Eq. 18), and
 *   - the D2Q5 temperature solver of Sec. 2.2 (Eqs. 24-36: shift N_T of
 *     Eq. 31 with the heat capacity ratio sigma, relaxation Eq. 28,
 *     streaming Eq. 35),
 * with walls treated by non-equilibrium extrapolation (Sec. 3).
 *
 * Conventions for every entry point:
 *   - Return CLB_OK (0) on success or a negative CLB_ERR_* code; no C++
 *     exception crosses the ABI.  clb_last_error() gives a message.
 *   - Host arrays of nodal fields are (ny, nx) row-major, x fastest, FP64,
 *     caller-owned; the library copies what it needs and keeps no pointer.
 *   - The handle owns all device memory; clb_destroy frees it.
 *   - All work is issued on the CUDA stream given to clb_init (NULL: the
 *     legacy default stream).  Calls that return host data synchronise that
 *     stream; clb_step does not.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef CLB_H
#define CLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CLB_OK 0
#define CLB_ERR_ARG (-1)      /* invalid argument or parameter */
#define CLB_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define CLB_ERR_OOM (-3)      /* device or host allocation failed */
#define CLB_ERR_UNSTABLE (-4) /* non-finite value found in the fields */
#define CLB_ERR_STATE (-5)    /* checkpoint does not match this handle */
#define CLB_ERR_TIMEOUT (-6)  /* a bounded wait on the GPU expired (persistent batch) */

/* Sides, in this order everywhere: west (x = 0), east (x = nx-1),
 * south (y = 0), north (y = ny-1).  Gravity points along -y. */
enum { CLB_W = 0, CLB_E = 1, CLB_S = 2, CLB_N = 3 };
enum { CLB_PERIODIC = 0, CLB_WALL = 1 };
enum { CLB_ADIABATIC = 0, CLB_ISOTHERMAL = 1 };
/* Arithmetic / storage form of the distributions (reductions stay FP64).
 *   CLB_F64  : FP64 storage and arithmetic; 232 B per node update.
 *   CLB_F16S : each distribution stored in FP16 as its deviation from the
 *              rest state (w_i rho_0 for f, the D2Q5 equilibrium at u = 0,
 *              T = T0 for g), arithmetic in FP32; 60 B per node update.
 *              The rest population's deviation is O(dT), so T is quantised
 *              at ~2e-4 dT every step: steady Nusselt numbers carry
 *              errors of 1e-4 to a few 1e-2 and visible noise.
 *   CLB_F16N : each post-collision value stored in FP16 as its deviation
 *              from the local equilibrium of the node that wrote it, plus
 *              that node's (rho - 1, u, T - T0) in FP16 as the baseline;
 *              FP32 arithmetic; 76 B per node update.
 * Both FP16 forms store the deviations times 2^12 with unbiased stochastic
 * rounding, seeded by the node and a per-buffer step counter (runs are
 * deterministic, and checkpoints carry the counter). */
enum { CLB_F64 = 0, CLB_F16S = 1, CLB_F16N = 2 };

/* Boundary specification.  Opposite sides must both be periodic or both
 * walls; a walled direction needs at least 4 nodes.  Wall nodes lie on the
 * boundary lines and are rebuilt every step by non-equilibrium extrapolation
 * from the inward neighbour: velocity (u[s], v[s]); temperature T[s] if
 * thermal[s] == CLB_ISOTHERMAL, else zero normal gradient extrapolated to
 * second order.  At a corner the W/E wall's velocity is used and an
 * isothermal wall wins over an adiabatic one (W/E first). */
typedef struct {
    int32_t kind[4];
    double u[4], v[4];
    int32_t thermal[4];
    double T[4];
} clb_bc;

/* Physical setup (Eq. 38 groups; Sec. 3 model constants).  Fill with
 * clb_params_default and override.
 *   Ra, Da, Pr, J, Gamma, sigma : Eq. 38 groups and the heat capacity ratio
 *   Ma    : Mach number of Eq. 46 (0.1)
 *   L     : characteristic length in lattice units (<= 0: ny - 1)
 *   nu    : > 0 fixes the fluid viscosity directly (channel flows,
 *           1/s_v = 1/2 + J nu / c_s^2); <= 0 uses Eq. 46
 *   dT, T0, T_init : temperature difference, reference and initial value
 *   ax, ay: external acceleration a (Eq. 4, G = -g beta (T - T0) + a)
 *   varpi : D2Q5 parameter (c_sT^2 = varpi / 2), 1/4
 *   s3, s4: free relaxation rates of Eq. 15, 1.2 and 1.8
 *   sb    : bulk relaxation rate s_b of Eq. 15 (s+ = (s_b + s_v)/2,
 *           s- = (s_b - s_v)/2 act on k~20, k~02).  > 0: used as given.
 *           <= 0 (default): s_b = s_v as in Sec. 3, raised to 1.2 when
 *           s_v < 1.2 -- with s3 = 1.2, s4 = 1.8 the linearised scheme is
 *           unstable for s_b below 1.19, and Eq. 46 gives s_v < 1.2 at low
 *           Ra or large L.  s_b only sets the bulk viscosity, which does not
 *           enter the incompressible equations (Eqs. 1-3).
 *   forchheimer : 1 = Ergun F_phi of Eq. 5, 0 = F_phi = 0
 *   shift : 1 = porous shift matrices (Eqs. 14, 31); 0 = unit shifts, the
 *           non-orthogonal MRT limit named at the end of Sec. 2
 *   precision : CLB_F64, CLB_F16S or CLB_F16N
 * Fixed by the paper (Sec. 3): s_0 = s_1 = 1, zeta_T = zeta_e = zeta_nu = 1.
 * The permeability is K = Da L^2, uniform; F_phi(phi(x)) and every phi
 * factor are taken at the node. */
typedef struct {
    int32_t nx, ny;
    int32_t precision;
    int32_t forchheimer;
    int32_t shift;
    int32_t reserved;
    double Ra, Da, Pr, J, Gamma, sigma;
    double Ma, L, nu;
    double dT, T0, T_init;
    double ax, ay;
    double varpi, s3, s4;
    double sb;
} clb_params;

/* Lattice parameters the library derived from clb_params (read-only). */
typedef struct {
    double sb, sv, zeta_a;/* relaxation rates s_b, s_v (Eq. 15) and zeta_alpha (Eq. 28) */
    double nu, nu_e;      /* fluid and effective kinematic viscosity */
    double alpha, alpha_e;/* fluid and effective thermal diffusivity */
    double K, gbeta, L;   /* permeability, g*beta, characteristic length */
    int64_t pitch;        /* row pitch of the device arrays, in elements */
} clb_lattice;

typedef struct clb_handle clb_handle;

/* Paper defaults: 64 x 64, Ra 1e4, Da 1e-2, Pr 1, J = Gamma = sigma = 1,
 * Ma 0.1, dT 1, T0 = T_init = 0.5, varpi 1/4, s3 1.2, s4 1.8, sb automatic,
 * Forchheimer on, porous shift on, FP64. */
void clb_params_default(clb_params* p);

/* Cavity of Sec. 3.2: four no-slip walls, W at Th, E at Tc, S and N
 * adiabatic. */
void clb_bc_cavity(clb_bc* bc, double Th, double Tc);

/* Create a simulation.
 *   phi    : porosity per node, host, ny*nx values in (0, 1] (required)
 *   ay_row : optional host array of ny values; replaces p->ay row by row
 *            (a y-dependent external force such as Eq. 42); NULL = uniform
 *   bc     : boundary specification
 *   stream : cudaStream_t to issue all work on, or NULL
 * The state starts at rest: rho = 1, u = 0, T = T_init.  On failure *h is
 * NULL and clb_last_error(NULL) describes the problem.  Parameters and grid
 * size are validated (CLB_ERR_ARG) before phi is read and before any CUDA
 * call; the FP16 forms accept grids with 9 * ny * pitch < 2^31, pitch = nx
 * rounded up to a multiple of 64. */
int clb_init(clb_handle** h, const clb_params* p, const double* phi, const double* ay_row,
             const clb_bc* bc, void* stream);

/* Advance n >= 0 time steps (asynchronous on the handle's stream). */
int clb_step(clb_handle* h, int64_t n);

/* Reset the state to the local equilibria of the given host fields
 * (ny*nx each; rho and T required, ux/uy may be NULL for zero) and the
 * step counter to 0. */
int clb_set_fields(clb_handle* h, const double* rho, const double* ux, const double* uy,
                   const double* T);

/* Macroscopic fields at the current time level into caller-owned host
 * arrays of ny*nx values (any may be NULL): rho (Eq. 20), u (Eqs. 22-23),
 * T (Eq. 36); wall nodes report the imposed velocity and wall temperature.
 * Returns CLB_ERR_UNSTABLE if any value is not finite. */
int clb_macros(clb_handle* h, double* rho, double* ux, double* uy, double* T);

/* Same, into device arrays of ny*nx values each (any may be NULL); no
 * synchronisation and no finiteness check. */
int clb_macros_device(clb_handle* h, double* rho, double* ux, double* uy, double* T);

/* Mean Nusselt number of a wall (Sec. 3.2): Nu(s) = -L dT/dn / dT with the
 * one-sided second-order difference taken along x (W, E) or y (S, N),
 * averaged over the wall by the trapezoid rule; FP64 device reduction. */
int clb_nusselt(clb_handle* h, int32_t side, double* nu);

/* Relative change since the previous call (or since init / set_fields):
 * r_u = ||u^n - u^m||_2 / ||u^n||_2 and r_T likewise for T, over all nodes;
 * FP64 device reduction.  Returns CLB_ERR_UNSTABLE on non-finite fields. */
int clb_residual(clb_handle* h, double* r_u, double* r_T);

/* Time steps taken since init / set_fields / set_state. */
int64_t clb_time(const clb_handle* h);

/* Derived lattice parameters. */
int clb_lattice_params(const clb_handle* h, clb_lattice* out);

/* Checkpoint: bytes needed, copy out, copy in (same nx, ny, precision).
 * Resuming from a checkpoint reproduces the run bit for bit. */
size_t clb_state_bytes(const clb_handle* h);
int clb_get_state(clb_handle* h, void* buf, size_t bytes);
int clb_set_state(clb_handle* h, const void* buf, size_t bytes);

/* Wait for all work issued on the handle's stream.  Returns CLB_ERR_TIMEOUT
 * (once; the flag is cleared) if a bounded wait of the TMA-fed FP16N step
 * expired since the last check -- the state is then invalid.  clb_macros and
 * clb_nusselt report the same. */
int clb_sync(clb_handle* h);

/* FP16N form: the interior rows (1 .. ny - 2) of each step run a persistent
 * kernel fed by bulk tensor copies (TMA) into shared memory, the edge nodes
 * the per-thread kernel; the two paths give the same bits (the collision of
 * Eqs. 11-18 and 28-34 is the same code, only the loads differ).  This
 * selects the path: enable = 1 (available for FP16N with ny >= 3 and a
 * driver that encodes the tensor maps) or 0 (the default: the step is bound
 * by its arithmetic, and the per-thread kernel measured faster).
 * CLB_ERR_ARG when enabling it is not possible.  Drops the captured step
 * graphs. */
int clb_set_tma(clb_handle* h, int32_t enable);

/* Failure-path check of the TMA-fed step: runs one step of it into the idle
 * buffer (time and state unchanged) in which every CTA's first wait is on a
 * barrier that nothing completes, bounded by limit_cycles (>= 1) SM clock
 * cycles; a CTA whose wait expired waits for its own copies (with the normal
 * bound) before it exits.  Then reports like clb_sync: CLB_ERR_TIMEOUT when
 * the expiry was detected and reported (the expected result). */
int clb_tma_selftest(clb_handle* h, int64_t limit_cycles);

void clb_destroy(clb_handle* h);

/* ---------------------------------------------------------------- batches
 * A batch advances ncase independent simulations (uneven grids, their own
 * parameters, porosity and walls) with one launch per step.  All cases share
 * precision, shift and forchheimer.  Arrays of per-case inputs are indexed
 * by case; phi[c] points to case c's ny*nx host porosity.  Steps advance
 * every active case; clb_batch_set_active takes a flag per case (retired
 * cases keep their state and stop advancing; re-activated, they resume
 * from that state).  clb_batch_tune times each of the 12 candidate tilings
 * for `steps` steps (the cases advance meanwhile) and keeps the fastest;
 * *chosen receives its index, choice = 3 * shape + p: shapes 0-3 are blocks
 * of 64x2, 32x4, 16x8 and 8x16 threads (each thread one node pair in the
 * FP16 forms, one node in FP64), p selects 4, 16 or 64 tiles per CTA.
 * clb_batch_set_tiling fixes a choice without timing.  Results do not
 * depend on the tiling.  Other conventions as for
 * the single-case entry points.  The paper has no batched form; this is the
 * data-parallel way to run parameter studies such as its Table 1. */
typedef struct clb_batch clb_batch;
/* Launch modes of a batch (clb_batch_set_mode):
 *   CLB_BATCH_GRAPH      : (the default) one launch per step, replayed
 *                          from CUDA graphs of 32 steps;
 *   CLB_BATCH_PERSISTENT : one cooperative launch (all blocks resident)
 *                          per 32 steps, itself captured in a CUDA graph,
 *                          whose steps are separated by a grid barrier; the
 *                          blocks claim tiles from a counter.  If the
 *                          device cannot co-schedule the grid, the batch
 *                          falls back to CLB_BATCH_GRAPH.  A
 *                          barrier wait is bounded (about 2 s); if it
 *                          expires the launch stops, and the next call that
 *                          waits for the batch (clb_batch_sync,
 *                          clb_batch_nusselt, clb_batch_macros,
 *                          clb_batch_set_mode) returns CLB_ERR_TIMEOUT.
 * Both modes give identical results. */
enum { CLB_BATCH_GRAPH = 0, CLB_BATCH_PERSISTENT = 1 };
int clb_batch_init(clb_batch** b, int32_t ncase, const clb_params* p, const double* const* phi, const clb_bc* bc,
                   void* stream);
int clb_batch_step(clb_batch* b, int64_t n);
int clb_batch_set_active(clb_batch* b, const int32_t* active);
int clb_batch_tune(clb_batch* b, int32_t steps, int32_t* chosen);
int clb_batch_set_tiling(clb_batch* b, int32_t choice);
int clb_batch_set_mode(clb_batch* b, int32_t mode);
/* Failure-path self-test of the persistent mode's grid barrier: runs one
 * persistent step whose barrier waits for one block more than the launch
 * has, bounded by limit_cycles SM clock cycles (1 .. 4e9).  The wait
 * expires, every block returns, and the call reports CLB_ERR_TIMEOUT; the
 * step wrote only the buffer not in use, so the batch's state and time are
 * unchanged and the batch stays usable. */
int clb_batch_barrier_selftest(clb_batch* b, int64_t limit_cycles);
/* Mean Nusselt number of `side` for every case (host array of ncase values). */
int clb_batch_nusselt(clb_batch* b, int32_t side, double* nu);
/* Macroscopic fields of case c (host arrays of that case's ny*nx values). */
int clb_batch_macros(clb_batch* b, int32_t c, double* rho, double* ux, double* uy, double* T);
/* Nodes updated per batch step (active cases), and steps taken. */
int64_t clb_batch_nodes(const clb_batch* b);
int64_t clb_batch_time(const clb_batch* b);
int clb_batch_sync(clb_batch* b);
const char* clb_batch_last_error(const clb_batch* b);
void clb_batch_destroy(clb_batch* b);

/* Allocation-free Nusselt reduction.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code that
 * runs inside another framework's memory pool, which may already hold
 * nearly all device memory and must see every allocation, and loops where
 * an allocation's implicit device-wide synchronisation cannot be afforded.
 *
 * Computes the same mean Nusselt number as clb_nusselt (Nu = -L dT/dn / dT,
 * one-sided second-order difference, trapezoid rule along the wall) from a
 * temperature field the caller already holds on the device.
 *   T      : device pointer, ny*nx FP64 values, (ny, nx) row-major (for
 *            instance filled by clb_macros_device); read only
 *   side   : CLB_W, CLB_E, CLB_S or CLB_N
 *   L, dT  : characteristic length and temperature difference (> 0)
 *   nu     : device pointer to one double, written with the result
 *   stream : cudaStream_t the two kernels run on (NULL: legacy stream)
 * Asynchronous: nu holds the result once the stream reaches it.
 * Scratch: a fixed array of CLB_STATIC_MAX_PARTIALS doubles (8 KiB) in the
 * library's device memory, present on every GPU that loads the library
 * until the process exits, so walls longer than CLB_STATIC_MAX_WALL nodes
 * are rejected with CLB_ERR_ARG.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  A call looks up the array's device address
 * in the current context (cudaGetSymbolAddress, which allocates nothing)
 * and caches it per device; a call whose stream is being captured uses
 * that cache instead, so make one call on each device before any stream
 * capture (a first call during capture fails with CLB_ERR_ARG).  All calls
 * share the one array:
 * calls whose kernels can overlap on the GPU (different streams without
 * ordering between them) race and give wrong results.  Every slot a call
 * reads it has written itself, so nothing needs clearing between calls.
 * Errors: CLB_ERR_ARG (bad pointer, side or size), CLB_ERR_CUDA (also when
 * a CUDA error from earlier work was already pending: it is reported and
 * left in place); message in clb_last_error(NULL). */
#define CLB_STATIC_MAX_PARTIALS 1024
#define CLB_STATIC_MAX_WALL (CLB_STATIC_MAX_PARTIALS * 256)
int clb_nusselt_field_static(const double* T, int32_t nx, int32_t ny, int32_t side, double L, double dT,
                             double* nu, void* stream);

/* Check of the FP64 step's own reciprocal and square root (hardware
 * estimates refined by one third-order Newton-Raphson step) against CUDA's
 * IEEE division and sqrt.  For each of the n device values x[i] > 0 it
 * writes four device values out[4i .. 4i+3] = (step's 1/x, IEEE 1/x,
 * step's sqrt(x), IEEE sqrt(x)); asynchronous on `stream`.  A diagnostic:
 * the paper has no counterpart.  Errors: CLB_ERR_ARG, CLB_ERR_CUDA
 * (message in clb_last_error(NULL)). */
int clb_fp64_special_check(const double* x, int64_t n, double* out, void* stream);

/* Last error message of h, or of the calling thread's last failed
 * clb_init when h is NULL. */
const char* clb_last_error(const clb_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* CLB_H */
