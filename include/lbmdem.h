/*
 * lbmdem.h -- C ABI of the GB300 (sm_103a) coupled lattice-Boltzmann /
 * discrete-element time step of Cheng, Luding, Rivas, Harting, Magnanimo,
 * "Hydro-micromechanical modeling of wave propagation in saturated granular
 * media" (arXiv 1808.08921).
 *
 * One call of lbm_dem_step advances the state by n coupled steps.  Each
 * step, on the GPU and in this order:
 *   1. map update: re-test the nodes near sphere surfaces against the
 *      current sphere positions and convert nodes that were covered or
 *      uncovered (Section 2.3, Eqs. 16-17);
 *   2. BGK collide + stream of the D3Q19 fluid (Section 2.1, Eqs. 3-8);
 *   3. moving-wall half-way bounce-back on every fluid-solid link and the
 *      hydrodynamic force and torque on each sphere (Eqs. 14-15, 18-19);
 *      on even steps 2 and 3 can run as one kernel (link_mode below);
 *   4. the pressure inlet with the oscillating density (Section 2.4, Zou-He
 *      form for D3Q19, Eq. 25, Table 2) and the outlet;
 *   5. K velocity-Verlet substeps of the spheres with Hertz normal and
 *      incremental Mindlin tangential contacts under a Coulomb cap
 *      (Section 2.2, Eqs. 9-12), driven by the mean of the hydrodynamic
 *      force and torque of this and the previous step.
 * Lattice units throughout: dx = dt = 1, c_s^2 = 1/3 (Section 3).
 *
 * Conventions
 *  - Return value: 0 on success, a negative LBMDEM_ERR_* code otherwise;
 *    lbm_dem_last_error() gives a one-line description.
 *  - Host arrays are owned by the caller; the library copies in and out
 *    and keeps no host pointer.  Device memory is owned by the context.
 *  - Host inputs and outputs are FP64 whatever the storage precision.
 *  - Lattice arrays are C-order [x][y][z] with x the propagation axis
 *    (inlet at x = 0); vector fields are [3][x][y][z].  y and z are
 *    periodic.  Particle arrays are [n][3] ([n][4] for quaternions w,x,y,z).
 *  - All work is issued on the context's CUDA stream.  lbm_dem_step returns
 *    once the work is queued, except that with mobile spheres it reads a
 *    few bytes back at chunk boundaries to decide re-layouts (see below).
 *    Device-side failures (NaN, skin exceeded, capacity) are latched in a
 *    status word and reported by the next lbm_dem_status / read call.
 *  - Not thread-safe: one host thread per context at a time.
 */
#ifndef LBMDEM_H
#define LBMDEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define LBMDEM_OK 0
#define LBMDEM_ERR_INVALID_ARG (-1) /* a parameter or input array is out of range   */
#define LBMDEM_ERR_OOM (-2)         /* device allocation failed                      */
#define LBMDEM_ERR_CUDA (-3)        /* a CUDA runtime call failed                    */
#define LBMDEM_ERR_UNSTABLE (-4)    /* NaN/Inf in the fluid or the spheres           */
#define LBMDEM_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up            */
#define LBMDEM_ERR_STATE (-6)       /* call out of order (e.g. step before packing)  */
#define LBMDEM_ERR_CAPACITY (-7)    /* a device list overflowed (flips, neighbours)  */
#define LBMDEM_ERR_SKIN (-8)        /* a sphere moved beyond the re-layout skin      */
#define LBMDEM_ERR_NO_DEVICE (-9)   /* no sm_103-class CUDA device                   */

/* distribution storage (the arithmetic is FP32 in every case) */
#define LBMDEM_F32 0      /* f_i - w_i rho_f stored as FP32                  */
#define LBMDEM_BF16_DEV 1 /* f_i - w_i rho_f stored as BF16                 */
#define LBMDEM_F16_DEV 2  /* f_i - w_i rho_f stored as FP16 scaled by 2^12   */

/* x boundaries */
#define LBMDEM_INLET_PRESSURE 0 /* Section 2.4 pressure inlet at x = 0 with rho(t)   */
#define LBMDEM_X_WALL 1         /* resting half-way wall at x = -1/2                  */
#define LBMDEM_X_PERIODIC 2     /* periodic in x (settling-sphere box, Section 3.1)   */
#define LBMDEM_OUT_ZERO_GRAD 0  /* outlet copies the upstream node's unknowns         */
#define LBMDEM_OUT_RHO_F 1      /* outlet locked to rho_f (Section 3.2)               */
#define LBMDEM_OUT_WALL 2       /* resting half-way wall at x = nx - 1/2              */

/* source waveforms, Eq. 25 and Table 2 (RICKER is an addition) */
#define LBMDEM_SINE 0   /* rho_f + rho' sin(w t)                       */
#define LBMDEM_COSINE 1 /* rho_f + rho' (1 - cos(w t))                 */
#define LBMDEM_STEP 2   /* rho_f + rho'                                */
#define LBMDEM_RICKER 3 /* rho_f + rho' (1 - 2a^2) exp(-a^2), a = pi f (t - t0), f = w / 2pi */

typedef struct lbmdem_ctx lbmdem_ctx; /* opaque, library-owned */

typedef struct {
    int32_t nx, ny, nz;   /* lattice; nx = propagation axis; nx <= 4096, ny, nz <= 1024 */
    double tau;           /* BGK relaxation time, Eq. 4; must exceed 0.5              */
    double rho_f;         /* mean fluid density, Eq. 6                                */
    int32_t storage;      /* LBMDEM_F32 | LBMDEM_BF16_DEV | LBMDEM_F16_DEV            */
    int32_t inlet;        /* LBMDEM_INLET_PRESSURE | LBMDEM_X_WALL | LBMDEM_X_PERIODIC */
    int32_t outlet;       /* LBMDEM_OUT_*; ignored when x is periodic                 */
    int32_t dem_substeps; /* K >= 1 velocity-Verlet substeps per LBM step             */
    double E_p, nu_p;     /* contact Young modulus and Poisson ratio, Eqs. 11-12      */
    double mu;            /* Coulomb friction coefficient, Eq. 12                     */
    double rho_p;         /* solid density: m = rho_p 4/3 pi R^3, I = 2/5 m R^2       */
    double body_force[3]; /* F_g of Eq. 9 on every free sphere                        */
    int32_t probe_x;      /* plane whose fluid-mean density is recorded; -1 = off     */
    int32_t lbm_on;       /* 1 = coupled step; 0 = spheres only (dry packing)         */
    double skin;          /* lattice re-layout skin (lu), > 0; 0 picks 0.25           */
    double dem_skin;      /* neighbour-list skin (lu), > 0; 0 picks 0.5               */
    int32_t monitor_every;/* accumulate FP64 mass/momentum every M steps; 0 = off     */
    int32_t graph_steps;  /* steps per captured CUDA graph (even); 0 picks 16         */
    int32_t max_flips;    /* node conversions per step the scratch holds; 0 = auto    */
    int32_t tile;         /* threads per block of collide+stream: 64 (0), 128 or 256  */
    int32_t device;       /* CUDA device ordinal                                      */
    int32_t link_mode;    /* 2: an even step's links (Eqs. 14-15, 18-19) are taken inside
                             its collide+stream kernel, an odd step's by the link kernel;
                             1: the link kernel every step; 0 (default): 2 with FP32
                             storage and a largest sphere radius of 8 lattice units
                             or more, else 1.  Boxes narrower than 2 (R + skin + 2)
                             on a periodic axis, and packings of more than 16383
                             spheres, always take 1.  Same results up to FP32
                             summation order.                                          */
    void* cuda_stream;    /* cudaStream_t to issue on; NULL = a stream of the context */
} lbmdem_params;

/* Fill *p with the defaults above (tau 0.8, rho_f 1, K 10, Table 1 solids,
 * mu 0.3, zero-gradient outlet, sine source off).  Never fails. */
void lbm_dem_default_params(lbmdem_params* p);

/* Create a context: validates p, allocates nothing lattice-sized yet.
 * *out receives the context or NULL.  Errors: INVALID_ARG, NO_DEVICE, CUDA. */
int lbm_dem_init(const lbmdem_params* p, lbmdem_ctx** out);

/* Place n spheres (Section 2.2): centres X[n][3] (lattice units, any value;
 * y, z are wrapped periodically), radii R[n] > 0, velocities V[n][3] and
 * angular velocities Omega[n][3] (NULL = 0), fixed[n] (NULL = all free;
 * fixed spheres keep V = Omega = 0, Section 4.1).  Resets the fluid to rest
 * at rho_f, the time to t = 0 and the probe trace; paints the solid map
 * (Section 2.3) and builds the compact lattice, the surface and link lists,
 * the neighbour list and the initial contact forces on the GPU.
 * n = 0 gives a pure fluid.  Errors: INVALID_ARG (R <= 0, NaN, R + skin not
 * below half a periodic box, 2 R + dem_skin wider than a periodic box, pair
 * overlap >= min R), OOM, CUDA. */
int lbm_dem_set_packing(lbmdem_ctx* c, int32_t n, const double* X, const double* R,
                        const double* V, const double* Omega, const uint8_t* fixed);

/* Oscillating source of Eq. 25 / Table 2 at the inlet: rho(t) = rho_f +
 * amplitude * shape(omega t) while t <= t_n (t_n < 0: forever), rho_f after.
 * The write that produces state t+1 uses rho(t+1).  Default: amplitude 0. */
int lbm_dem_set_pressure_source(lbmdem_ctx* c, int32_t waveform, double amplitude,
                                double omega, int64_t t_n, double t0);

/* Advance n >= 0 coupled steps.  Errors: STATE (no packing), CUDA, and the
 * latched device status (UNSTABLE, SKIN, CAPACITY) when it is read back. */
int lbm_dem_step(lbmdem_ctx* c, int64_t n);

/* Rebuild the compact lattice, the surface and link lists and the neighbour
 * lists around the current sphere positions.  lbm_dem_step does this by
 * itself when a sphere has moved half its skin; the state must sit between
 * an odd and an even step (t even).  Errors: STATE (t odd or no packing). */
int lbm_dem_relayout(lbmdem_ctx* c);

/* Synchronise the stream and return the latched device status (0 or an
 * LBMDEM_ERR_* code); does not clear it. */
int lbm_dem_status(lbmdem_ctx* c);

/* Macroscopic fields of the current state (Eq. 7): rho[nx*ny*nz],
 * u[3*nx*ny*nz], solid[nx*ny*nz] (1 = solid); any pointer may be NULL.
 * Solid nodes report rho = u = 0 (Section 4.2).  Synchronises. */
int lbm_dem_read_fields(lbmdem_ctx* c, double* rho, double* u, uint8_t* solid);

/* Sphere state: X, V, Omega [n][3], quat [n][4], and the hydrodynamic force
 * and torque sums of the last step (Eqs. 18-19) F_hyd, T_hyd [n][3] (the
 * spheres are driven by the mean of the last two); NULL skips.
 * Synchronises. */
int lbm_dem_read_particles(lbmdem_ctx* c, double* X, double* V, double* Omega, double* quat,
                           double* F_hyd, double* T_hyd);

/* The same read-out without any allocation (the paper has no counterpart:
 * this serves callers that cannot allocate device memory at read time, such
 * as one whose device memory is committed to the lattice state, where a
 * cudaMalloc fails, or one that must not take the device-wide
 * synchronisation of cudaFree while other streams are busy).  Same
 * arguments, layouts and results as lbm_dem_read_particles; the values are
 * staged in a fixed device array of the library (19 doubles per sphere,
 * 9.5 MiB) instead of a buffer allocated per call.
 *  - At most 65536 spheres: a larger packing returns LBMDEM_ERR_CAPACITY
 *    with a message, and nothing is read.
 *  - The first call on a device looks up the array's device address (once
 *    per device and CUDA context, with that device current; again after the
 *    device's context was reset or replaced); make that first call before
 *    any stream capture on the device.
 *  - The array is shared by all calls on a device and keeps the last call's
 *    contents (every value copied out is written by the same call).  Calls
 *    whose GPU work overlaps (two contexts of one device used from two host
 *    threads) race on it.
 * Synchronises the context stream. */
int lbm_dem_read_particles_noalloc(lbmdem_ctx* c, double* X, double* V, double* Omega,
                                   double* quat, double* F_hyd, double* T_hyd);

/* Plane averages of the current state over the fluid nodes of every x plane
 * (the space-time data whose discrete Fourier transform gives the dispersion
 * relation, Section 3.2): rho[nx] = mean density, jx[nx] = mean
 * rho u_x (Eq. 7); NaN for a plane without fluid; either pointer may be NULL.
 * Synchronises. */
int lbm_dem_read_plane_means(lbmdem_ctx* c, double* rho, double* jx);

/* Probe trace: trace[k] = mean density over the fluid nodes of plane probe_x
 * entering step k (after that step's map update), k = 0 .. len-1.  Copies
 * min(len, max_len) values; *len receives the full length.  Synchronises. */
int lbm_dem_read_probe(lbmdem_ctx* c, double* trace, int64_t max_len, int64_t* len);

/* FP64 totals over the fluid accumulated at the last monitored step:
 * out[0] = sum rho, out[1..3] = sum rho u, out[4] = max |u|, out[5] = step. */
int lbm_dem_read_monitors(lbmdem_ctx* c, double out[6]);

/* Counters of the current layout: out[0] lattice nodes, [1] stored nodes,
 * [2] fluid nodes now, [3] surface nodes tracked for conversion, [4] fluid-
 * solid link records (links fixed until the next re-layout plus the links
 * whose solid end is re-decided every step), [5] neighbour-list entries,
 * [6] time step t, [7] re-layouts done, [8] node conversions so far, [9]
 * kernels launched by lbm_dem_step so far.  Synchronises. */
int lbm_dem_read_counters(lbmdem_ctx* c, int64_t out[10]);

/* Per-kernel timing with CUDA events on the context stream.  enable = 1
 * brackets every launch group of the following steps with event pairs;
 * lbm_dem_read_timing synchronises and returns, per group, the summed
 * milliseconds and the number of launches since the last read:
 * [0] collide+stream of the odd steps, [1] link kernel, [2] map update,
 * [3] inlet/outlet, [4] DEM substeps, [5] collide+stream of the even steps
 * (with the step's links where the even steps take them there: link_mode 2,
 * or 0 with FP32 storage). */
int lbm_dem_set_timing(lbmdem_ctx* c, int32_t enable);
int lbm_dem_read_timing(lbmdem_ctx* c, double ms[6], int64_t launches[6]);

/* Gradient of the probe-plane pressure misfit for a fixed packing (every
 * sphere fixed; the paper's pressure p = c_s^2 rho, Section 3, at the probe
 * plane of Section 3.2): runs `steps` coupled steps from the current state
 * (t even), L = sum_k (p(k) - target[k])^2 over the probe trace entries
 * p(k) = c_s^2 * trace[t0 + k], k = 0 .. steps-1, and the exact gradient of
 * that discrete L with respect to tau (Eq. 4) and the source amplitude rho'
 * (Eq. 25) by the adjoint of the step (hand-written reverse kernels), with
 * the populations checkpointed every `every` (even) steps and each segment
 * recomputed once.  Writes *loss, *dL_dtau, *dL_damp and, if not NULL,
 * trace_out[steps] = p(k).  Leaves the context at t0 + steps.  Device memory:
 * the checkpoints (steps / every population copies) and `every` FP32
 * snapshots.  Errors: INVALID_ARG, STATE (mobile spheres, no probe, odd t),
 * OOM, CUDA. */
int lbm_dem_adjoint(lbmdem_ctx* c, int64_t steps, int32_t every, const double* target, double* loss,
                    double* dL_dtau, double* dL_damp, double* trace_out);

/* The same misfit's gradient under a smooth surrogate of the coupling, with
 * respect to the sphere centres as well (not in the paper: with the binary
 * solid map of Eqs. 14-15 the misfit is piecewise constant in the centres,
 * so this entry point differentiates a surrogate from the family Section 1
 * names as the alternative, Noble and Torczynski's collision weighted by
 * the solid fraction of each cell).  Model: every node carries populations;
 * solid fraction eps = 1 - prod_p (1 - S(R_p - |x - X_p| + 1/2)), S the cubic
 * smoothstep (x ends fluid); collision g*_i = g_i - (1 - B)/tau (g_i - g^eq_i)
 * + B (g_opp(i) - g_i + w_i drho - g^eq_opp(i)), B = eps (tau - 1/2) /
 * ((1 - eps) + (tau - 1/2)); streaming, inlet and outlet as in the coupled
 * step; probe p(k) = c_s^2 times the mean density over every node of plane
 * probe_x.  The surrogate runs from rest at rho_f with the source at time 0
 * for `steps` steps on its own dense lattice (the context's state is left
 * unchanged), checkpointed every `every` (>= 1) steps: L = sum_k (p(k) -
 * target[k])^2, dL/dtau, dL/drho' and dL_dX[n][3] (NULL skips), trace_out
 * [steps] = p(k) (NULL skips); with all three gradient pointers NULL only
 * the forward run and the loss are computed.  Device memory, released on
 * return: (steps/every + every + 6) 19 N FP32 values plus N FP64,
 * N = nx ny nz (4 19 N FP32 for the forward alone).
 * Errors: INVALID_ARG, STATE (mobile spheres, no probe, resting-wall inlet),
 * OOM, CUDA. */
int lbm_dem_adjoint_psm(lbmdem_ctx* c, int64_t steps, int32_t every, const double* target, double* loss,
                        double* dL_dtau, double* dL_damp, double* dL_dX, double* trace_out);

/* ---- Batched columns ------------------------------------------------------
 * The paper's study of the acoustic source (Section 4.4: input waveforms and
 * frequencies of Table 2) runs one column per source; a batch advances many
 * such independent contexts (columns of any length, packing and source)
 * together, each by its own number of steps, in ONE launch of one CUDA
 * graph: each column is a parallel branch holding a device-side WHILE loop
 * (conditional graph node) over pairs of coupled steps and, for an odd
 * count, an IF node with the last step.  A control kernel ends a column's
 * loop when its steps are done, when its device status latches an error, or
 * when the batch's time limit (lbm_dem_batch_set_time_limit) has passed on
 * the GPU clock, which latches LBMDEM_ERR_TIMEOUT for that column.  The host
 * takes no part between launch and end: re-layout checks of mobile columns
 * run before the launch only (a sphere that moves beyond its skin inside the
 * launch latches LBMDEM_ERR_SKIN).  Per-kernel timing is not recorded inside
 * the batch graph.  The contexts stay owned by the caller and must outlive
 * the batch; use no context elsewhere while a batch call runs. */
typedef struct lbmdem_batch lbmdem_batch; /* opaque, library-owned */

/* Group n contexts (distinct, all on one device, each after set_packing).
 * Errors: INVALID_ARG (NULL, duplicates, mixed devices), STATE, CUDA. */
int lbm_dem_batch_create(lbmdem_ctx* const* cols, int32_t n, lbmdem_batch** out);

/* Wall-clock limit of every following lbm_dem_batch_step launch, in seconds
 * of GPU time from the launch (0 = none, the default).  A column whose loop
 * is still running when it passes stops between two steps and latches
 * LBMDEM_ERR_TIMEOUT; the other columns stop the same way.
 * Errors: INVALID_ARG (negative or not finite). */
int lbm_dem_batch_set_time_limit(lbmdem_batch* b, double seconds);

/* Advance column i by steps[i] >= 0 coupled steps in one graph launch
 * (asynchronous like lbm_dem_step; the graph is built for the call, after a
 * re-layout check and, for a column at an odd step, one single step).
 * Errors: INVALID_ARG, a column's latched status, CUDA. */
int lbm_dem_batch_step(lbmdem_batch* b, const int64_t* steps);

/* Wait for the batch and every column; returns the first column status
 * (0, or e.g. LBMDEM_ERR_TIMEOUT); a column whose loop stopped early is left
 * at the step it reached. */
int lbm_dem_batch_sync(lbmdem_batch* b);

/* Graph launches issued by lbm_dem_batch_step so far (-1 for NULL). */
int64_t lbm_dem_batch_graph_launches(const lbmdem_batch* b);

const char* lbm_dem_batch_last_error(const lbmdem_batch* b);

/* Release the batch's stream, events and graph (not the contexts). */
void lbm_dem_batch_destroy(lbmdem_batch* b);

/* One-line description of the last error on this context ("" if none). */
const char* lbm_dem_last_error(const lbmdem_ctx* c);

/* Release all device memory and the owned stream.  NULL is a no-op. */
void lbm_dem_destroy(lbmdem_ctx* c);

#ifdef __cplusplus
}
#endif
#endif /* LBMDEM_H */
