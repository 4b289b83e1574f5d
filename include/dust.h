/*
 * dust.h - C interface of the GB300 dust drag-coupling library.
 *
 * One call of dust_step() performs, for every grain, the particle part of
 * one hybrid time step of Mignone, Flock & Vaidya, "A Particle Module for
 * the PLUTO Code: III - Dust" (arXiv:1908.10793):
 *
 *   - gather of gas density and momentum-like velocity at the grain's
 *     half-step position with the paper's weights (Eq. Delta_vp; Sec. 3.4
 *     Eqs. weight, b0, b1, CIC/TSC_cylindrical; App. C);
 *   - the exponential-midpoint drift-kick-drift push (Eq. exp_midpoint,
 *     Eqs. phi1, h1, kick_modified; App. B.1 shearing box, App. B.2
 *     cylindrical and spherical);
 *   - deposition of the drag back-reaction on the grid (Eq.
 *     dust_feedback_final), in momentum and energy, into 64-bit fixed-point
 *     accumulators, and optionally its application to the gas momentum (the
 *     corrector term of the RK2 step, Sec. 3.1).
 *
 * Conventions
 *   - Zones are indexed i + n[0] * (j + n[1] * k) (Sec. 3.1, cell index
 *     i = (i,j,k)); a direction with n[d] == 1 is not gridded (2-D runs).
 *   - Grain coordinates q = (x1, x2, x3): Cartesian (x,y,z); cylindrical
 *     (R, phi, z); spherical (r, theta, phi).  Velocities passed in and out
 *     are physical components; internally the library evolves the
 *     momentum-like variables of Sec. 2.2 (l_phi = R v_phi; l_theta = r
 *     v_theta, l_phi = r sin(theta) v_phi).  In the shearing box with orbital
 *     advection (fargo = 1) velocities are the residual v' = v + q Omega x e_y
 *     (Sec. 2.1).
 *   - Every call returns an int status: DUST_OK (0) or a negative DUST_E*
 *     code; dust_last_error() gives a message.
 *   - Memory: the library owns all device memory of a context.  Inputs are
 *     copied in; getters copy into caller buffers.  A `mem` argument says
 *     whether caller pointers are host (DUST_MEM_HOST) or device
 *     (DUST_MEM_DEVICE) memory; device pointers must be valid on the
 *     context's device and their contents complete with respect to the
 *     context's stream.
 *   - All work is enqueued on the context's stream.  dust_step() does not
 *     wait for the GPU; dust_sync() waits and returns the device status
 *     words raised since the previous dust_sync().
 *   - One context must not be used from two host threads at the same time.
 */
#ifndef DUST_H
#define DUST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DUST_OK 0
#define DUST_EINVAL (-1)    /* bad argument, NaN/Inf input, size out of range   */
#define DUST_ENOMEM (-2)    /* device allocation failed                          */
#define DUST_ECUDA (-3)     /* a CUDA runtime call failed                        */
#define DUST_ECFL (-4)      /* a grain moved more than 1.8 zones in one step (Eq. particles_dt); results are still correct */
#define DUST_EOVERFLOW (-5) /* a fixed-point deposit piece exceeded 2^52 quanta */
#define DUST_ENAN (-6)      /* a NaN/Inf appeared on the device                  */
#define DUST_ETIMEOUT (-7)  /* a bounded device wait gave up; results are void  */
#define DUST_ESTATE (-8)    /* call out of order (e.g. dust_step before data)    */

/* ---- enumerations ------------------------------------------------------ */
enum { DUST_CARTESIAN = 0, DUST_SHEARING_BOX = 1, DUST_CYLINDRICAL = 2, DUST_SPHERICAL = 3 };
enum { DUST_BC_PERIODIC = 0, DUST_BC_OUTFLOW = 1 };
/* weighting factors (Sec. 3.4): DUST_WEIGHT_CIC and DUST_WEIGHT_TSC are the
 * b0 / b1 shapes integrated over each zone with the geometry's measure (Eqs.
 * weight, shape_curv; App. C).  DUST_WEIGHT_VOLUME is the traditional volume
 * weighting the paper compares against (Eq. CIC_vol): linear interpolation in
 * the volume coordinate (R^2, r^3, -cos theta) between the centres of the two
 * zones around the grain, with a ghost centre one edge-zone width beyond each
 * end of the grid; in directions whose volume coordinate is the coordinate
 * itself (all of them in Cartesian and shearing-box geometries) it is CIC.
 * Volume weighting runs on the tiled and per-grain kernels and computes its
 * weights in double precision. */
enum { DUST_WEIGHT_CIC = 0, DUST_WEIGHT_TSC = 1, DUST_WEIGHT_VOLUME = 2 };
/* stopping time: DUST_TAU_CONST tau_s = value; DUST_TAU_STOKES tau_s =
 * value / Omega_K (Omega_K = sqrt(GM / R^3) at the cylindrical radius of the
 * half-step position; shearing box: value / Omega); DUST_TAU_EPSTEIN tau_s =
 * value / rho_gathered (Epstein regime, Sec. 2: tau_s ~ 1/rho). */
enum { DUST_TAU_CONST = 0, DUST_TAU_STOKES = 1, DUST_TAU_EPSTEIN = 2 };
/* DUST_FP64: all arithmetic in double precision.  DUST_MIXED: positions in
 * double precision, momentum-like variables, gas fields, weights, gather and
 * push in single precision, deposit in 64-bit fixed point. */
enum { DUST_FP64 = 0, DUST_MIXED = 1 };
/* particle pusher: the exponential midpoint rule (Sec. 3.2.2, default) or the
 * semi-implicit drift-kick-drift scheme with the linearised drag kick
 * (Sec. 3.2.1; Cartesian and shearing-box geometries only). */
enum { DUST_PUSHER_EM = 0, DUST_PUSHER_SEMI_IMPLICIT = 1 };
enum { DUST_MEM_HOST = 0, DUST_MEM_DEVICE = 1 };
/* kernel choice.  DUST_KERNEL_PER_GRAIN: one thread per grain, every grain
 * quantises its own 27 x 4 deposit pieces into global 64-bit atomics (the
 * reference kernel; its integer grid does not depend on the store order).
 * DUST_KERNEL_TILED: one block per tile of zones, gas stencil and deposit in
 * shared memory, deposit quantised once per run (grains of one zone sharing
 * their half-step host zone).  DUST_KERNEL_SLAB (mixed precision, x gridded):
 * like the tiled kernel, but three lanes own one zone and keep its stencil
 * and its deposit in registers.  DUST_KERNEL_AUTO: the slab kernel where it
 * applies, else the tiled kernel. */
enum { DUST_KERNEL_AUTO = 0, DUST_KERNEL_PER_GRAIN = 1, DUST_KERNEL_TILED = 2, DUST_KERNEL_SLAB = 3 };

/* status flag bits returned in dust_stats.flags */
#define DUST_FLAG_NAN 1
#define DUST_FLAG_OVERFLOW 2
#define DUST_FLAG_CFL 4
#define DUST_FLAG_WRAP 8   /* a grain moved more than one period in one step */
#define DUST_FLAG_TIMEOUT 16 /* a bounded device wait gave up (a tile was skipped) */
#define DUST_FLAG_SPECIES 32 /* a grain's species index was >= n_species; the grain was left unchanged */

/* ---- descriptors -------------------------------------------------------- */
typedef struct dust_geometry {
    int kind;             /* DUST_CARTESIAN .. DUST_SPHERICAL                   */
    int fargo;            /* shearing box: 1 = orbital-advection (residual)
                             form, Eq. FARGO_SB_p; 0 = standard, Eq. standard_SB_p */
    double omega;         /* shearing box angular velocity Omega                */
    double q;             /* shearing box shear parameter q (3/2: Keplerian)    */
    double gm;            /* cylindrical / spherical point-mass GM (0 = none)   */
    int vertical_gravity; /* shearing box: -Omega^2 z term; cylindrical: z
                             component of the point-mass gravity                */
} dust_geometry;

typedef struct dust_grid {
    int n[3];              /* zones per direction, >= 1                         */
    const double *edges[3];/* host arrays of n[d] + 1 strictly increasing zone
                              edges; copied by dust_create                      */
    int bc[3];             /* DUST_BC_PERIODIC or DUST_BC_OUTFLOW per direction;
                              shearing-box x is shear-periodic when periodic    */
} dust_grid;

typedef struct dust_species {
    double mass;           /* grain (macro-particle) mass m_p                   */
    int tau_mode;          /* DUST_TAU_*                                        */
    double tau_value;      /* tau_s, St or the Epstein constant (may be +inf)  */
} dust_species;

typedef struct dust_options {
    int precision;         /* DUST_FP64 or DUST_MIXED                           */
    int weight;            /* DUST_WEIGHT_CIC, DUST_WEIGHT_TSC or DUST_WEIGHT_VOLUME */
    int feedback_apply;    /* 1: add the deposit to the gas momentum each step  */
    double quantum;        /* fixed-point quantum of the deposit (momentum
                              units); 0 = the default: 2^-44 * (largest
                              species mass) with DUST_FP64 (a grain's velocity
                              change of up to 256 code units per step stays
                              below 2^52 quanta, and zone sums of a few
                              thousand pieces fit int64), 2^-40 * (largest
                              species mass) with DUST_MIXED (still finer than
                              the single-precision sums it rounds)          */
    void *stream;          /* cudaStream_t to enqueue on; NULL = own stream     */
    int sort_interval;     /* re-sort grains by zone every k steps (0 = 1)      */
    int kernel;            /* DUST_KERNEL_*                                     */
    int device;            /* CUDA device ordinal                               */
    int timing;            /* 1: record device events around each kernel group
                              (read with dust_get_kernel_times)                */
    int tile[3];           /* zones per tile of the tiled kernel and of the
                              sort order (0 = default: 8x8x8 in 3-D, 16x16 in
                              2-D; clipped to the grid); each 0..1023, else
                              DUST_EINVAL                                     */
    int pusher;            /* DUST_PUSHER_EM (0) or DUST_PUSHER_SEMI_IMPLICIT */
    int gas_predictor;     /* 1: before each step, advance the gas by half a
                              step with the drag of the grains at x^n (Sec. 3.1,
                              Eqs. Delta_vp and f_D, tau_s <- max(tau_s, dt));
                              the step gathers from that prediction, and with
                              feedback_apply the deposit corrects the gas at
                              t^n, as the paper's predictor-corrector does for
                              the drag term (no hydrodynamic fluxes here).
                              In mixed precision on the slab kernel the
                              predictor sorts the grains by their zone at x^n
                              first (12 more bytes per grain of device
                              memory, 4 per sort key)                        */
    int host_io_async;     /* 0: calls with host memory (dust_load_particles,
                              dust_set_gas, dust_get_particles, dust_get_deposit
                              with DUST_MEM_HOST) return when their copies are
                              done.  1: they only enqueue them, on two copy
                              streams of the context with their own staging
                              areas (two for each output), so that one step's
                              read-back, the next step's load and the steps
                              themselves overlap.  Host buffers should then be
                              pinned; an input buffer must not be changed, and
                              an output buffer not read, before the next
                              dust_sync, which waits for every copy.  Invalid
                              grain or gas data is then reported by dust_sync
                              (DUST_EINVAL) instead of by the call, and invalid
                              grains are dropped as removed.  dust_get_gas stays
                              synchronous.                                    */
    int test_wait_timeout; /* testing only (0 otherwise): 1 makes the tile
                              kernels' bounded wait for their gas box run out
                              after 1 ms (the barrier expects more bytes than
                              the copy brings), so the failure path can be
                              checked without a GPU fault: the step's blocks
                              give up and dust_sync returns DUST_ETIMEOUT   */
    int batch_mode;        /* dust_batch_create only.  0: where every instance
                              allows it (mixed precision on the slab kernel,
                              exponential midpoint, no gas predictor, one
                              geometry: x-z shearing boxes in the orbital-
                              advection frame, or x-y Cartesian boxes),
                              each dust_batch_step call is one persistent
                              launch for all instances and steps; otherwise,
                              and with 1, a graph of per-instance kernels.
                              The batch's sort_interval k (0 = 1): the steps
                              s = 0, k, 2k, ... of a call sort first (the
                              graph sorts every step)                        */
} dust_options;

typedef struct dust_stats {
    int64_t n_stored;      /* grains held (active and removed)                  */
    int64_t n_active;      /* grains inside the domain                          */
    int64_t n_removed;     /* grains removed through outflow boundaries, total  */
    double max_cells_moved;/* largest per-step displacement seen, in zones      */
    int flags;             /* DUST_FLAG_* raised since the previous dust_sync   */
    int64_t steps;         /* steps taken                                       */
    double time;           /* simulation time                                   */
    double dt_dust;        /* dust time step of Eq. particles_dt (Sec. 3.5):
                              1.8 / max over grains and directions of
                              |v_d^{n+1/2}| / dl_d, from the largest displacement
                              of the steps since the previous dust_sync and the
                              last step's length (exact when those steps had
                              equal lengths); +inf if no grain moved.  In the
                              orbital-advection frame the displacement includes
                              the shear transport -q Omega x                  */
} dust_stats;

/* Device time per kernel group, summed over the steps since the last reset
 * (needs dust_options.timing = 1; launch counts are always kept). */
typedef struct dust_kernel_times {
    double step_ms;        /* gather-push-deposit kernel                        */
    double sort_ms;        /* zone sort: keys, scan, scatter                    */
    double other_ms;       /* deposit clear and feedback application            */
    int64_t step_launches; /* kernels launched by the library, per group        */
    int64_t sort_launches;
    int64_t other_launches;
    int64_t steps;
} dust_kernel_times;

typedef struct dust_ctx dust_ctx;

/* Create a context for one grid and set of species.  `species` has
 * n_species (1..16) entries; grains refer to them by index.  The grain
 * store is described in Sec. 3 (each particle carries x_p, v_p, tau_s,p,
 * m_p).  Errors: DUST_EINVAL (non-increasing edges, n[d] < 1, bad enums),
 * DUST_ECUDA, DUST_ENOMEM.  On error *out is NULL. */
int dust_create(dust_ctx **out, const dust_geometry *geom, const dust_grid *grid,
                const dust_species *species, int n_species, const dust_options *opt);

/* Set the gas: density rho and the physical velocity components v0, v1, v2
 * per zone (length = number of zones).  The library stores the density and
 * the momentum-like velocity p_g of Sec. 2.2, evaluated with the zone
 * centre radius (cylindrical l_g = R_i v_phi; spherical r_i v_theta,
 * r_i sin(theta_j) v_phi).  rho must be positive. */
int dust_set_gas(dust_ctx *ctx, const double *rho, const double *v0, const double *v1,
                 const double *v2, int mem);

/* Read the gas back (physical velocity components), e.g. after feedback. */
int dust_get_gas(dust_ctx *ctx, double *rho, double *v0, double *v1, double *v2, int mem);

/* Load n grains (replacing any held): coordinates q0..q2 and physical
 * velocities v0..v2 (float64, length n).  species: uint8 species index per
 * grain, or NULL for species 0.  param: per-grain stopping-time value
 * (overrides the species' tau_value), or NULL.  Grains get ids 0..n-1 in
 * load order.  Coordinates must lie inside the grid; NaN/Inf rejected. */
int dust_load_particles(dust_ctx *ctx, int64_t n, const double *q0, const double *q1,
                        const double *q2, const double *v0, const double *v1,
                        const double *v2, const uint8_t *species, const double *param,
                        int mem);

/* dust_load_particles with float32 velocity arrays v0..v2 (coordinates stay
 * float64): the grain state of Sec. 2 with velocities at the precision a
 * DUST_MIXED context stores them in, so a host that keeps them as float32
 * moves 12 bytes per grain fewer over the host link.  In a Cartesian or
 * shearing-box DUST_MIXED context the stored grains equal those of
 * dust_load_particles given the same velocities in float64; in curvilinear
 * geometry the momentum-like variables are formed from the float32 value.
 * Same layout, ownership, memory kinds and errors as dust_load_particles. */
int dust_load_particles_v32(dust_ctx *ctx, int64_t n, const double *q0, const double *q1,
                            const double *q2, const float *v0, const float *v1,
                            const float *v2, const uint8_t *species, const double *param,
                            int mem);

/* Advance every grain by one step of size dt (dt may be negative: the
 * scheme is time reversible, Sec. 3.2.2) and deposit the back-reaction of
 * that step; with feedback_apply the deposit is then added to the gas
 * momentum.  Asynchronous on the context stream. */
int dust_step(dust_ctx *ctx, double dt);

/* Allocation-free variant of one dust_step() of the one-thread-per-grain
 * kernel (DUST_KERNEL_PER_GRAIN, FP64, no zone sort, no feedback
 * application) on caller-owned device arrays.  The paper has no counterpart:
 * it exists for callers that cannot let a library allocate device memory
 * while they step (a host code that gives the device memory to its own pool
 * at start-up, or one whose other streams must not be stalled by the
 * device-wide synchronisation of cudaMalloc/cudaFree).  It calls no
 * cudaMalloc/cudaFree and no allocating library; its only scratch (grid
 * tables and status words, 512 KiB) is a fixed device array of the library.
 *
 *   geom, grid, species, n_species, weight: as for dust_create (host
 *       structs; grid edges are host arrays).  Each direction may have at
 *       most 2048 zones; a larger grid is rejected with DUST_EINVAL.
 *   quantum: fixed-point quantum of the deposit (0 = 2^-44 * largest mass).
 *   t, dt: time at the start of the step and step length (the shearing-box
 *       shift of Sec. 2.1 uses t).
 *   n: grains (0 <= n < 2^31).  q0..q2: device float64 [n] coordinates,
 *       updated in place (a grain removed through an outflow boundary gets
 *       q0 = NaN and is skipped by later calls); they must lie inside the
 *       grid or be NaN.  p0..p2: device float64 [n] momentum-like variables
 *       of Sec. 2.2 (cylindrical: v_R, R v_phi, v_z; spherical: v_r,
 *       r v_theta, r sin(theta) v_phi; shearing box with fargo = 1: the
 *       residual velocity), updated in place.  species_idx: device uint8 [n]
 *       or NULL (species 0); every index must be < n_species (a grain with a
 *       larger index is left unchanged and DUST_FLAG_SPECIES is raised in
 *       status_out).  param: device float64 [n] stopping-time values or
 *       NULL.
 *   gas: device float64 [ncell][4]: rho, then the momentum-like gas
 *       velocity p_g0..p_g2 of each zone (zone-centre radius factors).
 *   dep: device int64 [ncell][4], overwritten with this step's deposit in
 *       units of the quantum (channels as in dust_get_deposit).
 *   status_out: device uint32 [4] or NULL: DUST_FLAG_* bits, the largest
 *       displacement in zones (float bits), grains removed (low, high word).
 *   device: CUDA device ordinal (0..63), made current by the call.
 *   stream: cudaStream_t (NULL = the legacy default stream).
 *
 * Everything is enqueued on `stream`.  Each call writes the grid tables
 * into a static host image of the library and copies it asynchronously into
 * the scratch, then zeroes `dep`; the scratch's status words start at zero.
 * The image is page-locked (the first call registers it with
 * cudaHostRegister, which locks memory the library already holds and
 * allocates nothing), so the call does not wait for the GPU, with one
 * exception: before it rewrites the image it waits until the previous call's
 * copy, on whichever device, has run.  The first call on a device also
 * looks up the scratch's address (cudaGetSymbolAddress) and creates one
 * event; make that first call before any stream capture.  Calls from
 * several host threads are serialised by a lock; the scratch itself is
 * shared by all calls on a device, so calls whose kernels can overlap on the
 * GPU (two streams without ordering between them) race.  Errors:
 * DUST_EINVAL (bad descriptor, oversize grid, NULL array), DUST_ECUDA; the
 * message is dust_last_error(NULL). */
int dust_step_noalloc(const dust_geometry *geom, const dust_grid *grid,
                      const dust_species *species, int n_species, int weight,
                      double quantum, double t, double dt, int64_t n,
                      double *q0, double *q1, double *q2,
                      double *p0, double *p1, double *p2,
                      const uint8_t *species_idx, const double *param,
                      const double *gas, int64_t *dep, uint32_t *status_out,
                      int device, void *stream);

/* ---- batched stepping ---------------------------------------------------
 * Many independent contexts (instances with their own grids, sizes, species
 * and step lengths, e.g. a set of streaming-instability shearing boxes,
 * Sec. 4.3) advanced together, in one of two ways (dust_options.batch_mode):
 *  - one persistent launch per dust_batch_step call (the default where
 *    every instance allows it, see batch_mode): a cooperative kernel takes
 *    the sort, step and feedback work items of all instances and steps from
 *    one work list, each waiting (bounded in time) only for the work its
 *    instance's previous phase did; a wait that runs out makes every
 *    instance report DUST_ETIMEOUT at its next dust_sync;
 *  - a CUDA graph: dust_batch_step captures, once, one period of two steps
 *    of every instance (each instance a branch on its own stream: sort,
 *    deposit clear, step kernel, feedback, time advance) and replays it
 *    nsteps / 2 times with one launch each; an odd last step is taken with
 *    dust_step.  The graph is captured again when a dt changes, particles
 *    are reloaded, or a context was stepped on its own in between.
 * Results equal, bit for bit, those of calling dust_step on each context
 * with the same dt (the graph sorts before every step; the persistent launch
 * at the batch's sort interval, as contexts with that sort_interval do).
 * Per-group timing (dust_options.timing) is not recorded for batched steps.
 * Contexts must be on one device and on streams that can be captured (not
 * the legacy default stream); the batch does not own them and must be
 * destroyed before them. */
typedef struct dust_batch dust_batch;

/* insts: n (1..4096) distinct contexts.  opt may be NULL; opt->stream, if
 * set, is the stream the batch's work is launched on (else the batch creates
 * one); opt->batch_mode and opt->sort_interval choose the way (above).
 * Errors: DUST_EINVAL, DUST_ECUDA, DUST_ENOMEM (message:
 * dust_batch_last_error(NULL)). */
int dust_batch_create(dust_batch **out, dust_ctx *const *insts, int n, const dust_options *opt);

/* Advance every instance i by nsteps steps of length dt[i] (dt: n values).
 * Asynchronous: each context's stream is ordered after the batch's work, so
 * dust_sync and the getters on a context see its result.  Errors:
 * DUST_EINVAL, DUST_ESTATE (gas or particles missing), DUST_ECUDA. */
int dust_batch_step(dust_batch *b, const double *dt, int nsteps);

/* Message of the last error of a batch (NULL: of the last failed create). */
const char *dust_batch_last_error(const dust_batch *b);

/* Wait for the batch's work and free the batch (not its contexts). */
void dust_batch_destroy(dust_batch *b);

/* Wait for the context stream, fill *out (may be NULL) and return
 * DUST_ENAN / DUST_EOVERFLOW / DUST_ECFL if the matching flag was raised
 * since the previous dust_sync, else DUST_OK.  Flags are then cleared. */
int dust_sync(dust_ctx *ctx, dust_stats *out);

/* Deposit of the most recent step, channels (momentum-like 0..2, energy 3)
 * per zone: fixed ([ncell][4] int64, units of the quantum) and/or as_double
 * ([ncell][4], fixed * quantum); either may be NULL.  Channel c of zone i is
 * -sum_p m_p W_ip (dp_c - dt a_c) (Eq. dust_feedback_final times dV dt),
 * the impulse given to the gas; channel 3 is sum_c of that times dH/dp_c at
 * the half step (energy given to the gas).  *quantum_out may be NULL. */
int dust_get_deposit(dust_ctx *ctx, int64_t *fixed, double *as_double,
                     double *quantum_out, int mem);

/* Dust mass per zone of the grains as they are now (Sec. 3.4, Eq.
 * deposition with q_p = m_p), with the context's weighting (CIC, TSC or
 * volume weighting) at the stored positions; divided by the zone volume it
 * is the dust density the paper's rigid-disk test (Sec. 4.7) measures.
 * fixed: [ncell] int64 in units of the context's quantum read as a mass,
 * or NULL; as_double: [ncell], fixed * quantum, or NULL; *quantum_out may
 * be NULL.  Per grain, the non-host stencil zones get rint(W m / quantum)
 * and the host zone the rest of rint(m / quantum), so the zone sum equals
 * the grain sum exactly.  Zones beyond an outflow boundary fold onto the
 * edge zone.  Synchronous.  Errors: DUST_ESTATE (no particles loaded),
 * DUST_ECUDA, DUST_ENOMEM. */
int dust_get_mass_deposit(dust_ctx *ctx, int64_t *fixed, double *as_double,
                          double *quantum_out, int mem);

/* Copy the stored grains (current storage order, which the zone sort
 * permutes): coordinates, physical velocities and original ids (int64).
 * Removed grains are included with NaN coordinates, after the live ones and
 * in no particular order (the live ones are in zone-key, then id, order
 * after a sort).  cap = capacity of the
 * caller arrays; *n_out = grains written.  Any pointer but n_out may be
 * NULL. */
int dust_get_particles(dust_ctx *ctx, int64_t cap, double *q0, double *q1, double *q2,
                       double *v0, double *v1, double *v2, int64_t *ids, int64_t *n_out,
                       int mem);

/* dust_get_particles with float32 velocity arrays v0..v2 (coordinates stay
 * float64): each velocity is the float64 value dust_get_particles returns,
 * rounded to float32 (exact for the stored velocities of a Cartesian or
 * shearing-box DUST_MIXED context).  Same order, arguments and errors as
 * dust_get_particles. */
int dust_get_particles_v32(dust_ctx *ctx, int64_t cap, double *q0, double *q1, double *q2,
                           float *v0, float *v1, float *v2, int64_t *ids, int64_t *n_out,
                           int mem);

/* Wait for the context stream and return the per-group device times and
 * launch counts accumulated since the last reset; reset != 0 clears them. */
int dust_get_kernel_times(dust_ctx *ctx, dust_kernel_times *out, int reset);

/* Message of the last error on this context (static storage of the
 * context; NULL ctx gives the last dust_create error). */
const char *dust_last_error(const dust_ctx *ctx);

/* Free the context and all its device memory.  NULL is allowed. */
void dust_destroy(dust_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DUST_H */
