// Internal declarations of the dust library (not part of the C interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dust.h"

namespace dust {

constexpr int kMaxSpecies = 16;

enum GeomKind { GEOM_CART = 0, GEOM_SB = 1, GEOM_CYL = 2, GEOM_SPH = 3 };
enum EdgeKind { EDGE_UNIFORM = 0, EDGE_LOG = 1, EDGE_GENERAL = 2 };

// Status words on the device: [0] flag bits, [1] max zones moved (float
// bits, non-negative so integer max orders them), [2] removed this step
// (low), [3] high.
enum { ST_FLAGS = 0, ST_MAXMOVE = 1, ST_REMOVED_LO = 2, ST_REMOVED_HI = 3, ST_WORDS = 8 };

// Integer key that orders non-NaN doubles like their values (-0 and +0
// equal): comparisons of grain coordinates against zone edges run on the
// integer pipe instead of the (narrow) double-precision pipe.
__host__ __device__ __forceinline__ long long order_key(double x)
{
    union { double d; long long i; } u;
    u.d = x;
    long long b = u.i;
    if (b == (long long)0x8000000000000000ULL) b = 0;
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

struct GridDev {
    long long lo_key[3], hi_key[3];
    const long long *ekey[3];  // order_key of every edge
    int n[3];
    int bc[3];
    int edge_kind[3];
    const double *edges[3];  // device, n[d] + 1 each
    double lo[3], hi[3];
    double inv_d[3];         // uniform: n / (hi - lo); log: n / ln(hi / lo)
    float inv_df[3];
    float log_lo_f[3];
    const double *dvol[3];   // per-direction factors of the zone volume
    const float *dvol_f[3];
    const double *zc[3];     // zone centres (edges midpoint)
    const double *ziw[3];    // 1 / zone width
    const float *ziw_f[3];
    const float *znu_f[3];   // centre / width (curvilinear radial weights)
    const float *zlo_f[3];   // lower edge (polar-angle weights)
    const float *zc_f[3];    // zone centres, single precision
    int64_t ncell;
    // tile layout of the zone sort: tiles of T[0] x T[1] x T[2] zones; key of
    // zone (i,j,k) = tile index * tvol + position inside the tile
    int T[3];
    int nt[3];
    int tvol;
    int64_t nkeys;           // number of tiles * tvol (>= ncell)
};

__host__ __device__ __forceinline__ int64_t zone_key(const GridDev &g, int i, int j, int k)
{
    const int ti = i / g.T[0], tj = j / g.T[1], tk = k / g.T[2];
    const int li = i - ti * g.T[0], lj = j - tj * g.T[1], lk = k - tk * g.T[2];
    const int64_t tile = ti + (int64_t)g.nt[0] * (tj + (int64_t)g.nt[1] * tk);
    return tile * g.tvol + li + g.T[0] * (lj + g.T[1] * lk);
}

struct PhysDev {
    int geom;
    int fargo;
    int vgrav;
    int pusher;              // DUST_PUSHER_EM or DUST_PUSHER_SEMI_IMPLICIT
    double omega, qshear, gm;
    double q_om;             // q * Omega
    double jump_v;           // q * Omega * Lx (standard-frame v_y jump)
    double shift_mid;        // fmod(q Omega Lx (t + dt/2), Ly)
    double shift_end;        // fmod(q Omega Lx (t + dt), Ly)
    // single-precision copies for the mixed path
    float omega_f, qshear_f, gm_f, q_om_f, jump_v_f;
};

struct SpeciesDev {
    int n;
    double mass[kMaxSpecies];
    double tau[kMaxSpecies];
    int mode[kMaxSpecies];
    double mq[kMaxSpecies];   // mass / fixed-point quantum
    float mqf[kMaxSpecies];
    float tau_f[kMaxSpecies];
    // single-precision propagators of the step (Eqs. phi1, h1) for species
    // whose stopping time is the same for all their grains (constant tau;
    // constant Stokes number in Cartesian and shearing-box geometry),
    // computed in double precision on the host for the step's dt; bit s of
    // coef_const says species s has them
    unsigned coef_const;
    float tau_eff_f[kMaxSpecies], E_f[kMaxSpecies], cg_f[kMaxSpecies], h1_f[kMaxSpecies];
};

template <typename Real>
struct StoreDev {
    double *q[3];
    Real *p[3];
    uint8_t *species;        // may be null (all species 0)
    Real *param;             // may be null (species value)
    int32_t *id;
    int64_t n;
};

template <typename Real>
struct StepArgs {
    GridDev g;
    PhysDev ph;
    SpeciesDev sp;
    double t, dt;
    double inv_quantum;
    StoreDev<Real> s;
    const Real *gas;              // [ncell][4]: rho, p_g0, p_g1, p_g2
    unsigned long long *dep;      // [ncell][4] two's complement int64
    unsigned int *status;         // ST_WORDS words
    // null: the shear-periodic shifts are ph.shift_mid / ph.shift_end; else
    // device memory [t, shift_mid, shift_end] of the step (graph replays)
    const double *tdev;
};

template <typename Real>
struct TiledArgs {
    StepArgs<Real> s;
    const int32_t *key_off;       // [nkeys + 1] start of each key in the sorted store
    int tsc;                      // 1: TSC weights, 0: CIC
    int vol;                      // 1: volume weighting (Eq. CIC_vol) in the
                                  // curvilinear directions, CIC elsewhere (tsc 0)
    // optional: the step kernel predicts every grain's key for the next sort
    int emit_keys;
    int32_t *key_out;             // [n]
    int32_t *count_out;           // [nkeys + 2], zeroed before the step
    // optional: the sort's gather fused into the step.  The grain at sorted
    // position i is read from s at perm[i] and written, with id perm_id[i],
    // to dst at i (null: read and write s in place)
    const int32_t *perm;
    const int32_t *perm_id;
    StoreDev<Real> dst;
    // optional: tensor map (CUtensorMap, device memory) of s.gas viewed as a
    // 4-D array (channel, x, y, z); the tile kernels then stage their gas
    // box with one bulk tensor copy
    const void *gas_tmap;
    // limit of the wait for that copy (0: one second), and bytes the
    // barrier expects beyond the copy (0; > 0 only to test the timeout)
    unsigned long long wait_ns;
    unsigned int wait_extra_tx;
};

template <typename Real>
struct SortArgs {
    GridDev g;
    PhysDev ph;
    double dt;                    // step the key predicts (half drift of it)
    StoreDev<Real> src, dst;
    int32_t *key;                 // [n]
    int32_t *count;               // [nkeys + 1] key offsets after the scan
    int32_t *cursor;              // [nkeys + 1]
    int32_t *pair_id;             // [n] grain id at its sorted position
    int32_t *pair_src;            // [n] source position of that grain
    int64_t nkeys1;               // nkeys + 1 (the removed-grain key included)
    // zone segments too long for the warp's staging: [0] their count
    // (zeroed before the segment sort), [1 ..] their keys ([nkeys + 2])
    int32_t *big;
    // scratch of the block sort's merge passes, [n] each (free between the
    // scatter and the step: the key column and the other store's ids)
    int32_t *tmp_id, *tmp_src;
};

#ifdef __CUDACC__
// Feedback of zone c (a8): the deposited momentum-like impulse over rho dV
// added to the gas (the corrector term of the RK2 step, Sec. 3.1).
template <typename Real>
__device__ __forceinline__ void apply_feedback_zone(const GridDev &g, double quantum, Real *gas,
                                                    const unsigned long long *dep, int64_t c)
{
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int k = (int)(c / ((int64_t)g.n[0] * g.n[1]));
    const long long d0 = (long long)dep[4 * c + 0], d1 = (long long)dep[4 * c + 1],
                    d2 = (long long)dep[4 * c + 2];
    if ((d0 | d1 | d2) == 0) return;
    // each product and sum rounded on its own (no fused multiply-add), so
    // that every kernel that applies the feedback gives the same bits
    if (sizeof(Real) == 4) {
        const float s = (float)quantum /
                        ((float)gas[4 * c] * g.dvol_f[0][i] * g.dvol_f[1][j] * g.dvol_f[2][k]);
        gas[4 * c + 1] = (Real)__fadd_rn((float)gas[4 * c + 1], __fmul_rn((float)d0, s));
        gas[4 * c + 2] = (Real)__fadd_rn((float)gas[4 * c + 2], __fmul_rn((float)d1, s));
        gas[4 * c + 3] = (Real)__fadd_rn((float)gas[4 * c + 3], __fmul_rn((float)d2, s));
    } else {
        const double s = quantum / ((double)gas[4 * c] * g.dvol[0][i] * g.dvol[1][j] * g.dvol[2][k]);
        gas[4 * c + 1] = (Real)__dadd_rn((double)gas[4 * c + 1], __dmul_rn((double)d0, s));
        gas[4 * c + 2] = (Real)__dadd_rn((double)gas[4 * c + 2], __dmul_rn((double)d1, s));
        gas[4 * c + 3] = (Real)__dadd_rn((double)gas[4 * c + 3], __dmul_rn((double)d2, s));
    }
}

// Time of the next step of a context stepped from the device: t += dt, then
// the shear-periodic shifts of the step that starts at the new t, with the
// same operations as on the host: fmod(((q Omega) Lx) (t + dt/2), Ly).
__device__ __forceinline__ void advance_time(double *tm, double dt, double q_om_lx, double ly, int sb)
{
    const double t = __dadd_rn(tm[0], dt);
    tm[0] = t;
    if (sb) {
        tm[1] = fmod(__dmul_rn(q_om_lx, __dadd_rn(t, __dmul_rn(0.5, dt))), ly);
        tm[2] = fmod(__dmul_rn(q_om_lx, __dadd_rn(t, dt)), ly);
    }
}
#endif  // __CUDACC__

// ---- batched persistent step (dust_batch_step) ---------------------------
// One instance of a batch as the persistent kernel sees it: the step's
// arguments with the fields that change from step to step set per step from
// the buffers below.
struct BatchInst {
    TiledArgs<float> ta;         // the step's arguments (store, sort and count fields set per step)
    StoreDev<float> store[2];    // the two grain stores
    int32_t *count[2];           // [0]: offsets of the last sort, [1]: counts for the next sort (at the launch)
    int32_t *key, *cursor, *pair_id, *pair_src, *bigseg, *blocksums;
    double *time;                // [t, shift_mid, shift_end] of the step (the steps' tdev)
    double dt, q_om_lx, ly;
    double quantum;
    int sb;                      // shearing box: the shifts advance with t
    int cur;                     // current store at the launch
    int feedback;                // apply the deposit to the gas after each step
    int ntiles;
    int64_t n, nkeys, ncell;
};

// The tile shapes with a compiled copy of the slab tile function (TSC weights,
// exponential midpoint): 8^3 in 3-D, 32 x 16 and 16 x 16 zones in x-z.
enum SlabShapeId { SHAPE_ANY = 0, SHAPE_8C = 1, SHAPE_32X16 = 2, SHAPE_16X16 = 3 };

inline int slab_shape_id(const GridDev &g, int flat, int tsc, int mode)
{
    if (!tsc || mode != 1) return SHAPE_ANY;
    if (flat == 0 && g.T[0] == 8 && g.T[1] == 8 && g.T[2] == 8) return SHAPE_8C;
    if (flat == 1 && g.T[0] == 32 && g.T[1] == 1 && g.T[2] == 16) return SHAPE_32X16;
    if (flat == 1 && g.T[0] == 16 && g.T[1] == 1 && g.T[2] == 16) return SHAPE_16X16;
    return SHAPE_ANY;
}

// Phases of one step of one instance in the persistent kernel.
enum { BPH_SCANA = 0, BPH_SCANB, BPH_SCANC, BPH_SCATTER, BPH_SEG, BPH_ZERO, BPH_TILE, BPH_FB, BPH_N };

// One task of the persistent kernel's work list: phase p of step s for the
// instances of group g, as `items` consecutive work items from `begin`.  It
// starts once task `dep` (the group's previous task with items, or -1) has
// completed all its items.
struct BatchTask {
    int s, g, p;
    int begin, items;
    int dep;
};

struct BatchDev {
    const BatchInst *inst;
    int ninst;
    // the work list: tasks in round order (a group's phase p of step s in
    // round s * period + g + p; inside a round by phase), nitems work items
    // in all, taken by the blocks in turn from *grab
    const BatchTask *tasks;
    int ntasks, nitems;
    int *grab;                   // zero at launch
    int *done;                   // [ntasks] items completed, zero at launch
    // instances of group g: members[g * gmax + k], k < gcount[g]; their work
    // items per phase: prefix sums gpre[((sorted * BPH_N + p) * ngroups + g) * (gmax + 1) + k]
    const int *members, *gcount, *gpre;
    int ngroups, gmax;
    int nsteps;
    int sort_interval;           // steps s with s % sort_interval == 0 sort first
    int wait_extra;              // > 0 only to test the bounded wait
    unsigned long long wait_ns;  // limit of one wait for a task
    size_t ta_offset;            // where the block's copy of the step arguments sits in shared memory
    // the host's layout of the work list in one int table: tasks, members,
    // gcount, gpre (nstatic ints), then done and grab
    int off_tasks, off_members, off_gcount, off_gpre, nstatic;
};

// Work items per phase of one instance: chunks of the per-context kernels'
// blocks, kBatchChunks of them per item.
constexpr int kBatchScanChunk = 256 * 4;     // counts per scan chunk (256 threads x 4)
constexpr int kBatchScatterChunk = 256 * 4;  // grains per scatter chunk
constexpr int kBatchSegChunk = 256;          // keys per segment-sort chunk
constexpr int kBatchZeroChunk = 256 * 8;     // 8-byte words zeroed per chunk
constexpr int kBatchFbChunk = 256;           // zones per feedback chunk
constexpr int kBatchChunks = 8;              // chunks per work item
constexpr int kBatchBigItems = 8;            // items of the block sort per instance

// TX > 0: the copy for a TX x TY x TZ tile (every instance's, TSC weights).
template <int GEOM, int FLAT, int MODE, int TX = 0, int TY = 0, int TZ = 0>
cudaError_t launch_batch_persistent(const BatchDev &b, size_t smem, int grid, cudaStream_t s);

// Shared memory of one slab tile of this grid, and of the sort's staging.
size_t batch_tile_smem(const GridDev &g);
size_t batch_sort_smem();

// Grid size of the persistent kernel for this shared memory (all blocks
// resident at once), 0 if it cannot run.
template <int GEOM, int FLAT, int MODE, int TX = 0, int TY = 0, int TZ = 0>
int batch_persistent_grid(size_t smem);

// Launch wrappers, explicitly instantiated per geometry.
template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_step_per_grain(const StepArgs<Real> &a, cudaStream_t s);

template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_step_tiled(const TiledArgs<Real> &a, cudaStream_t s);

// FLAT: 0 = all directions gridded, 1 = y not gridded, 2 = z not gridded;
// MODE: 0 = pusher and frame at run time, 1 = exponential midpoint (and, in
// the shearing box, the orbital-advection frame), 2 = exponential midpoint
// in the standard shearing-box frame
template <int GEOM, int FLAT, int MODE>
cudaError_t launch_step_slab(const TiledArgs<float> &a, cudaStream_t s);

// Gas predictor on the slab layout (mixed precision), one per flat pattern.
template <int GEOM, int FLAT>
cudaError_t launch_predict_slab(const TiledArgs<float> &a, cudaStream_t s);

template <typename Real, int GEOM>
cudaError_t launch_sort_keys(const SortArgs<Real> &a, cudaStream_t s);

// Keys of the zones at x^n (the gas predictor's sort), one per geometry.
template <int GEOM>
cudaError_t launch_zone_keys(const SortArgs<float> &a, cudaStream_t s);

template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_predict_gas(const StepArgs<Real> &a, cudaStream_t s);

template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_predict_tiled(const TiledArgs<Real> &a, cudaStream_t s);

template <int GEOM>
cudaError_t launch_deposit_mass(const GridDev &g, const SpeciesDev &sp, int wk, int64_t n,
                                const double *const q[3], const uint8_t *species,
                                unsigned long long *out, unsigned int *status, cudaStream_t s);

template <typename Real>
cudaError_t launch_sort_scatter(const SortArgs<Real> &a, cudaStream_t s, bool gather);

cudaError_t launch_exclusive_scan(int32_t *data, int64_t n, int32_t *block_sums,
                                  cudaStream_t s);
int64_t scan_block_sums_size(int64_t n);

}  // namespace dust
