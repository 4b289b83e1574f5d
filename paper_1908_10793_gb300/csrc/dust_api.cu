// Host side of the C interface declared in include/dust.h: context
// management, data movement, unit conversion, step sequencing.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include <cuda.h>  // CUtensorMap and its enumerations (the encoder is fetched at run time)

#include "dust_internal.h"
#include "dust_worklist.h"

using namespace dust;

namespace {

enum { ST_LOAD_BAD = 4 };

thread_local std::string g_create_error;

}  // namespace

struct dust_ctx {
    int device = 0;
    dust_geometry geom{};
    dust_options opt{};
    int mixed = 1;
    size_t rsz = 4;
    int n[3] = {1, 1, 1};
    int bc[3] = {0, 0, 0};
    std::vector<double> edges[3];
    SpeciesDev sp{};
    int64_t ncell = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    GridDev g{};
    double *d_edges[3] = {nullptr, nullptr, nullptr};
    double *d_dvol[3] = {nullptr, nullptr, nullptr};
    float *d_dvol_f[3] = {nullptr, nullptr, nullptr};
    double *d_zc[3] = {nullptr, nullptr, nullptr};
    long long *d_ekey[3] = {nullptr, nullptr, nullptr};
    double *d_ziw[3] = {nullptr, nullptr, nullptr};
    float *d_ziw_f[3] = {nullptr, nullptr, nullptr};
    float *d_znu_f[3] = {nullptr, nullptr, nullptr};
    float *d_zlo_f[3] = {nullptr, nullptr, nullptr};
    float *d_zc_f[3] = {nullptr, nullptr, nullptr};
    bool need_sort = true;
    void *d_gas = nullptr;
    unsigned long long *d_dep = nullptr;
    // gas half-step predictor (dust_options.gas_predictor): its impulse and
    // the predicted gas the step gathers from
    unsigned long long *d_pred = nullptr;
    unsigned long long *d_mass = nullptr;   // dust_get_mass_deposit (on first use)
    void *d_gas_half = nullptr;
    // tensor maps (CUtensorMap, 64-byte aligned device memory) of d_gas [0]
    // and d_gas_half [1] for the tile kernels' bulk gas-box copy; null: none
    CUtensorMap *d_tmaps = nullptr;
    bool tmap_ok[2] = {false, false};
    unsigned int *d_status = nullptr;
    unsigned int *h_status = nullptr;

    double *d_q[2][3] = {};
    void *d_p[2][3] = {};
    uint8_t *d_species[2] = {nullptr, nullptr};
    void *d_param[2] = {nullptr, nullptr};
    int32_t *d_id[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t n_grains = 0, cap = 0;
    bool has_species = false, has_param = false;

    int32_t *d_key = nullptr, *d_count = nullptr, *d_cursor = nullptr, *d_blocksums = nullptr;
    int32_t *d_pair_id = nullptr, *d_pair_src = nullptr;
    // the gas predictor's own sort of the store by the zone at x^n (mixed
    // precision on the slab layout): keys, key offsets, (id, source) pairs
    int32_t *d_pkey = nullptr, *d_pcount = nullptr, *d_ppair_id = nullptr, *d_ppair_src = nullptr;
    // zone segments left to the block sort: count, then keys ([nkeys + 2])
    int32_t *d_bigseg = nullptr;
    // key counts for the next sort (d_count holds the current key offsets)
    int32_t *d_count_next = nullptr;
    bool keys_ready = false;   // d_key / d_count_next predicted by the last step
    double keys_dt = 0.0;      // the step length they were predicted for
    // steps replayed from a captured graph read their time from the device:
    // d_time = [t, shift_mid, shift_end, -]
    double *d_time = nullptr;
    bool capture_mode = false;  // enqueueing into a stream capture
    bool perm_pending = false;  // sorted order computed, gather left to the step
    uint64_t gen = 0;           // bumped when the grain store is reallocated
    double *d_stage = nullptr;
    size_t stage_bytes = 0;
    // asynchronous host I/O (dust_options.host_io_async): two copy streams
    // and staging areas, each with an event for "data in place" and one for
    // "free for reuse"; outputs alternate between two areas
    struct IoBuf {
        void *d = nullptr;
        size_t bytes = 0;
        cudaEvent_t ready = nullptr;
        cudaEvent_t done = nullptr;
        bool used = false;  // `done` recorded at least once
    };
    cudaStream_t io_in = nullptr, io_out = nullptr;
    IoBuf in_grains, in_gas, out_grains[2], out_dep[2];
    int out_flip = 0, dep_flip = 0;

    double t = 0.0;
    double last_dt = 0.0;       // length of the last step (dust time step estimate)
    int64_t steps = 0;
    int64_t removed_total = 0;
    float max_moved = 0.f;
    bool gas_set = false, particles_set = false, have_deposit = false;
    double quantum = 0.0;
    int sort_interval = 1;
    std::string err;

    // per-group device timing (dust_options.timing) and launch counts
    enum { GROUP_STEP = 0, GROUP_SORT = 1, GROUP_OTHER = 2, N_GROUPS = 3 };
    std::vector<cudaEvent_t> event_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[N_GROUPS];
    double group_ms[N_GROUPS] = {0, 0, 0};
    int64_t launches[N_GROUPS] = {0, 0, 0};
    int64_t timed_steps = 0;
};

namespace {

int fail(dust_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_error = buf;
    return code;
}

#define CU(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? DUST_ENOMEM : DUST_ECUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                    \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}

void dfree(void *p)
{
    if (p) cudaFree(p);
}

int edge_kind(const double *e, int n)
{
    if (n <= 1) return EDGE_UNIFORM;
    const double lo = e[0], hi = e[n];
    bool uni = true, lg = lo > 0.0;
    for (int i = 0; i <= n && (uni || lg); ++i) {
        const double u = lo + (hi - lo) * i / n;
        if (fabs(e[i] - u) > 1e-9 * (hi - lo) / n) uni = false;
        if (lg) {
            const double l = lo * pow(hi / lo, (double)i / n);
            if (fabs(e[i] - l) > 1e-9 * (e[i] * (pow(hi / lo, 1.0 / n) - 1.0))) lg = false;
        }
    }
    return uni ? EDGE_UNIFORM : (lg ? EDGE_LOG : EDGE_GENERAL);
}

// Checks of the geometry, grid, species and weight descriptors shared by
// dust_create and dust_step_noalloc; *ncell_out = number of zones.
int validate_descriptors(const dust_geometry *geom, const dust_grid *grid,
                         const dust_species *species, int n_species, int weight,
                         int64_t *ncell_out)
{
    if (!geom || !grid || !species) return fail(nullptr, DUST_EINVAL, "NULL descriptor");
    if (geom->kind < DUST_CARTESIAN || geom->kind > DUST_SPHERICAL)
        return fail(nullptr, DUST_EINVAL, "bad geometry kind %d", geom->kind);
    if (n_species < 1 || n_species > kMaxSpecies)
        return fail(nullptr, DUST_EINVAL, "n_species must be 1..%d", kMaxSpecies);
    if (weight != DUST_WEIGHT_CIC && weight != DUST_WEIGHT_TSC && weight != DUST_WEIGHT_VOLUME)
        return fail(nullptr, DUST_EINVAL, "bad weight");
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
        if (grid->n[d] < 1 || !grid->edges[d])
            return fail(nullptr, DUST_EINVAL, "direction %d: n < 1 or no edges", d);
        if (!std::isfinite(grid->edges[d][0]))
            return fail(nullptr, DUST_EINVAL, "direction %d: edges not finite", d);
        for (int i = 0; i < grid->n[d]; ++i)
            if (!(grid->edges[d][i] < grid->edges[d][i + 1]) || !std::isfinite(grid->edges[d][i + 1]))
                return fail(nullptr, DUST_EINVAL, "direction %d: edges not increasing", d);
        if (grid->bc[d] != DUST_BC_PERIODIC && grid->bc[d] != DUST_BC_OUTFLOW)
            return fail(nullptr, DUST_EINVAL, "direction %d: bad boundary kind", d);
        ncell *= grid->n[d];
    }
    if (ncell >= (int64_t)1 << 31) return fail(nullptr, DUST_EINVAL, "too many zones");
    if (geom->kind == DUST_CYLINDRICAL && grid->edges[0][0] <= 0.0)
        return fail(nullptr, DUST_EINVAL, "cylindrical R must be > 0");
    if (geom->kind == DUST_SPHERICAL &&
        (grid->edges[0][0] <= 0.0 || grid->edges[1][0] <= 0.0 ||
         grid->edges[1][grid->n[1]] >= M_PI))
        return fail(nullptr, DUST_EINVAL, "spherical r must be > 0 and theta in (0, pi)");
    if ((geom->kind == DUST_CYLINDRICAL || geom->kind == DUST_SPHERICAL))
        for (int s = 0; s < n_species; ++s)
            if (species[s].tau_mode == DUST_TAU_STOKES && !(geom->gm > 0.0))
                return fail(nullptr, DUST_EINVAL, "Stokes-number mode needs GM > 0");
    *ncell_out = ncell;
    return DUST_OK;
}

// Species constants; quantum <= 0 selects the default: 2^-44 * largest mass
// (FP64), 2^-40 * largest mass (mixed precision, default_exp -40).
SpeciesDev make_species(const dust_species *species, int n_species, double quantum,
                        double *quantum_out, int default_exp = -44)
{
    SpeciesDev sp{};
    double mmax = 0.0;
    sp.n = n_species;
    for (int s = 0; s < n_species; ++s) {
        sp.mass[s] = species[s].mass;
        sp.tau[s] = species[s].tau_value;
        sp.mode[s] = species[s].tau_mode;
        mmax = fmax(mmax, fabs(species[s].mass));
    }
    const double qu = quantum > 0.0 ? quantum : ldexp(mmax > 0 ? mmax : 1.0, default_exp);
    for (int s = 0; s < n_species; ++s) {
        sp.mq[s] = species[s].mass / qu;
        sp.mqf[s] = (float)sp.mq[s];
        sp.tau_f[s] = (float)sp.tau[s];
    }
    *quantum_out = qu;
    return sp;
}

// Propagators E = exp(-dt/tau), c_g = -expm1(-dt/tau), h1 = dt c_g/(dt/tau)
// (Eqs. phi1, h1) of every species whose stopping time does not depend on
// the grain, for a step of length dt, rounded once to single precision.
void species_coefficients(SpeciesDev &sp, int geom, double omega, double dt)
{
    sp.coef_const = 0u;
    for (int s = 0; s < sp.n; ++s) {
        double tau;
        if (sp.mode[s] == DUST_TAU_CONST) tau = sp.tau[s];
        else if (sp.mode[s] == DUST_TAU_STOKES && (geom == DUST_CARTESIAN || geom == DUST_SHEARING_BOX))
            tau = sp.tau[s] / omega;
        else continue;
        const double x = dt / tau;
        const double cg = -expm1(-x);
        sp.tau_eff_f[s] = (float)tau;
        sp.E_f[s] = (float)exp(-x);
        sp.cg_f[s] = (float)cg;
        sp.h1_f[s] = (float)(x == 0.0 ? dt : dt * cg / x);
        sp.coef_const |= 1u << s;
    }
}

// Scalar description of direction d of the grid (host side).
void grid_direction(GridDev &g, int d, const double *e, int n, int bc)
{
    g.n[d] = n;
    g.bc[d] = bc;
    g.lo[d] = e[0];
    g.hi[d] = e[n];
    g.edge_kind[d] = edge_kind(e, n);
    if (g.edge_kind[d] == EDGE_LOG) {
        g.inv_d[d] = n / log(e[n] / e[0]);
        g.log_lo_f[d] = logf((float)e[0]);
    } else {
        g.inv_d[d] = n / (e[n] - e[0]);
        g.log_lo_f[d] = 0.f;
    }
    g.inv_df[d] = (float)g.inv_d[d];
    g.lo_key[d] = order_key(e[0]);
    g.hi_key[d] = order_key(e[n]);
}

// Per-zone tables of one direction, written to host arrays: volume factors
// (Sec. 3.4: dR, d(R^2/2), d(r^3/3), -d cos(theta)), centres, inverse
// widths, centre / width, lower edges and edge order keys.
struct ZoneTables {
    double *dvol, *zc, *ziw;
    float *dvol_f, *ziw_f, *znu_f, *zlo_f, *zc_f;   // zlo_f: n + 1 entries
    long long *ekey;                                 // n + 1 entries
};

void fill_zone_tables(int kind, int d, const double *e, int n, const ZoneTables &t)
{
    for (int i = 0; i < n; ++i) {
        const double a = e[i], b = e[i + 1];
        double v = b - a;
        if (d == 0 && kind == DUST_CYLINDRICAL) v = 0.5 * (b * b - a * a);
        if (d == 0 && kind == DUST_SPHERICAL) v = (b * b * b - a * a * a) / 3.0;
        if (d == 1 && kind == DUST_SPHERICAL) v = cos(a) - cos(b);
        t.dvol[i] = v;
        t.dvol_f[i] = (float)v;
        t.zc[i] = 0.5 * (a + b);
        t.ziw[i] = 1.0 / (b - a);
        t.ziw_f[i] = (float)t.ziw[i];
        t.znu_f[i] = (float)(t.zc[i] * t.ziw[i]);
        t.zc_f[i] = (float)t.zc[i];
    }
    for (int i = 0; i <= n; ++i) {
        t.zlo_f[i] = (float)e[i];
        t.ekey[i] = order_key(e[i]);
    }
}

// --------------------------------------------------------- aux kernels ----

__device__ __forceinline__ double centre(const GridDev &g, int d, int i)
{
    return 0.5 * (g.edges[d][i] + g.edges[d][i + 1]);
}

// Physical gas velocity -> stored momentum-like velocity (Sec. 2.2), zone
// centre factors.
template <typename Real>
__global__ void set_gas_kernel(GridDev g, int geom, const double *rho, const double *v0,
                               const double *v1, const double *v2, Real *gas, unsigned int *st)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    double p0 = v0[c], p1 = v1[c], p2 = v2[c];
    const double r = rho[c];
    if (geom == GEOM_CYL) p1 *= centre(g, 0, i);
    if (geom == GEOM_SPH) {
        const double rc = centre(g, 0, i);
        p1 *= rc;
        p2 *= rc * sin(centre(g, 1, j));
    }
    if (!(r > 0.0) || !isfinite(r) || !isfinite(p0) || !isfinite(p1) || !isfinite(p2))
        atomicOr(&st[ST_LOAD_BAD], 1u);
    gas[4 * c + 0] = (Real)r;
    gas[4 * c + 1] = (Real)p0;
    gas[4 * c + 2] = (Real)p1;
    gas[4 * c + 3] = (Real)p2;
}

template <typename Real>
__global__ void get_gas_kernel(GridDev g, int geom, const Real *gas, double *rho, double *v0,
                               double *v1, double *v2)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    double p0 = gas[4 * c + 1], p1 = gas[4 * c + 2], p2 = gas[4 * c + 3];
    if (geom == GEOM_CYL) p1 /= centre(g, 0, i);
    if (geom == GEOM_SPH) {
        const double rc = centre(g, 0, i);
        p1 /= rc;
        p2 /= rc * sin(centre(g, 1, j));
    }
    if (rho) rho[c] = gas[4 * c + 0];
    if (v0) v0[c] = p0;
    if (v1) v1[c] = p1;
    if (v2) v2[c] = p2;
}

// Physical grain velocity -> momentum-like variables (Sec. 2.2).  VT: the
// type of the host's velocity arrays (double, or float for the store's own
// precision in mixed contexts).
template <typename Real, typename VT>
__global__ void load_kernel(GridDev g, int geom, int64_t n, const double *q0, const double *q1,
                            const double *q2, const VT *v0, const VT *v1,
                            const VT *v2, const uint8_t *species_in, int n_species,
                            const double *param_in, StoreDev<Real> s, unsigned int *st,
                            int drop_bad)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double x0 = q0[k], x1 = q1[k], x2 = q2[k];
    double p0 = (double)v0[k], p1 = (double)v1[k], p2 = (double)v2[k];
    bool bad = !(isfinite(x0) && isfinite(x1) && isfinite(x2) && isfinite(p0) &&
                 isfinite(p1) && isfinite(p2));
    bad |= !(x0 >= g.lo[0] && x0 < g.hi[0] && x1 >= g.lo[1] && x1 < g.hi[1] &&
             x2 >= g.lo[2] && x2 < g.hi[2]);
    if (geom == GEOM_CYL) p1 *= x0;
    if (geom == GEOM_SPH) {
        p1 *= x0;
        p2 *= x0 * sin(x1);
    }
    s.q[0][k] = x0; s.q[1][k] = x1; s.q[2][k] = x2;
    s.p[0][k] = (Real)p0; s.p[1][k] = (Real)p1; s.p[2][k] = (Real)p2;
    s.id[k] = (int32_t)k;
    if (s.species) {
        const uint8_t sp = species_in[k];
        if (sp >= n_species) bad = true;
        s.species[k] = sp;
    }
    if (s.param) {
        const double v = param_in[k];
        if (!(v >= 0.0) || isnan(v)) bad = true;
        s.param[k] = (Real)v;
    }
    if (bad) {
        atomicOr(&st[ST_LOAD_BAD], 1u);
        if (drop_bad) {
            // stored as a removed grain (NaN coordinate), species and
            // stopping-time value made harmless
            s.q[0][k] = __longlong_as_double(0x7ff8000000000000LL);
            if (s.species) s.species[k] = 0;
            if (s.param) s.param[k] = (Real)0;
            atomicAdd(reinterpret_cast<unsigned long long *>(&st[ST_REMOVED_LO]), 1ull);
        }
    }
}

template <typename Real, typename VT>
__global__ void get_particles_kernel(int geom, StoreDev<Real> s, double *q0, double *q1,
                                     double *q2, VT *v0, VT *v1, VT *v2, int64_t *ids)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.n) return;
    const double x0 = s.q[0][k], x1 = s.q[1][k], x2 = s.q[2][k];
    double p0 = s.p[0][k], p1 = s.p[1][k], p2 = s.p[2][k];
    if (geom == GEOM_CYL) p1 /= x0;
    if (geom == GEOM_SPH) {
        p1 /= x0;
        p2 /= x0 * sin(x1);
    }
    if (q0) q0[k] = x0;
    if (q1) q1[k] = x1;
    if (q2) q2[k] = x2;
    if (v0) v0[k] = (VT)p0;
    if (v1) v1[k] = (VT)p1;
    if (v2) v2[k] = (VT)p2;
    if (ids) ids[k] = s.id[k];
}

// Feedback on the gas momentum: rho p_g += dP / dV (corrector term of the
// RK2 step, Sec. 3.1; the gas is otherwise held fixed).
// Gas predicted to the half step: out = gas + impulse / (rho dV) in the three
// momentum-like channels (Sec. 3.1 predictor with the drag term only).
template <typename Real>
__global__ void predict_apply_kernel(GridDev g, double quantum, const Real *gas,
                                     const unsigned long long *imp, Real *out)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int k = (int)(c / ((int64_t)g.n[0] * g.n[1]));
    const double s = quantum / ((double)gas[4 * c] * g.dvol[0][i] * g.dvol[1][j] * g.dvol[2][k]);
    out[4 * c] = gas[4 * c];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
        out[4 * c + 1 + ch] = (Real)((double)gas[4 * c + 1 + ch] +
                                     (double)(long long)imp[4 * c + ch] * s);
}

template <typename Real>
__global__ void apply_feedback_kernel(GridDev g, double quantum, Real *gas,
                                      const unsigned long long *dep)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    apply_feedback_zone<Real>(g, quantum, gas, dep, c);
}

__global__ void dep_to_double_kernel(const unsigned long long *dep, int64_t n, double quantum,
                                     double *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = (double)(long long)dep[k] * quantum;
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <typename Real>
StoreDev<Real> store_of(dust_ctx *c, int which)
{
    StoreDev<Real> s;
    for (int d = 0; d < 3; ++d) {
        s.q[d] = c->d_q[which][d];
        s.p[d] = static_cast<Real *>(c->d_p[which][d]);
    }
    s.species = c->has_species ? c->d_species[which] : nullptr;
    s.param = c->has_param ? static_cast<Real *>(c->d_param[which]) : nullptr;
    s.id = c->d_id[which];
    s.n = c->n_grains;
    return s;
}

// Geometry constants of the step starting at t (the shear-periodic shifts of
// the shearing box at the half and the full step).
PhysDev make_phys(const dust_geometry &geo, const GridDev &g, double t, double dt)
{
    PhysDev ph{};
    ph.geom = geo.kind;
    ph.fargo = geo.fargo;
    ph.vgrav = geo.vertical_gravity;
    ph.omega = geo.omega;
    ph.qshear = geo.q;
    ph.gm = geo.gm;
    ph.q_om = geo.q * geo.omega;
    const double Lx = g.hi[0] - g.lo[0];
    const double Ly = g.hi[1] - g.lo[1];
    ph.jump_v = geo.q * geo.omega * Lx;
    if (geo.kind == DUST_SHEARING_BOX) {
        // same expression order as q Omega Lx t, reduced modulo Ly
        ph.shift_mid = fmod(geo.q * geo.omega * Lx * (t + 0.5 * dt), Ly);
        ph.shift_end = fmod(geo.q * geo.omega * Lx * (t + dt), Ly);
    }
    ph.omega_f = (float)ph.omega;
    ph.qshear_f = (float)ph.qshear;
    ph.gm_f = (float)ph.gm;
    ph.q_om_f = (float)ph.q_om;
    ph.jump_v_f = (float)ph.jump_v;
    return ph;
}

PhysDev phys_of(const dust_ctx *c, double t, double dt)
{
    PhysDev ph = make_phys(c->geom, c->g, t, dt);
    ph.pusher = c->opt.pusher;
    return ph;
}

int ensure_stage(dust_ctx *ctx, size_t bytes)
{
    if (ctx->stage_bytes >= bytes) return DUST_OK;
    dfree(ctx->d_stage);
    ctx->d_stage = nullptr;
    ctx->stage_bytes = 0;
    CU(cudaMalloc(reinterpret_cast<void **>(&ctx->d_stage), bytes));
    ctx->stage_bytes = bytes;
    return DUST_OK;
}

cudaEvent_t take_event(dust_ctx *ctx)
{
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records an event pair around a kernel group when timing is on.
struct GroupTimer {
    dust_ctx *ctx;
    int group;
    cudaEvent_t a = nullptr;
    GroupTimer(dust_ctx *c, int g) : ctx(c), group(g)
    {
        if (ctx->opt.timing && !ctx->capture_mode && (a = take_event(ctx)))
            cudaEventRecord(a, ctx->stream);
    }
    ~GroupTimer()
    {
        if (!a) return;
        cudaEvent_t b = take_event(ctx);
        if (!b) { ctx->event_pool.push_back(a); return; }
        cudaEventRecord(b, ctx->stream);
        ctx->pending[group].emplace_back(a, b);
    }
};

// Copy `count` doubles from caller memory into staging slot `slot` (device).
// Host array -> slot `slot` of the staging area (slots of count doubles; a
// float array uses the first half of its slot).
template <typename T>
const T *stage_in(dust_ctx *ctx, const T *src, int64_t count, int slot, int mem)
{
    if (!src) return nullptr;
    if (mem == DUST_MEM_DEVICE) return src;
    T *dst = reinterpret_cast<T *>(ctx->d_stage + (size_t)slot * count);
    cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
    return dst;
}

// ---- asynchronous host I/O helpers

int io_streams(dust_ctx *ctx)
{
    if (!ctx->io_in) CU(cudaStreamCreateWithFlags(&ctx->io_in, cudaStreamNonBlocking));
    if (!ctx->io_out) CU(cudaStreamCreateWithFlags(&ctx->io_out, cudaStreamNonBlocking));
    return DUST_OK;
}

// Makes b hold at least `bytes`; a reallocation first waits for its last use.
int io_ensure(dust_ctx *ctx, dust_ctx::IoBuf &b, size_t bytes)
{
    if (!b.ready) CU(cudaEventCreateWithFlags(&b.ready, cudaEventDisableTiming));
    if (!b.done) CU(cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming));
    if (b.bytes >= bytes) return DUST_OK;
    if (b.d) {
        if (b.used) CU(cudaEventSynchronize(b.done));
        CU(cudaFree(b.d));
        b.d = nullptr;
        b.bytes = 0;
    }
    CU(cudaMalloc(&b.d, bytes));
    b.bytes = bytes;
    return DUST_OK;
}

void io_free(dust_ctx::IoBuf &b)
{
    if (b.d) cudaFree(b.d);
    if (b.ready) cudaEventDestroy(b.ready);
    if (b.done) cudaEventDestroy(b.done);
    b = dust_ctx::IoBuf{};
}

// Input: after b's last consumer, copy the host arrays (src[k], bytes[k]) one
// after the other into b on the input copy stream; the context stream waits
// for them.  Returns the device address of each part in dev[k].
int io_stage_in(dust_ctx *ctx, dust_ctx::IoBuf &b, int parts, const void *const *src,
                const size_t *bytes, const void **dev)
{
    size_t total = 0;
    for (int k = 0; k < parts; ++k) total += (bytes[k] + 255) & ~(size_t)255;
    int r = io_ensure(ctx, b, total > 0 ? total : 256);
    if (r) return r;
    if (b.used) CU(cudaStreamWaitEvent(ctx->io_in, b.done, 0));
    size_t off = 0;
    for (int k = 0; k < parts; ++k) {
        if (!src[k]) { dev[k] = nullptr; continue; }
        void *d = static_cast<char *>(b.d) + off;
        CU(cudaMemcpyAsync(d, src[k], bytes[k], cudaMemcpyHostToDevice, ctx->io_in));
        dev[k] = d;
        off += (bytes[k] + 255) & ~(size_t)255;
    }
    CU(cudaEventRecord(b.ready, ctx->io_in));
    CU(cudaStreamWaitEvent(ctx->stream, b.ready, 0));
    return DUST_OK;
}

// The context stream has enqueued the last reader of input area b.
int io_consumed(dust_ctx *ctx, dust_ctx::IoBuf &b)
{
    CU(cudaEventRecord(b.done, ctx->stream));
    b.used = true;
    return DUST_OK;
}

// Output: the context stream waits until area b's previous read-back is done
// (before its producer kernel overwrites it).
int io_out_acquire(dust_ctx *ctx, dust_ctx::IoBuf &b, size_t bytes)
{
    int r = io_ensure(ctx, b, bytes);
    if (r) return r;
    if (b.used) CU(cudaStreamWaitEvent(ctx->stream, b.done, 0));
    return DUST_OK;
}

// Output: after the producer (enqueued on the context stream), copy the
// parts of b to the host on the output copy stream.
int io_stage_out(dust_ctx *ctx, dust_ctx::IoBuf &b, int parts, void *const *dst,
                 const void *const *dev, const size_t *bytes)
{
    CU(cudaEventRecord(b.ready, ctx->stream));
    CU(cudaStreamWaitEvent(ctx->io_out, b.ready, 0));
    for (int k = 0; k < parts; ++k)
        if (dst[k]) CU(cudaMemcpyAsync(dst[k], dev[k], bytes[k], cudaMemcpyDeviceToHost, ctx->io_out));
    CU(cudaEventRecord(b.done, ctx->io_out));
    b.used = true;
    return DUST_OK;
}

bool io_async(const dust_ctx *ctx, int mem)
{
    return ctx->opt.host_io_async && mem == DUST_MEM_HOST;
}

void free_store(dust_ctx *c)
{
    for (int w = 0; w < 2; ++w) {
        for (int d = 0; d < 3; ++d) {
            dfree(c->d_q[w][d]);
            dfree(c->d_p[w][d]);
            c->d_q[w][d] = nullptr;
            c->d_p[w][d] = nullptr;
        }
        dfree(c->d_species[w]);
        dfree(c->d_param[w]);
        dfree(c->d_id[w]);
        c->d_species[w] = nullptr;
        c->d_param[w] = nullptr;
        c->d_id[w] = nullptr;
    }
    dfree(c->d_key);
    dfree(c->d_pair_id);
    dfree(c->d_pair_src);
    dfree(c->d_pkey);
    dfree(c->d_ppair_id);
    dfree(c->d_ppair_src);
    c->d_pair_id = nullptr;
    c->d_pair_src = nullptr;
    c->d_key = nullptr;
    c->d_pkey = nullptr;
    c->d_ppair_id = nullptr;
    c->d_ppair_src = nullptr;
    c->cap = 0;
}

int alloc_store(dust_ctx *ctx, int64_t n)
{
    free_store(ctx);
    for (int w = 0; w < 2; ++w) {
        for (int d = 0; d < 3; ++d) {
            CU(dalloc(&ctx->d_q[w][d], n));
            CU(cudaMalloc(&ctx->d_p[w][d], n * ctx->rsz));
        }
        CU(dalloc(&ctx->d_id[w], n));
        if (ctx->has_species) CU(dalloc(&ctx->d_species[w], n));
        if (ctx->has_param) CU(cudaMalloc(&ctx->d_param[w], n * ctx->rsz));
    }
    CU(dalloc(&ctx->d_key, n));
    CU(dalloc(&ctx->d_pair_id, n));
    CU(dalloc(&ctx->d_pair_src, n));
    if (ctx->d_pcount) {
        CU(dalloc(&ctx->d_pkey, n));
        CU(dalloc(&ctx->d_ppair_id, n));
        CU(dalloc(&ctx->d_ppair_src, n));
    }
    ctx->cap = n;
    return DUST_OK;
}

template <typename Real>
int run_sort(dust_ctx *ctx, double dt, bool fused)
{
    SortArgs<Real> a;
    a.g = ctx->g;
    a.ph = phys_of(ctx, ctx->t, dt);
    a.dt = dt;
    a.src = store_of<Real>(ctx, ctx->cur);
    a.dst = store_of<Real>(ctx, 1 - ctx->cur);
    a.key = ctx->d_key;
    a.count = ctx->d_count_next;
    a.cursor = ctx->d_cursor;
    a.pair_id = ctx->d_pair_id;
    a.pair_src = ctx->d_pair_src;
    a.nkeys1 = ctx->g.nkeys + 1;
    a.big = ctx->d_bigseg;
    // scratch of the block sort: the key column (read by the scatter, next
    // written by the step) and the other store's ids (written after the sort)
    a.tmp_id = ctx->d_key;
    a.tmp_src = ctx->d_id[1 - ctx->cur];
    // counts of the nkeys + 1 keys and a zero: the exclusive scan then also
    // gives the end of the last (removed-grain) key's segment
    const int64_t m = ctx->g.nkeys + 2;
    GroupTimer timer(ctx, dust_ctx::GROUP_SORT);
    // keys predicted by the previous step for this dt are reused; otherwise
    // the key kernel computes them
    const bool reuse = ctx->keys_ready && ctx->keys_dt == dt;
    if (ctx->n_grains > 0) ctx->launches[dust_ctx::GROUP_SORT] += (reuse ? 7 : 8) - (fused ? 1 : 0);
    if (!reuse) {
        CU(cudaMemsetAsync(ctx->d_count_next, 0, m * sizeof(int32_t), ctx->stream));
        cudaError_t e = cudaSuccess;
        switch (ctx->geom.kind) {
        case DUST_CARTESIAN: e = launch_sort_keys<Real, GEOM_CART>(a, ctx->stream); break;
        case DUST_SHEARING_BOX: e = launch_sort_keys<Real, GEOM_SB>(a, ctx->stream); break;
        case DUST_CYLINDRICAL: e = launch_sort_keys<Real, GEOM_CYL>(a, ctx->stream); break;
        default: e = launch_sort_keys<Real, GEOM_SPH>(a, ctx->stream); break;
        }
        CU(e);
    }
    CU(launch_exclusive_scan(ctx->d_count_next, m, ctx->d_blocksums, ctx->stream));
    CU(cudaMemcpyAsync(ctx->d_cursor, ctx->d_count_next, m * sizeof(int32_t),
                       cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_bigseg, 0, sizeof(int32_t), ctx->stream));
    CU(launch_sort_scatter<Real>(a, ctx->stream, !fused));
    // fused: the step kernel moves the grains (and then flips the store)
    if (fused) ctx->perm_pending = true;
    else ctx->cur = 1 - ctx->cur;
    std::swap(ctx->d_count, ctx->d_count_next);
    ctx->keys_ready = false;
    return DUST_OK;
}

// Flat pattern the slab kernel supports for this grid: 0 (3-D), 1 (y not
// gridded), 2 (z not gridded); -1 = not supported (x not gridded, or 1-D).
inline int slab_flat(const GridDev &g)
{
    if (g.n[0] <= 1) return -1;
    if (g.n[1] > 1 && g.n[2] > 1) return 0;
    if (g.n[1] <= 1 && g.n[2] > 1) return 1;
    if (g.n[1] > 1 && g.n[2] <= 1) return 2;
    return -1;
}

// Slab kernel variant: the flat pattern, and the pusher / shearing-box frame
// fixed at compile time where the context allows (MODE, see launch_step_slab).
template <int GEOM, int FLAT>
cudaError_t launch_slab_mode(const TiledArgs<float> &ta, cudaStream_t s)
{
    const PhysDev &ph = ta.s.ph;
    if constexpr (GEOM == GEOM_CYL || GEOM == GEOM_SPH) {
        return launch_step_slab<GEOM, FLAT, 1>(ta, s);  // exponential midpoint only
    } else if constexpr (GEOM == GEOM_SB) {
        if (ph.pusher != DUST_PUSHER_EM) return launch_step_slab<GEOM, FLAT, 0>(ta, s);
        return ph.fargo ? launch_step_slab<GEOM, FLAT, 1>(ta, s) : launch_step_slab<GEOM, FLAT, 2>(ta, s);
    } else {
        return ph.pusher != DUST_PUSHER_EM ? launch_step_slab<GEOM, FLAT, 0>(ta, s)
                                           : launch_step_slab<GEOM, FLAT, 1>(ta, s);
    }
}

template <int GEOM>
cudaError_t launch_slab_geom(const TiledArgs<float> &ta, int flat, cudaStream_t s);

template <>
cudaError_t launch_slab_geom<GEOM_CART>(const TiledArgs<float> &ta, int flat, cudaStream_t s)
{
    return flat == 0 ? launch_slab_mode<GEOM_CART, 0>(ta, s) : launch_slab_mode<GEOM_CART, 2>(ta, s);
}
template <>
cudaError_t launch_slab_geom<GEOM_SB>(const TiledArgs<float> &ta, int flat, cudaStream_t s)
{
    return flat == 0 ? launch_slab_mode<GEOM_SB, 0>(ta, s)
                     : (flat == 1 ? launch_slab_mode<GEOM_SB, 1>(ta, s) : launch_slab_mode<GEOM_SB, 2>(ta, s));
}
template <>
cudaError_t launch_slab_geom<GEOM_CYL>(const TiledArgs<float> &ta, int, cudaStream_t s)
{
    return launch_slab_mode<GEOM_CYL, 0>(ta, s);
}
template <>
cudaError_t launch_slab_geom<GEOM_SPH>(const TiledArgs<float> &ta, int, cudaStream_t s)
{
    return launch_slab_mode<GEOM_SPH, 0>(ta, s);
}

// Whether volume weighting differs from CIC in this geometry (it has a
// curvilinear radius or polar angle); elsewhere it is CIC.
inline bool uses_volume_weights(int geom, int weight)
{
    return weight == DUST_WEIGHT_VOLUME && (geom == GEOM_CYL || geom == GEOM_SPH);
}

// Whether the slab kernel runs for this context: mixed precision, a
// supported flat pattern, and the geometry's instantiation.
inline bool slab_available(int geom, int flat)
{
    if (flat < 0) return false;
    if (geom == GEOM_CYL || geom == GEOM_SPH) return flat == 0;
    if (geom == GEOM_CART) return flat == 0 || flat == 2;
    return true;
}

template <typename Real, int GEOM>
cudaError_t launch_step_geom(const StepArgs<Real> &a, int weight, int kernel,
                             const int32_t *key_off, int32_t *key_out, int32_t *count_out,
                             const int32_t *perm, const int32_t *perm_id, const StoreDev<Real> &dst,
                             const void *gas_tmap, unsigned wait_extra_tx, cudaStream_t s)
{
    TiledArgs<Real> ta;
    ta.s = a;
    ta.gas_tmap = gas_tmap;
    ta.wait_extra_tx = wait_extra_tx;
    ta.wait_ns = wait_extra_tx ? 1000000ull : 0ull;  // the timeout test waits 1 ms
    ta.key_off = key_off;
    ta.tsc = weight == DUST_WEIGHT_TSC;
    const bool vol = (GEOM == GEOM_CYL || GEOM == GEOM_SPH) && weight == DUST_WEIGHT_VOLUME;
    ta.vol = vol ? 1 : 0;
    ta.emit_keys = key_out != nullptr;
    ta.key_out = key_out;
    ta.count_out = count_out;
    ta.perm = perm;
    ta.perm_id = perm_id;
    ta.dst = dst;
    if (kernel == DUST_KERNEL_PER_GRAIN) {
        if (perm) return cudaErrorInvalidValue;  // only the slab kernel gathers
        if constexpr (GEOM == GEOM_CYL || GEOM == GEOM_SPH)
            if (vol) return launch_step_per_grain<Real, GEOM, 2>(a, s);
        return weight == DUST_WEIGHT_TSC ? launch_step_per_grain<Real, GEOM, 1>(a, s)
                                         : launch_step_per_grain<Real, GEOM, 0>(a, s);
    }
    if constexpr (sizeof(Real) == 4) {
        const int flat = slab_flat(a.g);
        if ((kernel == DUST_KERNEL_AUTO || kernel == DUST_KERNEL_SLAB) && slab_available(GEOM, flat))
            return launch_slab_geom<GEOM>(ta, flat, s);
    }
    ta.emit_keys = 0;
    if (perm) return cudaErrorInvalidValue;  // only the slab kernel gathers
    if constexpr (GEOM == GEOM_CYL || GEOM == GEOM_SPH)
        if (vol) return launch_step_tiled<Real, GEOM, 2>(ta, s);
    return weight == DUST_WEIGHT_TSC ? launch_step_tiled<Real, GEOM, 1>(ta, s)
                                     : launch_step_tiled<Real, GEOM, 0>(ta, s);
}

// Whether the step kernel of this context predicts the next sort's keys: the
// slab kernel does (single-precision push, a supported flat pattern).
inline bool step_emits_keys(const dust_ctx *ctx)
{
    const int kn = ctx->opt.kernel;
    return ctx->mixed && (kn == DUST_KERNEL_AUTO || kn == DUST_KERNEL_SLAB) &&
           slab_available(ctx->geom.kind, slab_flat(ctx->g));
}

// Gas predictor of one geometry and weighting: the tiled kernel when tile
// arguments are given, else one thread per grain.
template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_predict_w(const StepArgs<Real> &pa, const TiledArgs<Real> *pt, cudaStream_t s)
{
    return pt ? launch_predict_tiled<Real, GEOM, WEIGHT>(*pt, s) : launch_predict_gas<Real, GEOM, WEIGHT>(pa, s);
}

template <typename Real, int GEOM>
cudaError_t launch_predict_g(int weight, const StepArgs<Real> &pa, const TiledArgs<Real> *pt, cudaStream_t s)
{
    if constexpr (GEOM == GEOM_CYL || GEOM == GEOM_SPH)
        if (weight == DUST_WEIGHT_VOLUME) return launch_predict_w<Real, GEOM, 2>(pa, pt, s);
    if (weight == DUST_WEIGHT_TSC) return launch_predict_w<Real, GEOM, 1>(pa, pt, s);
    return launch_predict_w<Real, GEOM, 0>(pa, pt, s);
}

template <typename Real>
cudaError_t launch_predict(int geom, int weight, const StepArgs<Real> &pa, const TiledArgs<Real> *pt,
                           cudaStream_t s)
{
    switch (geom) {
    case DUST_CARTESIAN: return launch_predict_g<Real, GEOM_CART>(weight, pa, pt, s);
    case DUST_SHEARING_BOX: return launch_predict_g<Real, GEOM_SB>(weight, pa, pt, s);
    case DUST_CYLINDRICAL: return launch_predict_g<Real, GEOM_CYL>(weight, pa, pt, s);
    default: return launch_predict_g<Real, GEOM_SPH>(weight, pa, pt, s);
    }
}

// The gas predictor's sort: the live store (the current store, before any
// pending gather) ordered by the key of the zone at x^n (zone_keys_kernel:
// the key kernel's keys with no drift), grains in id order inside a zone, as the pairs d_ppair_id /
// d_ppair_src with the zone offsets d_pcount.  The scratch of its block sort
// is the other store's id column, which the step writes afterwards.
int run_predictor_sort(dust_ctx *ctx)
{
    SortArgs<float> a;
    a.g = ctx->g;
    a.ph = phys_of(ctx, ctx->t, 0.0);
    a.dt = 0.0;
    a.src = store_of<float>(ctx, ctx->cur);
    a.dst = store_of<float>(ctx, 1 - ctx->cur);
    a.key = ctx->d_pkey;
    a.count = ctx->d_pcount;
    a.cursor = ctx->d_cursor;
    a.pair_id = ctx->d_ppair_id;
    a.pair_src = ctx->d_ppair_src;
    a.nkeys1 = ctx->g.nkeys + 1;
    a.big = ctx->d_bigseg;
    a.tmp_id = ctx->d_pkey;
    a.tmp_src = ctx->d_id[1 - ctx->cur];
    const int64_t m = ctx->g.nkeys + 2;
    CU(cudaMemsetAsync(ctx->d_pcount, 0, m * sizeof(int32_t), ctx->stream));
    cudaError_t e = cudaSuccess;
    switch (ctx->geom.kind) {
    case DUST_CARTESIAN: e = launch_zone_keys<GEOM_CART>(a, ctx->stream); break;
    case DUST_SHEARING_BOX: e = launch_zone_keys<GEOM_SB>(a, ctx->stream); break;
    case DUST_CYLINDRICAL: e = launch_zone_keys<GEOM_CYL>(a, ctx->stream); break;
    default: e = launch_zone_keys<GEOM_SPH>(a, ctx->stream); break;
    }
    CU(e);
    CU(launch_exclusive_scan(ctx->d_pcount, m, ctx->d_blocksums, ctx->stream));
    CU(cudaMemcpyAsync(ctx->d_cursor, ctx->d_pcount, m * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_bigseg, 0, sizeof(int32_t), ctx->stream));
    CU(launch_sort_scatter<float>(a, ctx->stream, false));
    if (ctx->n_grains > 0) ctx->launches[dust_ctx::GROUP_OTHER] += 7;
    return DUST_OK;
}

// Gas predictor on the slab layout, for the flat patterns the slab kernel has.
cudaError_t launch_predict_slab_any(int geom, const TiledArgs<float> &pt, int flat, cudaStream_t s)
{
    switch (geom) {
    case DUST_CARTESIAN:
        return flat == 0 ? launch_predict_slab<GEOM_CART, 0>(pt, s) : launch_predict_slab<GEOM_CART, 2>(pt, s);
    case DUST_SHEARING_BOX:
        return flat == 0 ? launch_predict_slab<GEOM_SB, 0>(pt, s)
                         : (flat == 1 ? launch_predict_slab<GEOM_SB, 1>(pt, s) : launch_predict_slab<GEOM_SB, 2>(pt, s));
    case DUST_CYLINDRICAL: return launch_predict_slab<GEOM_CYL, 0>(pt, s);
    default: return launch_predict_slab<GEOM_SPH, 0>(pt, s);
    }
}

template <typename Real>
int run_step(dust_ctx *ctx, double dt)
{
    StepArgs<Real> a;
    a.g = ctx->g;
    a.ph = phys_of(ctx, ctx->t, dt);
    a.sp = ctx->sp;
    species_coefficients(a.sp, ctx->geom.kind, ctx->geom.omega, dt);
    a.t = ctx->t;
    a.dt = dt;
    a.inv_quantum = 1.0 / ctx->quantum;
    a.s = store_of<Real>(ctx, ctx->cur);
    a.gas = static_cast<const Real *>(ctx->d_gas);
    a.dep = ctx->d_dep;
    a.status = ctx->d_status;
    a.tdev = ctx->capture_mode ? ctx->d_time : nullptr;
    {
        GroupTimer timer(ctx, dust_ctx::GROUP_OTHER);
        CU(cudaMemsetAsync(ctx->d_dep, 0, ctx->ncell * 4 * sizeof(unsigned long long), ctx->stream));
        if (ctx->opt.gas_predictor) {
            // predictor: drag of the grains at x^n advances the gas by dt/2;
            // the step gathers from the prediction, the feedback corrects the
            // gas at t^n
            CU(cudaMemsetAsync(ctx->d_pred, 0, ctx->ncell * 4 * sizeof(unsigned long long), ctx->stream));
            StepArgs<Real> pa = a;
            pa.dep = ctx->d_pred;
            cudaError_t pe;
            if (ctx->opt.kernel == DUST_KERNEL_PER_GRAIN) {
                // one thread per grain, global atomics (any store order)
                pe = launch_predict<Real>(ctx->geom.kind, ctx->opt.weight, pa, nullptr, ctx->stream);
            } else {
                // tiles of the last sort (through the pending permutation when
                // the step kernel finishes the sort); same integers
                TiledArgs<Real> pt{};
                pt.s = pa;
                pt.key_off = ctx->d_count;
                pt.perm = ctx->perm_pending ? ctx->d_pair_src : nullptr;
                // the predictor gathers the gas at t^n
                pt.gas_tmap = ctx->tmap_ok[0] ? static_cast<const void *>(ctx->d_tmaps) : nullptr;
                pt.wait_extra_tx = ctx->opt.test_wait_timeout ? 16u : 0u;
                pt.wait_ns = ctx->opt.test_wait_timeout ? 1000000ull : 0ull;
                pt.tsc = ctx->opt.weight == DUST_WEIGHT_TSC;
                pt.vol = uses_volume_weights(ctx->geom.kind, ctx->opt.weight) ? 1 : 0;
                if constexpr (sizeof(Real) == 4) {
                    // on the slab layout where the step runs the slab kernel,
                    // over the store sorted by the zone at x^n
                    if (step_emits_keys(ctx) && ctx->n_grains > 0) {
                        const int r = run_predictor_sort(ctx);
                        if (r) return r;
                        pt.key_off = ctx->d_pcount;
                        pt.perm = ctx->d_ppair_src;
                        pe = launch_predict_slab_any(ctx->geom.kind, pt, slab_flat(ctx->g), ctx->stream);
                    } else
                        pe = launch_predict<Real>(ctx->geom.kind, ctx->opt.weight, pa, &pt, ctx->stream);
                } else {
                    pe = launch_predict<Real>(ctx->geom.kind, ctx->opt.weight, pa, &pt, ctx->stream);
                }
            }
            CU(pe);
            predict_apply_kernel<Real><<<blocks_for(ctx->ncell), 256, 0, ctx->stream>>>(
                ctx->g, ctx->quantum, static_cast<const Real *>(ctx->d_gas), ctx->d_pred,
                static_cast<Real *>(ctx->d_gas_half));
            CU(cudaGetLastError());
            if (ctx->n_grains > 0) ctx->launches[dust_ctx::GROUP_OTHER] += 2;
            a.gas = static_cast<const Real *>(ctx->d_gas_half);
        }
    }
    cudaError_t e;
    GroupTimer *step_timer = new GroupTimer(ctx, dust_ctx::GROUP_STEP);
    if (ctx->n_grains > 0) ctx->launches[dust_ctx::GROUP_STEP] += 1;
    const int kn = ctx->opt.kernel;
    const int wt = ctx->opt.weight;
    const int32_t *ko = ctx->d_count;
    cudaStream_t st = ctx->stream;
    // the step before a sort predicts that sort's keys (for the same dt);
    // captured steps sort every step
    const bool emit = step_emits_keys(ctx) && ctx->n_grains > 0 &&
                      (ctx->capture_mode || (ctx->steps + 1) % ctx->sort_interval == 0);
    int32_t *kout = emit ? ctx->d_key : nullptr;
    int32_t *cout_ = emit ? ctx->d_count_next : nullptr;
    // a fused sort left its gather to this step: read the old store through
    // the permutation, write the other one
    const bool pend = ctx->perm_pending;
    const int32_t *perm = pend ? ctx->d_pair_src : nullptr;
    const int32_t *perm_id = pend ? ctx->d_pair_id : nullptr;
    const StoreDev<Real> dst = store_of<Real>(ctx, 1 - ctx->cur);
    if (emit)
        CU(cudaMemsetAsync(ctx->d_count_next, 0, (ctx->g.nkeys + 2) * sizeof(int32_t), st));
    // tensor map of the gas the step gathers from (the predicted gas or the
    // gas at t^n)
    const int tslot = ctx->opt.gas_predictor ? 1 : 0;
    const void *tmap = ctx->tmap_ok[tslot] ? static_cast<const void *>(ctx->d_tmaps + tslot) : nullptr;
    const unsigned xtx = ctx->opt.test_wait_timeout ? 16u : 0u;
    switch (ctx->geom.kind) {
    case DUST_CARTESIAN: e = launch_step_geom<Real, GEOM_CART>(a, wt, kn, ko, kout, cout_, perm, perm_id, dst, tmap, xtx, st); break;
    case DUST_SHEARING_BOX: e = launch_step_geom<Real, GEOM_SB>(a, wt, kn, ko, kout, cout_, perm, perm_id, dst, tmap, xtx, st); break;
    case DUST_CYLINDRICAL: e = launch_step_geom<Real, GEOM_CYL>(a, wt, kn, ko, kout, cout_, perm, perm_id, dst, tmap, xtx, st); break;
    default: e = launch_step_geom<Real, GEOM_SPH>(a, wt, kn, ko, kout, cout_, perm, perm_id, dst, tmap, xtx, st); break;
    }
    delete step_timer;
    CU(e);
    if (pend) {
        ctx->cur = 1 - ctx->cur;
        ctx->perm_pending = false;
    }
    ctx->keys_ready = emit;
    ctx->keys_dt = dt;
    if (ctx->opt.feedback_apply) {
        GroupTimer timer(ctx, dust_ctx::GROUP_OTHER);
        ctx->launches[dust_ctx::GROUP_OTHER] += 1;
        apply_feedback_kernel<Real><<<blocks_for(ctx->ncell), 256, 0, ctx->stream>>>(
            ctx->g, ctx->quantum, static_cast<Real *>(ctx->d_gas), ctx->d_dep);
        CU(cudaGetLastError());
    }
    return DUST_OK;
}

}  // namespace

// Tensor map of a gas array [ncell][4] (float in mixed precision, double in
// FP64) viewed as the 4-D array (channel, x, y, z), with the tile kernels'
// box (4, B0, B1, B2) (the tile plus its halo); written to device memory for
// the kernels.  The encoder is the driver's cuTensorMapEncodeTiled, fetched
// at run time.  Returns false (no bulk copy; plain loads) if anything is
// unavailable.
bool make_gas_tmap(dust_ctx *ctx, const void *gas, int slot)
{
    typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<EncodeTiled>(fn);
    }
    const GridDev &g = ctx->g;
    const cuuint64_t zone = 4 * (cuuint64_t)ctx->rsz;  // bytes per zone
    cuuint64_t dims[4] = {4, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    cuuint64_t strides[3] = {zone, zone * (cuuint64_t)g.n[0], zone * (cuuint64_t)g.n[0] * g.n[1]};
    cuuint32_t box[4] = {4, 1, 1, 1};
    for (int d = 0; d < 3; ++d) {
        box[d + 1] = (cuuint32_t)(g.T[d] + (g.n[d] > 1 ? 2 : 0));
        if (box[d + 1] > 256) return false;
    }
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUtensorMap map;
    const CUtensorMapDataType type = ctx->mixed ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    if (encode(&map, type, 4, const_cast<void *>(gas), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (!ctx->d_tmaps &&
        cudaMalloc(reinterpret_cast<void **>(&ctx->d_tmaps), 2 * sizeof(CUtensorMap)) != cudaSuccess)
        return false;
    return cudaMemcpy(ctx->d_tmaps + slot, &map, sizeof map, cudaMemcpyHostToDevice) == cudaSuccess;
}

// ================================================================ C API ====

extern "C" int dust_create(dust_ctx **out, const dust_geometry *geom, const dust_grid *grid,
                           const dust_species *species, int n_species, const dust_options *opt)
{
    if (!out) return fail(nullptr, DUST_EINVAL, "out is NULL");
    *out = nullptr;
    if (!geom || !grid || !species || !opt) return fail(nullptr, DUST_EINVAL, "NULL descriptor");
    if (opt->precision != DUST_FP64 && opt->precision != DUST_MIXED)
        return fail(nullptr, DUST_EINVAL, "bad precision");
    if (opt->pusher != DUST_PUSHER_EM && opt->pusher != DUST_PUSHER_SEMI_IMPLICIT)
        return fail(nullptr, DUST_EINVAL, "bad pusher");
    if (opt->gas_predictor != 0 && opt->gas_predictor != 1)
        return fail(nullptr, DUST_EINVAL, "gas_predictor must be 0 or 1");
    if (opt->host_io_async != 0 && opt->host_io_async != 1)
        return fail(nullptr, DUST_EINVAL, "host_io_async must be 0 or 1");
    if (opt->test_wait_timeout != 0 && opt->test_wait_timeout != 1)
        return fail(nullptr, DUST_EINVAL, "test_wait_timeout must be 0 or 1");
    // the slab kernel packs a zone's tile-local coordinates in 10-bit fields
    for (int d = 0; d < 3; ++d)
        if (opt->tile[d] < 0 || opt->tile[d] > 1023)
            return fail(nullptr, DUST_EINVAL, "tile[%d] must be 0 (default) or 1..1023 zones", d);
    if (opt->pusher == DUST_PUSHER_SEMI_IMPLICIT && geom->kind != DUST_CARTESIAN &&
        geom->kind != DUST_SHEARING_BOX)
        return fail(nullptr, DUST_EINVAL,
                    "the semi-implicit pusher is defined for Cartesian and shearing-box geometries");
    int64_t ncell = 0;
    const int rv = validate_descriptors(geom, grid, species, n_species, opt->weight, &ncell);
    if (rv) return rv;

    dust_ctx *ctx = new (std::nothrow) dust_ctx();
    if (!ctx) return fail(nullptr, DUST_ENOMEM, "host allocation failed");
    ctx->geom = *geom;
    ctx->opt = *opt;
    ctx->mixed = opt->precision == DUST_MIXED;
    ctx->rsz = ctx->mixed ? 4 : 8;
    ctx->device = opt->device;
    ctx->ncell = ncell;
    ctx->sort_interval = opt->sort_interval > 0 ? opt->sort_interval : 1;
    ctx->sp = make_species(species, n_species, opt->quantum, &ctx->quantum, ctx->mixed ? -40 : -44);

    auto bail = [&](int code) {
        std::string msg = ctx->err;
        dust_destroy(ctx);
        return fail(nullptr, code, "%s", msg.c_str());
    };
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        ctx->err = "cudaSetDevice failed";
        return bail(DUST_ECUDA);
    }
    if (opt->stream) {
        ctx->stream = static_cast<cudaStream_t>(opt->stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            ctx->err = "stream creation failed";
            return bail(DUST_ECUDA);
        }
        ctx->own_stream = true;
    }
    GridDev &g = ctx->g;
    g.ncell = ncell;
    for (int d = 0; d < 3; ++d) {
        const int n = grid->n[d];
        ctx->n[d] = n;
        ctx->bc[d] = grid->bc[d];
        ctx->edges[d].assign(grid->edges[d], grid->edges[d] + n + 1);
        const std::vector<double> &e = ctx->edges[d];
        grid_direction(g, d, e.data(), n, grid->bc[d]);
        std::vector<double> dv(n), zc(n), ziw(n);
        std::vector<float> dvf(n), ziwf(n), znuf(n), zlof(n + 1), zcf(n);
        std::vector<long long> ek(n + 1);
        fill_zone_tables(geom->kind, d, e.data(), n,
                         ZoneTables{dv.data(), zc.data(), ziw.data(), dvf.data(), ziwf.data(),
                                    znuf.data(), zlof.data(), zcf.data(), ek.data()});
        if (dalloc(&ctx->d_edges[d], n + 1) != cudaSuccess || dalloc(&ctx->d_dvol[d], n) != cudaSuccess ||
            dalloc(&ctx->d_dvol_f[d], n) != cudaSuccess || dalloc(&ctx->d_zc[d], n) != cudaSuccess ||
            dalloc(&ctx->d_ziw[d], n) != cudaSuccess || dalloc(&ctx->d_ziw_f[d], n) != cudaSuccess ||
            dalloc(&ctx->d_znu_f[d], n) != cudaSuccess || dalloc(&ctx->d_zlo_f[d], n + 1) != cudaSuccess ||
            dalloc(&ctx->d_ekey[d], n + 1) != cudaSuccess || dalloc(&ctx->d_zc_f[d], n) != cudaSuccess) {
            ctx->err = "device allocation of grid arrays failed";
            return bail(DUST_ENOMEM);
        }
        cudaMemcpy(ctx->d_edges[d], e.data(), (n + 1) * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_dvol[d], dv.data(), n * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_dvol_f[d], dvf.data(), n * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_zc[d], zc.data(), n * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_ziw[d], ziw.data(), n * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_ziw_f[d], ziwf.data(), n * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_znu_f[d], znuf.data(), n * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_zlo_f[d], zlof.data(), (n + 1) * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_zc_f[d], zcf.data(), n * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(ctx->d_ekey[d], ek.data(), (n + 1) * sizeof(long long), cudaMemcpyHostToDevice);
        g.zc_f[d] = ctx->d_zc_f[d];
        g.ekey[d] = ctx->d_ekey[d];
        g.edges[d] = ctx->d_edges[d];
        g.dvol[d] = ctx->d_dvol[d];
        g.dvol_f[d] = ctx->d_dvol_f[d];
        g.zc[d] = ctx->d_zc[d];
        g.ziw[d] = ctx->d_ziw[d];
        g.ziw_f[d] = ctx->d_ziw_f[d];
        g.znu_f[d] = ctx->d_znu_f[d];
        g.zlo_f[d] = ctx->d_zlo_f[d];
    }
    // tile layout: default 8^3 zones in 3-D, 16^2 in 2-D, 256 in 1-D
    {
        int nd = 0;
        for (int d = 0; d < 3; ++d) nd += grid->n[d] > 1;
        const int def = nd >= 3 ? 8 : (nd == 2 ? 16 : 256);
        g.tvol = 1;
        g.nkeys = 1;
        for (int d = 0; d < 3; ++d) {
            int t = opt->tile[d] > 0 ? opt->tile[d] : def;
            if (grid->n[d] <= 1) t = 1;
            if (t > grid->n[d]) t = grid->n[d];
            g.T[d] = t;
            g.nt[d] = (grid->n[d] + t - 1) / t;
            g.tvol *= t;
        }
        g.nkeys = (int64_t)g.nt[0] * g.nt[1] * g.nt[2] * g.tvol;
        if (g.nkeys + 2 >= ((int64_t)1 << 31)) {
            ctx->err = "too many sort keys for this tile layout";
            return bail(DUST_EINVAL);
        }
        const size_t smem = (size_t)(g.T[0] + (grid->n[0] > 1 ? 2 : 0)) *
                            (g.T[1] + (grid->n[1] > 1 ? 2 : 0)) *
                            (g.T[2] + (grid->n[2] > 1 ? 2 : 0)) * (4 * ctx->rsz + 32) +
                            256 * (8 + 13 * ctx->rsz + 64) + 16;
        if (smem > 220 * 1024) {
            ctx->err = "tile too large for shared memory";
            return bail(DUST_EINVAL);
        }
    }
    const int64_t nk = g.nkeys;
    if (cudaMalloc(&ctx->d_gas, ncell * 4 * ctx->rsz) != cudaSuccess ||
        dalloc(&ctx->d_dep, ncell * 4) != cudaSuccess ||
        (opt->gas_predictor && (dalloc(&ctx->d_pred, ncell * 4) != cudaSuccess ||
                                cudaMalloc(&ctx->d_gas_half, ncell * 4 * ctx->rsz) != cudaSuccess ||
                                (ctx->mixed && dalloc(&ctx->d_pcount, nk + 2) != cudaSuccess))) ||
        dalloc(&ctx->d_status, ST_WORDS) != cudaSuccess ||
        dalloc(&ctx->d_count, nk + 2) != cudaSuccess ||
        dalloc(&ctx->d_count_next, nk + 2) != cudaSuccess ||
        dalloc(&ctx->d_time, 4) != cudaSuccess ||
        dalloc(&ctx->d_cursor, nk + 2) != cudaSuccess ||
        dalloc(&ctx->d_bigseg, nk + 2) != cudaSuccess ||
        dalloc(&ctx->d_blocksums, scan_block_sums_size(nk + 2)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void **>(&ctx->h_status), ST_WORDS * sizeof(unsigned)) !=
            cudaSuccess) {
        ctx->err = "device allocation failed";
        return bail(DUST_ENOMEM);
    }
    cudaMemset(ctx->d_gas, 0, ncell * 4 * ctx->rsz);
    cudaMemset(ctx->d_dep, 0, ncell * 4 * sizeof(unsigned long long));
    ctx->tmap_ok[0] = make_gas_tmap(ctx, ctx->d_gas, 0);
    if (ctx->d_gas_half) ctx->tmap_ok[1] = make_gas_tmap(ctx, ctx->d_gas_half, 1);
    cudaMemset(ctx->d_status, 0, ST_WORDS * sizeof(unsigned));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        ctx->err = "device initialisation failed";
        return bail(DUST_ECUDA);
    }
    *out = ctx;
    return DUST_OK;
}

extern "C" int dust_set_gas(dust_ctx *ctx, const double *rho, const double *v0, const double *v1,
                            const double *v2, int mem)
{
    if (!ctx) return DUST_EINVAL;
    if (!rho || !v0 || !v1 || !v2) return fail(ctx, DUST_EINVAL, "NULL gas array");
    CU(cudaSetDevice(ctx->device));
    const int64_t nc = ctx->ncell;
    if (io_async(ctx, mem)) {
        // enqueue only; invalid values are reported by dust_sync
        int r = io_streams(ctx);
        if (r) return r;
        const void *src[4] = {rho, v0, v1, v2};
        const size_t by[4] = {nc * sizeof(double), nc * sizeof(double), nc * sizeof(double),
                              nc * sizeof(double)};
        const void *dv[4];
        r = io_stage_in(ctx, ctx->in_gas, 4, src, by, dv);
        if (r) return r;
        const double *a = static_cast<const double *>(dv[0]), *b = static_cast<const double *>(dv[1]),
                     *c = static_cast<const double *>(dv[2]), *d = static_cast<const double *>(dv[3]);
        if (ctx->mixed)
            set_gas_kernel<float><<<blocks_for(nc), 256, 0, ctx->stream>>>(
                ctx->g, ctx->geom.kind, a, b, c, d, static_cast<float *>(ctx->d_gas), ctx->d_status);
        else
            set_gas_kernel<double><<<blocks_for(nc), 256, 0, ctx->stream>>>(
                ctx->g, ctx->geom.kind, a, b, c, d, static_cast<double *>(ctx->d_gas), ctx->d_status);
        CU(cudaGetLastError());
        r = io_consumed(ctx, ctx->in_gas);
        if (r) return r;
        ctx->gas_set = true;
        return DUST_OK;
    }
    if (mem == DUST_MEM_HOST) {
        int r = ensure_stage(ctx, 4 * nc * sizeof(double));
        if (r) return r;
    }
    const double *a = stage_in(ctx, rho, nc, 0, mem), *b = stage_in(ctx, v0, nc, 1, mem),
                 *c = stage_in(ctx, v1, nc, 2, mem), *d = stage_in(ctx, v2, nc, 3, mem);
    CU(cudaMemsetAsync(ctx->d_status + ST_LOAD_BAD, 0, sizeof(unsigned), ctx->stream));
    if (ctx->mixed)
        set_gas_kernel<float><<<blocks_for(nc), 256, 0, ctx->stream>>>(
            ctx->g, ctx->geom.kind, a, b, c, d, static_cast<float *>(ctx->d_gas), ctx->d_status);
    else
        set_gas_kernel<double><<<blocks_for(nc), 256, 0, ctx->stream>>>(
            ctx->g, ctx->geom.kind, a, b, c, d, static_cast<double *>(ctx->d_gas), ctx->d_status);
    CU(cudaGetLastError());
    unsigned bad = 0;
    CU(cudaMemcpyAsync(&bad, ctx->d_status + ST_LOAD_BAD, sizeof bad, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (bad) return fail(ctx, DUST_EINVAL, "gas density must be positive and all values finite");
    ctx->gas_set = true;
    return DUST_OK;
}

extern "C" int dust_get_gas(dust_ctx *ctx, double *rho, double *v0, double *v1, double *v2, int mem)
{
    if (!ctx) return DUST_EINVAL;
    CU(cudaSetDevice(ctx->device));
    const int64_t nc = ctx->ncell;
    double *outs[4] = {rho, v0, v1, v2};
    double *dev[4] = {rho, v0, v1, v2};
    if (mem == DUST_MEM_HOST) {
        int r = ensure_stage(ctx, 4 * nc * sizeof(double));
        if (r) return r;
        for (int k = 0; k < 4; ++k) dev[k] = outs[k] ? ctx->d_stage + k * nc : nullptr;
    }
    if (ctx->mixed)
        get_gas_kernel<float><<<blocks_for(nc), 256, 0, ctx->stream>>>(
            ctx->g, ctx->geom.kind, static_cast<const float *>(ctx->d_gas), dev[0], dev[1], dev[2], dev[3]);
    else
        get_gas_kernel<double><<<blocks_for(nc), 256, 0, ctx->stream>>>(
            ctx->g, ctx->geom.kind, static_cast<const double *>(ctx->d_gas), dev[0], dev[1], dev[2], dev[3]);
    CU(cudaGetLastError());
    if (mem == DUST_MEM_HOST)
        for (int k = 0; k < 4; ++k)
            if (outs[k])
                CU(cudaMemcpyAsync(outs[k], dev[k], nc * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DUST_OK;
}

// dust_load_particles and dust_load_particles_v32: VT is the type of the
// velocity arrays.
template <typename VT>
int load_particles_impl(dust_ctx *ctx, int64_t n, const double *q0, const double *q1, const double *q2,
                        const VT *v0, const VT *v1, const VT *v2, const uint8_t *species,
                        const double *param, int mem)
{
    if (!ctx) return DUST_EINVAL;
    if (n < 0 || n >= ((int64_t)1 << 31) - 1) return fail(ctx, DUST_EINVAL, "bad grain count");
    if (n > 0 && (!q0 || !q1 || !q2 || !v0 || !v1 || !v2))
        return fail(ctx, DUST_EINVAL, "NULL particle array");
    CU(cudaSetDevice(ctx->device));
    const bool hs = species != nullptr, hp = param != nullptr;
    const bool async = io_async(ctx, mem);
    if (n > ctx->cap || hs != ctx->has_species || hp != ctx->has_param) {
        // the store is about to be replaced: finish the work that reads it
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->has_species = hs;
        ctx->has_param = hp;
        int r = alloc_store(ctx, n > 0 ? n : 1);
        if (r) return r;
    }
    ctx->n_grains = n;
    ctx->cur = 0;
    ctx->need_sort = true;
    ctx->keys_ready = false;
    ctx->perm_pending = false;
    ctx->gen += 1;
    if (n > 0) {
        const uint8_t *sp_dev = species;
        const double *a, *b, *c, *pp;
        const VT *d, *e, *f;
        if (async) {
            // enqueue only: copies on the input stream; invalid grains are
            // dropped and reported by dust_sync
            int r = io_streams(ctx);
            if (r) return r;
            const size_t nb = n * sizeof(double), nv = n * sizeof(VT);
            const void *src[8] = {q0, q1, q2, v0, v1, v2, param, species};
            const size_t by[8] = {nb, nb, nb, nv, nv, nv, nb, (size_t)n};
            const void *dv[8];
            r = io_stage_in(ctx, ctx->in_grains, 8, src, by, dv);
            if (r) return r;
            a = static_cast<const double *>(dv[0]);
            b = static_cast<const double *>(dv[1]);
            c = static_cast<const double *>(dv[2]);
            d = static_cast<const VT *>(dv[3]);
            e = static_cast<const VT *>(dv[4]);
            f = static_cast<const VT *>(dv[5]);
            pp = static_cast<const double *>(dv[6]);
            sp_dev = static_cast<const uint8_t *>(dv[7]);
        } else {
            if (mem == DUST_MEM_HOST) {
                const size_t need = (7 * n) * sizeof(double) + (hs ? n : 0) + 16;
                int r = ensure_stage(ctx, need);
                if (r) return r;
            }
            a = stage_in(ctx, q0, n, 0, mem);
            b = stage_in(ctx, q1, n, 1, mem);
            c = stage_in(ctx, q2, n, 2, mem);
            d = stage_in(ctx, v0, n, 3, mem);
            e = stage_in(ctx, v1, n, 4, mem);
            f = stage_in(ctx, v2, n, 5, mem);
            pp = stage_in(ctx, param, n, 6, mem);
            if (hs && mem == DUST_MEM_HOST) {
                uint8_t *dst = reinterpret_cast<uint8_t *>(ctx->d_stage + 7 * n);
                CU(cudaMemcpyAsync(dst, species, n, cudaMemcpyHostToDevice, ctx->stream));
                sp_dev = dst;
            }
            CU(cudaMemsetAsync(ctx->d_status + ST_LOAD_BAD, 0, sizeof(unsigned), ctx->stream));
        }
        if (ctx->mixed)
            load_kernel<float, VT><<<blocks_for(n), 256, 0, ctx->stream>>>(
                ctx->g, ctx->geom.kind, n, a, b, c, d, e, f, sp_dev, ctx->sp.n, pp,
                store_of<float>(ctx, 0), ctx->d_status, async ? 1 : 0);
        else
            load_kernel<double, VT><<<blocks_for(n), 256, 0, ctx->stream>>>(
                ctx->g, ctx->geom.kind, n, a, b, c, d, e, f, sp_dev, ctx->sp.n, pp,
                store_of<double>(ctx, 0), ctx->d_status, async ? 1 : 0);
        CU(cudaGetLastError());
        if (async) {
            int r = io_consumed(ctx, ctx->in_grains);
            if (r) return r;
            ctx->particles_set = true;
            return DUST_OK;
        }
        unsigned bad = 0;
        CU(cudaMemcpyAsync(&bad, ctx->d_status + ST_LOAD_BAD, sizeof bad, cudaMemcpyDeviceToHost,
                           ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        if (bad) {
            ctx->particles_set = false;
            return fail(ctx, DUST_EINVAL,
                        "grain data must be finite, inside the grid, with valid species/param");
        }
    }
    ctx->particles_set = true;
    return DUST_OK;
}

extern "C" int dust_load_particles(dust_ctx *ctx, int64_t n, const double *q0, const double *q1,
                                   const double *q2, const double *v0, const double *v1,
                                   const double *v2, const uint8_t *species, const double *param,
                                   int mem)
{
    return load_particles_impl<double>(ctx, n, q0, q1, q2, v0, v1, v2, species, param, mem);
}

extern "C" int dust_load_particles_v32(dust_ctx *ctx, int64_t n, const double *q0, const double *q1,
                                       const double *q2, const float *v0, const float *v1,
                                       const float *v2, const uint8_t *species, const double *param,
                                       int mem)
{
    return load_particles_impl<float>(ctx, n, q0, q1, q2, v0, v1, v2, species, param, mem);
}

extern "C" int dust_step(dust_ctx *ctx, double dt)
{
    if (!ctx) return DUST_EINVAL;
    if (!std::isfinite(dt)) return fail(ctx, DUST_EINVAL, "dt must be finite");
    if (!ctx->gas_set || !ctx->particles_set)
        return fail(ctx, DUST_ESTATE, "set the gas and load particles before stepping");
    CU(cudaSetDevice(ctx->device));
    int r;
    if (ctx->need_sort || ctx->steps % ctx->sort_interval == 0) {
        const bool fused = step_emits_keys(ctx);  // the slab kernel will move the grains
        r = ctx->mixed ? run_sort<float>(ctx, dt, fused) : run_sort<double>(ctx, dt, fused);
        if (r) return r;
        ctx->need_sort = false;
    }
    r = ctx->mixed ? run_step<float>(ctx, dt) : run_step<double>(ctx, dt);
    if (r) return r;
    ctx->t += dt;
    ctx->last_dt = dt;
    ctx->steps += 1;
    ctx->timed_steps += 1;
    ctx->have_deposit = true;
    return DUST_OK;
}

extern "C" int dust_get_kernel_times(dust_ctx *ctx, dust_kernel_times *out, int reset)
{
    if (!ctx) return DUST_EINVAL;
    CU(cudaSetDevice(ctx->device));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int g = 0; g < dust_ctx::N_GROUPS; ++g) {
        for (auto &pr : ctx->pending[g]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) ctx->group_ms[g] += ms;
            ctx->event_pool.push_back(pr.first);
            ctx->event_pool.push_back(pr.second);
        }
        ctx->pending[g].clear();
    }
    if (out) {
        out->step_ms = ctx->group_ms[dust_ctx::GROUP_STEP];
        out->sort_ms = ctx->group_ms[dust_ctx::GROUP_SORT];
        out->other_ms = ctx->group_ms[dust_ctx::GROUP_OTHER];
        out->step_launches = ctx->launches[dust_ctx::GROUP_STEP];
        out->sort_launches = ctx->launches[dust_ctx::GROUP_SORT];
        out->other_launches = ctx->launches[dust_ctx::GROUP_OTHER];
        out->steps = ctx->timed_steps;
    }
    if (reset) {
        for (int g = 0; g < dust_ctx::N_GROUPS; ++g) {
            ctx->group_ms[g] = 0.0;
            ctx->launches[g] = 0;
        }
        ctx->timed_steps = 0;
    }
    return DUST_OK;
}

extern "C" int dust_sync(dust_ctx *ctx, dust_stats *out)
{
    if (!ctx) return DUST_EINVAL;
    CU(cudaSetDevice(ctx->device));
    // pending asynchronous host copies
    if (ctx->io_in) CU(cudaStreamSynchronize(ctx->io_in));
    if (ctx->io_out) CU(cudaStreamSynchronize(ctx->io_out));
    CU(cudaMemcpyAsync(ctx->h_status, ctx->d_status, ST_WORDS * sizeof(unsigned),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    unsigned st[ST_WORDS];
    memcpy(st, ctx->h_status, sizeof st);
    CU(cudaMemsetAsync(ctx->d_status, 0, 4 * sizeof(unsigned), ctx->stream));
    const bool load_bad = ctx->opt.host_io_async && st[ST_LOAD_BAD];
    if (load_bad) CU(cudaMemsetAsync(ctx->d_status + ST_LOAD_BAD, 0, sizeof(unsigned), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const unsigned long long rem =
        (unsigned long long)st[ST_REMOVED_LO] | ((unsigned long long)st[ST_REMOVED_HI] << 32);
    ctx->removed_total += (int64_t)rem;
    float mv;
    memcpy(&mv, &st[ST_MAXMOVE], sizeof mv);
    ctx->max_moved = fmaxf(ctx->max_moved, mv);
    int flags = (int)st[ST_FLAGS];
    if (mv > 1.8f) flags |= DUST_FLAG_CFL;
    if (out) {
        out->n_stored = ctx->n_grains;
        out->n_removed = ctx->removed_total;
        out->n_active = ctx->n_grains - ctx->removed_total;
        out->max_cells_moved = ctx->max_moved;
        out->flags = flags;
        out->steps = ctx->steps;
        out->time = ctx->t;
        // Eq. particles_dt: the largest displacement of these steps in zones
        // is dt max_{p,d} |v_d^{n+1/2}| / dl_d
        out->dt_dust = mv > 0.f ? 1.8 * fabs(ctx->last_dt) / (double)mv : INFINITY;
    }
    if (load_bad)
        return fail(ctx, DUST_EINVAL,
                    "invalid grain or gas data in an asynchronous load (invalid grains were dropped)");
    if (flags & DUST_FLAG_TIMEOUT)
        return fail(ctx, DUST_ETIMEOUT, "a bounded device wait gave up; the step's results are void");
    if (flags & DUST_FLAG_NAN) return fail(ctx, DUST_ENAN, "NaN/Inf produced on the device");
    if (flags & DUST_FLAG_OVERFLOW)
        return fail(ctx, DUST_EOVERFLOW, "fixed-point deposit piece beyond 2^52 quanta");
    if (flags & DUST_FLAG_CFL)
        return fail(ctx, DUST_ECFL, "a grain moved %.3g zones in one step (limit 1.8)", mv);
    return DUST_OK;
}

extern "C" int dust_get_deposit(dust_ctx *ctx, int64_t *fixed, double *as_double,
                                double *quantum_out, int mem)
{
    if (!ctx) return DUST_EINVAL;
    if (quantum_out) *quantum_out = ctx->quantum;
    if (!fixed && !as_double) return DUST_OK;
    CU(cudaSetDevice(ctx->device));
    const int64_t m = ctx->ncell * 4;
    if (io_async(ctx, mem)) {
        // enqueue only: snapshot into one of two staging areas (the next
        // step overwrites the deposit), read back on the output stream
        int r = io_streams(ctx);
        if (r) return r;
        dust_ctx::IoBuf &b = ctx->out_dep[ctx->dep_flip];
        ctx->dep_flip ^= 1;
        r = io_out_acquire(ctx, b, 2 * m * sizeof(int64_t));
        if (r) return r;
        int64_t *fx = fixed ? static_cast<int64_t *>(b.d) : nullptr;
        double *dd = as_double ? reinterpret_cast<double *>(static_cast<int64_t *>(b.d) + m) : nullptr;
        if (fixed)
            CU(cudaMemcpyAsync(fx, ctx->d_dep, m * sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx->stream));
        if (as_double) {
            dep_to_double_kernel<<<blocks_for(m), 256, 0, ctx->stream>>>(ctx->d_dep, m, ctx->quantum, dd);
            CU(cudaGetLastError());
        }
        void *dst[2] = {fixed, as_double};
        const void *src[2] = {fx, dd};
        const size_t by[2] = {m * sizeof(int64_t), m * sizeof(double)};
        return io_stage_out(ctx, b, 2, dst, src, by);
    }
    const cudaMemcpyKind kind = mem == DUST_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (fixed) CU(cudaMemcpyAsync(fixed, ctx->d_dep, m * sizeof(int64_t), kind, ctx->stream));
    if (as_double) {
        double *dst = as_double;
        if (mem == DUST_MEM_HOST) {
            int r = ensure_stage(ctx, m * sizeof(double));
            if (r) return r;
            dst = ctx->d_stage;
        }
        dep_to_double_kernel<<<blocks_for(m), 256, 0, ctx->stream>>>(ctx->d_dep, m, ctx->quantum, dst);
        CU(cudaGetLastError());
        if (mem == DUST_MEM_HOST)
            CU(cudaMemcpyAsync(as_double, dst, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return DUST_OK;
}

extern "C" int dust_get_mass_deposit(dust_ctx *ctx, int64_t *fixed, double *as_double,
                                     double *quantum_out, int mem)
{
    if (!ctx) return DUST_EINVAL;
    if (quantum_out) *quantum_out = ctx->quantum;
    if (!fixed && !as_double) return DUST_OK;
    if (!ctx->particles_set) return fail(ctx, DUST_ESTATE, "load particles first");
    CU(cudaSetDevice(ctx->device));
    const int64_t nc = ctx->ncell;
    if (!ctx->d_mass) CU(dalloc(&ctx->d_mass, nc));
    CU(cudaMemsetAsync(ctx->d_mass, 0, nc * sizeof(unsigned long long), ctx->stream));
    const double *q[3];
    const uint8_t *species = nullptr;
    if (ctx->mixed) {
        const StoreDev<float> st = store_of<float>(ctx, ctx->cur);
        for (int d = 0; d < 3; ++d) q[d] = st.q[d];
        species = st.species;
    } else {
        const StoreDev<double> st = store_of<double>(ctx, ctx->cur);
        for (int d = 0; d < 3; ++d) q[d] = st.q[d];
        species = st.species;
    }
    // the current store holds every grain (when a sort's gather is pending,
    // in the previous order; the per-grain rule does not depend on it)
    cudaError_t e;
    const int wk = ctx->opt.weight;
    switch (ctx->geom.kind) {
    case DUST_CARTESIAN: e = launch_deposit_mass<GEOM_CART>(ctx->g, ctx->sp, wk, ctx->n_grains, q, species, ctx->d_mass, ctx->d_status, ctx->stream); break;
    case DUST_SHEARING_BOX: e = launch_deposit_mass<GEOM_SB>(ctx->g, ctx->sp, wk, ctx->n_grains, q, species, ctx->d_mass, ctx->d_status, ctx->stream); break;
    case DUST_CYLINDRICAL: e = launch_deposit_mass<GEOM_CYL>(ctx->g, ctx->sp, wk, ctx->n_grains, q, species, ctx->d_mass, ctx->d_status, ctx->stream); break;
    default: e = launch_deposit_mass<GEOM_SPH>(ctx->g, ctx->sp, wk, ctx->n_grains, q, species, ctx->d_mass, ctx->d_status, ctx->stream); break;
    }
    CU(e);
    const cudaMemcpyKind kind = mem == DUST_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (fixed) CU(cudaMemcpyAsync(fixed, ctx->d_mass, nc * sizeof(int64_t), kind, ctx->stream));
    if (as_double) {
        double *dst = as_double;
        if (mem == DUST_MEM_HOST) {
            int r = ensure_stage(ctx, nc * sizeof(double));
            if (r) return r;
            dst = ctx->d_stage;
        }
        dep_to_double_kernel<<<blocks_for(nc), 256, 0, ctx->stream>>>(ctx->d_mass, nc, ctx->quantum, dst);
        CU(cudaGetLastError());
        if (mem == DUST_MEM_HOST)
            CU(cudaMemcpyAsync(as_double, dst, nc * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return DUST_OK;
}

// The read-back kernel into dev[0..5] (positions, then velocities of type VT)
// and ids.
template <typename VT>
void launch_get_particles(dust_ctx *ctx, void *const dev[6], int64_t *dids)
{
    const int64_t n = ctx->n_grains;
    double *q[3] = {static_cast<double *>(dev[0]), static_cast<double *>(dev[1]), static_cast<double *>(dev[2])};
    VT *v[3] = {static_cast<VT *>(dev[3]), static_cast<VT *>(dev[4]), static_cast<VT *>(dev[5])};
    if (ctx->mixed)
        get_particles_kernel<float, VT><<<blocks_for(n), 256, 0, ctx->stream>>>(
            ctx->geom.kind, store_of<float>(ctx, ctx->cur), q[0], q[1], q[2], v[0], v[1], v[2], dids);
    else
        get_particles_kernel<double, VT><<<blocks_for(n), 256, 0, ctx->stream>>>(
            ctx->geom.kind, store_of<double>(ctx, ctx->cur), q[0], q[1], q[2], v[0], v[1], v[2], dids);
}

// dust_get_particles and dust_get_particles_v32: VT is the type of the
// velocity arrays.
template <typename VT>
int get_particles_impl(dust_ctx *ctx, int64_t cap, double *q0, double *q1, double *q2, VT *v0, VT *v1,
                       VT *v2, int64_t *ids, int64_t *n_out, int mem)
{
    if (!ctx || !n_out) return DUST_EINVAL;
    *n_out = 0;
    const int64_t n = ctx->n_grains;
    if (cap < n) return fail(ctx, DUST_EINVAL, "capacity %lld < %lld grains", (long long)cap, (long long)n);
    if (n == 0) return DUST_OK;
    CU(cudaSetDevice(ctx->device));
    // the velocity columns use the first half of their double-sized slots
    // when VT is float
    void *outs[6] = {q0, q1, q2, v0, v1, v2};
    void *dev[6] = {q0, q1, q2, v0, v1, v2};
    const size_t esz[6] = {sizeof(double), sizeof(double), sizeof(double), sizeof(VT), sizeof(VT), sizeof(VT)};
    int64_t *dids = ids;
    if (io_async(ctx, mem)) {
        // enqueue only: convert into one of two staging areas, read back on
        // the output stream (done at the next dust_sync)
        int r = io_streams(ctx);
        if (r) return r;
        dust_ctx::IoBuf &b = ctx->out_grains[ctx->out_flip];
        ctx->out_flip ^= 1;
        r = io_out_acquire(ctx, b, 7 * n * sizeof(double));
        if (r) return r;
        double *base = static_cast<double *>(b.d);
        for (int k = 0; k < 6; ++k) dev[k] = outs[k] ? static_cast<void *>(base + k * n) : nullptr;
        dids = ids ? reinterpret_cast<int64_t *>(base + 6 * n) : nullptr;
        launch_get_particles<VT>(ctx, dev, dids);
        CU(cudaGetLastError());
        void *dst[7] = {q0, q1, q2, v0, v1, v2, ids};
        const void *src[7] = {dev[0], dev[1], dev[2], dev[3], dev[4], dev[5], dids};
        size_t by[7];
        for (int k = 0; k < 6; ++k) by[k] = n * esz[k];
        by[6] = n * sizeof(int64_t);
        r = io_stage_out(ctx, b, 7, dst, src, by);
        if (r) return r;
        *n_out = n;
        return DUST_OK;
    }
    if (mem == DUST_MEM_HOST) {
        int r = ensure_stage(ctx, 7 * n * sizeof(double));
        if (r) return r;
        for (int k = 0; k < 6; ++k) dev[k] = outs[k] ? static_cast<void *>(ctx->d_stage + k * n) : nullptr;
        dids = ids ? reinterpret_cast<int64_t *>(ctx->d_stage + 6 * n) : nullptr;
    }
    launch_get_particles<VT>(ctx, dev, dids);
    CU(cudaGetLastError());
    if (mem == DUST_MEM_HOST) {
        for (int k = 0; k < 6; ++k)
            if (outs[k])
                CU(cudaMemcpyAsync(outs[k], dev[k], n * esz[k], cudaMemcpyDeviceToHost, ctx->stream));
        if (ids) CU(cudaMemcpyAsync(ids, dids, n * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    *n_out = n;
    return DUST_OK;
}

extern "C" int dust_get_particles(dust_ctx *ctx, int64_t cap, double *q0, double *q1, double *q2,
                                  double *v0, double *v1, double *v2, int64_t *ids,
                                  int64_t *n_out, int mem)
{
    return get_particles_impl<double>(ctx, cap, q0, q1, q2, v0, v1, v2, ids, n_out, mem);
}

extern "C" int dust_get_particles_v32(dust_ctx *ctx, int64_t cap, double *q0, double *q1, double *q2,
                                      float *v0, float *v1, float *v2, int64_t *ids,
                                      int64_t *n_out, int mem)
{
    return get_particles_impl<float>(ctx, cap, q0, q1, q2, v0, v1, v2, ids, n_out, mem);
}

extern "C" const char *dust_last_error(const dust_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

extern "C" void dust_destroy(dust_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (cudaStream_t io : {ctx->io_in, ctx->io_out})
        if (io) {
            cudaStreamSynchronize(io);
            cudaStreamDestroy(io);
        }
    io_free(ctx->in_grains);
    io_free(ctx->in_gas);
    for (int k = 0; k < 2; ++k) {
        io_free(ctx->out_grains[k]);
        io_free(ctx->out_dep[k]);
    }
    free_store(ctx);
    for (int d = 0; d < 3; ++d) {
        dfree(ctx->d_edges[d]);
        dfree(ctx->d_dvol[d]);
        dfree(ctx->d_dvol_f[d]);
        dfree(ctx->d_zc[d]);
        dfree(ctx->d_ekey[d]);
        dfree(ctx->d_ziw[d]);
        dfree(ctx->d_ziw_f[d]);
        dfree(ctx->d_znu_f[d]);
        dfree(ctx->d_zlo_f[d]);
        dfree(ctx->d_zc_f[d]);
    }
    dfree(ctx->d_gas);
    dfree(ctx->d_dep);
    dfree(ctx->d_pred);
    dfree(ctx->d_pcount);
    dfree(ctx->d_gas_half);
    dfree(ctx->d_tmaps);
    dfree(ctx->d_status);
    dfree(ctx->d_count);
    dfree(ctx->d_count_next);
    dfree(ctx->d_time);
    dfree(ctx->d_cursor);
    dfree(ctx->d_bigseg);
    dfree(ctx->d_blocksums);
    dfree(ctx->d_stage);
    dfree(ctx->d_mass);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    for (int g = 0; g < dust_ctx::N_GROUPS; ++g)
        for (auto &pr : ctx->pending[g]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

// ------------------------------------------------------- batched steps ----
//
// A batch steps many independent contexts (instances of different grids,
// sizes and species) with one graph launch per two steps.  The graph is
// captured once from the contexts' own streams: each instance is a branch
// (sort, deposit clear, step, feedback, time advance, twice), so the
// instances run concurrently and the per-kernel launch cost is paid once per
// capture.  Captured steps read their time and shear-periodic shifts from
// the device (a small kernel advances them), sort before every step and let
// the step kernel predict the next sort's keys.  Two steps make one period
// because the sort alternates the grain store and the key-count buffers.

struct dust_batch {
    int device = 0;
    std::vector<dust_ctx *> ctx;
    cudaStream_t root = nullptr;
    bool own_root = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    std::vector<cudaEvent_t> join;
    // what the captured graph assumed about each instance
    std::vector<double> dt;
    std::vector<uint64_t> gen;
    std::vector<int> cur;
    std::vector<int32_t *> count;
    std::vector<std::array<int64_t, dust_ctx::N_GROUPS>> period_launches;
    std::string err;
    // one persistent launch for all instances (batch_persistent_kernel):
    // the instances' descriptors (page-locked host copy, device copy), the
    // work list, and a graph of the call (descriptor copy, counter reset,
    // the launch) per work list
    int mode = 0;               // 0: persistent where the instances allow it; 1: graph
    int sort_interval = 1;
    int test_timeout = 0;
    BatchInst *h_inst = nullptr, *d_inst = nullptr;
    // the work list of the captured launch (tasks, groups, item prefix
    // sums; then the completion counts and the item counter, zeroed by the
    // graph) and its shape
    int *d_tab = nullptr;
    size_t tab_cap = 0;
    std::vector<int> tab;
    BatchDev pdev{};
    cudaEvent_t inst_copied = nullptr;
    cudaGraph_t pgraph = nullptr;
    cudaGraphExec_t pexec = nullptr;
    int pvariant = -1;
    size_t psmem = 0;
    int pgrid = 0;
};

namespace {

thread_local std::string g_batch_error;

int bfail(dust_batch *b, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    g_batch_error = buf;
    return code;
}

#define BCU(call)                                                                    \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return bfail(b, DUST_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

__global__ void set_time_kernel(double *tm, double t, double shift_mid, double shift_end)
{
    tm[0] = t;
    tm[1] = shift_mid;
    tm[2] = shift_end;
}

// t += dt, then the shifts of the step that starts at the new t, with the
// same operations as make_phys: fmod(((q Omega) Lx) (t + dt/2), Ly).
__global__ void time_advance_kernel(double *tm, double dt, double q_om_lx, double ly, int sb)
{
    advance_time(tm, dt, q_om_lx, ly, sb);
}

// Keys of the first sort of a captured period, computed now for the current
// store (the graph's sorts reuse the keys the previous step predicted).
template <typename Real>
int prime_keys(dust_ctx *ctx, double dt)
{
    SortArgs<Real> a;
    a.g = ctx->g;
    a.ph = phys_of(ctx, ctx->t, dt);
    a.dt = dt;
    a.src = store_of<Real>(ctx, ctx->cur);
    a.dst = store_of<Real>(ctx, 1 - ctx->cur);
    a.key = ctx->d_key;
    a.count = ctx->d_count_next;
    a.cursor = ctx->d_cursor;
    a.pair_id = ctx->d_pair_id;
    a.pair_src = ctx->d_pair_src;
    a.nkeys1 = ctx->g.nkeys + 1;
    a.big = ctx->d_bigseg;
    a.tmp_id = ctx->d_key;
    a.tmp_src = ctx->d_id[1 - ctx->cur];
    CU(cudaMemsetAsync(ctx->d_count_next, 0, (ctx->g.nkeys + 2) * sizeof(int32_t), ctx->stream));
    cudaError_t e;
    switch (ctx->geom.kind) {
    case DUST_CARTESIAN: e = launch_sort_keys<Real, GEOM_CART>(a, ctx->stream); break;
    case DUST_SHEARING_BOX: e = launch_sort_keys<Real, GEOM_SB>(a, ctx->stream); break;
    case DUST_CYLINDRICAL: e = launch_sort_keys<Real, GEOM_CYL>(a, ctx->stream); break;
    default: e = launch_sort_keys<Real, GEOM_SPH>(a, ctx->stream); break;
    }
    CU(e);
    if (ctx->n_grains > 0) ctx->launches[dust_ctx::GROUP_SORT] += 1;
    ctx->keys_ready = true;
    ctx->keys_dt = dt;
    return DUST_OK;
}

// Enqueue one period (two steps) of a context into the running capture.
template <typename Real>
int capture_period(dust_ctx *ctx, double dt)
{
    const double Lx = ctx->g.hi[0] - ctx->g.lo[0], Ly = ctx->g.hi[1] - ctx->g.lo[1];
    const double q_om_lx = ctx->geom.q * ctx->geom.omega * Lx;
    const int sb = ctx->geom.kind == DUST_SHEARING_BOX;
    for (int k = 0; k < 2; ++k) {
        int r = run_sort<Real>(ctx, dt, step_emits_keys(ctx));
        if (r) return r;
        r = run_step<Real>(ctx, dt);
        if (r) return r;
        time_advance_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_time, dt, q_om_lx, Ly, sb);
        CU(cudaGetLastError());
    }
    return DUST_OK;
}

void drop_graph(dust_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

int capture(dust_batch *b, const double *dt)
{
    drop_graph(b);
    const size_t n = b->ctx.size();
    // host state the capture changes and a failed capture must restore
    struct Saved { int cur; int32_t *count, *count_next; bool keys_ready; double keys_dt;
                   int64_t launches[dust_ctx::N_GROUPS]; };
    std::vector<Saved> saved(n);
    for (size_t i = 0; i < n; ++i) {
        dust_ctx *c = b->ctx[i];
        saved[i] = Saved{c->cur, c->d_count, c->d_count_next, c->keys_ready, c->keys_dt, {}};
        for (int g = 0; g < dust_ctx::N_GROUPS; ++g) saved[i].launches[g] = c->launches[g];
    }
    auto restore = [&](bool state) {
        for (size_t i = 0; i < n; ++i) {
            dust_ctx *c = b->ctx[i];
            c->capture_mode = false;
            c->perm_pending = false;
            for (int g = 0; g < dust_ctx::N_GROUPS; ++g) c->launches[g] = saved[i].launches[g];
            if (!state) continue;
            c->cur = saved[i].cur;
            c->d_count = saved[i].count;
            c->d_count_next = saved[i].count_next;
            c->keys_ready = saved[i].keys_ready;
            c->keys_dt = saved[i].keys_dt;
        }
    };
    BCU(cudaStreamBeginCapture(b->root, cudaStreamCaptureModeThreadLocal));
    int rc = DUST_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->root);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->ctx[i]->stream, b->fork, 0);
    for (size_t i = 0; i < n && e == cudaSuccess && rc == DUST_OK; ++i) {
        dust_ctx *c = b->ctx[i];
        c->capture_mode = true;
        rc = c->mixed ? capture_period<float>(c, dt[i]) : capture_period<double>(c, dt[i]);
        c->capture_mode = false;
        if (rc == DUST_OK) {
            for (int g = 0; g < dust_ctx::N_GROUPS; ++g)
                b->period_launches[i][g] = c->launches[g] - saved[i].launches[g];
            e = cudaEventRecord(b->join[i], c->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->root, b->join[i], 0);
        } else {
            b->err = c->err;
        }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->root, &graph);
    if (rc != DUST_OK || e != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        restore(true);
        if (rc != DUST_OK) return bfail(b, rc, "capture: %s", b->err.c_str());
        return bfail(b, DUST_ECUDA, "capture: %s",
                     cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    // the period leaves every store, count buffer and key flag as it found
    // them; launch counts are added per replay
    restore(false);
    b->graph = graph;
    BCU(cudaGraphInstantiate(&b->exec, b->graph, 0));
    for (size_t i = 0; i < n; ++i) {
        dust_ctx *c = b->ctx[i];
        b->dt[i] = dt[i];
        b->gen[i] = c->gen;
        b->cur[i] = c->cur;
        b->count[i] = c->d_count;
    }
    return DUST_OK;
}

// ---- the persistent path

// Kernel variant of the persistent launch for these instances, -1 if they
// cannot share it: all mixed precision on the slab kernel (which predicts
// the next sort's keys), the exponential-midpoint pusher, no gas predictor,
// and one of the two instantiated geometries: x-z shearing boxes in the
// orbital-advection frame (variant 0; 2 and 3 when every instance has the
// 32 x 16 or the 16 x 16 tile with TSC weights, which have compiled copies)
// or x-y Cartesian boxes (variant 1).
int persistent_variant(const dust_batch *b)
{
    int v = -1, shape = -1;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        const dust_ctx *c = b->ctx[i];
        if (!step_emits_keys(c) || c->opt.gas_predictor || c->opt.pusher != DUST_PUSHER_EM) return -1;
        const int flat = slab_flat(c->g);
        int vi = -1;
        if (c->geom.kind == DUST_SHEARING_BOX && c->geom.fargo && flat == 1) vi = 0;
        else if (c->geom.kind == DUST_CARTESIAN && flat == 2) vi = 1;
        if (vi < 0 || (v >= 0 && vi != v)) return -1;
        v = vi;
        const int si = slab_shape_id(c->g, flat, c->opt.weight == DUST_WEIGHT_TSC, 1);
        shape = (shape < 0 || shape == si) ? si : SHAPE_ANY;
    }
    if (v == 0 && shape == SHAPE_32X16) return 2;
    if (v == 0 && shape == SHAPE_16X16) return 3;
    return v;
}

int grid_of(int variant, size_t smem)
{
    switch (variant) {
    case 0: return batch_persistent_grid<GEOM_SB, 1, 1>(smem);
    case 2: return batch_persistent_grid<GEOM_SB, 1, 1, 32, 1, 16>(smem);
    case 3: return batch_persistent_grid<GEOM_SB, 1, 1, 16, 1, 16>(smem);
    default: return batch_persistent_grid<GEOM_CART, 2, 1>(smem);
    }
}

cudaError_t launch_variant(int variant, const BatchDev &d, size_t smem, int grid, cudaStream_t st)
{
    switch (variant) {
    case 0: return launch_batch_persistent<GEOM_SB, 1, 1>(d, smem, grid, st);
    case 2: return launch_batch_persistent<GEOM_SB, 1, 1, 32, 1, 16>(d, smem, grid, st);
    case 3: return launch_batch_persistent<GEOM_SB, 1, 1, 16, 1, 16>(d, smem, grid, st);
    default: return launch_batch_persistent<GEOM_CART, 2, 1>(d, smem, grid, st);
    }
}

// Descriptor of instance c for a launch of steps of length dt starting at
// its current time.
BatchInst batch_inst_of(dust_ctx *c, double dt, int test_timeout)
{
    BatchInst I{};
    TiledArgs<float> &ta = I.ta;
    StepArgs<float> &a = ta.s;
    a.g = c->g;
    a.ph = phys_of(c, c->t, dt);
    a.sp = c->sp;
    species_coefficients(a.sp, c->geom.kind, c->geom.omega, dt);
    a.t = c->t;
    a.dt = dt;
    a.inv_quantum = 1.0 / c->quantum;
    a.s = store_of<float>(c, c->cur);
    a.gas = static_cast<const float *>(c->d_gas);
    a.dep = c->d_dep;
    a.status = c->d_status;
    a.tdev = c->d_time;
    ta.tsc = c->opt.weight == DUST_WEIGHT_TSC;
    ta.vol = uses_volume_weights(c->geom.kind, c->opt.weight) ? 1 : 0;
    ta.gas_tmap = c->tmap_ok[0] ? static_cast<const void *>(c->d_tmaps) : nullptr;
    ta.wait_extra_tx = (c->opt.test_wait_timeout || test_timeout) ? 16u : 0u;
    ta.wait_ns = (c->opt.test_wait_timeout || test_timeout) ? 1000000ull : 0ull;
    for (int w = 0; w < 2; ++w) I.store[w] = store_of<float>(c, w);
    I.count[0] = c->d_count;
    I.count[1] = c->d_count_next;
    I.key = c->d_key;
    I.cursor = c->d_cursor;
    I.pair_id = c->d_pair_id;
    I.pair_src = c->d_pair_src;
    I.bigseg = c->d_bigseg;
    I.blocksums = c->d_blocksums;
    I.time = c->d_time;
    I.dt = dt;
    I.q_om_lx = c->geom.q * c->geom.omega * (c->g.hi[0] - c->g.lo[0]);
    I.ly = c->g.hi[1] - c->g.lo[1];
    I.sb = c->geom.kind == DUST_SHEARING_BOX;
    I.quantum = c->quantum;
    I.cur = c->cur;
    I.feedback = c->opt.feedback_apply;
    I.ntiles = c->g.nt[0] * c->g.nt[1] * c->g.nt[2];
    I.n = c->n_grains;
    I.nkeys = c->g.nkeys;
    I.ncell = c->ncell;
    return I;
}

void drop_persistent(dust_batch *b)
{
    if (b->pexec) cudaGraphExecDestroy(b->pexec);
    if (b->pgraph) cudaGraphDestroy(b->pgraph);
    b->pexec = nullptr;
    b->pgraph = nullptr;
    b->tab.clear();
}

// nsteps steps of every instance as one persistent launch (see
// dust_batch.cu).  Steps s with s % sort_interval == 0 of the call sort
// first; the step before a sort predicts its keys.
int step_persistent(dust_batch *b, const double *dt, int nsteps)
{
    const size_t n = b->ctx.size();
    const int K = b->sort_interval;
    // keys for the first sort (the previous call's last step, or now)
    for (size_t i = 0; i < n; ++i) {
        dust_ctx *c = b->ctx[i];
        if (c->n_grains > 0 && !(c->keys_ready && c->keys_dt == dt[i]) && !c->perm_pending) {
            const int r = prime_keys<float>(c, dt[i]);
            if (r) return bfail(b, r, "context %zu: %s", i, c->err.c_str());
        }
        if (c->perm_pending) return bfail(b, DUST_ESTATE, "context %zu: a sort is pending", i);
    }
    // descriptors and work list
    if (b->inst_copied) BCU(cudaEventSynchronize(b->inst_copied));
    size_t slab = 0;
    for (size_t i = 0; i < n; ++i) {
        dust_ctx *c = b->ctx[i];
        b->h_inst[i] = batch_inst_of(c, dt[i], b->test_timeout);
        slab = std::max(slab, batch_tile_smem(c->g));
    }
    std::vector<int> tab;
    BatchDev d{};
    if (!work_list(b->h_inst, n, nsteps, K, tab, d)) return bfail(b, DUST_EINVAL, "too many work items");
    // shared memory: the largest tile layout (or the sort's staging), then
    // the block's copy of the step arguments
    const size_t ta_off = (std::max(slab, batch_sort_smem()) + 15) & ~(size_t)15;
    const size_t smem = ta_off + sizeof(TiledArgs<float>) + 16;  // + the item counter's broadcast
    if (smem != b->psmem) {
        b->psmem = smem;
        b->pgrid = grid_of(b->pvariant, smem);
        drop_persistent(b);
    }
    if (b->pgrid <= 0) return bfail(b, DUST_EINVAL, "the persistent kernel does not fit on the device");
    // each instance's time of this call, after its pending work
    for (size_t i = 0; i < n; ++i) {
        dust_ctx *c = b->ctx[i];
        const PhysDev ph = phys_of(c, c->t, dt[i]);
        set_time_kernel<<<1, 1, 0, c->stream>>>(c->d_time, c->t, ph.shift_mid, ph.shift_end);
        BCU(cudaGetLastError());
        BCU(cudaEventRecord(b->join[i], c->stream));
        BCU(cudaStreamWaitEvent(b->root, b->join[i], 0));
    }
    if (!b->pexec || tab != b->tab || d.nsteps != b->pdev.nsteps || d.sort_interval != b->pdev.sort_interval) {
        // a new work list: its static part copied once, a new graph
        drop_persistent(b);
        const size_t nstatic = (size_t)d.nstatic, ntotal = tab.size() + (size_t)d.ntasks + 1;
        if (ntotal > b->tab_cap) {
            if (b->d_tab) BCU(cudaFree(b->d_tab));
            b->d_tab = nullptr;
            b->tab_cap = 0;
            BCU(cudaMalloc(reinterpret_cast<void **>(&b->d_tab), ntotal * sizeof(int)));
            b->tab_cap = ntotal;
        }
        BCU(cudaMemcpyAsync(b->d_tab, tab.data(), nstatic * sizeof(int), cudaMemcpyHostToDevice, b->root));
        BCU(cudaStreamSynchronize(b->root));
        d.inst = b->d_inst;
        d.ninst = (int)n;
        d.tasks = reinterpret_cast<const BatchTask *>(b->d_tab + d.off_tasks);
        d.members = b->d_tab + d.off_members;
        d.gcount = b->d_tab + d.off_gcount;
        d.gpre = b->d_tab + d.off_gpre;
        d.done = b->d_tab + nstatic;
        d.grab = d.done + d.ntasks;
        d.wait_extra = b->test_timeout ? 1 : 0;
        d.wait_ns = b->test_timeout ? 1000000ull : 4000000000ull;
        d.ta_offset = ta_off;
        cudaStream_t cs = nullptr;
        BCU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_inst, b->h_inst, n * sizeof(BatchInst),
                                                  cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.done, 0, ((size_t)d.ntasks + 1) * sizeof(int), cs);
        if (e == cudaSuccess) e = launch_variant(b->pvariant, d, smem, b->pgrid, cs);
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(b, DUST_ECUDA, "persistent launch capture: %s",
                         cudaGetErrorString(e != cudaSuccess ? e : ee));
        }
        b->pgraph = g;
        BCU(cudaGraphInstantiate(&b->pexec, g, 0));
        b->tab.swap(tab);
        b->pdev = d;
    }
    BCU(cudaGraphLaunch(b->pexec, b->root));
    BCU(cudaEventRecord(b->inst_copied, b->root));
    BCU(cudaEventRecord(b->done, b->root));
    // host state of every context after the call
    const int sorts = (nsteps + K - 1) / K;
    for (size_t i = 0; i < n; ++i) {
        dust_ctx *c = b->ctx[i];
        BCU(cudaStreamWaitEvent(c->stream, b->done, 0));
        if (sorts & 1) {
            c->cur = 1 - c->cur;
            std::swap(c->d_count, c->d_count_next);
        }
        c->keys_ready = (nsteps % K) == 0 && c->n_grains > 0;
        c->keys_dt = dt[i];
        c->perm_pending = false;
        for (int s = 0; s < nsteps; ++s) c->t += dt[i];
        c->last_dt = dt[i];
        c->steps += nsteps;
        c->timed_steps += nsteps;
        c->have_deposit = true;
        c->need_sort = false;
    }
    b->ctx[0]->launches[dust_ctx::GROUP_STEP] += 1;
    return DUST_OK;
}

}  // namespace

extern "C" int dust_batch_create(dust_batch **out, dust_ctx *const *insts, int n,
                                 const dust_options *opt)
{
    if (!out) return bfail(nullptr, DUST_EINVAL, "out is NULL");
    *out = nullptr;
    if (!insts || n < 1 || n > 4096) return bfail(nullptr, DUST_EINVAL, "need 1..4096 contexts");
    for (int i = 0; i < n; ++i) {
        if (!insts[i]) return bfail(nullptr, DUST_EINVAL, "context %d is NULL", i);
        for (int j = 0; j < i; ++j)
            if (insts[j] == insts[i]) return bfail(nullptr, DUST_EINVAL, "context %d appears twice", i);
        if (insts[i]->device != insts[0]->device)
            return bfail(nullptr, DUST_EINVAL, "contexts on different devices");
    }
    dust_batch *b = new (std::nothrow) dust_batch();
    if (!b) return bfail(nullptr, DUST_ENOMEM, "host allocation failed");
    b->device = insts[0]->device;
    b->ctx.assign(insts, insts + n);
    b->dt.assign(n, 0.0);
    b->gen.assign(n, 0);
    b->cur.assign(n, -1);
    b->count.assign(n, nullptr);
    b->period_launches.assign(n, {});
    b->join.assign(n, nullptr);
    auto bail = [&](const char *what) {
        std::string m = what;
        dust_batch_destroy(b);
        return bfail(nullptr, DUST_ECUDA, "%s", m.c_str());
    };
    if (cudaSetDevice(b->device) != cudaSuccess) return bail("cudaSetDevice failed");
    if (opt && opt->stream) {
        b->root = static_cast<cudaStream_t>(opt->stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking) != cudaSuccess)
            return bail("stream creation failed");
        b->own_root = true;
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess)
        return bail("event creation failed");
    for (int i = 0; i < n; ++i)
        if (cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess)
            return bail("event creation failed");
    if (opt) {
        b->mode = opt->batch_mode;
        b->sort_interval = opt->sort_interval > 0 ? opt->sort_interval : 1;
        b->test_timeout = opt->test_wait_timeout;
    }
    b->pvariant = b->mode == 0 ? persistent_variant(b) : -1;
    if (b->pvariant >= 0) {
        if (cudaMallocHost(reinterpret_cast<void **>(&b->h_inst), n * sizeof(BatchInst)) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void **>(&b->d_inst), n * sizeof(BatchInst)) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->inst_copied, cudaEventDisableTiming) != cudaSuccess)
            return bail("allocation for the persistent launch failed");
    }
    *out = b;
    return DUST_OK;
}

extern "C" int dust_batch_step(dust_batch *b, const double *dt, int nsteps)
{
    if (!b) return bfail(nullptr, DUST_EINVAL, "batch is NULL");
    if (nsteps < 0 || (nsteps > 0 && !dt)) return bfail(b, DUST_EINVAL, "bad nsteps or dt");
    const size_t n = b->ctx.size();
    for (size_t i = 0; i < n; ++i) {
        if (nsteps > 0 && !std::isfinite(dt[i])) return bfail(b, DUST_EINVAL, "dt[%zu] not finite", i);
        if (!b->ctx[i]->gas_set || !b->ctx[i]->particles_set)
            return bfail(b, DUST_ESTATE, "context %zu: set the gas and load particles first", i);
    }
    if (nsteps == 0) return DUST_OK;
    BCU(cudaSetDevice(b->device));
    if (b->pvariant >= 0 && persistent_variant(b) == b->pvariant) return step_persistent(b, dt, nsteps);
    const int pairs = nsteps / 2;
    if (pairs > 0) {
        // keys for the first captured sort
        for (size_t i = 0; i < n; ++i) {
            dust_ctx *c = b->ctx[i];
            if (step_emits_keys(c) && c->n_grains > 0 && !(c->keys_ready && c->keys_dt == dt[i])) {
                const int r = c->mixed ? prime_keys<float>(c, dt[i]) : prime_keys<double>(c, dt[i]);
                if (r) return bfail(b, r, "context %zu: %s", i, c->err.c_str());
            }
        }
        bool fresh = b->exec != nullptr;
        for (size_t i = 0; i < n && fresh; ++i) {
            const dust_ctx *c = b->ctx[i];
            fresh = b->dt[i] == dt[i] && b->gen[i] == c->gen && b->cur[i] == c->cur &&
                    b->count[i] == c->d_count;
        }
        if (!fresh) {
            const int r = capture(b, dt);
            if (r) return r;
        }
        // each instance's time of this call, after its pending work
        for (size_t i = 0; i < n; ++i) {
            dust_ctx *c = b->ctx[i];
            const PhysDev ph = phys_of(c, c->t, dt[i]);
            set_time_kernel<<<1, 1, 0, c->stream>>>(c->d_time, c->t, ph.shift_mid, ph.shift_end);
            BCU(cudaGetLastError());
            BCU(cudaEventRecord(b->join[i], c->stream));
            BCU(cudaStreamWaitEvent(b->root, b->join[i], 0));
        }
        for (int k = 0; k < pairs; ++k) BCU(cudaGraphLaunch(b->exec, b->root));
        BCU(cudaEventRecord(b->done, b->root));
        for (size_t i = 0; i < n; ++i) {
            dust_ctx *c = b->ctx[i];
            BCU(cudaStreamWaitEvent(c->stream, b->done, 0));
            for (int s = 0; s < 2 * pairs; ++s) c->t += dt[i];
            c->last_dt = dt[i];
            c->steps += 2 * pairs;
            c->timed_steps += 2 * pairs;
            c->have_deposit = true;
            c->need_sort = false;
            for (int g = 0; g < dust_ctx::N_GROUPS; ++g)
                c->launches[g] += b->period_launches[i][g] * pairs;
        }
    }
    if (nsteps % 2) {
        for (size_t i = 0; i < n; ++i) {
            const int r = dust_step(b->ctx[i], dt[i]);
            if (r) return bfail(b, r, "context %zu: %s", i, b->ctx[i]->err.c_str());
        }
    }
    return DUST_OK;
}

extern "C" const char *dust_batch_last_error(const dust_batch *b)
{
    return b ? b->err.c_str() : g_batch_error.c_str();
}

extern "C" void dust_batch_destroy(dust_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->root) cudaStreamSynchronize(b->root);
    drop_graph(b);
    drop_persistent(b);
    if (b->h_inst) cudaFreeHost(b->h_inst);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_tab) cudaFree(b->d_tab);
    if (b->inst_copied) cudaEventDestroy(b->inst_copied);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->own_root && b->root) cudaStreamDestroy(b->root);
    delete b;
}

// ------------------------------------------------ allocation-free step ----
//
// dust_step_noalloc is for callers that cannot let the library allocate
// device memory while they step.  One kind is a host code that hands the
// device's memory to its own pool when it starts: a later cudaMalloc fails or
// breaks the budget that pool was sized for.  Another keeps work running on
// other streams: cudaMalloc and cudaFree synchronise the whole device and
// would stall that work.  Here the grains, the gas and the deposit are the
// caller's device arrays, and the only scratch the kernel needs (the grid
// tables and the status words) lives in a fixed device array of this library.

namespace {

constexpr int kNoAllocMaxZones = 2048;               // zones per direction
constexpr size_t kNoAllocScratchBytes = 512 * 1024;  // fits 3 x 2048-zone tables
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

// Device address of g_noalloc_scratch per device ordinal (null until the
// first call on that device looks it up).
void *g_noalloc_addr[kNoAllocMaxDevices];
// Host image of the scratch contents, copied to the device by each call.  It
// is page-locked once (cudaHostRegister of this existing array, no
// allocation), so the copy runs asynchronously; the next call waits for the
// event recorded after the copy before it rewrites the image.
alignas(4096) unsigned char g_noalloc_image[kNoAllocScratchBytes];
bool g_noalloc_image_locked = false;
cudaEvent_t g_noalloc_copied[kNoAllocMaxDevices];
// one call at a time writes the image and enqueues its copy
std::mutex g_noalloc_mutex;

// Byte offsets inside the scratch: status words, then per direction the grid
// tables, each region on a 256-byte boundary.
struct NoAllocLayout {
    size_t status;
    size_t edges[3], ekey[3], dvol[3], zc[3], ziw[3];
    size_t dvol_f[3], ziw_f[3], znu_f[3], zlo_f[3], zc_f[3];
    size_t total;
};

NoAllocLayout noalloc_layout(const int n[3])
{
    NoAllocLayout L{};
    size_t off = 0;
    auto take = [&off](size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    };
    L.status = take(ST_WORDS * sizeof(unsigned));
    for (int d = 0; d < 3; ++d) {
        const size_t m = (size_t)n[d];
        L.edges[d] = take((m + 1) * sizeof(double));
        L.ekey[d] = take((m + 1) * sizeof(long long));
        L.dvol[d] = take(m * sizeof(double));
        L.zc[d] = take(m * sizeof(double));
        L.ziw[d] = take(m * sizeof(double));
        L.dvol_f[d] = take(m * sizeof(float));
        L.ziw_f[d] = take(m * sizeof(float));
        L.znu_f[d] = take(m * sizeof(float));
        L.zlo_f[d] = take((m + 1) * sizeof(float));
        L.zc_f[d] = take(m * sizeof(float));
    }
    L.total = off;
    return L;
}

template <int GEOM>
cudaError_t launch_noalloc(const StepArgs<double> &a, int weight, cudaStream_t s)
{
    if constexpr (GEOM == GEOM_CYL || GEOM == GEOM_SPH)
        if (weight == DUST_WEIGHT_VOLUME) return launch_step_per_grain<double, GEOM, 2>(a, s);
    return weight == DUST_WEIGHT_TSC ? launch_step_per_grain<double, GEOM, 1>(a, s)
                                     : launch_step_per_grain<double, GEOM, 0>(a, s);
}

}  // namespace

extern "C" int dust_step_noalloc(const dust_geometry *geom, const dust_grid *grid,
                                 const dust_species *species, int n_species, int weight,
                                 double quantum, double t, double dt, int64_t n,
                                 double *q0, double *q1, double *q2,
                                 double *p0, double *p1, double *p2,
                                 const uint8_t *species_idx, const double *param,
                                 const double *gas, int64_t *dep, uint32_t *status_out,
                                 int device, void *stream)
{
    dust_ctx *ctx = nullptr;  // errors are reported through dust_last_error(NULL)
    int64_t ncell = 0;
    const int rv = validate_descriptors(geom, grid, species, n_species, weight, &ncell);
    if (rv) return rv;
    for (int d = 0; d < 3; ++d)
        if (grid->n[d] > kNoAllocMaxZones)
            return fail(nullptr, DUST_EINVAL,
                        "direction %d has %d zones; dust_step_noalloc holds grid tables for at "
                        "most %d zones per direction",
                        d, grid->n[d], kNoAllocMaxZones);
    if (!std::isfinite(t) || !std::isfinite(dt) || !(quantum >= 0.0))
        return fail(nullptr, DUST_EINVAL, "t and dt must be finite and quantum >= 0");
    if (n < 0 || n >= ((int64_t)1 << 31))
        return fail(nullptr, DUST_EINVAL, "grain count out of range");
    if (!gas || !dep || (n > 0 && (!q0 || !q1 || !q2 || !p0 || !p1 || !p2)))
        return fail(nullptr, DUST_EINVAL, "NULL device array");
    if (device < 0 || device >= kNoAllocMaxDevices)
        return fail(nullptr, DUST_EINVAL, "device ordinal out of range");
    const NoAllocLayout L = noalloc_layout(grid->n);
    if (L.total > kNoAllocScratchBytes)
        return fail(nullptr, DUST_EINVAL, "grid tables exceed the %zu-byte scratch",
                    kNoAllocScratchBytes);

    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    CU(cudaSetDevice(device));
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    // setup: once per process, page-lock the host image; once per device, the
    // scratch's device address and the event that marks the image's copy
    if (!g_noalloc_image_locked) {
        CU(cudaHostRegister(g_noalloc_image, sizeof(g_noalloc_image), cudaHostRegisterPortable));
        g_noalloc_image_locked = true;
    }
    if (!g_noalloc_addr[device]) {
        void *addr = nullptr;
        CU(cudaGetSymbolAddress(&addr, g_noalloc_scratch));
        CU(cudaEventCreateWithFlags(&g_noalloc_copied[device], cudaEventDisableTiming));
        g_noalloc_addr[device] = addr;
    }
    unsigned char *base = static_cast<unsigned char *>(g_noalloc_addr[device]);
    unsigned char *img = g_noalloc_image;
    // the previous call's copy (on whichever device) reads the image: wait
    // until it has run before writing the image again
    for (int dv = 0; dv < kNoAllocMaxDevices; ++dv)
        if (g_noalloc_copied[dv]) CU(cudaEventSynchronize(g_noalloc_copied[dv]));

    StepArgs<double> a{};
    GridDev &g = a.g;
    g.ncell = ncell;
    std::memset(img + L.status, 0, ST_WORDS * sizeof(unsigned));  // status words start at zero
    for (int d = 0; d < 3; ++d) {
        const int m = grid->n[d];
        const double *e = grid->edges[d];
        grid_direction(g, d, e, m, grid->bc[d]);
        std::memcpy(img + L.edges[d], e, (m + 1) * sizeof(double));
        fill_zone_tables(geom->kind, d, e, m,
                         ZoneTables{reinterpret_cast<double *>(img + L.dvol[d]),
                                    reinterpret_cast<double *>(img + L.zc[d]),
                                    reinterpret_cast<double *>(img + L.ziw[d]),
                                    reinterpret_cast<float *>(img + L.dvol_f[d]),
                                    reinterpret_cast<float *>(img + L.ziw_f[d]),
                                    reinterpret_cast<float *>(img + L.znu_f[d]),
                                    reinterpret_cast<float *>(img + L.zlo_f[d]),
                                    reinterpret_cast<float *>(img + L.zc_f[d]),
                                    reinterpret_cast<long long *>(img + L.ekey[d])});
        g.edges[d] = reinterpret_cast<const double *>(base + L.edges[d]);
        g.ekey[d] = reinterpret_cast<const long long *>(base + L.ekey[d]);
        g.dvol[d] = reinterpret_cast<const double *>(base + L.dvol[d]);
        g.zc[d] = reinterpret_cast<const double *>(base + L.zc[d]);
        g.ziw[d] = reinterpret_cast<const double *>(base + L.ziw[d]);
        g.dvol_f[d] = reinterpret_cast<const float *>(base + L.dvol_f[d]);
        g.ziw_f[d] = reinterpret_cast<const float *>(base + L.ziw_f[d]);
        g.znu_f[d] = reinterpret_cast<const float *>(base + L.znu_f[d]);
        g.zlo_f[d] = reinterpret_cast<const float *>(base + L.zlo_f[d]);
        g.zc_f[d] = reinterpret_cast<const float *>(base + L.zc_f[d]);
        // the per-grain kernel has no tiles: one zone per key
        g.T[d] = 1;
        g.nt[d] = m;
    }
    g.tvol = 1;
    g.nkeys = ncell;
    double qu = 0.0;
    a.sp = make_species(species, n_species, quantum, &qu);
    a.ph = make_phys(*geom, g, t, dt);
    a.t = t;
    a.dt = dt;
    a.inv_quantum = 1.0 / qu;
    a.s.q[0] = q0; a.s.q[1] = q1; a.s.q[2] = q2;
    a.s.p[0] = p0; a.s.p[1] = p1; a.s.p[2] = p2;
    a.s.species = const_cast<uint8_t *>(species_idx);
    a.s.param = const_cast<double *>(param);
    a.s.id = nullptr;
    a.s.n = n;
    a.gas = gas;
    a.dep = reinterpret_cast<unsigned long long *>(dep);
    a.status = reinterpret_cast<unsigned *>(base + L.status);

    // tables and zeroed status words in one copy; the deposit starts at zero
    CU(cudaMemcpyAsync(base, img, L.total, cudaMemcpyHostToDevice, st));
    CU(cudaEventRecord(g_noalloc_copied[device], st));
    CU(cudaMemsetAsync(dep, 0, (size_t)ncell * 4 * sizeof(int64_t), st));
    cudaError_t e;
    switch (geom->kind) {
    case DUST_CARTESIAN: e = launch_noalloc<GEOM_CART>(a, weight, st); break;
    case DUST_SHEARING_BOX: e = launch_noalloc<GEOM_SB>(a, weight, st); break;
    case DUST_CYLINDRICAL: e = launch_noalloc<GEOM_CYL>(a, weight, st); break;
    default: e = launch_noalloc<GEOM_SPH>(a, weight, st); break;
    }
    CU(e);
    if (status_out)
        CU(cudaMemcpyAsync(status_out, base + L.status, 4 * sizeof(unsigned),
                           cudaMemcpyDeviceToDevice, st));
    return DUST_OK;
}
