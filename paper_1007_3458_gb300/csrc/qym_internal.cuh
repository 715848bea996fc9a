// qym_internal.cuh -- device helpers and launch declarations shared by the
// libqym translation units (sm_103a). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qym.h"

namespace qym {

constexpr double kPi = 3.14159265358979323846;
constexpr int kHermMaxClusters = 160;  // entries of Dev::hcl (2 x 152 CTAs in clusters of 2 or more)

// ---------------------------------------------------------------- layout
// Device state of a context. Rows of all systems are concatenated; each
// system's star sits at its first row with Q = v = 0. Positions and
// velocities are float64 structure-of-arrays [3][rows].
struct Dev {
    int64_t rows = 0;
    int32_t nsys = 0;
    int64_t *offsets = nullptr;   // [nsys+1]
    int32_t *sys_of = nullptr;    // [rows] system of each row
    double *m = nullptr;          // [rows]
    double *q = nullptr, *v = nullptr;     // [3][rows] current state (DH)
    double *q1 = nullptr, *v1 = nullptr;   // [3][rows] Kepler output / step scratch
    double *rH = nullptr;         // [rows] Hill radius used by this step's encounter test
    double *rH_fixed = nullptr;   // [rows] Hill radii computed at init (hill_fixed)
    // kick operand packs, float32 (rebuilt from the FP64 state every step)
    float4 *pk_pos = nullptr;     // (x_hi, y_hi, z_hi, G m)
    float4 *pk_lo = nullptr;      // (x_lo, y_lo, z_lo, c = 2 rho^2, rho the crude reach)
    float *amag = nullptr;        // [rows] |a_int| of the last kick
    float *rH_bound = nullptr;    // [rows] Hill radius bound used by the crude test
    double *apart = nullptr;      // [splits][3][rows] kick partial accelerations
    int32_t splits = 1;
    int32_t *kick_cnt = nullptr;  // arrivals per i-block: with it the kick's last CTA of
                                  // each i-block adds the slots into slot 0 (kick.cu)
    int32_t *wh_flag = nullptr;   // [nsys] 1: this step of the system is integrated whole
                                  // by the Hermite (whole.cu); its sets are not
    double *vpre = nullptr;       // [3][rows] velocities entering the first kick
    // kick work items (one CTA each): (i0, i1, j0, j1) and the partial slot
    int4 *items = nullptr;
    int32_t *item_slot = nullptr;
    int32_t nitems = 0;
    // momentum reduction
    int4 *mchunks = nullptr;      // (row0, row1, sys, -) chunks of at most 1024 rows
    int32_t nmchunks = 0;
    double *mpart = nullptr;      // [nmchunks][3]
    int32_t *sys_chunk0 = nullptr;  // [nsys+1] first chunk of each system
    double *S = nullptr;          // [nsys][3] sum of m v over bodies
    // encounters
    int2 *cand = nullptr;         // crude candidate pairs (i < j)
    int64_t max_cand = 0;
    int4 *fchunk = nullptr;       // (i, j0, j1, -): j chunks [j0, j1) of row i whose crude
                                  // minimum fell below c_i, re-tested pair by pair
    int64_t max_fchunk = 0;
    int2 *enc = nullptr;          // rigorous encounter pairs
    int64_t max_enc = 0;
    int32_t *rescan = nullptr;    // rows whose crude bounds were exceeded
    int32_t *set_start = nullptr; // [max_sets+1]
    int32_t *set_mem = nullptr;   // [max_members]
    double *rcrit = nullptr;      // [max_sets]
    int32_t max_sets = 0, max_members = 0;
    // Hermite schedule: block steps of the set each row was in during the
    // last step (0 for rows in no set), the per-CTA queue of sets in order of
    // predicted cost, and the set each thread-block cluster takes (-1: none)
    int32_t *hcost = nullptr;     // [rows]
    int32_t *hsetcost = nullptr;  // [max_sets] largest hcost over each set's members
                                  // (raised by the set builder, cleared by the plan)
    int32_t *hq = nullptr;        // [max_sets]
    int32_t *hcl = nullptr;       // [kHermMaxClusters]
    int32_t *uf = nullptr;        // [rows] union-find parents, kept at -1 when idle
    int64_t *log = nullptr;       // [max_log][3] encounter records of one qym_step call
    int64_t max_log = 0;
    // heavy bodies of each system (mixed kick: their pull is summed in FP64)
    int32_t *heavy_rows = nullptr;   // ascending rows, system by system
    int32_t *heavy_start = nullptr;  // [nsys+1]
    double *heavy_thr = nullptr;     // [nsys] mass threshold (+inf: no split)
    double *kmu = nullptr;           // [nsys][3] mu = G m0, sqrt(mu), 1/mu (E_Kep)
    double *hfac = nullptr;          // [rows] (m / 3 m0)^(1/3): r_H = |Q| hfac (0 for stars)
    int32_t heavy_split = 0;         // 1 when the kick in use is the mixed one
    int32_t escape_reach = 0;        // 1: the crude reach is the escape-velocity one
    // counters (device): see Counters below
    unsigned long long *ctr = nullptr;
    int32_t *status = nullptr;    // QYM_ST_* bits
    // a system's step split over several GPUs: this context computes the
    // rows [own_lo, own_hi) (kick rows, finisher, Kepler drift, the
    // candidates of those rows, the Hermite of the sets whose lowest row is
    // among them); own_hi = 0: every row
    int64_t own_lo = 0, own_hi = 0;
    int32_t *set_root = nullptr;  // [max_sets] lowest row of each set (sets are numbered by it)
    int32_t log_refine = 1;       // the rigorous test logs its pairs (0: the split's import does)
    // order of the bodies in the kick's packs and partial sums (sort.cu):
    // position p holds row perm[p], row r sits at position inv[r]; NULL: row order
    int32_t *perm = nullptr, *inv = nullptr;
    int32_t *vmax = nullptr; // [nsys] largest |v| after the first kick (float bits), for the
                             // binned search; NULL: not kept
    float4 *far = nullptr;   // [rows] (offset from the tile's reference point, G m) in that order
    float4 *tile = nullptr;  // [3 x tiles] reference point and radius, box min, box max
};

// device counters, indices into Dev::ctr
enum Ctr : int {
    C_NCAND = 0,     // candidates this step (reset per step)
    C_NENC,          // encounter pairs this step (reset per step)
    C_NRESCAN,       // rows to re-search this step (reset per step)
    C_NSETS,         // sets this step (written by the set builder)
    C_NMEM,          // set members this step
    C_LOG,           // records in the encounter log (per qym_step call)
    C_SUM_CAND,      // running sums over the steps of one qym_step call
    C_SUM_ENC,
    C_SUM_SETS,
    C_MAX_SET,
    C_SUM_KITER,
    C_SUM_HSTEPS,
    C_SUM_RESCAN,
    C_STEP,          // step index within the current qym_step call
    C_MAX_HSET,      // most Hermite steps taken by one set in one step
    C_HSMALL,        // next set for the Hermite kernel's per-CTA queue (reset per step)
    C_NFCHUNK,       // flagged (row, j chunk) entries of the last search kick
    C_FCDONE,        // CTAs of the chunk re-test done (its last CTA resets both)
    C_HNQ,           // sets in the Hermite kernel's per-CTA queue this step
    C_NACTIVE,       // overlapping tile pairs of the binned search (reset per step)
    C_COUNT
};

// ---------------------------------------------------------------- helpers
// one MUFU instruction; inputs here are squared separations, never denormal
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct alignas(32) D4 {
    double x, y, z, w;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// split a double into a float pair with hi + lo == x to ~2^-48 relative
__device__ __forceinline__ void split_ds(double x, float &hi, float &lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

// FP64 pull of the heavy bodies hs[0..nh) (ascending rows, i excluded) on
// the body at (x, y, z): sum -G m_h (r_i - r_h) / |r_i - r_h|^3
__device__ __forceinline__ void heavy_pull(const int32_t *hs, int nh, int64_t i, double x,
                                           double y, double z, const double *q, const double *m,
                                           int64_t R, double G, double &ax, double &ay,
                                           double &az) {
    for (int k = 0; k < nh; ++k) {
        int64_t h = hs[k];
        if (h == i) continue;
        double dx = x - q[h], dy = y - q[R + h], dz = z - q[2 * R + h];
        double r2 = dx * dx + dy * dy + dz * dz;
        double ri = rsqrt(r2);
        double s = G * m[h] * (ri * ri) * ri;
        ax -= s * dx;
        ay -= s * dy;
        az -= s * dz;
    }
}

// the calling thread's context-free error message (qym_last_error(NULL))
void set_thread_error(const std::string &msg);

// ---------------------------------------------------------------- launches
// Each returns cudaSuccess or the launch error. All work goes on `st`.

// kepler.cu
struct KeplerArgs {
    int64_t n;            // bodies
    const double *q0, *v0; // [3][ld] inputs
    double *q1, *v1;       // [3][ld] outputs
    int64_t ld;            // leading dimension (stride between x, y, z blocks)
    const int64_t *rows;   // optional row map: body k is row rows[k]; NULL: row row0 + k
    int64_t row0;
    double mu, sqmu, imu, dt;   // mu with sqrt(mu) and 1/mu (all rows, when kmu is NULL)
    int32_t solver, guess, max_iter;
    const float *mlp_w;    // guess network weights (QYM_GUESS_MLP) or NULL
    double *x_out;         // [n] or NULL
    double *x0_out;        // [n] starting guesses, or NULL
    // training rows (u1..u4, t) [log_cap][5], or NULL; row of body k:
    // (*log_base + *log_step) * n + k, or k when log_step is NULL
    float *log;
    int64_t log_cap;
    const unsigned long long *log_base, *log_step;
    int32_t *iters;        // [n] or NULL
    int32_t *status;       // or NULL
    unsigned long long *iter_sum;  // or NULL
    // per-row mu, sqrt(mu), 1/mu: kmu[3 sys_of[row] + 0..2] when kmu != NULL
    const int32_t *sys_of;
    const double *kmu;
};
cudaError_t launch_kepler(const KeplerArgs &a, cudaStream_t st);

// mlp.cu: learned Kepler guess, inference and training
size_t mlp_workspace_bytes();
cudaError_t launch_mlp_forward(int64_t n, const float *w, const float *u, float *y, cudaStream_t st);
cudaError_t launch_mlp_grad(int64_t n, const float *w, const float *rows, float *grad, float *loss,
                            void *work, cudaStream_t st);
cudaError_t launch_mlp_adam(float *w, float *m, float *v, const float *grad, int64_t t, float lr,
                            float beta1, float beta2, float eps, cudaStream_t st);
cudaError_t launch_mlp_train(float *w, float *m, float *v, int64_t t0, const float *rows, int64_t n,
                             int64_t batch, int32_t epochs, float lr, float lr_final, float *losses,
                             void *work, cudaStream_t st);

// step kernels (step.cu)
cudaError_t launch_momentum(const Dev &d, cudaStream_t st);
// kick_span: the time of the kick(s) between this pack and the Kepler drift
// (tau/2, or tau when two half kicks are merged); it sizes the crude reach
cudaError_t launch_drift_pack_from(const Dev &d, const double *qs, const double *vs,
                                   double h_close, double h_open, double tau, double a_E,
                                   double G, int flag_next, int hill_fixed, cudaStream_t st,
                                   double kick_span, double a_allow = 1.01);
// a_allow: the bound on |a| / |a of the last kick| that the crude reach of the
// preceding pack assumed (checked when check != 0)
// skip_whole: leave v of the systems flagged in d.wh_flag (their step was
// integrated whole: no second kick)
cudaError_t launch_kick_finish_v(const Dev &d, double *v, const double *q, double dt, double G,
                                 int check, int hill_fixed, cudaStream_t st,
                                 double a_allow = 1.01, int skip_whole = 0);
cudaError_t launch_hill_init(const Dev &d, double G, cudaStream_t st);
cudaError_t launch_to_dh_impl(const Dev &d, int inverse, double *vout, double *mt_scratch,
                              cudaStream_t st);

// kick.cu
struct KickTune {
    int32_t threads = 128;  // threads per CTA
    int32_t ipt = 2;        // i rows per thread
    int32_t splits = 1;     // j splits per system
};
// flag: what a pass over the tiles does
enum KickMode {
    KICK_FORCE = 0,        // the interaction sums only
    KICK_SEARCH = 1,       // the sums and the crude encounter search
    KICK_SEARCH_ONLY = 2,  // the crude encounter search alone (no sums written)
};
cudaError_t launch_kick_tiles(const Dev &d, int prec, int flag, double G, int threads, int ipt,
                              cudaStream_t st);
cudaError_t launch_accel_single(int64_t rows, const double *m, const double *q, double *a,
                                double G, int prec, double heavy_mass, void *work,
                                size_t work_bytes, cudaStream_t st);
size_t accel_single_workspace(int64_t rows, int prec);
// items of the i rows in [i_lo, i_hi) (default: all rows) against all j
void kick_items_host(const int64_t *offsets, int32_t nsys, const KickTune &t,
                     int4 *items, int32_t *slots, int32_t *nitems, int32_t *splits_used,
                     int32_t max_items, int64_t i_lo = 0, int64_t i_hi = INT64_MAX,
                     int32_t align = 1);
constexpr int kKickTile = 256;  // j rows per shared-memory tile of the kick
int32_t kick_items_count(const int64_t *offsets, int32_t nsys, const KickTune &t,
                         int64_t i_lo = 0, int64_t i_hi = INT64_MAX);

// sort.cu: Morton order of a system's bodies for the kick
struct SortScratch {
    int *box;              // [6]
    uint32_t *k0, *k1;     // [rows] keys
    int32_t *v0, *v1;      // [rows] rows
    uint32_t *hist;        // [256 * sort_blocks(rows)]
};
int64_t sort_blocks(int64_t n);
cudaError_t launch_sort_rows(int64_t rows, const double *q, const SortScratch &s, int32_t *perm,
                             int32_t *inv, cudaStream_t st);

// search.cu: candidates by spatial binning after the Kepler drift
struct SearchArgs {
    double tau, a_E;
    float4 *box_lo, *box_hi; // [rows] widened boxes by position
    float4 *x0h, *x0l, *x1h, *x1l, *v0f, *v1f;  // [rows] by position (x0h.w: a_E r_H)
    int *tbox_bits;          // [6 x tiles] tile boxes: min x, y, z, -max x, y, z as ordered
                             // integer images (reset to INT_MAX every step)
    const int32_t *tile0;    // [nsys] first tile of each system
    const int4 *tiles;       // (system, p0, p1, -)
    int32_t ntiles;
    const int2 *tpairs;      // (tile I, tile J), I <= J, same system
    int64_t ntpairs;
    int2 *active;            // [ntpairs] tile pairs whose boxes overlap (count: C_NACTIVE)
};
cudaError_t launch_binned_search(const Dev &d, const SearchArgs &s, double tau, double a_E,
                                 cudaStream_t st);
void search_tiles_host(const int64_t *offsets, int32_t nsys, std::vector<int4> &tiles,
                       std::vector<int2> &tpairs);

// encounter.cu
struct SetScratch {
    int32_t *blk, *sid, *size, *fill;
    unsigned long long *rc_bits;
};
cudaError_t launch_refine(const Dev &d, double tau, double a_E, cudaStream_t st);
cudaError_t launch_sets_impl(const Dev &d, double a_H, const SetScratch &s, cudaStream_t st);
cudaError_t launch_pair_test(int64_t rows, const double *q0, const double *v0, const double *q1,
                             const double *v1, const double *rH, double tau, double a_E,
                             int64_t npairs, const int32_t *pairs, double *d2, int32_t *flag,
                             cudaStream_t st);

// hermite.cu
cudaError_t hermite_prepare();
cudaError_t launch_transition(int64_t n, const double *s, double rc, double *K, double *Kp,
                              double *Kpp, cudaStream_t st);
cudaError_t launch_hermite(const Dev &d, const qym_params &p, double tau, cudaStream_t st);

// whole.cu: the whole-system Hermite (Sec. 2.3, last paragraph)
enum WholeCtl { WC_NA = 0, WC_DONE, WC_NCH, WC_COUNT };
struct WholeArgs {
    int64_t R;           // rows of the context's [3][R] arrays
    int64_t r0;          // the system's star row; its bodies are rows r0+1 .. r0+nb
    int64_t ld;          // stride of the scratch arrays' coordinates
    int32_t nb;          // bodies
    int32_t grid;        // CTAs of the force kernel
    const double *m;
    double G, m0, eps2, eta, eta_s, T, sg, tick;
    int64_t max_steps;   // block steps
    double *x, *u, *xp, *up, *a0, *j0;  // [3][ld]
    // the prediction split into float hi + lo parts for the light partners'
    // FP32 pair terms: (x, y, z, G m) and (x, y, z, -) of the position, the
    // velocity's the same; heavy bodies (m >= heavy_thr) enter at G m = 0 and
    // are summed in FP64 over `heavy` instead
    float4 *pf_hi, *pf_lo, *vf_hi, *vf_lo;  // [ld]
    double heavy_thr;
    const int32_t *heavy;  // the system's heavy bodies (indices of its bodies, ascending)
    int32_t nheavy;
    double *part;        // [max(grid, nb)][6] partner-range sums
    long long *ti;       // [nb] time of each body (ticks of |tau| 2^-48)
    int32_t *lev;        // [nb] step level
    int32_t *act;        // [nb] bodies of the block step
    int32_t *ctl;        // [WC_COUNT]
    long long *tn, *steps;
    int32_t *status;
};
cudaError_t launch_wh_trigger(const Dev &d, double planet_mass, int32_t *flag, cudaStream_t st);
cudaError_t launch_wh_start(const WholeArgs &w, const double *q, const double *vpre, cudaStream_t st);
cudaError_t launch_wh_blocks(const WholeArgs &w, int nblocks, cudaStream_t st);
cudaError_t launch_wh_store(const WholeArgs &w, double *q1, double *v1, cudaStream_t st);

// energy.cu
int32_t energy_items_host(const int64_t *offsets, int32_t nsys, int4 *items, int32_t *isys,
                          int32_t *item0);
cudaError_t launch_energy_items(int32_t nitems, const int4 *items, const int32_t *isys,
                                const int32_t *item0, int32_t nsys, const int64_t *offsets,
                                int64_t R, const double *m, const double *q, const double *v,
                                double G, double *part, double *E, cudaStream_t st);

}  // namespace qym
