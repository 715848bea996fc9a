// api.cu -- the C ABI of libqym (include/qym.h): context creation, the step
// loop, state and encounter transfer, energy, and the device-level calls.
//
// The step (Sec. 2, Eq. 5 and the procedure of Sec. 2.3) runs entirely on the
// device, with no host round trip inside a qym_step call: the first step's
// opening drift, then per step
//   kick 1 (crude encounter search fused) -> finish -> Kepler drift ->
//   rigorous test -> encounter sets -> Hermite (with K corrections) ->
//   pack -> kick 2 -> finish -> momentum -> closing + next opening drift.
// Identical steps are captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qym_internal.cuh"

using namespace qym;

static thread_local std::string g_err;

namespace qym {
// the message qym_last_error(NULL) returns, for context-free calls of other
// translation units
void set_thread_error(const std::string &msg) { g_err = msg; }
}  // namespace qym

// A piece of a step call captured as a CUDA graph for the tau it was taken
// with, and the kernels one replay launches
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    double tau = 0.0;
    int64_t launches = 0;
};

struct qym_ctx {
    qym_params p;
    cudaStream_t stream = nullptr;
    Dev d;
    std::vector<int64_t> h_offsets;
    void *arena = nullptr;
    KickTune tune;
    // energy
    int4 *eitems = nullptr;
    int32_t *eisys = nullptr, *eitem0 = nullptr;
    double *epart = nullptr, *E = nullptr;
    int32_t neitems = 0;
    double *mt = nullptr;  // [nsys] total masses
    void *flush = nullptr; // L2 flush buffer (params.l2_flush_bytes)
    SetScratch ss;
    bool amag_valid = false;
    // captured pieces of a call: an interior step, the closing step, the
    // call's opening (counters, [Morton order,] drift) with and without the sort
    StepGraph g_step, g_last, g_open[2];
    StepGraph g_upload;  // qym_set_state after its check: the state in, converted, ordered
    qym_stats stats;
    std::string err;
    int32_t status_bits = 0;
    int32_t items_cap = 0, splits_cap = 0;  // sizes of the item and partial buffers
    int32_t *kick_cnt = nullptr;            // per i-block arrival counters of the kick
    int64_t n_heavy = 0;    // heavy bodies over all systems
    int64_t launches = 0;   // kernels enqueued by the current qym_step call
    // learned Kepler guess and the log of Kepler solves
    float *mlp_w = nullptr;      // [QYM_MLP_NW] device weights (arena)
    bool mlp_set = false;
    float *klog = nullptr;       // caller's device rows [klog_cap][5], or NULL
    int64_t klog_cap = 0;
    unsigned long long klog_steps = 0;   // steps logged so far
    unsigned long long *klog_base = nullptr;  // device copy of klog_steps (arena)
    int32_t *hflag = nullptr;    // state upload: bit 1 non-finite position, bit 2 velocity
    // caller's device arrays receiving the encounter test's inputs of the
    // last step of each qym_step call (q0, v0, q1, v1 [3][rows], rH [rows])
    double *snap[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // the step of one system split over several GPUs (qym_split_*)
    int32_t split_rank = 0, split_world = 0;  // world 0: not split
    bool split_fresh = false;   // this run's first kick has no |a| of an earlier one
    int64_t *owned_info = nullptr;  // device [2]: first member and count of the own sets
    // the kick's Morton order of the bodies (one system, mixed kick)
    bool sort_rows = false;
    bool sort_current = false;  // the order was taken from the present state (set_state)
    SortScratch sortw{};
    // binned encounter search (params.search == QYM_SEARCH_BINNED)
    bool binned = false;
    SearchArgs sarg{};
    int32_t nstiles = 0;
    int64_t nstpairs = 0;
    // whole-system Hermite (params.whole_hermite): scratch for the largest
    // system, the star masses, this qym_step call's counts
    WholeArgs wh{};
    int64_t wh_nbmax = 0;
    std::vector<double> h_m0;
    std::vector<int32_t> h_wh_heavy;      // each system's heavy bodies (indices of its bodies)
    std::vector<int64_t> h_wh_heavy_off;  // [nsys+1] their ranges
    int32_t *wh_heavy = nullptr;          // device copy
    std::vector<int32_t> h_wh_flag;
    int64_t wh_steps = 0, wh_hsteps = 0, wh_hmax = 0;
};

#define FAIL(ctx, code, msg)                         \
    do {                                             \
        std::string _m = (msg);                      \
        if (ctx) ((qym_ctx *)(ctx))->err = _m;       \
        else g_err = _m;                             \
        return (code);                               \
    } while (0)

#define CK(ctx, call)                                                                  \
    do {                                                                               \
        cudaError_t _e = (call);                                                       \
        if (_e != cudaSuccess)                                                         \
            FAIL(ctx, QYM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));  \
    } while (0)

extern "C" qym_status qym_default_params(qym_params *p) {
    if (!p) FAIL(nullptr, QYM_EINVAL, "qym_default_params: NULL params");
    std::memset(p, 0, sizeof(*p));
    p->G = 1.0;
    p->a_E = 3.0;
    p->a_H = 1.0;
    p->eps_H = 1e-6;
    p->eta = 0.02;
    p->eta_s = 0.01;
    p->kick_prec = QYM_KICK_MIXED;
    p->solver = QYM_SOLVER_LAGUERRE;
    p->guess = QYM_GUESS_STANDARD;
    p->encounters = 1;
    p->coords = 0;
    p->hill_fixed = 0;
    p->max_kepler_iter = 50;
    p->device = 0;
    p->max_hermite_steps = 100000;
    p->max_candidates = 0;
    p->max_encounters = 0;
    p->max_log = 0;
    p->l2_flush_bytes = 0;
    p->heavy_mass = 1e-7;
    p->search = QYM_SEARCH_AUTO;
    p->whole_hermite = 0;
    p->planet_mass = 1e-7;
    return QYM_OK;
}

static bool valid_params(const qym_params *p, std::string &why) {
    if (!(p->G > 0.0)) { why = "G must be > 0"; return false; }
    if (!(p->a_E >= 0.0) || !(p->a_H > 0.0)) { why = "a_E >= 0 and a_H > 0 required"; return false; }
    if (!(p->eps_H >= 0.0)) { why = "eps_H must be >= 0"; return false; }
    if (!(p->eta > 0.0) || !(p->eta_s > 0.0)) { why = "eta, eta_s must be > 0"; return false; }
    if (p->kick_prec != QYM_KICK_FP64 && p->kick_prec != QYM_KICK_MIXED) { why = "kick_prec"; return false; }
    if (p->solver != QYM_SOLVER_LAGUERRE && p->solver != QYM_SOLVER_NEWTON &&
        p->solver != QYM_SOLVER_NEWTON32) { why = "solver"; return false; }
    if (p->guess < 0 || p->guess > 2) { why = "guess"; return false; }
    if (p->max_kepler_iter < 1) { why = "max_kepler_iter must be >= 1"; return false; }
    if (p->max_hermite_steps < 1) { why = "max_hermite_steps must be >= 1"; return false; }
    if (p->max_candidates < 0 || p->max_encounters < 0 || p->max_log < 0) { why = "capacities"; return false; }
    if (p->l2_flush_bytes < 0 || p->l2_flush_bytes > ((int64_t)1 << 34)) { why = "l2_flush_bytes"; return false; }
    if (p->merge_kicks != 0 && p->merge_kicks != 1) { why = "merge_kicks must be 0 or 1"; return false; }
    if (p->search != QYM_SEARCH_FUSED && p->search != QYM_SEARCH_BINNED &&
        p->search != QYM_SEARCH_AUTO && p->search != QYM_SEARCH_ESCAPE) {
        why = "search must be QYM_SEARCH_AUTO, QYM_SEARCH_FUSED, QYM_SEARCH_BINNED or QYM_SEARCH_ESCAPE";
        return false;
    }
    if (p->hermite_cluster != 0 && p->hermite_cluster != 2 && p->hermite_cluster != 4 &&
        p->hermite_cluster != 8) {
        why = "hermite_cluster must be 0, 2, 4 or 8";
        return false;
    }
    if (p->whole_hermite != 0 && p->whole_hermite != 1) { why = "whole_hermite must be 0 or 1"; return false; }
    if (!(p->planet_mass >= 0.0) || !std::isfinite(p->planet_mass)) { why = "planet_mass must be >= 0"; return false; }
    if (p->whole_hermite && p->merge_kicks) {
        why = "whole_hermite needs the paper's two kicks per step (merge_kicks = 0)";
        return false;
    }
    return true;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// bodies from which a single system's kick holds them in Morton order
constexpr int64_t kSortMinBodies = 2048;
// bodies from which QYM_SEARCH_AUTO takes the binned search for one system
constexpr int64_t kBinnedMinBodies = 65536;
// steps between re-sorts inside one qym_step call (bodies drift apart slowly;
// the order only affects speed)
constexpr int64_t kSortEvery = 32;

// ------------------------------------------------------------------ arena
struct Carver {
    char *base;
    size_t off = 0;
    bool dry;
    template <class T>
    T *take(size_t n) {
        size_t o = off;
        off = al256(off + sizeof(T) * (n ? n : 1));
        return dry ? nullptr : (T *)(base + o);
    }
};

static void choose_slot_sums(qym_ctx *c);

// the captured steps, dropped whenever what they hold by value changes (the
// launch shape, the log and snapshot pointers, tau)
static void drop_graph(StepGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
}
static void drop_graphs(qym_ctx *c) {
    drop_graph(c->g_step);
    drop_graph(c->g_last);
    drop_graph(c->g_open[0]);
    drop_graph(c->g_open[1]);
    drop_graph(c->g_upload);
}

// Replay g, capturing it first from `enqueue` (which counts its launches in
// c->launches) when it is missing or was taken with another tau.
template <class F>
static cudaError_t replay(qym_ctx *c, StepGraph &g, double tau, F &&enqueue) {
    cudaStream_t st = c->stream;
    if (g.exec && g.tau != tau) drop_graph(g);
    cudaError_t e;
    if (!g.exec) {
        cudaGraph_t gr;
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal))) return e;
        const int64_t before = c->launches;
        e = enqueue();
        g.launches = c->launches - before;
        c->launches = before;
        const cudaError_t e2 = cudaStreamEndCapture(st, &gr);
        if (e != cudaSuccess) {
            if (e2 == cudaSuccess) cudaGraphDestroy(gr);
            return e;
        }
        if (e2 != cudaSuccess) return e2;
        e = cudaGraphInstantiate(&g.exec, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return e;
        }
        g.tau = tau;
    }
    if ((e = cudaGraphLaunch(g.exec, st))) return e;
    c->launches += g.launches;
    return cudaSuccess;
}

static void carve_all(qym_ctx *c, Carver &k) {
    Dev &d = c->d;
    const int64_t R = d.rows;
    d.offsets = k.take<int64_t>(d.nsys + 1);
    d.sys_of = k.take<int32_t>(R);
    d.m = k.take<double>(R);
    d.q = k.take<double>(3 * R);
    d.v = k.take<double>(3 * R);
    d.q1 = k.take<double>(3 * R);
    d.v1 = k.take<double>(3 * R);
    d.rH = k.take<double>(R);
    d.rH_fixed = k.take<double>(R);
    d.pk_pos = k.take<float4>(R);
    d.pk_lo = k.take<float4>(R);
    d.amag = k.take<float>(R);
    d.rH_bound = k.take<float>(R);
    d.apart = k.take<double>((size_t)3 * R * c->splits_cap);
    d.items = k.take<int4>(c->items_cap);
    d.item_slot = k.take<int32_t>(c->items_cap);
    c->kick_cnt = k.take<int32_t>(c->items_cap);  // zero with the arena
    d.mchunks = k.take<int4>(d.nmchunks);
    d.mpart = k.take<double>(3 * (size_t)d.nmchunks);
    d.sys_chunk0 = k.take<int32_t>(d.nsys + 1);
    d.S = k.take<double>(3 * (size_t)d.nsys);
    d.heavy_rows = k.take<int32_t>(c->n_heavy);
    d.heavy_start = k.take<int32_t>(d.nsys + 1);
    d.heavy_thr = k.take<double>(d.nsys);
    d.kmu = k.take<double>(3 * (size_t)d.nsys);
    d.hfac = k.take<double>(R);
    d.cand = k.take<int2>(d.max_cand);
    d.fchunk = k.take<int4>(d.max_fchunk);
    d.enc = k.take<int2>(d.max_enc);
    d.rescan = k.take<int32_t>(R);
    d.set_start = k.take<int32_t>((size_t)d.max_sets + 1);
    d.set_mem = k.take<int32_t>(d.max_members);
    d.rcrit = k.take<double>(d.max_sets);
    d.set_root = k.take<int32_t>(d.max_sets);
    d.hcost = k.take<int32_t>(R);
    d.hq = k.take<int32_t>(d.max_sets);
    d.hsetcost = k.take<int32_t>(d.max_sets);
    d.hcl = k.take<int32_t>(kHermMaxClusters);
    d.uf = k.take<int32_t>(R);
    d.log = k.take<int64_t>(3 * (size_t)d.max_log);
    d.ctr = k.take<unsigned long long>(C_COUNT);
    d.status = k.take<int32_t>(1);
    c->ss.blk = k.take<int32_t>((R + 1023) / 1024 + 1);
    c->ss.sid = k.take<int32_t>(R);
    c->ss.size = k.take<int32_t>(R + 1);
    c->ss.fill = k.take<int32_t>(R + 1);
    c->ss.rc_bits = k.take<unsigned long long>(R + 1);
    c->eitems = k.take<int4>(c->neitems);
    c->eisys = k.take<int32_t>(c->neitems);
    c->eitem0 = k.take<int32_t>(d.nsys + 1);
    c->epart = k.take<double>(c->neitems);
    c->E = k.take<double>(d.nsys);
    c->mt = k.take<double>(d.nsys);
    c->mlp_w = k.take<float>(QYM_MLP_NW);
    c->klog_base = k.take<unsigned long long>(1);
    c->hflag = k.take<int32_t>(1);
    c->owned_info = k.take<int64_t>(2);
    if (c->sort_rows) {
        d.perm = k.take<int32_t>(R);
        d.inv = k.take<int32_t>(R);
        c->sortw.box = k.take<int>(8);
        c->sortw.k0 = k.take<uint32_t>(R);
        c->sortw.k1 = k.take<uint32_t>(R);
        c->sortw.v0 = k.take<int32_t>(R);
        c->sortw.v1 = k.take<int32_t>(R);
        c->sortw.hist = k.take<uint32_t>(256 * (size_t)sort_blocks(R));
        d.far = k.take<float4>(R);
        d.tile = k.take<float4>(3 * (size_t)((R - 1 + kKickTile - 1) / kKickTile));
    }
    if (c->p.whole_hermite) {
        WholeArgs &w = c->wh;
        const int64_t L = std::max<int64_t>(1, c->wh_nbmax);
        d.wh_flag = k.take<int32_t>(d.nsys);
        d.vpre = k.take<double>(3 * (size_t)R);
        w.grid = 8 * 152;
        w.x = k.take<double>(3 * (size_t)L);
        w.u = k.take<double>(3 * (size_t)L);
        w.xp = k.take<double>(3 * (size_t)L);
        w.up = k.take<double>(3 * (size_t)L);
        w.a0 = k.take<double>(3 * (size_t)L);
        w.j0 = k.take<double>(3 * (size_t)L);
        w.part = k.take<double>(6 * (size_t)std::max<int64_t>(L, w.grid));
        w.pf_hi = k.take<float4>(L);
        w.pf_lo = k.take<float4>(L);
        w.vf_hi = k.take<float4>(L);
        w.vf_lo = k.take<float4>(L);
        c->wh_heavy = k.take<int32_t>(std::max<size_t>(1, c->h_wh_heavy.size()));
        w.ti = k.take<long long>(L);
        w.lev = k.take<int32_t>(L);
        w.act = k.take<int32_t>(L);
        w.ctl = k.take<int32_t>(WC_COUNT);
        w.tn = k.take<long long>(1);
        w.steps = k.take<long long>(1);
        w.ld = L;
    }
    if (c->binned) {
        SearchArgs &a = c->sarg;
        d.vmax = k.take<int32_t>(d.nsys);
        a.box_lo = k.take<float4>(R);
        a.box_hi = k.take<float4>(R);
        a.x0h = k.take<float4>(R);
        a.x0l = k.take<float4>(R);
        a.x1h = k.take<float4>(R);
        a.x1l = k.take<float4>(R);
        a.v0f = k.take<float4>(R);
        a.v1f = k.take<float4>(R);
        a.tbox_bits = k.take<int>(6 * (size_t)c->nstiles);
        a.tile0 = k.take<int32_t>(d.nsys);
        a.tiles = k.take<int4>(c->nstiles);
        a.tpairs = k.take<int2>(c->nstpairs);
        a.active = k.take<int2>(c->nstpairs);
        a.ntiles = c->nstiles;
        a.ntpairs = c->nstpairs;
    }
}

// The caller's rows [R][3] <-> the device's [3][R]. The transposes run on the
// device, so a pinned host buffer goes to and from the GPU in one DMA each;
// between steps the kick's partial sums are idle and stage the rows.
// host rows [R][3] -> [3][R] with star rows zero; `bit` set in *bad for a
// non-finite value, and with `cur` (the state held now, [3][R]) `cbit` set
// when some value differs from it bit for bit
__global__ void k_soa_from_aos(int64_t R, const double *aos, double *soa, const int64_t *offsets,
                               const int32_t *sys_of, int32_t *bad, int32_t bit,
                               const double *cur = nullptr, int32_t cbit = 0) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const bool star = offsets[sys_of[r]] == r;  // star rows are held at zero
    for (int c = 0; c < 3; ++c) {
        const double x = star ? 0.0 : aos[3 * r + c];
        if (!isfinite(x)) atomicOr(bad, bit);
        if (cur && __double_as_longlong(x) != __double_as_longlong(cur[c * R + r]))
            atomicOr(bad, cbit);
        soa[c * R + r] = x;
    }
}

__global__ void k_aos_from_soa(int64_t R, const double *soa, double *aos) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    for (int c = 0; c < 3; ++c) aos[3 * r + c] = soa[c * R + r];
}

// Launch shape of the kick for this batch: enough CTAs to fill the GPU
// several times, each CTA at least a tile of j rows per split.
static KickTune default_tune(const std::vector<int64_t> &off, int prec) {
    KickTune t;
    t.threads = 128;
    t.ipt = prec == QYM_KICK_MIXED ? 2 : 1;
    int32_t nsys = (int32_t)off.size() - 1;
    int64_t ib = 0, nbmax = 0;
    for (int32_t s = 0; s < nsys; ++s) {
        int64_t nb = off[s + 1] - off[s] - 1;
        ib += (nb + t.threads * t.ipt - 1) / (t.threads * t.ipt);
        nbmax = std::max(nbmax, nb);
    }
    int64_t want = 4 * 152;
    int64_t sp = (want + ib - 1) / std::max<int64_t>(ib, 1);
    int64_t maxsp = std::max<int64_t>(1, nbmax / 256);
    t.splits = (int32_t)std::max<int64_t>(1, std::min(sp, maxsp));
    return t;
}

static qym_status upload_state(qym_ctx *c, const double *q, const double *v) {
    Dev &d = c->d;
    const int64_t R = d.rows;
    cudaStream_t st = c->stream;
    // rows land in the partial-sum buffer (at least 4 slots of [3][R]), are
    // transposed and checked into (q1, v1), and only a valid state replaces (q, v)
    double *sq = d.apart, *sv = d.apart + 3 * R;
    const unsigned g = (unsigned)((R + 255) / 256);
    CK(c, cudaMemcpyAsync(sq, q, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, st));
    CK(c, cudaMemcpyAsync(sv, v, sizeof(double) * 3 * R, cudaMemcpyHostToDevice, st));
    CK(c, cudaMemsetAsync(c->hflag, 0, sizeof(int32_t), st));
    k_soa_from_aos<<<g, 256, 0, st>>>(R, sq, d.q1, d.offsets, d.sys_of, c->hflag, 1, d.q, 4);
    k_soa_from_aos<<<g, 256, 0, st>>>(R, sv, d.v1, d.offsets, d.sys_of, c->hflag, 2);
    CK(c, cudaGetLastError());
    int32_t bad = 0;
    CK(c, cudaMemcpyAsync(&bad, c->hflag, sizeof(bad), cudaMemcpyDeviceToHost, st));
    CK(c, cudaStreamSynchronize(st));  // (the host arrays are free from here on)
    if (bad & 1) FAIL(c, QYM_EINVAL, "non-finite position");
    if (bad & 2) FAIL(c, QYM_EINVAL, "non-finite velocity");
    auto commit = [&]() -> cudaError_t {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(d.q, d.q1, sizeof(double) * 3 * R, cudaMemcpyDeviceToDevice, st)))
            return e;
        if ((e = cudaMemcpyAsync(d.v, d.v1, sizeof(double) * 3 * R, cudaMemcpyDeviceToDevice, st)))
            return e;
        if (c->p.coords == 0 && (e = launch_to_dh_impl(d, 0, nullptr, c->mt, st))) return e;
        if (c->p.hill_fixed && (e = launch_hill_init(d, c->p.G, st))) return e;
        if (d.perm && (e = launch_sort_rows(d.rows, d.q, c->sortw, d.perm, d.inv, st))) return e;
        return cudaSuccess;
    };
    const int64_t launches = c->launches;  // (the last step call's count stays)
    CK(c, replay(c, c->g_upload, 1.0, commit));
    c->launches = launches;
    c->sort_current = d.perm != nullptr;
    // The |a| of the last kick bounds the coming kick's (the crude search's
    // allowance) only at the same separations: kept when every position is
    // the one held before, bit for bit (a state read back and set again), so
    // that the next step fuses its search into the kick; any other state
    // makes that step search after its kick.
    if (bad & 4) c->amag_valid = false;
    return QYM_OK;
}

extern "C" qym_status qym_init(const qym_params *params, int32_t nsys, const int64_t *offsets,
                               const double *m, const double *q, const double *v, qym_ctx **out) {
    if (out) *out = nullptr;
    if (!params || !offsets || !m || !q || !v || !out)
        FAIL(nullptr, QYM_EINVAL, "qym_init: NULL argument");
    std::string why;
    if (!valid_params(params, why)) FAIL(nullptr, QYM_EINVAL, "qym_init: " + why);
    if (nsys < 1) FAIL(nullptr, QYM_EINVAL, "qym_init: nsys must be >= 1");
    if (offsets[0] != 0) FAIL(nullptr, QYM_EINVAL, "qym_init: offsets[0] must be 0");
    for (int32_t s = 0; s < nsys; ++s)
        if (offsets[s + 1] - offsets[s] < 2)
            FAIL(nullptr, QYM_EINVAL, "qym_init: every system needs a star and at least one body");
    const int64_t R = offsets[nsys];
    if (R >= (int64_t)1 << 31) FAIL(nullptr, QYM_EINVAL, "qym_init: too many rows (>= 2^31)");
    for (int32_t s = 0; s < nsys; ++s)
        if (!(m[offsets[s]] > 0.0)) FAIL(nullptr, QYM_EINVAL, "qym_init: star masses must be > 0");
    for (int64_t r = 0; r < R; ++r)
        if (!(m[r] >= 0.0) || !std::isfinite(m[r])) FAIL(nullptr, QYM_EINVAL, "qym_init: masses must be finite and >= 0");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        FAIL(nullptr, QYM_ENODEV, "qym_init: no CUDA device");
    if (params->device < 0 || params->device >= ndev) FAIL(nullptr, QYM_EINVAL, "qym_init: bad device");
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, params->device) != cudaSuccess || prop.major != 10 || prop.minor != 3)
        FAIL(nullptr, QYM_ENODEV, "qym_init: device is not sm_103 (GB300 class)");
    if (cudaSetDevice(params->device) != cudaSuccess) FAIL(nullptr, QYM_ECUDA, "cudaSetDevice failed");

    qym_ctx *c = new qym_ctx();
    c->p = *params;
    c->h_offsets.assign(offsets, offsets + nsys + 1);
    Dev &d = c->d;
    d.rows = R;
    d.nsys = nsys;
    if (params->whole_hermite) {
        c->h_m0.resize(nsys);
        c->h_wh_flag.assign(nsys, 0);
        c->h_wh_heavy_off.assign(nsys + 1, 0);
        for (int32_t s = 0; s < nsys; ++s) {
            c->h_m0[s] = m[offsets[s]];
            c->wh_nbmax = std::max<int64_t>(c->wh_nbmax, offsets[s + 1] - offsets[s] - 1);
            // heavy: m >= heavy_mass m0 (every body when heavy_mass <= 0)
            const double thr = params->heavy_mass > 0.0 ? params->heavy_mass * m[offsets[s]] : 0.0;
            for (int64_t r = offsets[s] + 1; r < offsets[s + 1]; ++r)
                if (m[r] >= thr) c->h_wh_heavy.push_back((int32_t)(r - offsets[s] - 1));
            c->h_wh_heavy_off[s + 1] = (int64_t)c->h_wh_heavy.size();
        }
    }
    c->tune = default_tune(c->h_offsets, params->kick_prec);
    d.nitems = kick_items_count(offsets, nsys, c->tune);
    d.splits = c->tune.splits;
    {
        // buffers large enough for every shape the tuner may try
        KickTune big;
        big.threads = 128;
        big.ipt = 1;
        big.splits = 16;
        // partial-sum slots: up to 128 for small batches, within ~0.5 GB
        int64_t by_mem = ((int64_t)1 << 29) / (24 * R);
        c->splits_cap = (int32_t)std::max<int64_t>(c->tune.splits, std::min<int64_t>(128, std::max<int64_t>(4, by_mem)));
        big.splits = c->splits_cap;
        c->items_cap = std::max(kick_items_count(offsets, nsys, big), d.nitems);
        c->items_cap = std::max(c->items_cap, kick_items_count(offsets, nsys, c->tune));
    }
    // momentum chunks, never crossing systems: about two per SM, of 512 to
    // 4096 rows (a CTA's FP64 reduction of its partial sums costs about as
    // much as 1024 rows of m v, so large inputs take large chunks; a small
    // one takes short ones, its time being the loads' latency)
    const int64_t kMomChunk = std::min<int64_t>(4096, std::max<int64_t>(512, (R / 304 + 255) / 256 * 256));
    std::vector<int4> mch;
    std::vector<int32_t> sc0(nsys + 1);
    for (int32_t s = 0; s < nsys; ++s) {
        sc0[s] = (int32_t)mch.size();
        for (int64_t r0 = offsets[s]; r0 < offsets[s + 1]; r0 += kMomChunk)
            mch.push_back(make_int4((int)r0, (int)std::min<int64_t>(r0 + kMomChunk, offsets[s + 1]), s, 0));
    }
    sc0[nsys] = (int32_t)mch.size();
    d.nmchunks = (int32_t)mch.size();
    d.max_cand = params->max_candidates ? params->max_candidates : std::max<int64_t>(1 << 20, 16 * R);
    // a flagged chunk holds a partner within the crude bound: at most two
    // records per candidate pair, plus a margin of one per row
    d.max_fchunk = d.max_cand + R;
    d.max_enc = params->max_encounters ? params->max_encounters : std::max<int64_t>(1 << 16, R);
    d.max_log = params->max_log ? params->max_log : (int64_t)1 << 22;
    d.max_sets = (int32_t)R;
    d.max_members = (int32_t)R;
    c->neitems = energy_items_host(offsets, nsys, nullptr, nullptr, nullptr);
    // heavy bodies per system (mixed kick): m >= heavy_mass m0, at most
    // QYM_HEAVY_CAP of them, else the system keeps all bodies in FP32
    std::vector<int32_t> hrows, hstart(nsys + 1);
    std::vector<double> hthr(nsys);
    const bool split = params->kick_prec == QYM_KICK_MIXED && params->heavy_mass > 0.0;
    for (int32_t s = 0; s < nsys; ++s) {
        hstart[s] = (int32_t)hrows.size();
        double thr = params->heavy_mass * m[offsets[s]];
        std::vector<int32_t> hs;
        if (split)
            for (int64_t r = offsets[s] + 1; r < offsets[s + 1]; ++r)
                if (m[r] >= thr) hs.push_back((int32_t)r);
        if (!split || hs.size() > QYM_HEAVY_CAP) {
            hthr[s] = INFINITY;
            hs.clear();
        } else {
            hthr[s] = thr;
        }
        hrows.insert(hrows.end(), hs.begin(), hs.end());
    }
    hstart[nsys] = (int32_t)hrows.size();
    c->n_heavy = (int64_t)hrows.size();
    // the Hill radius's mass factor (m / 3 m0)^(1/3) of every row (Eq. 9),
    // formed once: the FP64 cube root costs tens of FP64 instructions a row
    std::vector<double> hfac(R, 0.0);
    for (int32_t s = 0; s < nsys; ++s)
        for (int64_t r = offsets[s] + 1; r < offsets[s + 1]; ++r)
            hfac[r] = std::cbrt(m[r] / (3.0 * m[offsets[s]]));
    // E_Kep's mu = G m0 per system with sqrt(mu) and 1/mu (IEEE, as on the device)
    std::vector<double> kmu(3 * (size_t)nsys);
    for (int32_t s = 0; s < nsys; ++s) {
        const double mu = params->G * m[offsets[s]];
        kmu[3 * s] = mu;
        kmu[3 * s + 1] = std::sqrt(mu);
        kmu[3 * s + 2] = 1.0 / mu;
    }
    d.heavy_split = split ? 1 : 0;

    // one system of at least two tiles' worth of bodies, mixed kick: the kick
    // holds the bodies in Morton order (sort.cu)
    c->sort_rows = nsys == 1 && params->kick_prec == QYM_KICK_MIXED && R - 1 >= kSortMinBodies;
    // measured on one GB300 (same trajectories, so the same encounter work):
    // 16384-body disk 1.40 ms per step binned against 1.33 fused, the
    // 512-system ensemble 23.6 against 20.3 ms, the 262144-body disk 64.9
    // against 66.1 ms
    const bool auto_binned = nsys == 1 && R - 1 >= kBinnedMinBodies;
    c->binned = params->encounters &&
                (params->search == QYM_SEARCH_BINNED ||
                 (params->search == QYM_SEARCH_AUTO && auto_binned));
    d.escape_reach = params->encounters && params->search == QYM_SEARCH_ESCAPE ? 1 : 0;
    c->p.search = c->binned ? QYM_SEARCH_BINNED : (d.escape_reach ? QYM_SEARCH_ESCAPE : QYM_SEARCH_FUSED);
    std::vector<int4> stiles;
    std::vector<int2> stpairs;
    if (c->binned) {
        search_tiles_host(offsets, nsys, stiles, stpairs);
        c->nstiles = (int32_t)stiles.size();
        c->nstpairs = (int64_t)stpairs.size();
    }
    Carver dry{nullptr, 0, true};
    carve_all(c, dry);
    size_t bytes = dry.off;
    if (cudaMalloc(&c->arena, bytes) != cudaSuccess) {
        delete c;
        FAIL(nullptr, QYM_ENOMEM, "qym_init: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    Carver real{(char *)c->arena, 0, false};
    carve_all(c, real);
    choose_slot_sums(c);
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(c->arena);
        delete c;
        FAIL(nullptr, QYM_ECUDA, "qym_init: stream creation failed");
    }
    auto bail = [&](qym_status st) {
        g_err = c->err;
        qym_destroy(c);
        return st;
    };
#define CKI(call)                                                                         \
    do {                                                                                  \
        cudaError_t _e = (call);                                                          \
        if (_e != cudaSuccess) {                                                          \
            c->err = std::string(#call) + ": " + cudaGetErrorString(_e);                  \
            return bail(QYM_ECUDA);                                                       \
        }                                                                                 \
    } while (0)
    CKI(cudaMemsetAsync(c->arena, 0, bytes, c->stream));
    CKI(cudaMemsetAsync(d.uf, 0xff, sizeof(int32_t) * R, c->stream));
    // host-built tables
    std::vector<int32_t> sys_of(R);
    for (int32_t s = 0; s < nsys; ++s)
        for (int64_t r = offsets[s]; r < offsets[s + 1]; ++r) sys_of[r] = s;
    std::vector<int4> items(d.nitems);
    std::vector<int32_t> slots(d.nitems);
    int32_t ni = 0, spu = 0;
    kick_items_host(offsets, nsys, c->tune, items.data(), slots.data(), &ni, &spu, d.nitems, 0,
                    INT64_MAX, c->sort_rows ? kKickTile / 2 : 1);
    std::vector<int4> eit(c->neitems);
    std::vector<int32_t> eis(c->neitems), ei0(nsys + 1);
    energy_items_host(offsets, nsys, eit.data(), eis.data(), ei0.data());
    CKI(cudaMemcpyAsync(d.offsets, offsets, sizeof(int64_t) * (nsys + 1), cudaMemcpyHostToDevice, c->stream));
    if (!c->h_wh_heavy.empty())
        CKI(cudaMemcpyAsync(c->wh_heavy, c->h_wh_heavy.data(), sizeof(int32_t) * c->h_wh_heavy.size(),
                            cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.sys_of, sys_of.data(), sizeof(int32_t) * R, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.m, m, sizeof(double) * R, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.items, items.data(), sizeof(int4) * d.nitems, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.item_slot, slots.data(), sizeof(int32_t) * d.nitems, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.mchunks, mch.data(), sizeof(int4) * d.nmchunks, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.sys_chunk0, sc0.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(c->eitems, eit.data(), sizeof(int4) * c->neitems, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(c->eisys, eis.data(), sizeof(int32_t) * c->neitems, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(c->eitem0, ei0.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, c->stream));
    if (!hrows.empty())
        CKI(cudaMemcpyAsync(d.heavy_rows, hrows.data(), sizeof(int32_t) * hrows.size(), cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.heavy_start, hstart.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.heavy_thr, hthr.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.kmu, kmu.data(), sizeof(double) * 3 * nsys, cudaMemcpyHostToDevice, c->stream));
    CKI(cudaMemcpyAsync(d.hfac, hfac.data(), sizeof(double) * R, cudaMemcpyHostToDevice, c->stream));
    if (c->binned && c->nstiles) {
        std::vector<int32_t> t0(nsys);
        for (size_t t = stiles.size(); t-- > 0;) t0[stiles[t].x] = (int32_t)t;
        CKI(cudaMemcpyAsync((void *)c->sarg.tile0, t0.data(), sizeof(int32_t) * nsys,
                            cudaMemcpyHostToDevice, c->stream));
        CKI(cudaMemcpyAsync((void *)c->sarg.tiles, stiles.data(), sizeof(int4) * stiles.size(),
                            cudaMemcpyHostToDevice, c->stream));
        CKI(cudaMemcpyAsync((void *)c->sarg.tpairs, stpairs.data(), sizeof(int2) * stpairs.size(),
                            cudaMemcpyHostToDevice, c->stream));
    }
    CKI(cudaStreamSynchronize(c->stream));  // host vectors go out of scope below
    CKI(hermite_prepare());
    if (params->l2_flush_bytes > 0) CKI(cudaMalloc(&c->flush, (size_t)params->l2_flush_bytes));
#undef CKI
    qym_status st = upload_state(c, q, v);
    if (st != QYM_OK) return bail(st);
    std::memset(&c->stats, 0, sizeof(c->stats));
    c->stats.kick_tile_i = c->tune.threads * c->tune.ipt;
    c->stats.kick_tile_splits = c->tune.splits;
    *out = c;
    return QYM_OK;
}

extern "C" void qym_destroy(qym_ctx *c) {
    if (!c) return;
    drop_graphs(c);
    if (c->stream) {
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
    }
    if (c->arena) cudaFree(c->arena);
    if (c->flush) cudaFree(c->flush);
    delete c;
}

extern "C" qym_status qym_shape(const qym_ctx *c, int64_t *rows, int32_t *nsys) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_shape: NULL context");
    if (rows) *rows = c->d.rows;
    if (nsys) *nsys = c->d.nsys;
    return QYM_OK;
}

// ------------------------------------------------------------------ step
__global__ void k_step_begin(unsigned long long *ctr, int32_t *vmax, int32_t nsys, int *tbits,
                             int64_t ntb) {
    if (vmax)  // the binned search's largest |v| per system, raised by the first finisher
        for (int32_t s = threadIdx.x; s < nsys; s += blockDim.x) vmax[s] = 0;
    for (int64_t k = threadIdx.x; k < ntb; k += blockDim.x) tbits[k] = 0x7fffffff;  // tile boxes
    if (threadIdx.x) return;
    ctr[C_NCAND] = 0;
    ctr[C_NACTIVE] = 0;
    ctr[C_NENC] = 0;
    ctr[C_NRESCAN] = 0;
    ctr[C_NSETS] = 0;
    ctr[C_HSMALL] = 0;
    ctr[C_NFCHUNK] = 0;
    ctr[C_FCDONE] = 0;
}

__global__ void k_step_end(unsigned long long *ctr, int64_t max_cand, int64_t max_enc) {
    ctr[C_SUM_CAND] += ctr[C_NCAND];
    ctr[C_SUM_ENC] += ctr[C_NENC];
    ctr[C_SUM_RESCAN] += ctr[C_NRESCAN];
    ctr[C_STEP] += 1;
}

// one step whose opening drift has been applied: ends with the closing drift
// of this step plus, unless last, the opening drift of the next one
// E_Kep of every row over tau, (q, v) -> (q1, v1), with the context's solver,
// guess and solve log
static KeplerArgs step_kepler_args(qym_ctx *c, double tau) {
    Dev &d = c->d;
    const qym_params &p = c->p;
    KeplerArgs ka;
    std::memset(&ka, 0, sizeof(ka));
    ka.n = d.rows;
    ka.q0 = d.q; ka.v0 = d.v; ka.q1 = d.q1; ka.v1 = d.v1;
    ka.ld = d.rows;
    ka.dt = tau;
    ka.solver = p.solver;
    ka.guess = p.guess;
    ka.mlp_w = p.guess == QYM_GUESS_MLP ? c->mlp_w : nullptr;
    ka.max_iter = p.max_kepler_iter;
    if (c->klog) {
        ka.log = c->klog;
        ka.log_cap = c->klog_cap;
        ka.log_base = c->klog_base;
        ka.log_step = d.ctr + C_STEP;
    }
    ka.status = d.status;
    ka.iter_sum = d.ctr + C_SUM_KITER;
    ka.sys_of = d.sys_of;
    ka.kmu = d.kmu;
    return ka;
}

// kernels a search kick adds after the kick itself (the mixed kick's exact
// re-test of its flagged chunks)
static int search_retest(const qym_params &p, int flag) {
    return (flag && p.kick_prec == QYM_KICK_MIXED) ? 1 : 0;
}

// 1 when the first kick of a step carries the crude encounter search
// (QYM_SEARCH_FUSED); with QYM_SEARCH_BINNED the search follows the drift
static int fused_search(const qym_ctx *c) { return (c->p.encounters && !c->binned) ? 1 : 0; }

// the binned search's candidates, after the Kepler drift
static cudaError_t enqueue_binned_search(qym_ctx *c, double tau) {
    if (!c->binned) return cudaSuccess;
    c->launches += 3;
    return launch_binned_search(c->d, c->sarg, tau, c->p.a_E, c->stream);
}

// copies of the rigorous encounter test's inputs (qym_set_encounter_snapshot):
// (q, v) enter the Kepler drift, (q1, v1) its result, before the Hermite
static cudaError_t enqueue_snapshot(qym_ctx *c) {
    if (!c->snap[0]) return cudaSuccess;
    const Dev &d = c->d;
    const size_t b3 = sizeof(double) * 3 * (size_t)d.rows;
    const double *src[5] = {d.q, d.v, d.q1, d.v1, d.rH};
    for (int k = 0; k < 5; ++k) {
        cudaError_t e = cudaMemcpyAsync(c->snap[k], src[k], k < 4 ? b3 : b3 / 3,
                                        cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The opening kick of a step with the crude encounter search when no |a| of
// an earlier kick bounds this one (after qym_init or qym_set_state): the kick
// runs first, then the reaches are built from the kicked state (no |a|
// allowance needed) and a pass over the tiles runs the search alone.
static cudaError_t enqueue_fresh_search_kick(qym_ctx *c, double dt) {
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    cudaError_t e;
    if ((e = launch_kick_tiles(d, p.kick_prec, KICK_FORCE, p.G, c->tune.threads, c->tune.ipt, st)))
        return e;
    if ((e = launch_kick_finish_v(d, d.v, d.q, dt, p.G, 0, p.hill_fixed, st))) return e;
    if ((e = launch_drift_pack_from(d, d.q, d.v, 0.0, 0.0, dt, p.a_E, p.G, 2, p.hill_fixed, st,
                                    0.0)))
        return e;
    if ((e = launch_kick_tiles(d, p.kick_prec, KICK_SEARCH_ONLY, p.G, c->tune.threads,
                               c->tune.ipt, st)))
        return e;
    // kick, finish, pack, search [+ chunk re-test]
    c->launches += 4 + search_retest(p, 1);
    return cudaSuccess;
}

// Sec. 2.3, last paragraph: the systems whose sets put two planets in one set
// this step (the sets just built) are integrated whole by the Hermite into
// (q1, v1); the host reads the flags and drives the block steps in chunks of
// 32 (four kernels each), reading the done flag after each chunk.
static cudaError_t enqueue_whole(qym_ctx *c, double tau) {
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(d.wh_flag, 0, sizeof(int32_t) * d.nsys, st))) return e;
    if ((e = launch_wh_trigger(d, p.planet_mass, d.wh_flag, st))) return e;
    if ((e = cudaMemcpyAsync(c->h_wh_flag.data(), d.wh_flag, sizeof(int32_t) * d.nsys,
                             cudaMemcpyDeviceToHost, st)))
        return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    c->launches += 2;
    for (int32_t s = 0; s < d.nsys; ++s) {
        if (!c->h_wh_flag[s]) continue;
        WholeArgs w = c->wh;
        w.R = d.rows;
        w.r0 = c->h_offsets[s];
        w.nb = (int32_t)(c->h_offsets[s + 1] - w.r0 - 1);
        w.m = d.m;
        w.G = p.G;
        w.m0 = c->h_m0[s];
        w.eps2 = p.eps_H * p.eps_H;
        w.eta = p.eta;
        w.eta_s = p.eta_s;
        w.T = std::fabs(tau);
        w.sg = tau >= 0.0 ? 1.0 : -1.0;
        w.tick = w.T / (double)(1ll << 48);
        w.max_steps = p.max_hermite_steps;
        w.status = d.status;
        w.heavy_thr = p.heavy_mass > 0.0 ? p.heavy_mass * w.m0 : 0.0;
        w.heavy = c->wh_heavy + c->h_wh_heavy_off[s];
        w.nheavy = (int32_t)(c->h_wh_heavy_off[s + 1] - c->h_wh_heavy_off[s]);
        if ((e = launch_wh_start(w, d.q, d.vpre, st))) return e;
        c->launches += 4;
        int32_t done = 0;
        const int64_t chunks = p.max_hermite_steps / 32 + 2;
        for (int64_t k = 0; k < chunks && !done; ++k) {
            if ((e = launch_wh_blocks(w, 32, st))) return e;
            if ((e = cudaMemcpyAsync(&done, w.ctl + WC_DONE, sizeof(done), cudaMemcpyDeviceToHost, st)))
                return e;
            if ((e = cudaStreamSynchronize(st))) return e;
            c->launches += 4 * 32;
        }
        long long steps = 0;
        if ((e = cudaMemcpyAsync(&steps, w.steps, sizeof(steps), cudaMemcpyDeviceToHost, st))) return e;
        if ((e = launch_wh_store(w, d.q1, d.v1, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        c->launches += 1;
        c->wh_steps += 1;
        c->wh_hsteps += steps;
        c->wh_hmax = std::max<int64_t>(c->wh_hmax, steps);
    }
    return cudaSuccess;
}

static cudaError_t enqueue_step(qym_ctx *c, double tau, bool last, bool fresh = false) {
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    const int enc = p.encounters;
    cudaError_t e;
    if (c->flush) {
        if ((e = cudaMemsetAsync(c->flush, c->launches & 0xff, (size_t)p.l2_flush_bytes, st))) return e;
    }
    k_step_begin<<<1, 256, 0, st>>>(d.ctr, d.vmax, d.nsys, c->sarg.tbox_bits, c->binned ? 6 * (int64_t)c->nstiles : 0);
    const int fz = fused_search(c);
    // the velocities entering the first kick, for a whole-system Hermite
    if (p.whole_hermite &&
        (e = cudaMemcpyAsync(d.vpre, d.v, sizeof(double) * 3 * d.rows, cudaMemcpyDeviceToDevice, st)))
        return e;
    // item 2: kick tau/2, with the crude encounter search when it is fused
    if (fz && fresh) {
        if ((e = enqueue_fresh_search_kick(c, 0.5 * tau))) return e;
        c->launches -= 2 + search_retest(p, fz);  // counted below as kick and finish
    } else {
        if ((e = launch_kick_tiles(d, p.kick_prec, fz, p.G, c->tune.threads, c->tune.ipt, st)))
            return e;
        // the finisher records the step's Hill radii (and audits a fused search)
        if ((e = launch_kick_finish_v(d, d.v, d.q, 0.5 * tau, p.G, enc ? (fz ? 1 : 2) : 0,
                                      p.hill_fixed, st)))
            return e;
    }
    // item 3: Kepler drift over tau, (q, v) -> (q1, v1)
    if ((e = launch_kepler(step_kepler_args(c, tau), st))) return e;
    if (last && (e = enqueue_snapshot(c))) return e;
    if (enc) {
        // items 4-8: [binned search,] rigorous test, sets and r_crit, K corrections + Hermite
        if ((e = enqueue_binned_search(c, tau))) return e;
        if ((e = launch_refine(d, tau, p.a_E, st))) return e;
        if ((e = launch_sets_impl(d, p.a_H, c->ss, st))) return e;
        // (the sets of a system integrated whole are left out of the Hermite)
        if (p.whole_hermite && (e = enqueue_whole(c, tau))) return e;
        if ((e = launch_hermite(d, p, tau, st))) return e;
    }
    // (q1, v1) -> (q, v) and the float packs for the second kick
    if ((e = launch_drift_pack_from(d, d.q1, d.v1, 0.0, 0.0, tau, p.a_E, p.G, 0, p.hill_fixed, st,
                                    0.5 * tau)))
        return e;
    // item 9: kick tau/2 (not for a system integrated whole)
    if ((e = launch_kick_tiles(d, p.kick_prec, 0, p.G, c->tune.threads, c->tune.ipt, st))) return e;
    if ((e = launch_kick_finish_v(d, d.v, d.q, 0.5 * tau, p.G, 0, p.hill_fixed, st, 1.01,
                                  p.whole_hermite)))
        return e;
    // item 10 (and item 1 of the next step): drift tau/2 with S = sum m v
    if ((e = launch_momentum(d, st))) return e;
    if ((e = launch_drift_pack_from(d, d.q, d.v, 0.5 * tau, last ? 0.0 : 0.5 * tau, tau, p.a_E,
                                    p.G, (!last) && fz, p.hill_fixed, st, 0.5 * tau)))
        return e;
    k_step_end<<<1, 1, 0, st>>>(d.ctr, d.max_cand, d.max_enc);
    // begin, kick [+ chunk re-test], finish, Kepler, [refine 2, sets 7, Hermite plan, Hermite],
    // pack, kick, finish, momentum 2, drift, end
    c->launches += 12 + (enc ? 11 : 0) + search_retest(p, fz);
    return cudaGetLastError();
}

// ---- merged kicks (params.merge_kicks): the closing kick of a step and the
// opening kick of the next, at the same separations, become one kick of tau.
// The opening half kick of the first step (with the encounter search):
static cudaError_t enqueue_opening_kick(qym_ctx *c, double tau, bool fresh) {
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    cudaError_t e;
    k_step_begin<<<1, 256, 0, st>>>(d.ctr, d.vmax, d.nsys, c->sarg.tbox_bits, c->binned ? 6 * (int64_t)c->nstiles : 0);
    c->launches += 1;
    const int fz = fused_search(c);
    if (fz && fresh) return enqueue_fresh_search_kick(c, 0.5 * tau);
    if ((e = launch_kick_tiles(d, p.kick_prec, fz, p.G, c->tune.threads, c->tune.ipt, st)))
        return e;
    if ((e = launch_kick_finish_v(d, d.v, d.q, 0.5 * tau, p.G,
                                  p.encounters ? (fz ? 1 : 2) : 0, p.hill_fixed, st)))
        return e;
    c->launches += 2 + search_retest(p, fz);
    return cudaGetLastError();
}

// One step from its Kepler drift on: items 3-8, then either the merged kick of
// tau that closes this step and opens the next (momentum, drift tau, the next
// step's packs with its encounter search, kick, finish), or for the last step
// the closing half kick and half drift.
static cudaError_t enqueue_unit(qym_ctx *c, double tau, bool last) {
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    const int enc = p.encounters;
    cudaError_t e;
    if (c->flush) {
        if ((e = cudaMemsetAsync(c->flush, c->launches & 0xff, (size_t)p.l2_flush_bytes, st))) return e;
    }
    if ((e = launch_kepler(step_kepler_args(c, tau), st))) return e;
    if (last && (e = enqueue_snapshot(c))) return e;
    const int fz = fused_search(c);
    if (enc) {
        if ((e = enqueue_binned_search(c, tau))) return e;
        if ((e = launch_refine(d, tau, p.a_E, st))) return e;
        if ((e = launch_sets_impl(d, p.a_H, c->ss, st))) return e;
        if ((e = launch_hermite(d, p, tau, st))) return e;
    }
    k_step_end<<<1, 1, 0, st>>>(d.ctr, d.max_cand, d.max_enc);
    // (q1, v1) -> (q, v)
    if ((e = launch_drift_pack_from(d, d.q1, d.v1, 0.0, 0.0, tau, p.a_E, p.G, 0, p.hill_fixed, st,
                                    0.5 * tau)))
        return e;
    if (!last) {
        k_step_begin<<<1, 256, 0, st>>>(d.ctr, d.vmax, d.nsys, c->sarg.tbox_bits, c->binned ? 6 * (int64_t)c->nstiles : 0);
        if ((e = launch_momentum(d, st))) return e;
        // the last kick was a step earlier: its |a| bounds this one's only
        // loosely, so the crude reach allows twice it (and the finisher checks)
        if ((e = launch_drift_pack_from(d, d.q, d.v, 0.5 * tau, 0.5 * tau, tau, p.a_E, p.G, fz,
                                        p.hill_fixed, st, tau, 2.0)))
            return e;
        if ((e = launch_kick_tiles(d, p.kick_prec, fz, p.G, c->tune.threads, c->tune.ipt, st))) return e;
        if ((e = launch_kick_finish_v(d, d.v, d.q, tau, p.G, enc ? (fz ? 1 : 2) : 0, p.hill_fixed,
                                      st, 2.0)))
            return e;
        // Kepler, [refine 2, sets 7, Hermite plan, Hermite], end, copy, begin, momentum 2, drift, kick
        // [+ chunk re-test], finish
        c->launches += 9 + (enc ? 11 : 0) + search_retest(p, fz);
    } else {
        if ((e = launch_kick_tiles(d, p.kick_prec, 0, p.G, c->tune.threads, c->tune.ipt, st))) return e;
        if ((e = launch_kick_finish_v(d, d.v, d.q, 0.5 * tau, p.G, 0, p.hill_fixed, st))) return e;
        if ((e = launch_momentum(d, st))) return e;
        if ((e = launch_drift_pack_from(d, d.q, d.v, 0.5 * tau, 0.0, tau, p.a_E, p.G, 0,
                                        p.hill_fixed, st, 0.5 * tau)))
            return e;
        // Kepler, [refine 2, sets 7, Hermite plan, Hermite], end, copy, kick, finish, momentum 2, drift
        c->launches += 8 + (enc ? 11 : 0);
    }
    return cudaGetLastError();
}

static qym_status collect(qym_ctx *c, int64_t nsteps) {
    Dev &d = c->d;
    unsigned long long ctr[C_COUNT];
    int32_t status = 0;
    CK(c, cudaMemcpyAsync(ctr, d.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(&status, d.status, sizeof(status), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    qym_stats &s = c->stats;
    s.steps = nsteps ? nsteps : (int64_t)ctr[C_STEP];  // 0: a split run counts its own
    s.candidates = (int64_t)ctr[C_SUM_CAND];
    s.encounters = (int64_t)ctr[C_SUM_ENC];
    s.sets = (int64_t)ctr[C_SUM_SETS];
    s.max_set = (int64_t)ctr[C_MAX_SET];
    s.kepler_iters = (int64_t)ctr[C_SUM_KITER];
    s.hermite_steps = (int64_t)ctr[C_SUM_HSTEPS];
    s.rescans = (int64_t)ctr[C_SUM_RESCAN];
    s.status_bits = status;
    s.launches = c->launches;
    s.hermite_steps_max = (int64_t)ctr[C_MAX_HSET];
    s.kick_tile_i = c->tune.threads * c->tune.ipt;
    s.kick_tile_splits = c->tune.splits;
    s.whole_steps = (int32_t)c->wh_steps;
    s.hermite_steps += c->wh_hsteps;
    s.hermite_steps_max = std::max<int64_t>(s.hermite_steps_max, c->wh_hmax);
    c->status_bits = status;
    if (status & QYM_ST_NAN) FAIL(c, QYM_ENAN, "non-finite state after a Kepler drift");
    if (status & (QYM_ST_KEPLER_NOCONV | QYM_ST_HERMITE_CAP))
        FAIL(c, QYM_ENOCONV, status & QYM_ST_KEPLER_NOCONV ? "Kepler iteration cap reached"
                                                           : "Hermite step cap reached");
    if (status & (QYM_ST_CAND_OVERFLOW | QYM_ST_ENC_OVERFLOW | QYM_ST_SET_OVERFLOW | QYM_ST_UF_CAP))
        FAIL(c, QYM_EOVERFLOW, "encounter capacity exceeded (status bits " + std::to_string(status) + ")");
    return QYM_OK;
}

extern "C" qym_status qym_step(qym_ctx *c, double tau, int64_t nsteps) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_step: NULL context");
    if (!(tau != 0.0) || !std::isfinite(tau) || nsteps < 0)
        FAIL(c, QYM_EINVAL, "qym_step: tau must be finite and nonzero, nsteps >= 0");
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    CK(c, cudaSetDevice(p.device));
    if (nsteps == 0) {
        CK(c, cudaMemsetAsync(d.ctr, 0, sizeof(unsigned long long) * C_COUNT, st));
        CK(c, cudaMemsetAsync(d.status, 0, sizeof(int32_t), st));
        std::memset(&c->stats, 0, sizeof(c->stats));
        return QYM_OK;
    }
    if (p.guess == QYM_GUESS_MLP && !c->mlp_set)
        FAIL(c, QYM_EINVAL, "qym_step: QYM_GUESS_MLP needs a network (qym_set_mlp)");
    if (c->klog)
        CK(c, cudaMemcpyAsync(c->klog_base, &c->klog_steps, sizeof(c->klog_steps),
                              cudaMemcpyHostToDevice, st));
    c->launches = 0;
    c->wh_steps = c->wh_hsteps = c->wh_hmax = 0;
    // the kick's order from the positions at the start of the call (unless
    // set_state has just taken it)
    const bool sort = d.perm && !c->sort_current;
    c->sort_current = false;
    // without the |a| of an earlier kick the first search runs after its kick
    // (the escape-velocity reach needs none)
    const bool fresh = !c->amag_valid && !d.escape_reach;
    c->amag_valid = true;  // every kick's finisher records |a|
    // the call's counters, the order, and item 1 of the first step: drift tau/2
    auto opening = [&]() -> cudaError_t {
        cudaError_t e;
        if ((e = cudaMemsetAsync(d.ctr, 0, sizeof(unsigned long long) * C_COUNT, st))) return e;
        if ((e = cudaMemsetAsync(d.status, 0, sizeof(int32_t), st))) return e;
        if (sort) {
            if ((e = launch_sort_rows(d.rows, d.q, c->sortw, d.perm, d.inv, st))) return e;
            c->launches += 16;
        }
        if ((e = launch_momentum(d, st))) return e;
        if ((e = launch_drift_pack_from(d, d.q, d.v, 0.0, 0.5 * tau, tau, p.a_E, p.G,
                                        fused_search(c) && !fresh, p.hill_fixed, st, 0.5 * tau)))
            return e;
        c->launches += 3;
        return cudaSuccess;
    };
    CK(c, fresh ? opening() : replay(c, c->g_open[sort ? 1 : 0], tau, opening));
    int64_t rest = nsteps;  // steps (or merged units) still to enqueue
    if (p.merge_kicks) {
        CK(c, enqueue_opening_kick(c, tau, fresh));
    } else if (fresh) {
        CK(c, enqueue_step(c, tau, nsteps == 1, true));
        if (--rest == 0) {
            if (c->klog) c->klog_steps += (unsigned long long)nsteps;
            return collect(c, nsteps);
        }
    }
    const int64_t interior = rest - 1;
    auto one = [&]() -> cudaError_t {
        return p.merge_kicks ? enqueue_unit(c, tau, false) : enqueue_step(c, tau, false);
    };
    // (a whole-system Hermite reads the sets back mid-step: no graph; a lone
    // interior step is not worth a capture)
    const bool graphs = !p.whole_hermite;
    for (int64_t k = 0; k < interior; ++k) {
        if (d.perm && k > 0 && k % kSortEvery == 0) {
            // re-sort between steps and lay the packs of the coming kick out
            // again in the new order (the same values: no drift)
            CK(c, launch_sort_rows(d.rows, d.q, c->sortw, d.perm, d.inv, st));
            CK(c, launch_drift_pack_from(d, d.q, d.v, 0.0, 0.0, tau, p.a_E, p.G,
                                         fused_search(c), p.hill_fixed, st,
                                         p.merge_kicks ? tau : 0.5 * tau,
                                         p.merge_kicks ? 2.0 : 1.01));
            c->launches += 17;
        }
        if (graphs && (interior >= 2 || c->g_step.exec)) CK(c, replay(c, c->g_step, tau, one));
        else CK(c, one());
    }
    // the closing step (or unit) of the call
    auto last = [&]() -> cudaError_t {
        return p.merge_kicks ? enqueue_unit(c, tau, true) : enqueue_step(c, tau, true);
    };
    CK(c, graphs ? replay(c, c->g_last, tau, last) : last());
    if (c->klog) c->klog_steps += (unsigned long long)nsteps;
    return collect(c, nsteps);
}

// ------------------------------------------------------------------ state, energy
extern "C" qym_status qym_get_state(qym_ctx *c, double *q, double *v) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_get_state: NULL context");
    Dev &d = c->d;
    const int64_t R = d.rows;
    cudaStream_t st = c->stream;
    const unsigned g = (unsigned)((R + 255) / 256);
    // transposed into the (idle) partial-sum buffer, then one copy each
    double *aq = d.apart, *av = d.apart + 3 * R;
    if (q) {
        k_aos_from_soa<<<g, 256, 0, st>>>(R, d.q, aq);
        CK(c, cudaGetLastError());
        CK(c, cudaMemcpyAsync(q, aq, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, st));
    }
    if (v) {
        const double *src = d.v;
        if (c->p.coords == 0) {
            CK(c, launch_to_dh_impl(d, 1, d.v1, c->mt, st));
            src = d.v1;
        }
        k_aos_from_soa<<<g, 256, 0, st>>>(R, src, av);
        CK(c, cudaGetLastError());
        CK(c, cudaMemcpyAsync(v, av, sizeof(double) * 3 * R, cudaMemcpyDeviceToHost, st));
    }
    CK(c, cudaStreamSynchronize(st));
    return QYM_OK;
}

extern "C" qym_status qym_set_state(qym_ctx *c, const double *q, const double *v) {
    if (!c || !q || !v) FAIL(c, QYM_EINVAL, "qym_set_state: NULL argument");
    return upload_state(c, q, v);
}

extern "C" qym_status qym_get_order(qym_ctx *c, int32_t *order) {
    if (!c || !order) FAIL(c, QYM_EINVAL, "qym_get_order: NULL argument");
    Dev &d = c->d;
    if (d.perm) {
        CK(c, cudaMemcpyAsync(order, d.perm, sizeof(int32_t) * d.rows, cudaMemcpyDeviceToHost,
                              c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    } else {
        for (int64_t r = 0; r < d.rows; ++r) order[r] = (int32_t)r;
    }
    return QYM_OK;
}

extern "C" qym_status qym_energy(qym_ctx *c, double *E) {
    if (!c || !E) FAIL(c, QYM_EINVAL, "qym_energy: NULL argument");
    Dev &d = c->d;
    CK(c, launch_energy_items(c->neitems, c->eitems, c->eisys, c->eitem0, d.nsys, d.offsets, d.rows,
                              d.m, d.q, d.v, c->p.G, c->epart, c->E, c->stream));
    CK(c, cudaMemcpyAsync(E, c->E, sizeof(double) * d.nsys, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return QYM_OK;
}

extern "C" qym_status qym_get_params(const qym_ctx *c, qym_params *p) {
    if (!c || !p) FAIL(c, QYM_EINVAL, "qym_get_params: NULL argument");
    *p = c->p;
    return QYM_OK;
}

extern "C" qym_status qym_get_stats(qym_ctx *c, qym_stats *s) {
    if (!c || !s) FAIL(c, QYM_EINVAL, "qym_get_stats: NULL argument");
    *s = c->stats;
    return QYM_OK;
}

extern "C" qym_status qym_get_encounters(qym_ctx *c, int64_t *recs, int64_t cap, int64_t *count) {
    if (!c || !count || cap < 0 || (cap > 0 && !recs)) FAIL(c, QYM_EINVAL, "qym_get_encounters: bad argument");
    Dev &d = c->d;
    unsigned long long n = 0;
    CK(c, cudaMemcpyAsync(&n, d.ctr + C_LOG, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (n > (unsigned long long)d.max_log) n = d.max_log;
    std::vector<int64_t> h(3 * n);
    if (n) {
        CK(c, cudaMemcpyAsync(h.data(), d.log, sizeof(int64_t) * 3 * n, cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    std::vector<size_t> idx(n);
    for (size_t k = 0; k < n; ++k) idx[k] = k;
    std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
        for (int t = 0; t < 3; ++t)
            if (h[3 * a + t] != h[3 * b + t]) return h[3 * a + t] < h[3 * b + t];
        return false;
    });
    int64_t w = 0;
    for (size_t k = 0; k < n; ++k) {
        size_t a = idx[k];
        if (k > 0) {
            size_t b = idx[k - 1];
            if (h[3 * a] == h[3 * b] && h[3 * a + 1] == h[3 * b + 1] && h[3 * a + 2] == h[3 * b + 2])
                continue;  // a pair found by both the candidate list and a re-search
        }
        if (w < cap)
            for (int t = 0; t < 3; ++t) recs[3 * w + t] = h[3 * a + t];
        ++w;
    }
    *count = w;
    return QYM_OK;
}

extern "C" qym_status qym_set_mlp(qym_ctx *c, const float *weights, int64_t n) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_set_mlp: NULL context");
    if (!weights || n != QYM_MLP_NW)
        FAIL(c, QYM_EINVAL, "qym_set_mlp: expected " + std::to_string(QYM_MLP_NW) + " weights");
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(weights[i])) FAIL(c, QYM_EINVAL, "qym_set_mlp: non-finite weight");
    for (int i = 0; i < 4; ++i)
        if (!(weights[QYM_MLP_NW - 6 + i] > 0.0f)) FAIL(c, QYM_EINVAL, "qym_set_mlp: feature std must be > 0");
    CK(c, cudaSetDevice(c->p.device));
    CK(c, cudaMemcpyAsync(c->mlp_w, weights, sizeof(float) * QYM_MLP_NW, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    c->mlp_set = true;
    return QYM_OK;
}

extern "C" qym_status qym_set_kepler_log(qym_ctx *c, float *rows, int64_t cap) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_set_kepler_log: NULL context");
    if (cap < 0 || (cap > 0 && !rows)) FAIL(c, QYM_EINVAL, "qym_set_kepler_log: bad buffer");
    c->klog = cap > 0 ? rows : nullptr;
    c->klog_cap = cap;
    c->klog_steps = 0;
    drop_graphs(c);  // the step graphs hold the log pointers: capture again
    return QYM_OK;
}

static qym_status apply_tune(qym_ctx *c, const KickTune &t);

// ------------------------------------------------------------------ split step
// One system's step over several GPUs: every GPU holds the whole state, and
// computes the kick of its own contiguous block of rows against all rows
// (with the crude search of those rows), their kick finish and Kepler drift,
// the rigorous test of their candidates and the Hermite of the encounter sets
// whose lowest row is its own; the caller exchanges the results between the
// phases (qym_split_phase). Everything else (momentum, drifts, packs, the
// encounter sets) is computed on every GPU from identical data in a fixed
// order, so it agrees to the bit without a collective.

__global__ void k_owned_members(Dev d, int64_t *info) {
    // first member (in set_mem) and member count of the sets rooted in
    // [own_lo, own_hi); sets are numbered by their lowest row
    const int nall = (int)min((unsigned long long)d.max_sets, d.ctr[C_NSETS]);
    int a = 0, b = nall;
    while (a < b) { const int m = (a + b) >> 1; if (d.set_root[m] < d.own_lo) a = m + 1; else b = m; }
    const int lo = a;
    b = nall;
    while (a < b) { const int m = (a + b) >> 1; if (d.set_root[m] < d.own_hi) a = m + 1; else b = m; }
    const int hi = a;
    info[0] = lo < nall ? d.set_start[lo] : 0;
    info[1] = (lo < hi) ? (int64_t)d.set_start[hi] - d.set_start[lo] : 0;
}

// the gathered encounter pairs of every GPU become this step's list, and its
// records (step, i, j)
__global__ void k_import_encounters(Dev d, const int2 *pairs, int64_t n) {
    const int64_t cap = min(n, d.max_enc);
    const unsigned long long step = d.ctr[C_STEP];
    const unsigned long long l0 = d.ctr[C_LOG];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = pairs[k];
        if (k < cap) d.enc[k] = p;
        const unsigned long long l = l0 + (unsigned long long)k;
        if (l < (unsigned long long)d.max_log) {
            d.log[3 * l] = (int64_t)step;
            d.log[3 * l + 1] = p.x;
            d.log[3 * l + 2] = p.y;
        }
    }
}

__global__ void k_import_count(Dev d, int64_t n) {
    d.ctr[C_NENC] = (unsigned long long)n;
    if (n > d.max_enc) atomicOr(d.status, QYM_ST_ENC_OVERFLOW);
    const unsigned long long l = d.ctr[C_LOG] + (unsigned long long)n;
    if (l > (unsigned long long)d.max_log) atomicOr(d.status, QYM_ST_LOG_OVERFLOW);
    d.ctr[C_LOG] = l;
}

extern "C" qym_status qym_split_init(qym_ctx *c, int32_t rank, int32_t world) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_split_init: NULL context");
    if (c->d.nsys != 1) FAIL(c, QYM_EINVAL, "qym_split_init: one system per context");
    if (c->p.whole_hermite) FAIL(c, QYM_EINVAL, "qym_split_init: not with whole_hermite");
    if (world < 1 || rank < 0 || rank >= world) FAIL(c, QYM_EINVAL, "qym_split_init: bad rank or world");
    if (c->klog) FAIL(c, QYM_EINVAL, "qym_split_init: the Kepler solve log is not split");
    int64_t lo = 0, hi = 0;
    qym_split_rows(c->d.rows, rank, world, &lo, &hi);
    Dev &d = c->d;
    d.own_lo = lo;
    d.own_hi = hi;
    if (hi <= lo) d.own_hi = d.own_lo = d.rows;  // nothing of its own: past the last row
    d.log_refine = 0;
    d.perm = d.inv = nullptr;  // the split's kick items are in row order
    d.far = d.tile = nullptr;
    c->p.search = QYM_SEARCH_FUSED;  // the split's candidates come with each rank's kick
    d.escape_reach = 0;
    c->binned = false;
    c->split_rank = rank;
    c->split_world = world;
    c->amag_valid = false;
    qym_status st = apply_tune(c, c->tune);
    if (st != QYM_OK) return st;
    return QYM_OK;
}

extern "C" void qym_split_rows(int64_t rows, int32_t rank, int32_t world, int64_t *lo, int64_t *hi) {
    // the bodies (rows 1 .. rows-1) in contiguous blocks of equal size, the
    // last one shorter
    const int64_t nb = rows - 1;
    const int64_t blk = world > 0 ? (nb + world - 1) / world : nb;
    int64_t a = 1 + (int64_t)rank * blk, b = a + blk;
    if (a > rows) a = rows;
    if (b > rows) b = rows;
    if (lo) *lo = a;
    if (hi) *hi = b;
}

extern "C" qym_status qym_split_phase(qym_ctx *c, int32_t phase, double tau, int32_t last) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_split_phase: NULL context");
    if (!c->split_world) FAIL(c, QYM_EINVAL, "qym_split_phase: qym_split_init first");
    if (!(tau != 0.0) || !std::isfinite(tau)) FAIL(c, QYM_EINVAL, "qym_split_phase: bad tau");
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    const int enc = p.encounters;
    CK(c, cudaSetDevice(p.device));
    switch (phase) {
    case QYM_PHASE_OPEN: {
        if (p.guess == QYM_GUESS_MLP && !c->mlp_set)
            FAIL(c, QYM_EINVAL, "qym_split_phase: QYM_GUESS_MLP needs a network (qym_set_mlp)");
        CK(c, cudaMemsetAsync(d.ctr, 0, sizeof(unsigned long long) * C_COUNT, st));
        CK(c, cudaMemsetAsync(d.status, 0, sizeof(int32_t), st));
        c->split_fresh = !c->amag_valid;
        c->amag_valid = true;
        c->launches = 0;
        CK(c, launch_momentum(d, st));
        CK(c, launch_drift_pack_from(d, d.q, d.v, 0.0, 0.5 * tau, tau, p.a_E, p.G,
                                     enc && !c->split_fresh, p.hill_fixed, st, 0.5 * tau));
        c->launches += 3;
        break;
    }
    case QYM_PHASE_KICK1: {
        k_step_begin<<<1, 256, 0, st>>>(d.ctr, d.vmax, d.nsys, c->sarg.tbox_bits, c->binned ? 6 * (int64_t)c->nstiles : 0);
        const int flag = (enc && !c->split_fresh) ? KICK_SEARCH : KICK_FORCE;
        CK(c, launch_kick_tiles(d, p.kick_prec, flag, p.G, c->tune.threads, c->tune.ipt, st));
        CK(c, launch_kick_finish_v(d, d.v, d.q, 0.5 * tau, p.G, flag == KICK_SEARCH, p.hill_fixed, st));
        c->launches += 3 + search_retest(p, flag == KICK_SEARCH);
        break;
    }
    case QYM_PHASE_SEARCH: {
        // after a first kick without the search: the reaches from the kicked
        // state of every row, then the search of the own rows alone
        if (enc && c->split_fresh) {
            CK(c, launch_drift_pack_from(d, d.q, d.v, 0.0, 0.0, 0.5 * tau, p.a_E, p.G, 2,
                                         p.hill_fixed, st, 0.0));
            CK(c, launch_kick_tiles(d, p.kick_prec, KICK_SEARCH_ONLY, p.G, c->tune.threads,
                                    c->tune.ipt, st));
            c->launches += 2 + search_retest(p, 1);
        }
        c->split_fresh = false;
        break;
    }
    case QYM_PHASE_KEPLER: {
        KeplerArgs ka = step_kepler_args(c, tau);
        ka.n = d.own_hi - d.own_lo;
        ka.row0 = d.own_lo;
        ka.log = nullptr;
        CK(c, launch_kepler(ka, st));
        c->launches += 1;
        break;
    }
    case QYM_PHASE_REFINE: {
        if (enc) {
            CK(c, launch_refine(d, tau, p.a_E, st));
            c->launches += 2;
        }
        break;
    }
    case QYM_PHASE_HERMITE: {
        if (enc) {
            CK(c, launch_sets_impl(d, p.a_H, c->ss, st));
            CK(c, launch_hermite(d, p, tau, st));
            k_owned_members<<<1, 1, 0, st>>>(d, c->owned_info);
            CK(c, cudaGetLastError());
            c->launches += 12;
        }
        break;
    }
    case QYM_PHASE_KICK2: {
        CK(c, launch_drift_pack_from(d, d.q1, d.v1, 0.0, 0.0, tau, p.a_E, p.G, 0, p.hill_fixed, st,
                                     0.5 * tau));
        CK(c, launch_kick_tiles(d, p.kick_prec, KICK_FORCE, p.G, c->tune.threads, c->tune.ipt, st));
        CK(c, launch_kick_finish_v(d, d.v, d.q, 0.5 * tau, p.G, 0, p.hill_fixed, st));
        c->launches += 3;
        break;
    }
    case QYM_PHASE_CLOSE: {
        CK(c, launch_momentum(d, st));
        CK(c, launch_drift_pack_from(d, d.q, d.v, 0.5 * tau, last ? 0.0 : 0.5 * tau, tau, p.a_E,
                                     p.G, (!last) && enc, p.hill_fixed, st, 0.5 * tau));
        k_step_end<<<1, 1, 0, st>>>(d.ctr, d.max_cand, d.max_enc);
        CK(c, cudaGetLastError());
        c->launches += 4;
        if (last) return collect(c, (int64_t)0);
        break;
    }
    default:
        FAIL(c, QYM_EINVAL, "qym_split_phase: unknown phase");
    }
    CK(c, cudaGetLastError());
    return QYM_OK;
}

extern "C" qym_status qym_split_arrays(qym_ctx *c, qym_split_view *view) {
    if (!c || !view) FAIL(c, QYM_EINVAL, "qym_split_arrays: NULL argument");
    const Dev &d = c->d;
    view->rows = d.rows;
    view->own_lo = d.own_hi > 0 ? d.own_lo : 0;
    view->own_hi = d.own_hi > 0 ? d.own_hi : d.rows;
    view->q = d.q;
    view->v = d.v;
    view->q1 = d.q1;
    view->v1 = d.v1;
    view->rH = d.rH;
    view->amag = d.amag;
    view->hcost = d.hcost;
    view->enc = (int32_t *)d.enc;
    view->max_enc = d.max_enc;
    view->set_mem = d.set_mem;
    view->stream = (void *)c->stream;
    return QYM_OK;
}

extern "C" qym_status qym_split_encounter_count(qym_ctx *c, int64_t *n) {
    if (!c || !n) FAIL(c, QYM_EINVAL, "qym_split_encounter_count: NULL argument");
    unsigned long long k = 0;
    CK(c, cudaMemcpyAsync(&k, c->d.ctr + C_NENC, sizeof(k), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (k > (unsigned long long)c->d.max_enc) FAIL(c, QYM_EOVERFLOW, "encounter capacity exceeded");
    *n = (int64_t)k;
    return QYM_OK;
}

extern "C" qym_status qym_split_import_encounters(qym_ctx *c, const int32_t *pairs, int64_t n) {
    if (!c || n < 0 || (n > 0 && !pairs)) FAIL(c, QYM_EINVAL, "qym_split_import_encounters: bad argument");
    if (!c->split_world) FAIL(c, QYM_EINVAL, "qym_split_import_encounters: qym_split_init first");
    cudaStream_t st = c->stream;
    if (n > 0) {
        k_import_encounters<<<64, 256, 0, st>>>(c->d, (const int2 *)pairs, n);
        CK(c, cudaGetLastError());
    }
    k_import_count<<<1, 1, 0, st>>>(c->d, n);
    CK(c, cudaGetLastError());
    c->launches += 1 + (n > 0);
    return QYM_OK;
}

extern "C" qym_status qym_split_owned_members(qym_ctx *c, int64_t *first, int64_t *count) {
    if (!c || !first || !count) FAIL(c, QYM_EINVAL, "qym_split_owned_members: NULL argument");
    int64_t info[2] = {0, 0};
    if (c->p.encounters) {
        CK(c, cudaMemcpyAsync(info, c->owned_info, sizeof(info), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
    }
    *first = info[0];
    *count = info[1];
    return QYM_OK;
}

extern "C" qym_status qym_set_encounter_snapshot(qym_ctx *c, double *q0, double *v0, double *q1,
                                                 double *v1, double *rH) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_set_encounter_snapshot: NULL context");
    double *in[5] = {q0, v0, q1, v1, rH};
    int n = 0;
    for (int k = 0; k < 5; ++k) n += in[k] != nullptr;
    if (n != 0 && n != 5) FAIL(c, QYM_EINVAL, "qym_set_encounter_snapshot: all five arrays or none");
    for (int k = 0; k < 5; ++k) c->snap[k] = in[k];
    drop_graphs(c);  // the closing step's graph holds the snapshot copies
    return QYM_OK;
}

extern "C" const char *qym_last_error(const qym_ctx *c) {
    return c ? c->err.c_str() : g_err.c_str();
}

// ------------------------------------------------------------------ device-level calls
extern "C" qym_status qym_kepler_drift_dev(int64_t n, const double *q0, const double *v0, double *q1,
                                           double *v1, double mu, double dt, int32_t solver,
                                           int32_t guess, const float *mlp_w, int32_t max_iter,
                                           double *x_out, double *x0_out, int32_t *iters,
                                           float *log_rows, int32_t *status, void *stream) {
    if (n < 0 || !(mu > 0.0) || max_iter < 1 || !std::isfinite(dt))
        FAIL(nullptr, QYM_EINVAL, "qym_kepler_drift_dev: bad n, mu, dt or max_iter");
    if (solver != QYM_SOLVER_LAGUERRE && solver != QYM_SOLVER_NEWTON && solver != QYM_SOLVER_NEWTON32)
        FAIL(nullptr, QYM_EINVAL, "qym_kepler_drift_dev: solver");
    if (guess < QYM_GUESS_STANDARD || guess > QYM_GUESS_MLP)
        FAIL(nullptr, QYM_EINVAL, "qym_kepler_drift_dev: guess");
    if (n == 0) return QYM_OK;
    if (!q0 || !v0 || !q1 || !v1) FAIL(nullptr, QYM_EINVAL, "qym_kepler_drift_dev: NULL array");
    if (guess == QYM_GUESS_MLP && !mlp_w) FAIL(nullptr, QYM_EINVAL, "qym_kepler_drift_dev: mlp_w required");
    if (mlp_w && ((uintptr_t)mlp_w & 15))
        FAIL(nullptr, QYM_EINVAL, "qym_kepler_drift_dev: mlp_w must be 16-byte aligned");
    KeplerArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = n;
    a.q0 = q0; a.v0 = v0; a.q1 = q1; a.v1 = v1;
    a.ld = n;
    a.mu = mu;
    a.sqmu = std::sqrt(mu);
    a.imu = 1.0 / mu;
    a.dt = dt;
    a.solver = solver;
    a.guess = guess;
    a.max_iter = max_iter;
    a.mlp_w = guess == QYM_GUESS_MLP ? mlp_w : nullptr;
    a.x_out = x_out;
    a.x0_out = x0_out;
    a.iters = iters;
    a.status = status;
    a.log = log_rows;
    a.log_cap = log_rows ? n : 0;
    CK(nullptr, launch_kepler(a, (cudaStream_t)stream));
    return QYM_OK;
}

extern "C" qym_status qym_transition_dev(int64_t n, const double *s, double r_crit, double *K,
                                         double *Kp, double *Kpp, void *stream) {
    if (n < 0 || !(r_crit > 0.0)) FAIL(nullptr, QYM_EINVAL, "qym_transition_dev: bad n or r_crit");
    if (n == 0) return QYM_OK;
    if (!s || !K || !Kp || !Kpp) FAIL(nullptr, QYM_EINVAL, "qym_transition_dev: NULL array");
    CK(nullptr, launch_transition(n, s, r_crit, K, Kp, Kpp, (cudaStream_t)stream));
    return QYM_OK;
}

// ------------------------------------------------------------------ learned guess
static bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

extern "C" size_t qym_mlp_workspace_bytes(void) { return mlp_workspace_bytes(); }

extern "C" qym_status qym_mlp_forward_dev(int64_t n, const float *w, const float *u, float *y,
                                          void *stream) {
    if (n < 0) FAIL(nullptr, QYM_EINVAL, "qym_mlp_forward_dev: n < 0");
    if (n == 0) return QYM_OK;
    if (!w || !u || !y || !aligned16(w) || !aligned16(u))
        FAIL(nullptr, QYM_EINVAL, "qym_mlp_forward_dev: NULL or unaligned array");
    CK(nullptr, launch_mlp_forward(n, w, u, y, (cudaStream_t)stream));
    return QYM_OK;
}

extern "C" qym_status qym_mlp_grad_dev(int64_t n, const float *w, const float *rows, float *grad,
                                       float *loss, void *work, size_t work_bytes, void *stream) {
    if (n < 1) FAIL(nullptr, QYM_EINVAL, "qym_mlp_grad_dev: n < 1");
    if (!w || !rows || !grad || !work || !aligned16(w))
        FAIL(nullptr, QYM_EINVAL, "qym_mlp_grad_dev: NULL or unaligned array");
    if (work_bytes < mlp_workspace_bytes()) FAIL(nullptr, QYM_EINVAL, "qym_mlp_grad_dev: workspace too small");
    CK(nullptr, launch_mlp_grad(n, w, rows, grad, loss, work, (cudaStream_t)stream));
    return QYM_OK;
}

extern "C" qym_status qym_mlp_adam_dev(float *w, float *m, float *v, const float *grad, int64_t t,
                                       float lr, float beta1, float beta2, float eps, void *stream) {
    if (!w || !m || !v || !grad) FAIL(nullptr, QYM_EINVAL, "qym_mlp_adam_dev: NULL array");
    if (t < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        FAIL(nullptr, QYM_EINVAL, "qym_mlp_adam_dev: bad t, lr, betas or eps");
    CK(nullptr, launch_mlp_adam(w, m, v, grad, t, lr, beta1, beta2, eps, (cudaStream_t)stream));
    return QYM_OK;
}

extern "C" qym_status qym_mlp_train_dev(float *w, float *m, float *v, int64_t t0, const float *rows,
                                        int64_t n, int64_t batch, int32_t epochs, float lr,
                                        float lr_final, float *losses, void *work, size_t work_bytes,
                                        void *stream) {
    if (!w || !m || !v || !rows || !work || !aligned16(w))
        FAIL(nullptr, QYM_EINVAL, "qym_mlp_train_dev: NULL or unaligned array");
    if (n < 1 || batch < 1 || epochs < 0 || t0 < 0 || !(lr >= 0.0f) || !(lr_final >= 0.0f))
        FAIL(nullptr, QYM_EINVAL, "qym_mlp_train_dev: bad n, batch, epochs, t0 or learning rate");
    if (work_bytes < mlp_workspace_bytes()) FAIL(nullptr, QYM_EINVAL, "qym_mlp_train_dev: workspace too small");
    CK(nullptr, launch_mlp_train(w, m, v, t0, rows, n, batch, epochs, lr, lr_final, losses, work,
                                 (cudaStream_t)stream));
    return QYM_OK;
}

extern "C" size_t qym_accel_workspace_bytes(int64_t rows, int32_t prec) {
    return accel_single_workspace(rows, prec);
}

extern "C" qym_status qym_accel_dev(int64_t rows, const double *m, const double *q, double *a,
                                    double G, int32_t prec, double heavy_mass, void *work,
                                    size_t work_bytes, void *stream) {
    if (rows < 2 || !m || !q || !a || !work) FAIL(nullptr, QYM_EINVAL, "qym_accel_dev: bad argument");
    if (prec != QYM_KICK_FP64 && prec != QYM_KICK_MIXED) FAIL(nullptr, QYM_EINVAL, "qym_accel_dev: prec");
    if (work_bytes < accel_single_workspace(rows, prec)) FAIL(nullptr, QYM_EINVAL, "qym_accel_dev: workspace too small");
    if (rows >= (int64_t)1 << 31) FAIL(nullptr, QYM_EINVAL, "qym_accel_dev: too many rows");
    CK(nullptr, launch_accel_single(rows, m, q, a, G, prec, heavy_mass, work, work_bytes,
                                    (cudaStream_t)stream));
    return QYM_OK;
}

extern "C" qym_status qym_encounter_test_dev(int64_t rows, const double *q0, const double *v0,
                                             const double *q1, const double *v1, const double *rH,
                                             double tau, double a_E, int64_t npairs,
                                             const int32_t *pairs, double *d2, int32_t *flag,
                                             void *stream) {
    if (rows < 1 || npairs < 0) FAIL(nullptr, QYM_EINVAL, "qym_encounter_test_dev: bad sizes");
    if (npairs == 0) return QYM_OK;
    if (!q0 || !v0 || !q1 || !v1 || !rH || !pairs) FAIL(nullptr, QYM_EINVAL, "qym_encounter_test_dev: NULL array");
    CK(nullptr, launch_pair_test(rows, q0, v0, q1, v1, rH, tau, a_E, npairs, pairs, d2, flag,
                                 (cudaStream_t)stream));
    return QYM_OK;
}

extern "C" size_t qym_energy_workspace_bytes(int64_t rows) {
    if (rows < 2) return 0;
    int64_t off[2] = {0, rows};
    int32_t n = energy_items_host(off, 1, nullptr, nullptr, nullptr);
    return al256(sizeof(int4) * n) + al256(sizeof(int32_t) * n) + al256(sizeof(int32_t) * 2) +
           al256(sizeof(double) * n) + al256(sizeof(int64_t) * 2);
}

extern "C" qym_status qym_energy_dev(int64_t rows, const double *m, const double *q, const double *v,
                                     double G, double *E, void *work, size_t work_bytes,
                                     void *stream) {
    if (rows < 2 || !m || !q || !v || !E || !work) FAIL(nullptr, QYM_EINVAL, "qym_energy_dev: bad argument");
    if (work_bytes < qym_energy_workspace_bytes(rows)) FAIL(nullptr, QYM_EINVAL, "qym_energy_dev: workspace too small");
    int64_t off[2] = {0, rows};
    int32_t n = energy_items_host(off, 1, nullptr, nullptr, nullptr);
    std::vector<int4> it(n);
    std::vector<int32_t> is(n), i0(2);
    energy_items_host(off, 1, it.data(), is.data(), i0.data());
    char *w = (char *)work;
    int4 *d_it = (int4 *)w; w += al256(sizeof(int4) * n);
    int32_t *d_is = (int32_t *)w; w += al256(sizeof(int32_t) * n);
    int32_t *d_i0 = (int32_t *)w; w += al256(sizeof(int32_t) * 2);
    double *d_part = (double *)w; w += al256(sizeof(double) * n);
    int64_t *d_off = (int64_t *)w;
    cudaStream_t st = (cudaStream_t)stream;
    // the tables are staged through pageable memory; the copies complete
    // before this call returns
    CK(nullptr, cudaMemcpyAsync(d_it, it.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, st));
    CK(nullptr, cudaMemcpyAsync(d_is, is.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    CK(nullptr, cudaMemcpyAsync(d_i0, i0.data(), sizeof(int32_t) * 2, cudaMemcpyHostToDevice, st));
    CK(nullptr, cudaMemcpyAsync(d_off, off, sizeof(int64_t) * 2, cudaMemcpyHostToDevice, st));
    CK(nullptr, launch_energy_items(n, d_it, d_is, d_i0, 1, d_off, rows, m, q, v, G, d_part, E, st));
    CK(nullptr, cudaStreamSynchronize(st));
    return QYM_OK;
}

extern "C" qym_status qym_get_stream(const qym_ctx *c, void **stream) {
    if (!c || !stream) FAIL(c, QYM_EINVAL, "qym_get_stream: NULL argument");
    *stream = (void *)c->stream;
    return QYM_OK;
}

static int64_t pairs_per_kick(const qym_ctx *c) {
    int64_t t = 0;
    for (int32_t s = 0; s < c->d.nsys; ++s) {
        int64_t nb = c->h_offsets[s + 1] - c->h_offsets[s] - 1;
        t += nb * (nb - 1);
    }
    return t;
}

// the kick kernel alone on the current state (packs rebuilt first; the
// candidate counter is reset after, the velocities are not touched)
// Mean time of `reps` launches of the kick (flag: with the fused search),
// or with `finish` of a step's pair of kicks (the flag's kick and a plain
// one), each with its finisher (which sums the partial slots; dt = 0 leaves
// the velocities as they are), per kick.
static qym_status time_kick_shape(qym_ctx *c, int flag, int reps, const KickTune &t, double *ms,
                                  bool finish = false) {
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    CK(c, launch_drift_pack_from(d, d.q, d.v, 0.0, 0.0, 0.1, p.a_E, p.G, flag, p.hill_fixed, st,
                                 0.05));
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    auto one = [&](int f) -> cudaError_t {
        cudaError_t e = launch_kick_tiles(d, p.kick_prec, f, p.G, t.threads, t.ipt, st);
        if (e == cudaSuccess && finish) e = launch_kick_finish_v(d, d.v, d.q, 0.0, p.G, 0, p.hill_fixed, st);
        return e;
    };
    CK(c, one(flag));  // warm
    CK(c, cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) {
        CK(c, one(flag));
        if (finish) CK(c, one(0));
    }
    CK(c, cudaEventRecord(e1, st));
    CK(c, cudaEventSynchronize(e1));
    float f = 0.f;
    CK(c, cudaEventElapsedTime(&f, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(c, cudaMemsetAsync(d.ctr + C_NCAND, 0, sizeof(unsigned long long), st));
    CK(c, cudaMemsetAsync(d.status, 0, sizeof(int32_t), st));
    CK(c, cudaStreamSynchronize(st));
    *ms = (double)f / (finish ? 2 * reps : reps);
    return QYM_OK;
}

extern "C" qym_status qym_time_drift(qym_ctx *c, double tau, int32_t reps, double *ms_momentum,
                                     double *ms_drift) {
    if (!c || reps < 1 || !ms_momentum || !ms_drift || !(tau != 0.0) || !std::isfinite(tau))
        FAIL(c, QYM_EINVAL, "qym_time_drift: bad argument");
    CK(c, cudaSetDevice(c->p.device));
    Dev &d = c->d;
    const qym_params &p = c->p;
    cudaStream_t st = c->stream;
    const size_t b3 = sizeof(double) * 3 * (size_t)d.rows;
    // the drift reads (q1, v1), copies of the state (idle between steps)
    CK(c, cudaMemcpyAsync(d.q1, d.q, b3, cudaMemcpyDeviceToDevice, st));
    CK(c, cudaMemcpyAsync(d.v1, d.v, b3, cudaMemcpyDeviceToDevice, st));
    cudaEvent_t e0, e1, e2;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    CK(c, cudaEventCreate(&e2));
    CK(c, launch_momentum(d, st));  // warm
    CK(c, cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) CK(c, launch_momentum(d, st));
    CK(c, cudaEventRecord(e1, st));
    for (int r = 0; r < reps; ++r)
        CK(c, launch_drift_pack_from(d, d.q1, d.v1, 0.5 * tau, 0.5 * tau, tau, p.a_E, p.G, 0,
                                     p.hill_fixed, st, 0.5 * tau));
    CK(c, cudaEventRecord(e2, st));
    CK(c, cudaEventSynchronize(e2));
    float f01 = 0.f, f12 = 0.f;
    CK(c, cudaEventElapsedTime(&f01, e0, e1));
    CK(c, cudaEventElapsedTime(&f12, e1, e2));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    // the state back (the next call packs the kick's operands again)
    CK(c, cudaMemcpyAsync(d.q, d.q1, b3, cudaMemcpyDeviceToDevice, st));
    CK(c, cudaMemcpyAsync(d.v, d.v1, b3, cudaMemcpyDeviceToDevice, st));
    CK(c, cudaStreamSynchronize(st));
    *ms_momentum = (double)f01 / reps;
    *ms_drift = (double)f12 / reps;
    return QYM_OK;
}

extern "C" qym_status qym_time_kick(qym_ctx *c, int32_t with_search, int32_t reps,
                                    double *ms_per_launch, int64_t *pairs) {
    if (!c || reps < 1 || !ms_per_launch) FAIL(c, QYM_EINVAL, "qym_time_kick: bad argument");
    CK(c, cudaSetDevice(c->p.device));
    double ms = 0.0;
    qym_status s = time_kick_shape(c, with_search ? 1 : 0, reps, c->tune, &ms);
    if (s != QYM_OK) return s;
    *ms_per_launch = ms;
    if (pairs) *pairs = pairs_per_kick(c);
    return QYM_OK;
}

// Where the kick's partial slots are added: by the finisher (k_finish), or,
// once the slots outgrow half of the 129 MB L2, by each i-block's last CTA
// inside the kick, which discards the dead slots from L2 so that they never
// reach HBM (kick.cu). With the slots in L2 the finisher's sum spreads over
// every SM and costs nothing in HBM; the in-kick sum puts an i-block's FP64
// adds on one SM (14 us for 64 slots of 256 rows), which a short kick (the
// 16384-body disk: 0.14 ms) would feel.
constexpr int64_t kSlotSumInKickBytes = 64ll << 20;
static void choose_slot_sums(qym_ctx *c) {
    Dev &d = c->d;
    d.kick_cnt = 24 * d.rows * (int64_t)d.splits > kSlotSumInKickBytes ? c->kick_cnt : nullptr;
}

// rebuild the work items for a launch shape (device buffers sized for the
// largest item count and split count seen so far are reused when they fit)
static qym_status apply_tune(qym_ctx *c, const KickTune &t) {
    Dev &d = c->d;
    const int64_t ilo = d.own_hi > 0 ? d.own_lo : 0, ihi = d.own_hi > 0 ? d.own_hi : INT64_MAX;
    int32_t n = kick_items_count(c->h_offsets.data(), d.nsys, t, ilo, ihi);
    if (n > c->items_cap || t.splits > c->splits_cap) FAIL(c, QYM_EINVAL, "launch shape exceeds the item buffers");
    std::vector<int4> items(n ? n : 1);
    std::vector<int32_t> slots(n ? n : 1);
    int32_t ni = 0, spu = 0;
    kick_items_host(c->h_offsets.data(), d.nsys, t, items.data(), slots.data(), &ni, &spu, n, ilo,
                    ihi, d.perm ? kKickTile / 2 : 1);
    if (n) {
        CK(c, cudaMemcpyAsync(d.items, items.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, c->stream));
        CK(c, cudaMemcpyAsync(d.item_slot, slots.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    d.nitems = n;
    d.splits = t.splits;
    choose_slot_sums(c);
    c->tune = t;
    drop_graphs(c);  // the captured steps hold the old shape
    return QYM_OK;
}

extern "C" qym_status qym_set_kick_shape(qym_ctx *c, int32_t threads, int32_t ipt, int32_t splits) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_set_kick_shape: NULL context");
    const bool mixed = c->p.kick_prec == QYM_KICK_MIXED;
    if ((threads != 128 && threads != 256) || !(ipt == 1 || ipt == 2 || (mixed && ipt == 4)) ||
        splits < 1 || splits > c->splits_cap)
        FAIL(c, QYM_EINVAL, "qym_set_kick_shape: threads 128 or 256, ipt 1, 2 (or 4 for the mixed "
                            "kick), splits 1 .. the context's cap");
    CK(c, cudaSetDevice(c->p.device));
    KickTune t;
    t.threads = threads;
    t.ipt = ipt;
    t.splits = splits;
    qym_status s = apply_tune(c, t);
    if (s != QYM_OK) return s;
    c->stats.kick_tile_i = threads * ipt;
    c->stats.kick_tile_splits = splits;
    return QYM_OK;
}

extern "C" qym_status qym_autotune(qym_ctx *c) {
    if (!c) FAIL(nullptr, QYM_EINVAL, "qym_autotune: NULL context");
    CK(c, cudaSetDevice(c->p.device));
    const int mixed = c->p.kick_prec == QYM_KICK_MIXED;
    std::vector<KickTune> cands;
    for (int threads : {128, 256})
        for (int ipt : mixed ? std::vector<int>{1, 2, 4} : std::vector<int>{1, 2})
            for (int sp : {1, 2, 4, 8, 16, 32, 64, 128}) {
                KickTune t;
                t.threads = threads;
                t.ipt = ipt;
                t.splits = sp;
                if (sp > c->splits_cap) continue;
                if (kick_items_count(c->h_offsets.data(), c->d.nsys, t) > c->items_cap) continue;
                cands.push_back(t);
            }
    KickTune best = c->tune;
    double best_ms = 1e30;
    for (const KickTune &t : cands) {
        qym_status s = apply_tune(c, t);
        if (s != QYM_OK) return s;
        double ms = 0.0;
        // a step's two kicks with their finishers: more j-splits shorten a
        // kick's tail but give the finisher more partial slots to add
        s = time_kick_shape(c, fused_search(c), 3, t, &ms, true);
        if (s != QYM_OK) return s;
        if (ms < best_ms) { best_ms = ms; best = t; }
    }
    qym_status s = apply_tune(c, best);
    if (s != QYM_OK) return s;
    c->stats.kick_tile_i = best.threads * best.ipt;
    c->stats.kick_tile_splits = best.splits;
    c->amag_valid = false;
    return QYM_OK;
}
