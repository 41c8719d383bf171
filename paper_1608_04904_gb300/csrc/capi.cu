// capi.cu -- host side of the C ABI declared in include/rmpcd.h.
//
// Owns the device buffers of a system, validates parameters, precomputes the
// per-replica constants, and sequences the kernels of one collision interval
// (§1.1, §1.4 of the RMPCDMD paper, arXiv:1608.04904):
//   granular: stream -> shift_and_sort -> collide -> react
//   fused   : [prime] { md ; cellpass(collide, react, next flight + bin) }*
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rmpcd.h"
#include "rmpcd_kernels.cuh"

using namespace rmpcd;

struct rmpcd_system {
    bool mixed = false;
    int n_rep = 0;
    int cap = 64;
    cudaStream_t stream = nullptr;
    std::vector<rmpcd_params> params;
    std::vector<ReplicaDev> rep;
    std::vector<rmpcd_colloid> colloids;
    int n_total = 0, n_tiles = 0, n_col = 0, n_bond = 0, max_part = 0;
    int any_colloids = 0;
    Dev d{};
    // device allocations
    std::vector<void *> allocs;
    double *stage_x = nullptr, *stage_v = nullptr;
    uint8_t *stage_f = nullptr;
    uint32_t *stage_id = nullptr;
    int32_t *stage_cell = nullptr;
    // staging area of every replica's particles for the batch state calls
    // (allocated on the first host call when the system has several replicas)
    double *sa_x = nullptr, *sa_v = nullptr;
    uint8_t *sa_f = nullptr;
    uint32_t *sa_id = nullptr;
    int32_t *sa_cell = nullptr;
    cudaStream_t xfer = nullptr;   // copies of the batch state calls, beside the system's stream
    int cell_order = RMPCD_ORDER_LINEAR;
    int *cell_rank_dev = nullptr, *cell_key_dev = nullptr;   // Hilbert tables (built on first use)
    unsigned long long *prof_acc = nullptr;   // [PROF_MAX_BINS * PROF_FIELDS] slab-profile sums
    int *flat_fill = nullptr;                 // [n_rep] records placed by a flatten
    bool dry = false;          // sizing only (rmpcd_workspace_size): count bytes, allocate nothing
    size_t dry_bytes = 0;
    // pipeline state
    uint32_t step = 0;
    int cur = 0;        // record buffer holding the state
    int bcur = 0;       // count/bucket buffer of the next collision (fused)
    bool primed = false;       // bins for the collision of `step` exist
    bool in_rows = false;      // the state lives in record rows + near area (fused run), not in rec[cur]
    int md_sub_next = 0;       // next sub-step of an interval run by rmpcd_md_substep (0: none open)
    bool has_sort = false;
    uint32_t sort_step = 0;
    bool obs_valid = false;
    long long launches = 0;
    std::string err;
    // per-phase timers
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int phase; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    long long t_launches[4] = {0, 0, 0, 0};
    double t_ms[4] = {0, 0, 0, 0};
    // MD kernel: 1 = general, 2 = few-colloid (when every replica allows it)
    int md_kernel = 1;
    bool fast_ok = false;
    int md_kernel_req = 0;
    // MD cluster size: fixed (1, 2, 4, 8) or tuned on the first intervals
    int md_fixed = 0;
    bool md_tuned = false;
    int md_best = 4;
    int md_fast_max = 8;              // largest cluster the device runs for the few-colloid kernel
    std::vector<int> md_cand;         // cluster sizes the tuner tries
    int md_wide_grid = 0;             // co-resident CTAs of the wide MD kernel (0: unavailable)
    std::vector<int> wide_reps;       // replicas with colloids (wide kernel: one launch each)
    std::vector<Pending> md_trials;   // phase field holds the cluster size
    // CUDA graphs of one fused interval, one per (record, bucket) buffer
    // parity; built once the MD launch geometry is settled
    bool graphs_on = true;
    // bucket width: fixed, or picked from the densities and grown on the
    // largest cell count seen (bucket_cap = 0 at creation)
    bool cap_auto = false;
    unsigned int *maxcnt_host = nullptr;   // pinned: largest cell count of the last fused run
    cudaEvent_t maxcnt_ev = nullptr;
    bool maxcnt_pending = false;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int graph_nodes = 0;              // kernel launches per replay
    // rigid bead bodies: per replica host copy (n_beads = 0: none), the
    // device arrays (rebuilt when a body is set) and the colloid slot that
    // stands for each body in the near-list test
    struct BodyHost {
        rmpcd_body b{};
        std::vector<rmpcd_bead> beads;
        BodyDev dev{};
        std::vector<int> gstart;
        std::vector<unsigned short> glist;
    };
    std::vector<BodyHost> bodies;
    bool any_body = false;
    int nb_max = 0;
    int grid_room = 0;                // shared-memory room for the lookup grids (0: global)
    std::vector<void *> body_allocs;  // bead and grid arrays
    // bead networks (iterative RATTLE): per replica host copy (beads empty:
    // none), links grouped by colour, and the device arrays of all networks
    struct NetHost {
        std::vector<rmpcd_net_bead> beads;
        std::vector<int> la, lb, cs;
        std::vector<double> dl;
        NetDev dev{};
    };
    std::vector<NetHost> nets;
    bool any_net = false;
    size_t net_smem = 0;
    std::vector<void *> net_allocs;
    double *col_rc = nullptr;         // writable colloid constants (body slots)
    float *col_rb = nullptr;
    size_t work_bytes = 0;            // md_work size
};

static void drop_graphs(rmpcd_system *sys);

static cudaEvent_t pool_event(rmpcd_system *sys)
{
    if (!sys->ev_pool.empty()) {
        cudaEvent_t e = sys->ev_pool.back();
        sys->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Record the start event of a timed phase (no-op when timers are off).
static void tstart(rmpcd_system *sys, cudaEvent_t *a)
{
    *a = nullptr;
    if (!sys->timing) return;
    *a = pool_event(sys);
    cudaEventRecord(*a, sys->stream);
}

static void tstop(rmpcd_system *sys, int phase, cudaEvent_t a)
{
    if (!sys->timing || !a) return;
    cudaEvent_t b = pool_event(sys);
    cudaEventRecord(b, sys->stream);
    sys->pending.push_back({phase, a, b});
}

static std::string g_create_error;

namespace rmpcd {
// Message of a failure of a call that has no system (rmpcd_last_error(NULL)).
void note_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace rmpcd

// MD kernel choice (0 = the few-colloid kernel when allowed) and the cluster
// sizes the tuner tries for it.
// The wide kernel by default: mixed path, a few replicas (one cooperative
// launch each) with more colloids than the few-colloid kernel takes.
static bool wide_default(const rmpcd_system *sys)
{
    return sys->mixed && sys->md_wide_grid > 0 && !sys->fast_ok && sys->wide_reps.size() <= 4;
}

static void set_md_kernel(rmpcd_system *sys, int req)
{
    sys->md_kernel_req = req;
    sys->md_kernel = req ? req : (sys->fast_ok ? 2 : (wide_default(sys) ? 3 : 1));
    sys->md_cand.clear();
    if (sys->md_kernel == 3) {
        sys->md_cand = {1};   // one grid over all SMs: nothing to tune
        sys->md_best = 1;
        sys->md_tuned = true;
    } else if (sys->md_kernel == 2) {
        sys->md_cand = {2, 4, 8};
        if (sys->md_fast_max >= 16) sys->md_cand.push_back(16);
        sys->md_best = 8;
    } else {
        sys->md_cand = {1, 2, 4, 8};
        sys->md_best = 4;
    }
}

// Mixed-path colloid representation: unwrapped integer cell, FP32 offset in
// [0,1), wrapped integer cell, FP32 velocity.
static void split_colloid(const rmpcd_colloid &c, const rmpcd_params &p, int Xi[3], float Xf[3], int Ci[3], float Vf[3])
{
    for (int k = 0; k < 3; ++k) {
        double fl = floor(c.x[k]);
        Xi[k] = (int)fl;
        Xf[k] = (float)(c.x[k] - fl);
        if (Xf[k] >= 1.0f) { Xf[k] = 0.0f; Xi[k] += 1; }
        int m = Xi[k] % p.L[k];
        Ci[k] = m < 0 ? m + p.L[k] : m;
        Vf[k] = (float)c.v[k];
    }
}

static rmpcd_status fail(rmpcd_system *s, rmpcd_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf; else g_create_error = buf;
    return st;
}

static rmpcd_status cuda_check(rmpcd_system *s, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return RMPCD_OK;
    return fail(s, e == cudaErrorMemoryAllocation ? RMPCD_ENOMEM : RMPCD_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(expr)                                                       \
    do {                                                               \
        rmpcd_status _st = cuda_check(sys, (expr), #expr);             \
        if (_st != RMPCD_OK) return _st;                               \
    } while (0)

static rmpcd_status after_launch(rmpcd_system *sys, int n)
{
    sys->launches += n;
    return cuda_check(sys, cudaGetLastError(), "kernel launch");
}

template <typename T>
static rmpcd_status dalloc(rmpcd_system *sys, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    if (sys->dry) {
        sys->dry_bytes += (count * sizeof(T) + 255) / 256 * 256;
        return RMPCD_OK;
    }
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) return cuda_check(sys, e, "cudaMalloc");
    sys->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return RMPCD_OK;
}

static void fill_rep(ReplicaDev &rp, const rmpcd_params &p)
{
    std::memset(&rp, 0, sizeof rp);
    for (int k = 0; k < 3; ++k) rp.L[k] = p.L[k];
    rp.walls = p.walls ? 1 : 0;
    rp.nz = p.L[2] + rp.walls;
    rp.rho_wall = p.rho_wall;
    rp.n_md = p.n_md;
    rp.n_slabs = p.n_slabs;
    rp.n_part = p.n_solvent;
    rp.n_cells = p.L[0] * p.L[1] * rp.nz;
    rp.n_tiles = (rp.n_cells + CPT - 1) / CPT;
    rp.n_col = p.n_colloids;
    rp.n_bond = p.n_bonds;
    rp.body = -1;
    rp.net = -1;
    rp.bulk_on = p.bulk_rate > 0.0 ? 1 : 0;
    rp.has_g = (p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0) ? 1 : 0;
    rp.kT = p.kT;
    rp.tau = p.tau;
    rp.dt = p.tau / (double)p.n_md;
    rp.hdt = 0.5 * rp.dt;
    rp.ca = cos(p.alpha);
    rp.sa = sin(p.alpha);
    rp.omc = 1.0 - rp.ca;
    for (int k = 0; k < 3; ++k) rp.g[k] = p.g[k];
    rp.gnorm = sqrt(p.g[0] * p.g[0] + p.g[1] * p.g[1] + p.g[2] * p.g[2]);
    rp.cat_thr = p.cat_prob * 4294967296.0;
    rp.skin = p.skin;
    for (int k = 0; k < 4; ++k) {
        rp.slab_x0[k] = p.slab_x0[k];
        rp.slab_x1[k] = p.slab_x1[k];
        // integer cx: x0 <= cx  <=>  ceil(x0) <= cx,   cx < x1  <=>  cx < ceil(x1)
        rp.slab_lo[k] = (int)std::max(-1e9, std::min(1e9, ceil(p.slab_x0[k])));
        rp.slab_hi[k] = (int)std::max(-1e9, std::min(1e9, ceil(p.slab_x1[k])));
        rp.slab_sd[k] = sqrt(p.slab_kT[k] > 0.0 ? p.slab_kT[k] : 0.0);
        rp.slab_sd_f[k] = (float)rp.slab_sd[k];
    }
    rp.cc_eps = p.cc_eps;
    rp.cc_sigma = p.cc_sigma;
    rp.cc_rc = p.cc_rc;
    for (int k = 0; k < 4; ++k) rp.res_y[k] = p.res_y[k];
    rp.tau_f = (float)rp.tau;
    rp.dt_f = (float)rp.dt;
    rp.hdt_f = (float)rp.hdt;
    rp.ca_f = (float)rp.ca;
    rp.sa_f = (float)rp.sa;
    rp.omc_f = (float)rp.omc;
    for (int k = 0; k < 3; ++k) rp.g_f[k] = (float)p.g[k];
    rp.gnorm_f = (float)rp.gnorm;
    rp.skin_f = (float)rp.skin;
    rp.seed = (unsigned long long)p.seed;
}

static rmpcd_status validate(const rmpcd_params &p, int r, const rmpcd_colloid *cols, const rmpcd_bond *bonds)
{
    for (int k = 0; k < 3; ++k)
        if (p.L[k] < 2 || p.L[k] > 1023) return fail(nullptr, RMPCD_EINVAL, "replica %d: L[%d]=%d not in [2,1023]", r, k, p.L[k]);
    if (p.n_md < 1) return fail(nullptr, RMPCD_EINVAL, "replica %d: n_md must be >= 1", r);
    if (!(p.tau > 0.0) || !std::isfinite(p.tau)) return fail(nullptr, RMPCD_EINVAL, "replica %d: tau must be > 0", r);
    if (!(p.kT >= 0.0)) return fail(nullptr, RMPCD_EINVAL, "replica %d: kT must be >= 0", r);
    if (!std::isfinite(p.alpha)) return fail(nullptr, RMPCD_EINVAL, "replica %d: alpha not finite", r);
    if (p.n_solvent < 0 || p.n_solvent > (int)ID_MASK) return fail(nullptr, RMPCD_EINVAL, "replica %d: n_solvent out of range", r);
    if (p.n_colloids < 0 || p.n_colloids > MAXC)
        return fail(nullptr, RMPCD_EINVAL, "replica %d: n_colloids %d not in [0,%d]", r, p.n_colloids, MAXC);
    if (p.n_bonds < 0 || p.n_bonds > MAXB) return fail(nullptr, RMPCD_EINVAL, "replica %d: n_bonds not in [0,%d]", r, MAXB);
    if (p.n_slabs < 0 || p.n_slabs > 4) return fail(nullptr, RMPCD_EINVAL, "replica %d: n_slabs not in [0,4]", r);
    if (p.walls && p.g[2] != 0.0) return fail(nullptr, RMPCD_EINVAL, "replica %d: walls need g[2] = 0", r);
    if (p.walls && p.n_colloids > 0) return fail(nullptr, RMPCD_EINVAL, "replica %d: colloids with walls are not supported", r);
    if (p.walls && p.rho_wall < 0) return fail(nullptr, RMPCD_EINVAL, "replica %d: rho_wall < 0", r);
    if (!(p.cat_prob >= 0.0 && p.cat_prob <= 1.0)) return fail(nullptr, RMPCD_EINVAL, "replica %d: cat_prob not in [0,1]", r);
    if (!(p.skin >= 0.0)) return fail(nullptr, RMPCD_EINVAL, "replica %d: skin < 0", r);
    if (!(p.bulk_rate >= 0.0)) return fail(nullptr, RMPCD_EINVAL, "replica %d: bulk_rate < 0", r);
    for (int j = 0; j < p.n_colloids; ++j) {
        const rmpcd_colloid &c = cols[j];
        if (!(c.mass > 0.0) || !(c.sigma > 0.0)) return fail(nullptr, RMPCD_EINVAL, "replica %d colloid %d: mass and sigma must be > 0", r, j);
        if (2.0 * c.sigma * 1.1224620483093730 + 2.0 * p.skin >= (double)std::min(p.L[0], std::min(p.L[1], p.L[2])))
            return fail(nullptr, RMPCD_EINVAL, "replica %d colloid %d: box too small for the cut-off", r, j);
    }
    for (int k = 0; k < p.n_bonds; ++k) {
        const rmpcd_bond &b = bonds[k];
        if (b.a < 0 || b.b < 0 || b.a >= p.n_colloids || b.b >= p.n_colloids || b.a == b.b || !(b.d > 0.0))
            return fail(nullptr, RMPCD_EINVAL, "replica %d bond %d invalid", r, k);
    }
    for (int k = 0; k < 4; k += 2)
        if (p.res_y[k] < 0 || p.res_y[k] > p.res_y[k + 1] || p.res_y[k + 1] > p.L[1])
            return fail(nullptr, RMPCD_EINVAL, "replica %d: reservoir columns [%d, %d) not within [0, L[1]]", r,
                        p.res_y[k], p.res_y[k + 1]);
    return RMPCD_OK;
}

extern "C" {

const char *rmpcd_last_error(const rmpcd_system *sys)
{
    if (!sys) return g_create_error.c_str();
    return sys->err.c_str();
}

void rmpcd_destroy(rmpcd_system *sys)
{
    if (!sys) return;
    cudaStreamSynchronize(sys->stream);
    drop_graphs(sys);
    if (sys->maxcnt_host) cudaFreeHost(sys->maxcnt_host);
    if (sys->maxcnt_ev) cudaEventDestroy(sys->maxcnt_ev);
    for (void *p : sys->allocs) cudaFree(p);
    for (void *p : sys->body_allocs) cudaFree(p);
    for (void *p : sys->net_allocs) cudaFree(p);
    for (auto &q : sys->pending) { sys->ev_pool.push_back(q.a); sys->ev_pool.push_back(q.b); }
    for (auto &q : sys->md_trials) { sys->ev_pool.push_back(q.a); sys->ev_pool.push_back(q.b); }
    for (cudaEvent_t e : sys->ev_pool) cudaEventDestroy(e);
    if (sys->xfer) cudaStreamDestroy(sys->xfer);
    delete sys;
}

// Bucket width from the densities: 1.25 x the count above which a Poisson
// cell count at the densest replica's mean occurs with probability below
// 1e-4 over all cells of the system per collision (so that the largest
// counts stay below the 80 % growth threshold), as a multiple of 8, >= 16.
static int auto_cap(const rmpcd_params *p, int n_rep)
{
    long long cells = 0;
    double m = 0.0;
    for (int r = 0; r < n_rep; ++r) {
        const long long c = (long long)p[r].L[0] * p[r].L[1] * (p[r].L[2] + (p[r].walls ? 1 : 0));
        cells += c;
        if (c > 0) m = std::max(m, (double)p[r].n_solvent / (double)c);
    }
    if (m <= 0.0) return 16;
    // P(N > k) by summing the pmf upwards from the mean outwards (no underflow
    // for the densities of interest)
    int k = 0;
    double pmf = exp(-m), cdf = pmf;
    while (k < CP_MAX_CAP && (1.0 - cdf) * (double)cells >= 1e-4) {
        ++k;
        pmf *= m / (double)k;
        cdf += pmf;
    }
    int cap = std::max(16, (((k + 1) * 5 / 4 + 7) / 8) * 8);
    return std::min(cap, CP_MAX_CAP);
}

// Bytes of one buffer of cell rows at width cap: a record (fused run) or a
// slot number (flat layout) per place.
static size_t row_bytes(const rmpcd_system *sys, int cap)
{
    const size_t recsz = sys->mixed ? sizeof(RecM) : sizeof(RecD);
    return (size_t)sys->n_tiles * CPT * (size_t)cap * recsz;
}

static rmpcd_status flatten(rmpcd_system *sys);

// Re-allocate the rows for width `cap` (at a step boundary: a fused run's
// state is flattened first; pending bins are dropped and rebuilt by the next
// pass).
static rmpcd_status set_bucket_cap(rmpcd_system *sys, int cap)
{
    rmpcd_status st = flatten(sys);
    if (st != RMPCD_OK) return st;
    CK(cudaStreamSynchronize(sys->stream));
    drop_graphs(sys);
    const size_t ncells = (size_t)sys->n_tiles * CPT;
    for (int b = 0; b < 2; ++b) {
        auto it = std::find(sys->allocs.begin(), sys->allocs.end(), sys->d.brec[b]);
        if (it != sys->allocs.end()) sys->allocs.erase(it);
        cudaFree(sys->d.brec[b]);
        sys->d.brec[b] = nullptr;
        sys->d.bucket[b] = nullptr;
    }
    unsigned char *rows[2] = {nullptr, nullptr};
    st = dalloc(sys, &rows[0], row_bytes(sys, cap));
    if (st == RMPCD_OK) st = dalloc(sys, &rows[1], row_bytes(sys, cap));
    if (st != RMPCD_OK) return st;
    for (int b = 0; b < 2; ++b) {
        sys->d.brec[b] = rows[b];
        sys->d.bucket[b] = reinterpret_cast<int *>(rows[b]);
    }
    sys->cap = cap;
    sys->d.cap = cap;
    CK(cudaMemsetAsync(sys->d.count[0], 0, sizeof(int) * ncells, sys->stream));
    CK(cudaMemsetAsync(sys->d.count[1], 0, sizeof(int) * ncells, sys->stream));
    CK(cudaMemsetAsync(sys->d.ovf_n, 0, sizeof(unsigned int) * 2, sys->stream));
    CK(cudaMemsetAsync(sys->d.near_count, 0, sizeof(int) * sys->n_rep, sys->stream));
    sys->primed = false;
    return RMPCD_OK;
}

// The width that leaves headroom above a largest cell count m.
static int grown_cap(int m) { return std::min(CP_MAX_CAP, std::max(16, ((m * 3 / 2 + 7) / 8) * 8)); }

// Automatic width: the largest count of count buffer b, measured now
// (synchronises); true when the buckets had to grow (the bins are gone).
static rmpcd_status check_counts(rmpcd_system *sys, int b, bool *grew)
{
    *grew = false;
    CK(cudaMemsetAsync(sys->d.maxcnt, 0, sizeof(unsigned int), sys->stream));
    launch_count_max(sys->d, b, sys->stream);
    rmpcd_status st = after_launch(sys, 1);
    if (st != RMPCD_OK) return st;
    CK(cudaMemcpyAsync(sys->maxcnt_host, sys->d.maxcnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemsetAsync(sys->d.maxcnt, 0, sizeof(unsigned int), sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    const int m = (int)*sys->maxcnt_host;
    if (m * 5 > sys->cap * 4 && sys->cap < CP_MAX_CAP) {
        if ((st = set_bucket_cap(sys, grown_cap(m))) != RMPCD_OK) return st;
        // the binning just measured is discarded and redone: an overflow it
        // latched is not an error of the run
        CK(cudaMemsetAsync(sys->d.err + ERR_OVERFLOW, 0, sizeof(unsigned int), sys->stream));
        *grew = true;
    }
    return RMPCD_OK;
}

// rmpcd_create, or with dry != NULL only its validation and the sum of its
// device buffers (nothing allocated, no CUDA call).
static rmpcd_status create_system(rmpcd_system **out, int32_t precision, int32_t n_replicas,
                                  const rmpcd_params *params, const rmpcd_colloid *colloids, const rmpcd_bond *bonds,
                                  int32_t bucket_cap, void *stream, size_t *dry)
{
    if (!out) return fail(nullptr, RMPCD_EINVAL, "out is NULL");
    *out = nullptr;
    if (precision != RMPCD_FP64 && precision != RMPCD_MIXED) return fail(nullptr, RMPCD_EINVAL, "unknown precision %d", precision);
    if (n_replicas < 1 || !params) return fail(nullptr, RMPCD_EINVAL, "need n_replicas >= 1 and params");
    const int max_cap = CP_MAX_CAP;
    const bool cap_auto = bucket_cap == 0;
    if (cap_auto) bucket_cap = auto_cap(params, n_replicas);
    if (bucket_cap < 1 || bucket_cap > max_cap)
        return fail(nullptr, RMPCD_EINVAL, "bucket_cap %d not in [1,%d] (0 = automatic)", bucket_cap, max_cap);
    long long n_total = 0, n_tiles = 0, n_col = 0, n_bond = 0;
    for (int r = 0; r < n_replicas; ++r) {
        if ((params[r].n_colloids > 0 && !colloids) || (params[r].n_bonds > 0 && !bonds))
            return fail(nullptr, RMPCD_EINVAL, "replica %d: colloid or bond array missing", r);
        rmpcd_status st = validate(params[r], r, colloids ? colloids + n_col : nullptr, bonds ? bonds + n_bond : nullptr);
        if (st != RMPCD_OK) return st;
        n_total += params[r].n_solvent;
        const long long nz = params[r].L[2] + (params[r].walls ? 1 : 0);
        n_tiles += ((long long)params[r].L[0] * params[r].L[1] * nz + CPT - 1) / CPT;
        n_col += params[r].n_colloids;
        n_bond += params[r].n_bonds;
    }
    if (n_total > 0x7FFFFFF0ll) return fail(nullptr, RMPCD_EINVAL, "too many solvent particles");
    if (n_tiles * CPT * (long long)bucket_cap > 0x7FFFFFFFll) return fail(nullptr, RMPCD_EINVAL, "cells x bucket_cap too large");

    rmpcd_system *sys = new rmpcd_system();
    sys->dry = dry != nullptr;
    sys->mixed = precision == RMPCD_MIXED;
    sys->n_rep = n_replicas;
    sys->cap = bucket_cap;
    sys->cap_auto = cap_auto;
    sys->stream = static_cast<cudaStream_t>(stream);
    sys->params.assign(params, params + n_replicas);
    sys->n_total = (int)n_total;
    sys->n_tiles = (int)n_tiles;
    sys->n_col = (int)n_col;
    sys->n_bond = (int)n_bond;
    if (n_col > 0) sys->colloids.assign(colloids, colloids + n_col);

    // per-replica constants and layout
    sys->rep.resize(n_replicas);
    std::vector<int> tile_rep((size_t)n_tiles);
    int part_off = 0, tile_off = 0, col_off = 0, bond_off = 0;
    for (int r = 0; r < n_replicas; ++r) {
        ReplicaDev &rp = sys->rep[r];
        fill_rep(rp, params[r]);
        rp.part_off = part_off;
        rp.tile_off = tile_off;
        rp.cell_off = tile_off * CPT;
        rp.col_off = col_off;
        rp.bond_off = bond_off;
        rp.thr_off = r * (CP_MAX_CELL + 1);   // sized for any cell count
        for (int t = 0; t < rp.n_tiles; ++t) tile_rep[tile_off + t] = r;
        part_off += rp.n_part;
        tile_off += rp.n_tiles;
        col_off += rp.n_col;
        bond_off += rp.n_bond;
        sys->max_part = std::max(sys->max_part, rp.n_part);
        if (rp.n_col > 0) sys->any_colloids = 1;
    }
    sys->fast_ok = true;
    for (int r = 0; r < n_replicas; ++r)
        if (params[r].n_colloids > MD_FAST_NC || params[r].cc_rc > 0.0 || params[r].n_bonds > 1)
            sys->fast_ok = false;
    // bulk reaction thresholds: accept iff draw < (1 - exp(-k N_B tau)) 2^32;
    // for an integer draw that is draw < ceil((1 - exp(-k N_B tau)) 2^32)
    std::vector<unsigned long long> thr((size_t)n_replicas * (CP_MAX_CELL + 1));
    for (int r = 0; r < n_replicas; ++r)
        for (int nb = 0; nb <= CP_MAX_CELL; ++nb)
            thr[(size_t)r * (CP_MAX_CELL + 1) + nb] = (unsigned long long)ceil(
                (1.0 - exp(-params[r].bulk_rate * (double)nb * params[r].tau)) * 4294967296.0);
    // colloid constants
    std::vector<double> cM(n_col), cS(n_col), cEA(n_col), cEB(n_col), cR2(n_col), cR(n_col), cX(3 * n_col), cV(3 * n_col);
    std::vector<float> fS(n_col), fEA(n_col), fEB(n_col), fR2(n_col), fR(n_col);
    std::vector<int> cCat(n_col), cXi(3 * n_col), cCi(3 * n_col);
    std::vector<float> cXf(3 * n_col), cVf(3 * n_col), cRb(n_col), cIM(n_col);
    std::vector<int> col_rep(n_col);
    for (int r = 0, j = 0; r < n_replicas; ++r)
        for (int k = 0; k < params[r].n_colloids; ++k) col_rep[j++] = r;
    for (long long j = 0; j < n_col; ++j) {
        const rmpcd_colloid &c = colloids[j];
        const rmpcd_params &pr = params[col_rep[j]];
        split_colloid(c, pr, &cXi[3 * j], &cXf[3 * j], &cCi[3 * j], &cVf[3 * j]);
        const double gn = sqrt(pr.g[0] * pr.g[0] + pr.g[1] * pr.g[1] + pr.g[2] * pr.g[2]);
        cRb[j] = (float)(sqrt(c.sigma * c.sigma * cbrt(2.0)) + 0.5 * gn * pr.tau * pr.tau + pr.skin);
        cIM[j] = (float)(1.0 / c.mass);
        cM[j] = c.mass; cS[j] = c.sigma; cEA[j] = c.eps_A; cEB[j] = c.eps_B;
        cR2[j] = c.sigma * c.sigma * cbrt(2.0);
        cR[j] = sqrt(cR2[j]);
        fS[j] = (float)c.sigma; fEA[j] = (float)c.eps_A; fEB[j] = (float)c.eps_B;
        fR2[j] = (float)cR2[j]; fR[j] = (float)cR[j];
        cCat[j] = c.catalytic ? 1 : 0;
        for (int k = 0; k < 3; ++k) { cX[3 * j + k] = c.x[k]; cV[3 * j + k] = c.v[k]; }
    }
    std::vector<BondDev> bd(n_bond);
    for (long long k = 0; k < n_bond; ++k) bd[k] = BondDev{bonds[k].a, bonds[k].b, bonds[k].d};

    rmpcd_status st = RMPCD_OK;
    Dev &d = sys->d;
    const size_t recsz = sys->mixed ? sizeof(RecM) : sizeof(RecD);
    const long long ncells = (long long)n_tiles * CPT;
    ReplicaDev *drep = nullptr;
    int *dtile = nullptr;
    unsigned long long *dthr = nullptr;
    double *dM, *dS, *dEA, *dEB, *dR2, *dR;
    float *dfS, *dfEA, *dfEB, *dfR2, *dfR;
    int *dCat;
    float *dRb, *dIM;
    BondDev *dB;
    unsigned char *r0, *r1, *work;
#define AL(p, n) if (st == RMPCD_OK) st = dalloc(sys, p, (size_t)(n))
    AL(&drep, n_replicas);
    AL(&dtile, n_tiles);
    AL(&r0, recsz * n_total);
    AL(&r1, recsz * n_total);
    AL(&d.count[0], ncells);
    AL(&d.count[1], ncells);
    // cell rows: a fused run's records, or the flat layout's slot numbers
    // (same memory; one layout in use at a time)
    unsigned char *rows0 = nullptr, *rows1 = nullptr;
    AL(&rows0, (size_t)ncells * bucket_cap * recsz);
    AL(&rows1, (size_t)ncells * bucket_cap * recsz);
    // overflow lists: entries (and a fused run's records) of cells beyond
    // bucket_cap (rare at the automatic width; a fixed narrow width leans on
    // them)
    const long long ovf_cap = 1024 + n_total / 8;
    AL(&d.ovf[0], ovf_cap);
    AL(&d.ovf[1], ovf_cap);
    AL(&d.ovf_n, 2);
    unsigned char *orec0 = nullptr, *orec1 = nullptr, *nrec = nullptr;
    AL(&orec0, (size_t)ovf_cap * recsz);
    AL(&orec1, (size_t)ovf_cap * recsz);
    AL(&nrec, (size_t)recsz * n_total);   // the near area of a fused run
    AL(&sys->flat_fill, n_replicas);
    AL(&d.near_list, n_total);
    AL(&d.near_count, n_replicas);
    AL(&d.tile_state, n_tiles);
    AL(&d.ticket, 4);
    AL(&d.err, ERR_COUNT);
    AL(&d.obs_part, (size_t)n_tiles * 8);
    AL(&d.obs_out, (size_t)n_replicas * 8);
    AL(&dthr, thr.size());
    // colloid arrays hold one spare slot per replica (n_col + r) for a body
    const long long n_slot = n_col + n_replicas;
    AL(&d.colX, 3 * n_slot);
    AL(&d.colV, 3 * n_slot);
    AL(&dM, n_slot); AL(&dS, n_slot); AL(&dEA, n_slot); AL(&dEB, n_slot); AL(&dR2, n_slot); AL(&dR, n_slot);
    AL(&dfS, n_slot); AL(&dfEA, n_slot); AL(&dfEB, n_slot); AL(&dfR2, n_slot); AL(&dfR, n_slot);
    AL(&dCat, n_slot);
    AL(&d.colXi, 3 * n_slot);
    AL(&d.colCi, 3 * n_slot);
    AL(&d.colXf, 3 * n_slot);
    AL(&d.md_wide, 1);
    AL(&d.ctl, 1);
    AL(&d.maxcnt, 1);
    AL(&d.colVf, 3 * n_slot);
    AL(&dRb, n_slot);
    AL(&dIM, n_slot);
    AL(&dB, n_bond);
    AL(&d.body, n_replicas);
    AL(&d.net, n_replicas);
    sys->work_bytes = (sys->mixed ? 64 : 80) * (size_t)(sys->any_colloids ? n_total : 1);
    AL(&work, sys->work_bytes);
    unsigned char *colsave = nullptr;
    AL(&colsave, md_col_state_bytes(sys->mixed) * (size_t)n_replicas);
    AL(&sys->prof_acc, (size_t)PROF_MAX_BINS * PROF_FIELDS);
    AL(&sys->stage_x, 3 * (size_t)sys->max_part);
    AL(&sys->stage_v, 3 * (size_t)sys->max_part);
    AL(&sys->stage_f, (size_t)sys->max_part);
    AL(&sys->stage_id, (size_t)sys->max_part);
    AL(&sys->stage_cell, (size_t)sys->max_part);
#undef AL
    if (sys->dry) {
        *dry = sys->dry_bytes;
        delete sys;
        return RMPCD_OK;
    }
    if (st != RMPCD_OK) {
        g_create_error = sys->err;
        rmpcd_destroy(sys);
        return st;
    }
    cudaStream_t s = sys->stream;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (st == RMPCD_OK && bytes) st = cuda_check(sys, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s), "upload");
    };
    auto zero = [&](void *dst, size_t bytes) {
        if (st == RMPCD_OK && bytes) st = cuda_check(sys, cudaMemsetAsync(dst, 0, bytes, s), "memset");
    };
    up(drep, sys->rep.data(), sizeof(ReplicaDev) * n_replicas);
    up(dtile, tile_rep.data(), sizeof(int) * n_tiles);
    up(dthr, thr.data(), sizeof(unsigned long long) * thr.size());
    up(d.colX, cX.data(), sizeof(double) * cX.size());
    up(d.colV, cV.data(), sizeof(double) * cV.size());
    up(dM, cM.data(), sizeof(double) * n_col); up(dS, cS.data(), sizeof(double) * n_col);
    up(dEA, cEA.data(), sizeof(double) * n_col); up(dEB, cEB.data(), sizeof(double) * n_col);
    up(dR2, cR2.data(), sizeof(double) * n_col); up(dR, cR.data(), sizeof(double) * n_col);
    up(dfS, fS.data(), sizeof(float) * n_col); up(dfEA, fEA.data(), sizeof(float) * n_col);
    up(dfEB, fEB.data(), sizeof(float) * n_col); up(dfR2, fR2.data(), sizeof(float) * n_col);
    up(dfR, fR.data(), sizeof(float) * n_col);
    up(dCat, cCat.data(), sizeof(int) * n_col);
    up(d.colXi, cXi.data(), sizeof(int) * 3 * n_col);
    up(d.colCi, cCi.data(), sizeof(int) * 3 * n_col);
    up(d.colXf, cXf.data(), sizeof(float) * 3 * n_col);
    up(d.colVf, cVf.data(), sizeof(float) * 3 * n_col);
    up(dRb, cRb.data(), sizeof(float) * n_col);
    up(dIM, cIM.data(), sizeof(float) * n_col);
    up(dB, bd.data(), sizeof(BondDev) * n_bond);
    zero(r0, recsz * n_total);
    zero(r1, recsz * n_total);
    zero(d.count[0], sizeof(int) * ncells);
    zero(d.count[1], sizeof(int) * ncells);
    zero(d.ovf_n, sizeof(unsigned int) * 2);
    zero(d.near_count, sizeof(int) * n_replicas);
    zero(d.tile_state, sizeof(unsigned long long) * n_tiles);
    zero(d.ticket, sizeof(unsigned int) * 4);
    zero(d.err, sizeof(unsigned int) * ERR_COUNT);
    zero(d.obs_out, sizeof(double) * 8 * n_replicas);
    if (st == RMPCD_OK) zero(d.md_wide, sizeof(MdWideGlobal));
    if (st == RMPCD_OK) zero(d.ctl, sizeof(Ctl));
    if (st == RMPCD_OK) zero(d.maxcnt, sizeof(unsigned int));
    if (st == RMPCD_OK && cudaMallocHost(&sys->maxcnt_host, sizeof(unsigned int)) != cudaSuccess) st = RMPCD_ENOMEM;
    if (st == RMPCD_OK && cudaEventCreateWithFlags(&sys->maxcnt_ev, cudaEventDisableTiming) != cudaSuccess)
        st = RMPCD_ECUDA;
    if (st == RMPCD_OK) st = cuda_check(sys, cudaStreamSynchronize(s), "create sync");
    if (st != RMPCD_OK) {
        g_create_error = sys->err;
        rmpcd_destroy(sys);
        return st;
    }
    d.rep = drep;
    d.tile_rep = dtile;
    d.rec[0] = r0;
    d.rec[1] = r1;
    d.brec[0] = rows0;
    d.brec[1] = rows1;
    d.bucket[0] = reinterpret_cast<int *>(rows0);
    d.bucket[1] = reinterpret_cast<int *>(rows1);
    d.orec[0] = orec0;
    d.orec[1] = orec1;
    d.near_rec = nrec;
    d.bulk_thr = dthr;
    d.colM = dM; d.colSig = dS; d.colEpsA = dEA; d.colEpsB = dEB; d.colRc2 = dR2; d.colRc = dR;
    d.colSig_f = dfS; d.colEpsA_f = dfEA; d.colEpsB_f = dfEB; d.colRc2_f = dfR2; d.colRc_f = dfR;
    d.colCat = dCat;
    d.colRb_f = dRb;
    sys->col_rc = dR;
    sys->col_rb = dRb;
    sys->bodies.resize(n_replicas);
    sys->nets.resize(n_replicas);
    d.colInvM_f = dIM;
    d.bonds = dB;
    d.md_work = work;
    d.md_col_save = colsave;
    d.cap = bucket_cap;
    d.ovf_cap = (int)ovf_cap;
    d.lb_limit = LB_SPIN_LIMIT;
    d.lb_stall = 0;
    d.many_col = 0;
    for (int r = 0; r < n_replicas; ++r)
        if (params[r].n_colloids >= CP_NEAR_CAND_MIN) d.many_col = 1;
    d.n_rep = n_replicas;
    d.n_tiles = (int)n_tiles;
    d.n_total = (int)n_total;
    if (sys->fast_ok && sys->any_colloids) sys->md_fast_max = md_fast_max_cluster(sys->mixed);
    if (sys->mixed && sys->any_colloids) sys->md_wide_grid = md_wide_grid();
    for (int r = 0; r < n_replicas; ++r)
        if (params[r].n_colloids > 0) sys->wide_reps.push_back(r);
    set_md_kernel(sys, 0);
    *out = sys;
    return RMPCD_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// pipeline helpers
// ----------------------------------------------------------------------------
// Drop the captured interval graphs (the MD launch geometry changed).
static void drop_graphs(rmpcd_system *sys)
{
    for (auto &row : sys->graph)
        for (auto &g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

// Back to the flat layout: a fused run's state is flattened (sorted on the
// grid of its last collision); pending bins of a primed run are dropped.
static rmpcd_status unprime(rmpcd_system *sys)
{
    if (sys->md_sub_next != 0)
        return fail(sys, RMPCD_ESTATE, "an interval is being sub-stepped (rmpcd_md_substep): run its last sub-step first");
    if (sys->in_rows) return flatten(sys);
    if (!sys->primed) return RMPCD_OK;
    const size_t ncells = (size_t)sys->n_tiles * CPT;
    CK(cudaMemsetAsync(sys->d.count[0], 0, sizeof(int) * ncells, sys->stream));
    CK(cudaMemsetAsync(sys->d.count[1], 0, sizeof(int) * ncells, sys->stream));
    CK(cudaMemsetAsync(sys->d.ovf_n, 0, sizeof(unsigned int) * 2, sys->stream));
    CK(cudaMemsetAsync(sys->d.near_count, 0, sizeof(int) * sys->n_rep, sys->stream));
    sys->primed = false;
    return RMPCD_OK;
}

// Bin the stored state on the grid of collision `grid_step` into count/bucket
// buffer `b` and run one cell pass with `opts` over it.
static rmpcd_status rebin_pass(rmpcd_system *sys, uint32_t grid_step, int opts, int b)
{
    launch_particles(sys->mixed, sys->d, PM_BIN, grid_step, sys->cur, b, sys->stream);
    rmpcd_status st = after_launch(sys, 1);
    if (st != RMPCD_OK) return st;
    if (sys->cap_auto) {
        bool grew = false;
        if ((st = check_counts(sys, b, &grew)) != RMPCD_OK) return st;
        if (grew) {
            launch_particles(sys->mixed, sys->d, PM_BIN, grid_step, sys->cur, b, sys->stream);
            if ((st = after_launch(sys, 1)) != RMPCD_OK) return st;
        }
    }
    CellPassArgs a{opts, grid_step, b, b ^ 1, sys->cur, sys->cur ^ 1};
    launch_cellpass(sys->mixed, sys->d, a, sys->stream);
    st = after_launch(sys, 1);
    if (st != RMPCD_OK) return st;
    if (opts & CP_WRITE) sys->cur ^= 1;
    return RMPCD_OK;
}

// A fused run's state (the record rows of buffer bcur, their overflow records
// and the near area) back into the flat slots of rec[cur], sorted on the grid
// of the last collision.  Sorting restores the canonical order (cell, id);
// positions have not moved since that collision, so every particle's cell
// key is the one it collided in.
static rmpcd_status flatten(rmpcd_system *sys)
{
    if (!sys->in_rows) return RMPCD_OK;
    sys->in_rows = false;
    sys->primed = false;
    const size_t ncells = (size_t)sys->n_tiles * CPT;
    CK(cudaMemsetAsync(sys->flat_fill, 0, sizeof(int) * sys->n_rep, sys->stream));
    launch_flatten(sys->mixed, sys->d, sys->bcur, sys->cur, sys->flat_fill, sys->stream);
    rmpcd_status st = after_launch(sys, 4);
    if (st != RMPCD_OK) return st;
    CK(cudaMemsetAsync(sys->d.count[0], 0, sizeof(int) * ncells, sys->stream));
    CK(cudaMemsetAsync(sys->d.count[1], 0, sizeof(int) * ncells, sys->stream));
    CK(cudaMemsetAsync(sys->d.ovf_n, 0, sizeof(unsigned int) * 2, sys->stream));
    CK(cudaMemsetAsync(sys->d.near_count, 0, sizeof(int) * sys->n_rep, sys->stream));
    if (!sys->has_sort) return RMPCD_OK;
    return rebin_pass(sys, sys->sort_step, CP_WRITE, 0);
}

static rmpcd_status check_errors(rmpcd_system *sys)
{
    unsigned int e[ERR_COUNT];
    CK(cudaMemcpyAsync(e, sys->d.err, sizeof e, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    bool any = false;
    for (int k = 0; k < ERR_COUNT; ++k) any |= e[k] != 0;
    if (!any) return RMPCD_OK;
    CK(cudaMemsetAsync(sys->d.err, 0, sizeof e, sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    if (e[ERR_TIMEOUT]) return fail(sys, RMPCD_ETIMEOUT, "a cell-pass look-back wait timed out; the state is invalid");
    if (e[ERR_OVERFLOW])
        return fail(sys, RMPCD_EOVERFLOW,
                    "a cell held %u particles: beyond the %d a cell may hold, or the overflow list past bucket_cap %d "
                    "(%d entries) ran full; the state is invalid", e[ERR_OVERFLOW], CP_MAX_CELL, sys->cap,
                    sys->d.ovf_cap);
    if (e[ERR_BOUNDS]) return fail(sys, RMPCD_ESTATE, "inconsistent bins (slot out of range); the state is invalid");
    if (e[ERR_RATTLE])
        return fail(sys, RMPCD_ESTATE, "a bead network's RATTLE stage did not converge within max_sweeps");
    if (e[ERR_SKIN]) return fail(sys, RMPCD_ESKIN, "a colloid moved further than skin in one interval (%u times)", e[ERR_SKIN]);
    return fail(sys, RMPCD_ESTATE, "device error");
}

extern "C" {

rmpcd_status rmpcd_create(rmpcd_system **out, int32_t precision, int32_t n_replicas, const rmpcd_params *params,
                          const rmpcd_colloid *colloids, const rmpcd_bond *bonds, int32_t bucket_cap, void *stream)
{
    return create_system(out, precision, n_replicas, params, colloids, bonds, bucket_cap, stream, nullptr);
}

rmpcd_status rmpcd_workspace_size(int32_t precision, int32_t n_replicas, const rmpcd_params *params,
                                  const rmpcd_colloid *colloids, const rmpcd_bond *bonds, int32_t bucket_cap,
                                  size_t *bytes)
{
    if (!bytes) return fail(nullptr, RMPCD_EINVAL, "bytes is NULL");
    *bytes = 0;
    rmpcd_system *tmp = nullptr;
    return create_system(&tmp, precision, n_replicas, params, colloids, bonds, bucket_cap, nullptr, bytes);
}

rmpcd_status rmpcd_set_state(rmpcd_system *sys, int32_t replica, const double *x, const double *v,
                             const uint8_t *flags, int64_t n, int32_t on_device)
{
    if (!sys) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    const ReplicaDev &rp = sys->rep[replica];
    if (n != rp.n_part) return fail(sys, RMPCD_EINVAL, "n = %lld but replica %d has %d particles", (long long)n, replica, rp.n_part);
    if (n > 0 && (!x || !v)) return fail(sys, RMPCD_EINVAL, "x and v are required");
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    const double *dx = x, *dv = v;
    const uint8_t *df = flags;
    if (!on_device && n > 0) {
        CK(cudaMemcpyAsync(sys->stage_x, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, sys->stream));
        CK(cudaMemcpyAsync(sys->stage_v, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, sys->stream));
        if (flags) CK(cudaMemcpyAsync(sys->stage_f, flags, n, cudaMemcpyHostToDevice, sys->stream));
        dx = sys->stage_x;
        dv = sys->stage_v;
        df = flags ? sys->stage_f : nullptr;
    }
    // the other replicas' records live in the current buffer too
    launch_set_state(sys->mixed, sys->d, replica, (int)n, dx, dv, df, sys->cur, sys->stream);
    st = after_launch(sys, n > 0 ? 1 : 0);
    if (st != RMPCD_OK) return st;
    if (!on_device) CK(cudaStreamSynchronize(sys->stream));   // host buffers may go away
    sys->has_sort = false;
    sys->obs_valid = false;
    return RMPCD_OK;
}

rmpcd_status rmpcd_get_state(rmpcd_system *sys, int32_t replica, double *x, double *v, uint8_t *flags,
                             uint32_t *id, int32_t *cell, int64_t n, int32_t on_device)
{
    if (!sys) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    const ReplicaDev &rp = sys->rep[replica];
    if (n != rp.n_part) return fail(sys, RMPCD_EINVAL, "n = %lld but replica %d has %d particles", (long long)n, replica, rp.n_part);
    rmpcd_status st0 = unprime(sys);   // a fused run's state, flattened and sorted
    if (st0 != RMPCD_OK) return st0;
    if (n > 0) {
        double *ox = x, *ov = v;
        uint8_t *of = flags;
        uint32_t *oi = id;
        int32_t *oc = cell;
        if (!on_device) {
            ox = x ? sys->stage_x : nullptr;
            ov = v ? sys->stage_v : nullptr;
            of = flags ? sys->stage_f : nullptr;
            oi = id ? sys->stage_id : nullptr;
            oc = cell ? sys->stage_cell : nullptr;
        }
        launch_get_state(sys->mixed, sys->d, replica, (int)n, sys->cur, ox, ov, of, oi, oc, sys->has_sort ? 1 : 0,
                         sys->sort_step, sys->stream);
        rmpcd_status st = after_launch(sys, 1);
        if (st != RMPCD_OK) return st;
        if (!on_device) {
            if (x) CK(cudaMemcpyAsync(x, sys->stage_x, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, sys->stream));
            if (v) CK(cudaMemcpyAsync(v, sys->stage_v, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, sys->stream));
            if (flags) CK(cudaMemcpyAsync(flags, sys->stage_f, n, cudaMemcpyDeviceToHost, sys->stream));
            if (id) CK(cudaMemcpyAsync(id, sys->stage_id, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, sys->stream));
            if (cell) CK(cudaMemcpyAsync(cell, sys->stage_cell, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, sys->stream));
        }
    }
    return check_errors(sys);
}

// The batch calls' staging area: the per-replica one when a single replica
// holds every particle, else n_total particles allocated once.
static rmpcd_status ensure_stage_all(rmpcd_system *sys)
{
    if (sys->sa_x) return RMPCD_OK;
    if (sys->n_total <= sys->max_part) {
        sys->sa_x = sys->stage_x;
        sys->sa_v = sys->stage_v;
        sys->sa_f = sys->stage_f;
        sys->sa_id = sys->stage_id;
        sys->sa_cell = sys->stage_cell;
        return RMPCD_OK;
    }
    const size_t n = (size_t)sys->n_total;
    rmpcd_status st = dalloc(sys, &sys->sa_x, 3 * n);
    if (st == RMPCD_OK) st = dalloc(sys, &sys->sa_v, 3 * n);
    if (st == RMPCD_OK) st = dalloc(sys, &sys->sa_f, n);
    if (st == RMPCD_OK) st = dalloc(sys, &sys->sa_id, n);
    if (st == RMPCD_OK) st = dalloc(sys, &sys->sa_cell, n);
    if (st != RMPCD_OK) {
        // keep nothing half-made (the buffers stay in allocs until destroy)
        sys->sa_x = sys->sa_v = nullptr;
        sys->sa_f = nullptr;
        sys->sa_id = nullptr;
        sys->sa_cell = nullptr;
        cudaGetLastError();
        return fail(sys, RMPCD_ENOMEM, "staging area of %d particles for the batch state calls", sys->n_total);
    }
    return RMPCD_OK;
}

// Replica groups of the batch state calls: consecutive replicas of about
// n_total / XFER_GROUPS particles.  A group's copy overlaps the kernels of
// its neighbour group, so the state kernels hide under the host copies.
static constexpr int XFER_GROUPS = 8;
static void xfer_groups(const rmpcd_system *sys, std::vector<int> &bounds)
{
    bounds.assign(1, 0);
    const long long target = std::max(1ll, (long long)sys->n_total / XFER_GROUPS);
    long long acc = 0;
    for (int r = 0; r < sys->n_rep; ++r) {
        acc += sys->rep[r].n_part;
        if (r + 1 == sys->n_rep || acc >= target * (long long)bounds.size()) bounds.push_back(r + 1);
    }
}

static rmpcd_status ensure_xfer(rmpcd_system *sys)
{
    if (!sys->xfer) CK(cudaStreamCreateWithFlags(&sys->xfer, cudaStreamNonBlocking));
    return RMPCD_OK;
}

rmpcd_status rmpcd_set_state_all(rmpcd_system *sys, const double *x, const double *v, const uint8_t *flags,
                                 int64_t n, int32_t on_device)
{
    if (!sys) return RMPCD_EINVAL;
    if (n != sys->n_total) return fail(sys, RMPCD_EINVAL, "n = %lld but the system has %d particles", (long long)n, sys->n_total);
    if (n > 0 && (!x || !v)) return fail(sys, RMPCD_EINVAL, "x and v are required");
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    const bool staged = !on_device && n > 0;
    if (staged) {
        if ((st = ensure_stage_all(sys)) != RMPCD_OK) return st;
        if ((st = ensure_xfer(sys)) != RMPCD_OK) return st;
    }
    const double *dx = staged ? sys->sa_x : x, *dv = staged ? sys->sa_v : v;
    const uint8_t *df = flags ? (staged ? sys->sa_f : flags) : nullptr;
    std::vector<int> gb;
    xfer_groups(sys, gb);
    std::vector<cudaEvent_t> evs;
    if (staged) {
        // the copies start after the work already on the system's stream
        // (which may still read the staging area)
        evs.push_back(pool_event(sys));
        CK(cudaEventRecord(evs.back(), sys->stream));
        CK(cudaStreamWaitEvent(sys->xfer, evs.back(), 0));
    }
    long long off = 0;
    for (size_t g = 0; g + 1 < gb.size(); ++g) {
        long long cnt = 0;
        for (int r = gb[g]; r < gb[g + 1]; ++r) cnt += sys->rep[r].n_part;
        if (staged && cnt > 0) {
            const size_t o = (size_t)off, m = (size_t)cnt;
            CK(cudaMemcpyAsync(sys->sa_x + 3 * o, x + 3 * o, sizeof(double) * 3 * m, cudaMemcpyHostToDevice, sys->xfer));
            CK(cudaMemcpyAsync(sys->sa_v + 3 * o, v + 3 * o, sizeof(double) * 3 * m, cudaMemcpyHostToDevice, sys->xfer));
            if (flags) CK(cudaMemcpyAsync(sys->sa_f + o, flags + o, m, cudaMemcpyHostToDevice, sys->xfer));
            evs.push_back(pool_event(sys));
            CK(cudaEventRecord(evs.back(), sys->xfer));
            CK(cudaStreamWaitEvent(sys->stream, evs.back(), 0));
        }
        for (int r = gb[g]; r < gb[g + 1]; ++r) {
            const int nr = sys->rep[r].n_part;
            if (nr > 0) {
                launch_set_state(sys->mixed, sys->d, r, nr, dx + 3 * off, dv + 3 * off, df ? df + off : nullptr,
                                 sys->cur, sys->stream);
                if ((st = after_launch(sys, 1)) != RMPCD_OK) return st;
            }
            off += nr;
        }
    }
    if (staged) CK(cudaStreamSynchronize(sys->stream));   // the host arrays may be reused
    for (cudaEvent_t e : evs) sys->ev_pool.push_back(e);
    sys->has_sort = false;
    sys->obs_valid = false;
    return RMPCD_OK;
}

rmpcd_status rmpcd_get_state_all(rmpcd_system *sys, double *x, double *v, uint8_t *flags, uint32_t *id,
                                 int32_t *cell, int64_t n, int32_t on_device)
{
    if (!sys) return RMPCD_EINVAL;
    if (n != sys->n_total) return fail(sys, RMPCD_EINVAL, "n = %lld but the system has %d particles", (long long)n, sys->n_total);
    rmpcd_status st = unprime(sys);   // a fused run's state, flattened and sorted
    if (st != RMPCD_OK) return st;
    std::vector<cudaEvent_t> evs;
    if (n > 0) {
        const bool staged = !on_device;
        if (staged) {
            if ((st = ensure_stage_all(sys)) != RMPCD_OK) return st;
            if ((st = ensure_xfer(sys)) != RMPCD_OK) return st;
        }
        double *ox = x ? (staged ? sys->sa_x : x) : nullptr;
        double *ov = v ? (staged ? sys->sa_v : v) : nullptr;
        uint8_t *of = flags ? (staged ? sys->sa_f : flags) : nullptr;
        uint32_t *oi = id ? (staged ? sys->sa_id : id) : nullptr;
        int32_t *oc = cell ? (staged ? sys->sa_cell : cell) : nullptr;
        std::vector<int> gb;
        xfer_groups(sys, gb);
        long long off = 0;
        for (size_t g = 0; g + 1 < gb.size(); ++g) {
            const long long g0 = off;
            for (int r = gb[g]; r < gb[g + 1]; ++r) {
                const int nr = sys->rep[r].n_part;
                if (nr > 0) {
                    launch_get_state(sys->mixed, sys->d, r, nr, sys->cur, ox ? ox + 3 * off : nullptr,
                                     ov ? ov + 3 * off : nullptr, of ? of + off : nullptr, oi ? oi + off : nullptr,
                                     oc ? oc + off : nullptr, sys->has_sort ? 1 : 0, sys->sort_step, sys->stream);
                    if ((st = after_launch(sys, 1)) != RMPCD_OK) return st;
                }
                off += nr;
            }
            if (staged && off > g0) {
                // this group's copies run beside the next group's kernels
                evs.push_back(pool_event(sys));
                CK(cudaEventRecord(evs.back(), sys->stream));
                CK(cudaStreamWaitEvent(sys->xfer, evs.back(), 0));
                const size_t o = (size_t)g0, m = (size_t)(off - g0);
                if (x) CK(cudaMemcpyAsync(x + 3 * o, sys->sa_x + 3 * o, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, sys->xfer));
                if (v) CK(cudaMemcpyAsync(v + 3 * o, sys->sa_v + 3 * o, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, sys->xfer));
                if (flags) CK(cudaMemcpyAsync(flags + o, sys->sa_f + o, m, cudaMemcpyDeviceToHost, sys->xfer));
                if (id) CK(cudaMemcpyAsync(id + o, sys->sa_id + o, sizeof(uint32_t) * m, cudaMemcpyDeviceToHost, sys->xfer));
                if (cell) CK(cudaMemcpyAsync(cell + o, sys->sa_cell + o, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, sys->xfer));
            }
        }
        if (staged) {
            // the system's stream (and so the error check below) waits for the copies
            evs.push_back(pool_event(sys));
            CK(cudaEventRecord(evs.back(), sys->xfer));
            CK(cudaStreamWaitEvent(sys->stream, evs.back(), 0));
        }
    }
    const rmpcd_status rc = check_errors(sys);
    for (cudaEvent_t e : evs) sys->ev_pool.push_back(e);
    return rc;
}

rmpcd_status rmpcd_set_colloids(rmpcd_system *sys, int32_t replica, const rmpcd_colloid *c, int32_t n)
{
    if (!sys) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    const ReplicaDev &rp = sys->rep[replica];
    const int ncol = sys->params[replica].n_colloids;
    if (n != ncol || (n > 0 && !c)) return fail(sys, RMPCD_EINVAL, "replica %d has %d colloids", replica, ncol);
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    std::vector<double> X(3 * n), V(3 * n);
    std::vector<int> Xi(3 * n), Ci(3 * n);
    std::vector<float> Xf(3 * n), Vf(3 * n);
    for (int j = 0; j < n; ++j) {
        for (int k = 0; k < 3; ++k) { X[3 * j + k] = c[j].x[k]; V[3 * j + k] = c[j].v[k]; }
        split_colloid(c[j], sys->params[replica], &Xi[3 * j], &Xf[3 * j], &Ci[3 * j], &Vf[3 * j]);
    }
    if (n > 0) {
        const size_t o = 3 * (size_t)rp.col_off;
        cudaStream_t s = sys->stream;
        CK(cudaMemcpyAsync(sys->d.colX + o, X.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(sys->d.colV + o, V.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(sys->d.colXi + o, Xi.data(), sizeof(int) * 3 * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(sys->d.colCi + o, Ci.data(), sizeof(int) * 3 * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(sys->d.colXf + o, Xf.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(sys->d.colVf + o, Vf.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    return RMPCD_OK;
}

rmpcd_status rmpcd_get_colloids(rmpcd_system *sys, int32_t replica, rmpcd_colloid *c, int32_t n)
{
    if (!sys) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    const ReplicaDev &rp = sys->rep[replica];
    const int ncol = sys->params[replica].n_colloids;
    if (n != ncol || (n > 0 && !c)) return fail(sys, RMPCD_EINVAL, "replica %d has %d colloids", replica, ncol);
    std::vector<double> X(3 * n + 1), V(3 * n + 1);
    std::vector<int> Xi(3 * n + 1);
    std::vector<float> Xf(3 * n + 1), Vf(3 * n + 1);
    if (n > 0) {
        const size_t o = 3 * (size_t)rp.col_off;
        cudaStream_t s = sys->stream;
        if (sys->mixed) {
            CK(cudaMemcpyAsync(Xi.data(), sys->d.colXi + o, sizeof(int) * 3 * n, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(Xf.data(), sys->d.colXf + o, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(Vf.data(), sys->d.colVf + o, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, s));
        } else {
            CK(cudaMemcpyAsync(X.data(), sys->d.colX + o, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(V.data(), sys->d.colV + o, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
        }
    }
    rmpcd_status st = check_errors(sys);
    for (int j = 0; j < n; ++j) {
        c[j] = sys->colloids[rp.col_off + j];
        for (int k = 0; k < 3; ++k) {
            if (sys->mixed) {
                c[j].x[k] = (double)Xi[3 * j + k] + (double)Xf[3 * j + k];
                c[j].v[k] = (double)Vf[3 * j + k];
            } else {
                c[j].x[k] = X[3 * j + k];
                c[j].v[k] = V[3 * j + k];
            }
        }
    }
    return st;
}

// Index of cell (x, y, z) on the 3-D Hilbert curve through the 2^m cube, by
// Skilling's transpose method ("Programming the Hilbert curve", AIP Conf.
// Proc. 707, 2004): undo the excess rotations and reflections from the
// coarsest level down, Gray-code across the axes, then read the bits level
// by level, x before y before z.
static uint64_t hilbert3(int m, uint32_t x, uint32_t y, uint32_t z)
{
    if (m <= 0) return 0;
    uint32_t a[3] = {x, y, z};
    for (int lev = m - 1; lev >= 1; --lev) {
        const uint32_t bit = 1u << lev, low = bit - 1u;
        for (int k = 0; k < 3; ++k) {
            if (a[k] & bit) {
                a[0] ^= low;
            } else {
                const uint32_t sw = (a[0] ^ a[k]) & low;
                a[0] ^= sw;
                a[k] ^= sw;
            }
        }
    }
    a[1] ^= a[0];
    a[2] ^= a[1];
    uint32_t flip = 0;
    for (int lev = m - 1; lev >= 1; --lev)
        if (a[2] & (1u << lev)) flip ^= (1u << lev) - 1u;
    uint64_t h = 0;
    for (int lev = m - 1; lev >= 0; --lev)
        for (int k = 0; k < 3; ++k) h = (h << 1) | (((a[k] ^ flip) >> lev) & 1u);
    return h;
}

// Place of every cell key k = x + L0 (y + L1 z) of a grid in the given order.
static void cell_places(const int32_t dims[3], int order, std::vector<int64_t> &place)
{
    const int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
    place.resize((size_t)n);
    if (order == RMPCD_ORDER_LINEAR) {
        for (int64_t k = 0; k < n; ++k) place[(size_t)k] = k;
        return;
    }
    int m = 0;
    while ((1 << m) < std::max(dims[0], std::max(dims[1], dims[2]))) ++m;
    std::vector<std::pair<uint64_t, int64_t>> hk((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        const uint32_t x = (uint32_t)(k % dims[0]), y = (uint32_t)((k / dims[0]) % dims[1]);
        const uint32_t z = (uint32_t)(k / ((int64_t)dims[0] * dims[1]));
        hk[(size_t)k] = {hilbert3(m, x, y, z), k};
    }
    std::sort(hk.begin(), hk.end());
    for (int64_t r = 0; r < n; ++r) place[(size_t)hk[(size_t)r].second] = r;
}

rmpcd_status rmpcd_cell_places(const int32_t dims[3], int32_t order, int64_t *place)
{
    if (!dims || !place) return RMPCD_EINVAL;
    if (order != RMPCD_ORDER_LINEAR && order != RMPCD_ORDER_HILBERT) return RMPCD_EINVAL;
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || dims[0] > 1023 || dims[1] > 1023 || dims[2] > 1023)
        return RMPCD_EINVAL;
    if ((int64_t)dims[0] * dims[1] * dims[2] > (1ll << 28)) return RMPCD_EINVAL;   // host work bound
    std::vector<int64_t> p;
    cell_places(dims, order, p);
    std::copy(p.begin(), p.end(), place);
    return RMPCD_OK;
}

rmpcd_status rmpcd_set_cell_order(rmpcd_system *sys, int32_t order)
{
    if (!sys) return RMPCD_EINVAL;
    if (order != RMPCD_ORDER_LINEAR && order != RMPCD_ORDER_HILBERT)
        return fail(sys, RMPCD_EINVAL, "cell order %d is neither linear nor Hilbert", order);
    if (order == sys->cell_order) return RMPCD_OK;
    // a fused run's rows are binned in the old order: back to the flat layout first
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    if (order == RMPCD_ORDER_HILBERT && !sys->cell_rank_dev) {
        const size_t nc = (size_t)sys->n_tiles * CPT;
        std::vector<int> rank(nc), key(nc);
        for (int r = 0; r < sys->n_rep; ++r) {
            const ReplicaDev &rp = sys->rep[r];
            const int32_t dims[3] = {rp.L[0], rp.L[1], rp.nz};
            std::vector<int64_t> place;
            cell_places(dims, order, place);
            const size_t off = (size_t)rp.cell_off, padded = (size_t)rp.n_tiles * CPT;
            for (size_t k = 0; k < padded; ++k) rank[off + k] = key[off + k] = (int)k;   // padding: itself
            for (size_t k = 0; k < place.size(); ++k) {
                rank[off + k] = (int)place[k];
                key[off + (size_t)place[k]] = (int)k;
            }
        }
        if ((st = dalloc(sys, &sys->cell_rank_dev, nc)) != RMPCD_OK) return st;
        if ((st = dalloc(sys, &sys->cell_key_dev, nc)) != RMPCD_OK) return st;
        CK(cudaMemcpyAsync(sys->cell_rank_dev, rank.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, sys->stream));
        CK(cudaMemcpyAsync(sys->cell_key_dev, key.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, sys->stream));
        CK(cudaStreamSynchronize(sys->stream));
    }
    sys->cell_order = order;
    sys->d.cell_rank = order == RMPCD_ORDER_HILBERT ? sys->cell_rank_dev : nullptr;
    sys->d.cell_key = order == RMPCD_ORDER_HILBERT ? sys->cell_key_dev : nullptr;
    drop_graphs(sys);   // the captured intervals hold the old tables
    sys->has_sort = false;
    sys->obs_valid = false;
    return RMPCD_OK;
}

rmpcd_status rmpcd_get_cell_order(rmpcd_system *sys, int32_t *order)
{
    if (!sys || !order) return RMPCD_EINVAL;
    *order = sys->cell_order;
    return RMPCD_OK;
}

rmpcd_status rmpcd_set_step(rmpcd_system *sys, uint32_t step)
{
    if (!sys) return RMPCD_EINVAL;
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    sys->step = step;
    launch_set_step(sys->d, step, sys->stream);
    return after_launch(sys, 1);
}

rmpcd_status rmpcd_get_step(const rmpcd_system *sys, uint32_t *step)
{
    if (!sys || !step) return RMPCD_EINVAL;
    *step = sys->step;
    return RMPCD_OK;
}

rmpcd_status rmpcd_stream(rmpcd_system *sys)
{
    if (!sys) return RMPCD_EINVAL;
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    launch_particles(sys->mixed, sys->d, PM_STREAM, sys->step, sys->cur, 0, sys->stream);
    if ((st = after_launch(sys, sys->n_total > 0 ? 1 : 0)) != RMPCD_OK) return st;
    if (sys->any_colloids) {
        const int cs = sys->md_fixed ? sys->md_fixed : sys->md_best;
        if (sys->md_kernel == 3)
            launch_md_wide(sys->d, sys->wide_reps, sys->md_wide_grid, sys->step, sys->cur, 0, 0, sys->stream);
        else if (sys->md_kernel == 2) launch_md_fast(sys->mixed, sys->d, sys->step, sys->cur, 0, 0, cs, sys->stream);
        else launch_md(sys->mixed, sys->d, sys->step, sys->cur, 0, 0, cs, sys->stream);
        if ((st = after_launch(sys, sys->md_kernel == 3 ? (int)sys->wide_reps.size() : 1)) != RMPCD_OK) return st;
    }
    if (sys->any_body) {
        launch_md_body(sys->mixed, sys->d, sys->nb_max, sys->grid_room, sys->step, sys->cur, 0, 0, sys->stream);
        if ((st = after_launch(sys, 1)) != RMPCD_OK) return st;
    }
    if (sys->any_net) {
        launch_md_network(sys->d, sys->net_smem, sys->step, sys->cur, 0, 0, sys->stream);
        if ((st = after_launch(sys, 1)) != RMPCD_OK) return st;
    }
    sys->has_sort = false;
    sys->obs_valid = false;
    return RMPCD_OK;
}

rmpcd_status rmpcd_md_substep(rmpcd_system *sys, int32_t k)
{
    if (!sys) return RMPCD_EINVAL;
    if (sys->any_body || sys->any_net)
        return fail(sys, RMPCD_EINVAL, "rmpcd_md_substep: not for replicas with a rigid body or a bead network");
    int n_md = 0;
    for (const auto &rp : sys->rep) n_md = std::max(n_md, rp.n_md);
    if (k < 0 || k >= n_md) return fail(sys, RMPCD_EINVAL, "sub-step %d outside 0..%d", k, n_md - 1);
    if (k != sys->md_sub_next)
        return fail(sys, RMPCD_ESTATE, "sub-step %d out of order: the next sub-step is %d", k, sys->md_sub_next);
    rmpcd_status st;
    if (k == 0) {
        // the interval starts: far particles fly, near particles join the near area
        if ((st = unprime(sys)) != RMPCD_OK) return st;
        launch_particles(sys->mixed, sys->d, PM_STREAM, sys->step, sys->cur, 0, sys->stream);
        if ((st = after_launch(sys, sys->n_total > 0 ? 1 : 0)) != RMPCD_OK) return st;
    }
    if (sys->any_colloids) {
        launch_md_range(sys->mixed, sys->d, sys->step, sys->cur, 0, 0, 1, k, k + 1, sys->stream);
        if ((st = after_launch(sys, 1)) != RMPCD_OK) return st;
    }
    sys->md_sub_next = (k + 1 < n_md) ? k + 1 : 0;
    sys->has_sort = false;
    sys->obs_valid = false;
    return RMPCD_OK;
}

rmpcd_status rmpcd_shift_and_sort(rmpcd_system *sys)
{
    if (!sys) return RMPCD_EINVAL;
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    if ((st = rebin_pass(sys, sys->step, CP_WRITE, 0)) != RMPCD_OK) return st;
    sys->has_sort = true;
    sys->sort_step = sys->step;
    sys->obs_valid = false;
    return RMPCD_OK;
}

static rmpcd_status sorted_op(rmpcd_system *sys, int opts, const char *name)
{
    if (!sys) return RMPCD_EINVAL;
    if (!sys->has_sort || sys->sort_step != sys->step)
        return fail(sys, RMPCD_ESTATE, "%s needs the state sorted on the grid of the current step (call rmpcd_shift_and_sort)", name);
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    if ((st = rebin_pass(sys, sys->step, CP_WRITE | opts, 0)) != RMPCD_OK) return st;
    sys->obs_valid = false;
    return RMPCD_OK;
}

rmpcd_status rmpcd_collide(rmpcd_system *sys) { return sorted_op(sys, CP_COLLIDE, "rmpcd_collide"); }
rmpcd_status rmpcd_react(rmpcd_system *sys) { return sorted_op(sys, CP_REACT, "rmpcd_react"); }

// Cluster size of the next MD launch; while tuning, each size in turn with a
// CUDA event pair around the launch.
static int md_cluster_for_launch(rmpcd_system *sys, cudaEvent_t *a)
{
    *a = nullptr;
    if (sys->md_fixed) return sys->md_fixed;
    if (sys->md_tuned) return sys->md_best;
    const int cs = sys->md_cand[sys->md_trials.size() % sys->md_cand.size()];
    *a = pool_event(sys);
    cudaEventRecord(*a, sys->stream);
    return cs;
}

static void md_trial_done(rmpcd_system *sys, int cs, cudaEvent_t a)
{
    if (!a) return;
    cudaEvent_t b = pool_event(sys);
    cudaEventRecord(b, sys->stream);
    sys->md_trials.push_back({cs, a, b});
    if (sys->md_trials.size() < 3 * sys->md_cand.size()) return;
    // three launches of each size: keep the size with the smallest median
    cudaEventSynchronize(b);
    double best_t = 1e30;
    for (int c : sys->md_cand) {
        std::vector<float> t;
        for (auto &q : sys->md_trials)
            if (q.phase == c) {
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, q.a, q.b);
                t.push_back(ms);
            }
        std::sort(t.begin(), t.end());
        const double med = t.empty() ? 1e30 : t[t.size() / 2];
        if (med < best_t) { best_t = med; sys->md_best = c; }
    }
    for (auto &q : sys->md_trials) { sys->ev_pool.push_back(q.a); sys->ev_pool.push_back(q.b); }
    sys->md_trials.clear();
    sys->md_tuned = true;
}

// The launches of one fused interval on buffers (cur, bcur), the step taken
// from the control block (STEP_DEVICE) and advanced by the cell pass; timers
// and the MD tuner wrap the launches when active.  Returns the launch count.
static int launch_interval(rmpcd_system *sys, int cur, int bcur, bool instrument)
{
    int n = 0;
    cudaEvent_t ev = nullptr, tev = nullptr;
    if (sys->any_colloids) {
        const int cs = instrument ? md_cluster_for_launch(sys, &tev) : (sys->md_fixed ? sys->md_fixed : sys->md_best);
        if (instrument) tstart(sys, &ev);
        if (sys->md_kernel == 3) {
            launch_md_wide(sys->d, sys->wide_reps, sys->md_wide_grid, STEP_DEVICE, cur, bcur, 1, sys->stream);
            n += (int)sys->wide_reps.size();
        } else {
            if (sys->md_kernel == 2) launch_md_fast(sys->mixed, sys->d, STEP_DEVICE, cur, bcur, 1, cs, sys->stream);
            else launch_md(sys->mixed, sys->d, STEP_DEVICE, cur, bcur, 1, cs, sys->stream);
            n += 1;
        }
        if (instrument) {
            tstop(sys, 1, ev);
            md_trial_done(sys, cs, tev);
        }
    }
    if (sys->any_body) {
        if (instrument) tstart(sys, &ev);
        launch_md_body(sys->mixed, sys->d, sys->nb_max, sys->grid_room, STEP_DEVICE, cur, bcur, 1, sys->stream);
        if (instrument) tstop(sys, 1, ev);
        n += 1;
    }
    if (sys->any_net) {
        if (instrument) tstart(sys, &ev);
        launch_md_network(sys->d, sys->net_smem, STEP_DEVICE, cur, bcur, 1, sys->stream);
        if (instrument) tstop(sys, 1, ev);
        n += 1;
    }
    // record rows bcur -> rows bcur ^ 1 and the near area (the flat buffers
    // are not touched)
    CellPassArgs a{CP_FLIGHT | CP_COLLIDE | CP_REACT | CP_NEXT | CP_ADVANCE, STEP_DEVICE, bcur, bcur ^ 1, cur, cur ^ 1};
    if (instrument) tstart(sys, &ev);
    launch_cellpass(sys->mixed, sys->d, a, sys->stream);
    if (instrument) tstop(sys, 2, ev);
    return n + 1;
}

// The graph of one fused interval on buffers (cur, bcur), captured on first
// use; nullptr when capture is not possible on this stream.
static cudaGraphExec_t interval_graph(rmpcd_system *sys, int cur, int bcur)
{
    cudaGraphExec_t &ge = sys->graph[cur][bcur];
    if (ge) return ge;
    if (sys->stream == nullptr) return nullptr;   // the legacy default stream cannot be captured
    if (cudaStreamBeginCapture(sys->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const int n = launch_interval(sys, cur, bcur, false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(sys->stream, &g);
    if (e == cudaSuccess && g) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ge = nullptr;
        return nullptr;
    }
    sys->graph_nodes = n;
    return ge;
}

rmpcd_status rmpcd_step(rmpcd_system *sys, int32_t n_intervals)
{
    if (!sys) return RMPCD_EINVAL;
    if (n_intervals < 0) return fail(sys, RMPCD_EINVAL, "n_intervals < 0");
    if (sys->md_sub_next != 0)
        return fail(sys, RMPCD_ESTATE, "an interval is being sub-stepped (rmpcd_md_substep): run its last sub-step first");
    if (n_intervals == 0) return RMPCD_OK;
    rmpcd_status st;
    cudaEvent_t ev;
    if (sys->cap_auto && sys->maxcnt_pending && cudaEventQuery(sys->maxcnt_ev) == cudaSuccess) {
        // the largest cell count of the last run: grow before it overflows
        sys->maxcnt_pending = false;
        const int m = (int)*sys->maxcnt_host;
        if (m * 5 > sys->cap * 4 && sys->cap < CP_MAX_CAP && (st = set_bucket_cap(sys, grown_cap(m))) != RMPCD_OK)
            return st;
    }
    for (int attempt = 0; !sys->primed && attempt < 8; ++attempt) {
        // bins for the collision of `step`: far particles at their flown
        // position, near particles through the MD kernel
        tstart(sys, &ev);
        launch_particles(sys->mixed, sys->d, PM_PRIME, sys->step, sys->cur, sys->bcur, sys->stream);
        tstop(sys, 0, ev);
        if ((st = after_launch(sys, sys->n_total > 0 ? 1 : 0)) != RMPCD_OK) return st;
        sys->primed = true;
        if (sys->cap_auto) {
            // a fresh state: measure the first binning before any pass uses it
            bool grew = false;
            if ((st = check_counts(sys, sys->bcur, &grew)) != RMPCD_OK) return st;
        }
    }
    int left = n_intervals;
    while (left > 0) {
        // a captured graph of the interval once nothing on the host side
        // watches single launches (timers, the MD tuner)
        const bool settled = !sys->any_colloids || sys->md_fixed || sys->md_tuned;
        cudaGraphExec_t ge = nullptr;
        if (sys->graphs_on && settled && !sys->timing) ge = interval_graph(sys, sys->cur, sys->bcur);
        if (ge) {
            CK(cudaGraphLaunch(ge, sys->stream));
            if ((st = after_launch(sys, sys->graph_nodes)) != RMPCD_OK) return st;
        } else {
            const int n = launch_interval(sys, sys->cur, sys->bcur, true);
            if ((st = after_launch(sys, n)) != RMPCD_OK) return st;
        }
        sys->bcur ^= 1;
        sys->in_rows = true;
        sys->sort_step = sys->step;
        sys->step += 1u;
        left -= 1;
    }
    if (sys->cap_auto && !sys->maxcnt_pending) {
        CK(cudaMemcpyAsync(sys->maxcnt_host, sys->d.maxcnt, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                           sys->stream));
        CK(cudaMemsetAsync(sys->d.maxcnt, 0, sizeof(unsigned int), sys->stream));
        CK(cudaEventRecord(sys->maxcnt_ev, sys->stream));
        sys->maxcnt_pending = true;
    }
    sys->has_sort = true;
    sys->obs_valid = false;   // observables are computed on request
    return RMPCD_OK;
}

rmpcd_status rmpcd_set_wait_test(rmpcd_system *sys, int32_t max_polls, int32_t stall)
{
    if (!sys) return RMPCD_EINVAL;
    if (max_polls < 0) return fail(sys, RMPCD_EINVAL, "max_polls %d < 0", max_polls);
    drop_graphs(sys);   // the kernels take Dev by value: captured launches hold the old limit
    sys->d.lb_limit = max_polls == 0 ? LB_SPIN_LIMIT : max_polls;
    sys->d.lb_stall = stall != 0 ? 1 : 0;
    return RMPCD_OK;
}

rmpcd_status rmpcd_get_bucket_cap(const rmpcd_system *sys, int32_t *cap)
{
    if (!sys || !cap) return RMPCD_EINVAL;
    *cap = sys->cap;
    return RMPCD_OK;
}

// Capture and replay of fused intervals as CUDA graphs (on by default).
rmpcd_status rmpcd_set_graphs(rmpcd_system *sys, int32_t on)
{
    if (!sys) return RMPCD_EINVAL;
    sys->graphs_on = on != 0;
    return RMPCD_OK;
}

rmpcd_status rmpcd_observables(rmpcd_system *sys, int32_t replica, rmpcd_obs *out)
{
    if (!sys || !out) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    rmpcd_status st;
    if (!sys->obs_valid) {
        if (!sys->has_sort) return fail(sys, RMPCD_ESTATE, "no collision grid yet: sort or step first");
        // the flat state, rebinned on the grid of the last sort
        if ((st = unprime(sys)) != RMPCD_OK) return st;
        if ((st = rebin_pass(sys, sys->sort_step, CP_OBS, 0)) != RMPCD_OK) return st;
        launch_obs_reduce(sys->d, sys->stream);
        if ((st = after_launch(sys, 1)) != RMPCD_OK) return st;
        sys->obs_valid = true;
    }
    double o[8];
    CK(cudaMemcpyAsync(o, sys->d.obs_out + 8 * replica, sizeof o, cudaMemcpyDeviceToHost, sys->stream));
    st = check_errors(sys);
    std::memset(out, 0, sizeof *out);
    out->n_cells_used = (int64_t)o[1];
    out->temperature = o[1] > 0 ? o[0] / (3.0 * o[1]) : 0.0;
    out->momentum[0] = o[2];
    out->momentum[1] = o[3];
    out->momentum[2] = o[4];
    out->kinetic = o[5];
    out->n_B = (int64_t)o[6];
    out->n_solvent = (int64_t)o[7];
    out->step = sys->sort_step;
    return st;
}

static_assert(RMPCD_MAX_PROFILE_BINS <= PROF_MAX_BINS, "profile bins exceed the kernel's shared sums");

rmpcd_status rmpcd_profile(rmpcd_system *sys, int32_t replica, int32_t axis, int32_t n_bins, rmpcd_profile_bin *out)
{
    if (!sys || !out) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    if (axis < 0 || axis > 2) return fail(sys, RMPCD_EINVAL, "axis %d is not 0, 1 or 2", axis);
    if (n_bins < 1 || n_bins > RMPCD_MAX_PROFILE_BINS)
        return fail(sys, RMPCD_EINVAL, "n_bins %d outside 1..%d", n_bins, RMPCD_MAX_PROFILE_BINS);
    const size_t words = (size_t)n_bins * PROF_FIELDS;
    rmpcd_status st0 = unprime(sys);   // the flat state
    if (st0 != RMPCD_OK) return st0;
    CK(cudaMemsetAsync(sys->prof_acc, 0, words * sizeof(unsigned long long), sys->stream));
    launch_profile(sys->mixed, sys->d, replica, sys->rep[replica].n_part, sys->cur, axis, n_bins, sys->prof_acc,
                   sys->stream);
    rmpcd_status st = after_launch(sys, 1);
    if (st != RMPCD_OK) return st;
    std::vector<unsigned long long> h(words);
    CK(cudaMemcpyAsync(h.data(), sys->prof_acc, words * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       sys->stream));
    st = check_errors(sys);   // synchronises
    for (int b = 0; b < n_bins; ++b) {
        const unsigned long long *a = h.data() + (size_t)b * PROF_FIELDS;
        rmpcd_profile_bin &o = out[b];
        o.n = (int64_t)a[0];
        o.n_B = (int64_t)a[1];
        for (int k = 0; k < 3; ++k) {
            o.v_sum[k] = (double)(long long)a[2 + k] * 0x1p-32;
            o.v2_sum[k] = (double)(long long)a[5 + k] * 0x1p-24;
        }
    }
    return st;
}

rmpcd_status rmpcd_sync(rmpcd_system *sys)
{
    if (!sys) return RMPCD_EINVAL;
    return check_errors(sys);
}

rmpcd_status rmpcd_enable_timers(rmpcd_system *sys, int32_t on)
{
    if (!sys) return RMPCD_EINVAL;
    sys->timing = on != 0;
    return RMPCD_OK;
}

rmpcd_status rmpcd_read_timers(rmpcd_system *sys, rmpcd_timers *out, int32_t reset)
{
    if (!sys || !out) return RMPCD_EINVAL;
    CK(cudaStreamSynchronize(sys->stream));
    for (auto &q : sys->pending) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, q.a, q.b));
        sys->t_ms[q.phase] += ms;
        sys->t_launches[q.phase] += 1;
        sys->ev_pool.push_back(q.a);
        sys->ev_pool.push_back(q.b);
    }
    sys->pending.clear();
    for (int k = 0; k < 4; ++k) {
        out->launches[k] = sys->t_launches[k];
        out->ms[k] = sys->t_ms[k];
        if (reset) { sys->t_launches[k] = 0; sys->t_ms[k] = 0.0; }
    }
    return RMPCD_OK;
}

rmpcd_status rmpcd_set_tuning(rmpcd_system *sys, int32_t md_cluster, int32_t md_kernel)
{
    if (!sys) return RMPCD_EINVAL;
    if (md_kernel < 0 || md_kernel > 3) return fail(sys, RMPCD_EINVAL, "md_kernel must be 0, 1, 2 or 3");
    if (md_kernel == 2 && !sys->fast_ok)
        return fail(sys, RMPCD_EINVAL, "the few-colloid MD kernel needs <= %d colloids, <= 1 bond and no "
                    "colloid-colloid potential", MD_FAST_NC);
    if (md_kernel == 3 && !(sys->mixed && sys->md_wide_grid > 0))
        return fail(sys, RMPCD_EINVAL, "the wide MD kernel needs the mixed path and cooperative launch");
    const int kern = md_kernel ? md_kernel : (sys->fast_ok ? 2 : (wide_default(sys) ? 3 : 1));
    if (kern == 3 && md_cluster > 1)
        return fail(sys, RMPCD_EINVAL, "the wide MD kernel takes no cluster size (0 or 1)");
    const int maxc = kern == 2 ? sys->md_fast_max : 8;
    if (md_cluster != 0 && md_cluster != 1 && md_cluster != 2 && md_cluster != 4 && md_cluster != 8 &&
        !(md_cluster == 16 && maxc >= 16))
        return fail(sys, RMPCD_EINVAL, "md_cluster must be 0 (tune), 1, 2, 4, 8%s", maxc >= 16 ? " or 16" : "");
    set_md_kernel(sys, md_kernel);
    drop_graphs(sys);
    sys->md_fixed = md_cluster;
    if (md_cluster == 0) {
        sys->md_tuned = false;
        for (auto &q : sys->md_trials) { sys->ev_pool.push_back(q.a); sys->ev_pool.push_back(q.b); }
        sys->md_trials.clear();
    }
    return RMPCD_OK;
}

rmpcd_status rmpcd_get_tuning(const rmpcd_system *sys, int32_t *md_cluster, int32_t *md_kernel)
{
    if (!sys || !md_cluster) return RMPCD_EINVAL;
    *md_cluster = sys->md_fixed ? sys->md_fixed : (sys->md_tuned ? sys->md_best : 0);
    if (md_kernel) *md_kernel = sys->md_kernel;
    return RMPCD_OK;
}

rmpcd_status rmpcd_launch_count(const rmpcd_system *sys, int64_t *count)
{
    if (!sys || !count) return RMPCD_EINVAL;
    *count = sys->launches;
    return RMPCD_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// rigid bead bodies
// ----------------------------------------------------------------------------
// Lookup grid of a body in its frame: gn^3 cubic cells of side h over
// [glo, glo + gn h)^3 around the centre; cell c lists, in ascending order,
// every bead whose distance to the cell's box is below the cut-off plus a
// margin.  The margin covers the FP32 rounding of a particle's body-frame
// position and of its cell index, so a bead within the cut-off of a particle
// is always in the particle's list, and a particle outside the grid reaches
// no bead.
static void build_body_grid(rmpcd_system::BodyHost &H)
{
    BodyDev &D = H.dev;
    const double margin = 0.0625;
    const double B = D.reach + margin;
    const double h0 = std::max(0.5, 2.0 * B / 32.0);
    const int gn = std::max(1, (int)ceil(2.0 * B / h0));
    D.gn = gn;
    D.glo = (float)(-B);
    D.ginv = (float)(1.0 / h0);
    const double lo = (double)D.glo, h = 1.0 / (double)D.ginv;
    const double rcm = sqrt(D.rc2) + margin;
    const int ncell = gn * gn * gn;
    std::vector<std::vector<unsigned short>> lists((size_t)ncell);
    for (int j = 0; j < D.nb; ++j) {
        const double *b = H.beads[j].b;
        int a[3], e[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = std::max(0, (int)floor((b[k] - rcm - lo) / h));
            e[k] = std::min(gn - 1, (int)floor((b[k] + rcm - lo) / h));
        }
        for (int iz = a[2]; iz <= e[2]; ++iz)
            for (int iy = a[1]; iy <= e[1]; ++iy)
                for (int ix = a[0]; ix <= e[0]; ++ix) {
                    const int id[3] = {ix, iy, iz};
                    double dd = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        const double c0 = lo + id[k] * h, c1 = c0 + h;
                        const double t = b[k] < c0 ? c0 - b[k] : (b[k] > c1 ? b[k] - c1 : 0.0);
                        dd += t * t;
                    }
                    if (dd < rcm * rcm) lists[(size_t)ix + gn * ((size_t)iy + gn * iz)].push_back((unsigned short)j);
                }
    }
    H.gstart.assign((size_t)ncell + 1, 0);
    H.glist.clear();
    for (int c = 0; c < ncell; ++c) {
        H.gstart[c] = (int)H.glist.size();
        H.glist.insert(H.glist.end(), lists[c].begin(), lists[c].end());
    }
    H.gstart[ncell] = (int)H.glist.size();
}

// Concatenated bead and grid arrays of all bodies (offsets written into each
// body's constants), uploaded into fresh buffers.
static rmpcd_status upload_bodies(rmpcd_system *sys)
{
    std::vector<double> bb, be;
    std::vector<float> bef;
    std::vector<int> bc, gs;
    std::vector<unsigned short> gl;
    sys->nb_max = 0;
    long long grid_entries = 0;
    for (auto &H : sys->bodies) {
        if (H.beads.empty()) continue;
        H.dev.bead_off = (int)bc.size();
        H.dev.gstart_off = (int)gs.size();
        H.dev.glist_off = (int)gl.size();
        for (const rmpcd_bead &e : H.beads) {
            for (int k = 0; k < 3; ++k) bb.push_back(e.b[k]);
            be.push_back(e.eps_A);
            be.push_back(e.eps_B);
            bef.push_back((float)e.eps_A);
            bef.push_back((float)e.eps_B);
            bc.push_back(e.catalytic ? 1 : 0);
        }
        gs.insert(gs.end(), H.gstart.begin(), H.gstart.end());
        gl.insert(gl.end(), H.glist.begin(), H.glist.end());
        sys->nb_max = std::max(sys->nb_max, H.dev.nb);
        grid_entries = std::max(grid_entries, (long long)(H.gstart.size() + H.glist.size()));
    }
    // 16-bit offsets in shared memory need every list below 65536 entries
    bool small = true;
    for (auto &H : sys->bodies)
        if (!H.beads.empty() && H.glist.size() >= 65536) small = false;
    sys->grid_room = small ? md_body_grid_room(sys->mixed, sys->nb_max, grid_entries) : 0;
    CK(cudaStreamSynchronize(sys->stream));
    for (void *p : sys->body_allocs) cudaFree(p);
    sys->body_allocs.clear();
    auto put = [&](const void **dst, const void *src, size_t bytes) -> rmpcd_status {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) return cuda_check(sys, e, "cudaMalloc (bodies)");
        sys->body_allocs.push_back(p);
        *dst = p;
        return cuda_check(sys, cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, sys->stream), "upload (bodies)");
    };
    rmpcd_status st = RMPCD_OK;
    Dev &d = sys->d;
    if (st == RMPCD_OK) st = put(reinterpret_cast<const void **>(&d.bead_b), bb.data(), sizeof(double) * bb.size());
    if (st == RMPCD_OK) st = put(reinterpret_cast<const void **>(&d.bead_eps), be.data(), sizeof(double) * be.size());
    if (st == RMPCD_OK) st = put(reinterpret_cast<const void **>(&d.bead_eps_f), bef.data(), sizeof(float) * bef.size());
    if (st == RMPCD_OK) st = put(reinterpret_cast<const void **>(&d.bead_cat), bc.data(), sizeof(int) * bc.size());
    if (st == RMPCD_OK) st = put(reinterpret_cast<const void **>(&d.grid_start), gs.data(), sizeof(int) * gs.size());
    if (st == RMPCD_OK)
        st = put(reinterpret_cast<const void **>(&d.grid_list), gl.data(), sizeof(unsigned short) * gl.size());
    return st;
}

// Centre of mass (sum in bead order) and reach (largest bead distance from it
// plus the cut-off) of a network, as the FP64 definition computes them.
static void net_com_reach(const std::vector<rmpcd_net_bead> &bd, double rc2, double X[3], double *reach)
{
    double s[3] = {0.0, 0.0, 0.0}, m = 0.0;
    for (const auto &b : bd) {
        m = m + b.mass;
        for (int t = 0; t < 3; ++t) s[t] = s[t] + b.mass * b.x[t];
    }
    for (int t = 0; t < 3; ++t) X[t] = s[t] / m;
    double rmax = 0.0;
    for (const auto &b : bd) {
        double e2 = 0.0;
        for (int t = 0; t < 3; ++t) { const double e = b.x[t] - X[t]; e2 = e2 + e * e; }
        if (sqrt(e2) > rmax) rmax = sqrt(e2);
    }
    *reach = rmax + sqrt(rc2);
}

// The arrays of every network, concatenated into fresh device buffers (the
// offsets go into each network's constants), and the constants themselves.
static rmpcd_status upload_networks(rmpcd_system *sys)
{
    std::vector<double> x, v, m, eps, dl;
    std::vector<int> cat, la, lb, cs;
    std::vector<NetDev> all(sys->n_rep);
    size_t smem = 0;
    for (int r = 0; r < sys->n_rep; ++r) {
        auto &H = sys->nets[r];
        if (H.beads.empty()) continue;
        H.dev.bead_off = (int)m.size();
        H.dev.link_off = (int)dl.size();
        H.dev.color_off = (int)cs.size();
        for (const auto &b : H.beads) {
            for (int t = 0; t < 3; ++t) { x.push_back(b.x[t]); v.push_back(b.v[t]); }
            m.push_back(b.mass);
            eps.push_back(b.eps_A);
            eps.push_back(b.eps_B);
            cat.push_back(b.catalytic ? 1 : 0);
        }
        la.insert(la.end(), H.la.begin(), H.la.end());
        lb.insert(lb.end(), H.lb.begin(), H.lb.end());
        dl.insert(dl.end(), H.dl.begin(), H.dl.end());
        cs.insert(cs.end(), H.cs.begin(), H.cs.end());
        all[r] = H.dev;
        smem = std::max(smem, md_network_smem(H.dev.nb, H.dev.nl, H.dev.ncol));
    }
    CK(cudaStreamSynchronize(sys->stream));
    for (void *p : sys->net_allocs) cudaFree(p);
    sys->net_allocs.clear();
    auto put = [&](void **dst, const void *src, size_t bytes) -> rmpcd_status {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) return cuda_check(sys, e, "cudaMalloc (networks)");
        sys->net_allocs.push_back(p);
        *dst = p;
        return cuda_check(sys, cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, sys->stream), "upload (networks)");
    };
    rmpcd_status st = RMPCD_OK;
    Dev &d = sys->d;
    void *p = nullptr;
    if (st == RMPCD_OK && (st = put(&p, x.data(), sizeof(double) * x.size())) == RMPCD_OK) d.net_x = (double *)p;
    if (st == RMPCD_OK && (st = put(&p, v.data(), sizeof(double) * v.size())) == RMPCD_OK) d.net_v = (double *)p;
    if (st == RMPCD_OK && (st = put(&p, m.data(), sizeof(double) * m.size())) == RMPCD_OK) d.net_m = (const double *)p;
    if (st == RMPCD_OK && (st = put(&p, eps.data(), sizeof(double) * eps.size())) == RMPCD_OK) d.net_eps = (const double *)p;
    if (st == RMPCD_OK && (st = put(&p, cat.data(), sizeof(int) * cat.size())) == RMPCD_OK) d.net_cat = (const int *)p;
    if (st == RMPCD_OK && (st = put(&p, la.data(), sizeof(int) * la.size())) == RMPCD_OK) d.net_la = (const int *)p;
    if (st == RMPCD_OK && (st = put(&p, lb.data(), sizeof(int) * lb.size())) == RMPCD_OK) d.net_lb = (const int *)p;
    if (st == RMPCD_OK && (st = put(&p, dl.data(), sizeof(double) * dl.size())) == RMPCD_OK) d.net_d = (const double *)p;
    if (st == RMPCD_OK && (st = put(&p, cs.data(), sizeof(int) * cs.size())) == RMPCD_OK) d.net_cs = (const int *)p;
    if (st != RMPCD_OK) return st;
    CK(cudaMemcpyAsync(d.net, all.data(), sizeof(NetDev) * sys->n_rep, cudaMemcpyHostToDevice, sys->stream));
    sys->net_smem = smem;
    CK(prepare_md_network(smem));
    return RMPCD_OK;
}

// The current bead states of every network, from the device into the host
// copies (before the arrays are rebuilt).
static rmpcd_status fetch_networks(rmpcd_system *sys)
{
    if (!sys->any_net) return RMPCD_OK;
    CK(cudaStreamSynchronize(sys->stream));
    for (auto &H : sys->nets) {
        if (H.beads.empty()) continue;
        const int nb = (int)H.beads.size();
        std::vector<double> x(3 * nb), v(3 * nb);
        CK(cudaMemcpy(x.data(), sys->d.net_x + 3 * H.dev.bead_off, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(v.data(), sys->d.net_v + 3 * H.dev.bead_off, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost));
        for (int j = 0; j < nb; ++j)
            for (int t = 0; t < 3; ++t) { H.beads[j].x[t] = x[3 * j + t]; H.beads[j].v[t] = v[3 * j + t]; }
    }
    return RMPCD_OK;
}

extern "C" {

rmpcd_status rmpcd_set_network(rmpcd_system *sys, int32_t replica, const rmpcd_net_bead *beads, int32_t n_beads,
                               const rmpcd_bond *links, const int32_t *colors, int32_t n_links, double sigma,
                               double tol, int32_t max_sweeps)
{
    if (!sys) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    if (sys->mixed) return fail(sys, RMPCD_EINVAL, "a bead network needs an FP64 system");
    const rmpcd_params &p = sys->params[replica];
    if (p.n_colloids != 0 || p.n_bonds != 0 || p.walls || !sys->bodies[replica].beads.empty())
        return fail(sys, RMPCD_EINVAL, "replica %d: a network needs a replica with no colloids, bonds, walls or body",
                    replica);
    if (n_beads < 1 || n_beads > RMPCD_MAX_NET_BEADS || !beads)
        return fail(sys, RMPCD_EINVAL, "n_beads %d not in [1,%d]", n_beads, RMPCD_MAX_NET_BEADS);
    if (n_links < 0 || (n_links > 0 && (!links || !colors))) return fail(sys, RMPCD_EINVAL, "links and colors required");
    if (!(sigma > 0.0) || !std::isfinite(sigma) || !(tol > 0.0) || !(max_sweeps >= 1))
        return fail(sys, RMPCD_EINVAL, "need sigma > 0, tol > 0, max_sweeps >= 1");
    for (int j = 0; j < n_beads; ++j) {
        const rmpcd_net_bead &b = beads[j];
        bool ok = b.mass > 0.0 && std::isfinite(b.mass) && b.eps_A >= 0.0 && b.eps_B >= 0.0 &&
                  std::isfinite(b.eps_A) && std::isfinite(b.eps_B);
        for (int t = 0; t < 3; ++t) ok = ok && std::isfinite(b.x[t]) && std::isfinite(b.v[t]);
        if (!ok) return fail(sys, RMPCD_EINVAL, "bead %d: finite state, mass > 0 and epsilons >= 0 required", j);
    }
    int ncol = 0;
    for (int k = 0; k < n_links; ++k) {
        const rmpcd_bond &l = links[k];
        if (l.a < 0 || l.b < 0 || l.a >= n_beads || l.b >= n_beads || l.a == l.b || !(l.d > 0.0) || !std::isfinite(l.d) ||
            colors[k] < 0 || colors[k] >= 4 * n_beads)
            return fail(sys, RMPCD_EINVAL, "link %d invalid", k);
        ncol = std::max(ncol, colors[k] + 1);
    }
    // links of one colour must share no bead
    std::vector<int> seen((size_t)ncol * n_beads, 0);
    for (int k = 0; k < n_links; ++k)
        for (int e : {links[k].a, links[k].b}) {
            int &s = seen[(size_t)colors[k] * n_beads + e];
            if (s) return fail(sys, RMPCD_EINVAL, "link %d: bead %d appears twice in colour %d", k, e, colors[k]);
            s = 1;
        }
    const double rc2 = sigma * sigma * cbrt(2.0);
    std::vector<rmpcd_net_bead> bd(beads, beads + n_beads);
    double X[3], reach;
    net_com_reach(bd, rc2, X, &reach);
    if (2.0 * reach + 2.0 * p.skin >= (double)std::min(p.L[0], std::min(p.L[1], p.L[2])))
        return fail(sys, RMPCD_EINVAL, "replica %d: box too small for the network's reach", replica);
    if (md_network_smem(n_beads, n_links, ncol) > 200 * 1024)
        return fail(sys, RMPCD_EINVAL, "network too large for shared memory");
    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    CK(cudaStreamSynchronize(sys->stream));
    drop_graphs(sys);
    if ((st = fetch_networks(sys)) != RMPCD_OK) return st;
    auto &H = sys->nets[replica];
    H.beads = bd;
    H.la.clear(); H.lb.clear(); H.dl.clear(); H.cs.assign(1, 0);
    for (int c = 0; c < ncol; ++c) {
        for (int k = 0; k < n_links; ++k)
            if (colors[k] == c) { H.la.push_back(links[k].a); H.lb.push_back(links[k].b); H.dl.push_back(links[k].d); }
        H.cs.push_back((int)H.la.size());
    }
    std::memset(&H.dev, 0, sizeof H.dev);
    H.dev.nb = n_beads;
    H.dev.nl = n_links;
    H.dev.ncol = ncol;
    H.dev.max_sweeps = max_sweeps;
    H.dev.sigma = sigma;
    H.dev.rc2 = rc2;
    H.dev.tol = tol;
    sys->any_net = true;
    if ((st = upload_networks(sys)) != RMPCD_OK) return st;
    // the network's colloid slot: centre of mass and reach for the near test
    const int g = sys->n_col + replica;
    cudaStream_t s = sys->stream;
    CK(cudaMemcpyAsync(sys->d.colX + 3 * g, X, sizeof(double) * 3, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sys->col_rc + g, &reach, sizeof(double), cudaMemcpyHostToDevice, s));
    ReplicaDev &rp = sys->rep[replica];
    rp.n_col = 1;
    rp.col_off = g;
    rp.net = replica;
    CK(cudaMemcpyAsync(const_cast<ReplicaDev *>(sys->d.rep) + replica, &rp, sizeof rp, cudaMemcpyHostToDevice, s));
    // working state of the near particles
    const size_t need = 80 * (size_t)std::max(sys->n_total, 1);
    if (sys->work_bytes < need) {
        CK(cudaStreamSynchronize(s));
        auto it = std::find(sys->allocs.begin(), sys->allocs.end(), sys->d.md_work);
        if (it != sys->allocs.end()) sys->allocs.erase(it);
        cudaFree(sys->d.md_work);
        sys->d.md_work = nullptr;
        unsigned char *w = nullptr;
        if ((st = dalloc(sys, &w, need)) != RMPCD_OK) return st;
        sys->d.md_work = w;
        sys->work_bytes = need;
    }
    CK(cudaStreamSynchronize(s));
    return RMPCD_OK;
}

rmpcd_status rmpcd_get_network(rmpcd_system *sys, int32_t replica, double *x, double *v, int32_t n_beads)
{
    if (!sys) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    const auto &H = sys->nets[replica];
    if (H.beads.empty()) return fail(sys, RMPCD_EINVAL, "replica %d has no network", replica);
    if (n_beads != (int)H.beads.size() || !x || !v)
        return fail(sys, RMPCD_EINVAL, "replica %d's network has %d beads", replica, (int)H.beads.size());
    const size_t o = 3 * (size_t)H.dev.bead_off;
    CK(cudaMemcpyAsync(x, sys->d.net_x + o, sizeof(double) * 3 * n_beads, cudaMemcpyDeviceToHost, sys->stream));
    CK(cudaMemcpyAsync(v, sys->d.net_v + o, sizeof(double) * 3 * n_beads, cudaMemcpyDeviceToHost, sys->stream));
    return check_errors(sys);
}

rmpcd_status rmpcd_set_body(rmpcd_system *sys, int32_t replica, const rmpcd_body *body, const rmpcd_bead *beads)
{
    if (!sys) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    if (!body || !beads) return fail(sys, RMPCD_EINVAL, "body and beads are required");
    const rmpcd_params &p = sys->params[replica];
    if (p.n_colloids != 0 || p.n_bonds != 0 || p.walls || !sys->nets[replica].beads.empty())
        return fail(sys, RMPCD_EINVAL, "replica %d: a body needs a replica created with no colloids, bonds, walls or network",
                    replica);
    const int nb = body->n_beads;
    if (nb < 1 || nb > RMPCD_MAX_BEADS) return fail(sys, RMPCD_EINVAL, "n_beads %d not in [1,%d]", nb, RMPCD_MAX_BEADS);
    const double mb = body->bead_mass, sig = body->sigma;
    if (!(mb > 0.0) || !(sig > 0.0) || !std::isfinite(mb) || !std::isfinite(sig))
        return fail(sys, RMPCD_EINVAL, "bead_mass and sigma must be finite and > 0");
    bool fin = true;
    for (int k = 0; k < 3; ++k) fin = fin && std::isfinite(body->x[k]) && std::isfinite(body->v[k]) && std::isfinite(body->l[k]);
    for (int k = 0; k < 4; ++k) fin = fin && std::isfinite(body->q[k]);
    if (!fin) return fail(sys, RMPCD_EINVAL, "body state not finite");
    const double qn = body->q[0] * body->q[0] + body->q[1] * body->q[1] + body->q[2] * body->q[2] + body->q[3] * body->q[3];
    if (!(fabs(qn - 1.0) <= 1e-9)) return fail(sys, RMPCD_EINVAL, "q must be a unit quaternion");
    // mass, principal moments and reach, computed as the FP64 definition does
    double I[3] = {0.0, 0.0, 0.0}, off[3] = {0.0, 0.0, 0.0}, sum[3] = {0.0, 0.0, 0.0}, bmax = 0.0;
    for (int j = 0; j < nb; ++j) {
        const double *b = beads[j].b;
        if (!std::isfinite(b[0]) || !std::isfinite(b[1]) || !std::isfinite(b[2]) || !std::isfinite(beads[j].eps_A) ||
            !std::isfinite(beads[j].eps_B) || beads[j].eps_A < 0.0 || beads[j].eps_B < 0.0)
            return fail(sys, RMPCD_EINVAL, "bead %d: position and epsilons must be finite, epsilons >= 0", j);
        I[0] = I[0] + mb * (b[1] * b[1] + b[2] * b[2]);
        I[1] = I[1] + mb * (b[2] * b[2] + b[0] * b[0]);
        I[2] = I[2] + mb * (b[0] * b[0] + b[1] * b[1]);
        off[0] += mb * b[0] * b[1];
        off[1] += mb * b[0] * b[2];
        off[2] += mb * b[1] * b[2];
        for (int k = 0; k < 3; ++k) sum[k] += b[k];
        const double r = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        if (r > bmax) bmax = r;
    }
    if (!(I[0] > 0.0 && I[1] > 0.0 && I[2] > 0.0)) return fail(sys, RMPCD_EINVAL, "principal moments must be > 0");
    for (int k = 0; k < 3; ++k) {
        if (!(fabs(sum[k]) <= 1e-9 * nb * bmax)) return fail(sys, RMPCD_EINVAL, "beads are not centred on the centre of mass");
        if (!(fabs(off[k]) <= 1e-9 * (I[0] + I[1] + I[2])))
            return fail(sys, RMPCD_EINVAL, "beads are not in the principal frame (off-diagonal inertia)");
    }
    const double rc2 = sig * sig * cbrt(2.0);
    const double reach = bmax + sqrt(rc2);
    if (2.0 * reach + 2.0 * p.skin >= (double)std::min(p.L[0], std::min(p.L[1], p.L[2])))
        return fail(sys, RMPCD_EINVAL, "replica %d: box too small for the body's reach", replica);

    rmpcd_status st = unprime(sys);
    if (st != RMPCD_OK) return st;
    CK(cudaStreamSynchronize(sys->stream));
    drop_graphs(sys);
    // the other bodies' state lives on the device
    std::vector<BodyDev> all(sys->n_rep);
    CK(cudaMemcpy(all.data(), sys->d.body, sizeof(BodyDev) * sys->n_rep, cudaMemcpyDeviceToHost));
    for (int r = 0; r < sys->n_rep; ++r)
        if (!sys->bodies[r].beads.empty()) {
            BodyDev &D = sys->bodies[r].dev;
            for (int k = 0; k < 3; ++k) { D.X[k] = all[r].X[k]; D.V[k] = all[r].V[k]; D.l[k] = all[r].l[k]; }
            for (int k = 0; k < 4; ++k) D.q[k] = all[r].q[k];
        }
    rmpcd_system::BodyHost &H = sys->bodies[replica];
    H.b = *body;
    H.beads.assign(beads, beads + nb);
    BodyDev &D = H.dev;
    std::memset(&D, 0, sizeof D);
    for (int k = 0; k < 3; ++k) { D.X[k] = body->x[k]; D.V[k] = body->v[k]; D.l[k] = body->l[k]; D.I[k] = I[k]; }
    for (int k = 0; k < 4; ++k) D.q[k] = body->q[k];
    D.M = (double)nb * mb;
    D.sigma = sig;
    D.rc2 = rc2;
    D.reach = reach;
    D.sigma_f = (float)sig;
    D.rc2_f = (float)rc2;
    D.nb = nb;
    build_body_grid(H);
    if ((st = upload_bodies(sys)) != RMPCD_OK) return st;
    for (int r = 0; r < sys->n_rep; ++r) all[r] = sys->bodies[r].dev;
    CK(cudaMemcpyAsync(sys->d.body, all.data(), sizeof(BodyDev) * sys->n_rep, cudaMemcpyHostToDevice, sys->stream));

    // the body's colloid slot: centre and reach for the near-list test
    const int g = sys->n_col + replica;
    rmpcd_colloid c{};
    for (int k = 0; k < 3; ++k) { c.x[k] = body->x[k]; c.v[k] = body->v[k]; }
    int Xi[3], Ci[3];
    float Xf[3], Vf[3];
    split_colloid(c, p, Xi, Xf, Ci, Vf);
    const double gn = sqrt(p.g[0] * p.g[0] + p.g[1] * p.g[1] + p.g[2] * p.g[2]);
    const float rb = (float)(reach + 0.5 * gn * p.tau * p.tau + p.skin);
    cudaStream_t s = sys->stream;
    CK(cudaMemcpyAsync(sys->d.colX + 3 * g, c.x, sizeof(double) * 3, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sys->d.colV + 3 * g, c.v, sizeof(double) * 3, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sys->d.colXi + 3 * g, Xi, sizeof Xi, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sys->d.colXf + 3 * g, Xf, sizeof Xf, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sys->d.colCi + 3 * g, Ci, sizeof Ci, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sys->d.colVf + 3 * g, Vf, sizeof Vf, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sys->col_rc + g, &reach, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sys->col_rb + g, &rb, sizeof(float), cudaMemcpyHostToDevice, s));
    ReplicaDev &rp = sys->rep[replica];
    rp.n_col = 1;
    rp.col_off = g;
    rp.body = replica;
    CK(cudaMemcpyAsync(const_cast<ReplicaDev *>(sys->d.rep) + replica, &rp, sizeof rp, cudaMemcpyHostToDevice, s));
    // working state of the near particles (the mixed body kernel keeps its
    // per-sub-step list of particles in reach of a bead past its 32-byte records)
    const size_t need = (sys->mixed ? 64 : 80) * (size_t)std::max(sys->n_total, 1);
    if (sys->work_bytes < need) {
        CK(cudaStreamSynchronize(s));
        auto it = std::find(sys->allocs.begin(), sys->allocs.end(), sys->d.md_work);
        if (it != sys->allocs.end()) sys->allocs.erase(it);
        cudaFree(sys->d.md_work);
        sys->d.md_work = nullptr;
        unsigned char *w = nullptr;
        if ((st = dalloc(sys, &w, need)) != RMPCD_OK) return st;
        sys->d.md_work = w;
        sys->work_bytes = need;
    }
    CK(prepare_md_body(sys->mixed, sys->nb_max, sys->grid_room));
    sys->any_body = true;
    CK(cudaStreamSynchronize(s));
    return RMPCD_OK;
}

rmpcd_status rmpcd_get_body(rmpcd_system *sys, int32_t replica, rmpcd_body *out)
{
    if (!sys || !out) return RMPCD_EINVAL;
    if (replica < 0 || replica >= sys->n_rep) return fail(sys, RMPCD_EINVAL, "replica %d out of range", replica);
    const rmpcd_system::BodyHost &H = sys->bodies[replica];
    if (H.beads.empty()) return fail(sys, RMPCD_EINVAL, "replica %d has no body", replica);
    BodyDev D;
    CK(cudaMemcpyAsync(&D, sys->d.body + replica, sizeof D, cudaMemcpyDeviceToHost, sys->stream));
    rmpcd_status st = check_errors(sys);
    *out = H.b;
    for (int k = 0; k < 3; ++k) { out->x[k] = D.X[k]; out->v[k] = D.V[k]; out->l[k] = D.l[k]; }
    for (int k = 0; k < 4; ++k) out->q[k] = D.q[k];
    return st;
}

}  // extern "C"
