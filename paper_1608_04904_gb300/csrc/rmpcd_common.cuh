// rmpcd_common.cuh -- device data layout and per-particle arithmetic shared by
// the sm_103a kernels of the MPCD collision-interval update.
//
// Method: de Buyl, Huang & Deprez, RMPCDMD (arXiv:1608.04904), §1.1 and §1.4.
// Units: cell side 1, solvent mass 1.
//
// Two storage precisions:
//   mixed: 32-byte record {packed integer cell (10/10/10 bits), FP32 offset in
//          the cell [0,1)^3, FP32 velocity, id+flags}; arithmetic in FP32.
//   fp64 : 64-byte record {FP64 position, id+flags, FP64 velocity}.
// The id+flags word holds the particle id in bits 0..28 and the flags
// B (species), TAG (inside a catalytic range) and PROP (already moved through
// the current interval by the MD kernel) in bits 29..31.
//
// FP64 arithmetic is written with explicit fma() where a fused multiply-add is
// meant and is compiled with --fmad=false, so every other product and sum is
// rounded where written.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rmpcd {

constexpr int CPT = 128;           // cells per tile of the cell pass
constexpr int PROF_MAX_BINS = 512; // most bins of one slab profile
constexpr int PROF_FIELDS = 8;     // count, B count, sum v_k (3), sum v_k^2 (3)
constexpr int CP_THREADS = 256;    // threads per cell-pass CTA
constexpr int CP_WARPS = CP_THREADS / 32;
constexpr int CP_STAGE_M = 6;      // particles a cell-pass thread stages at once (mixed records)
constexpr int CP_STAGE_D = 6;      // particles a cell-pass thread stages at once (fp64 records)
constexpr int CP_MAX_CAP = 768;    // largest bucket_cap
constexpr int CP_MAX_CELL = 1536;  // most particles one cell may hold (the cell pass stages a cell at once)
constexpr int CP_NEAR_CAND_MIN = 5;   // colloids from which the mixed cell pass filters them per batch
constexpr int MD_THREADS = 1024;   // threads of the near-field MD CTA (one per replica)
constexpr int MAXC = 64;           // colloids per replica handled by the MD CTA
constexpr int MAXB = 16;           // bonds per replica
constexpr int MAXBEADS = 1024;     // beads of a rigid body

constexpr uint32_t F_B = 1u << 29;
constexpr uint32_t F_TAG = 1u << 30;
constexpr uint32_t F_PROP = 1u << 31;
constexpr uint32_t ID_MASK = (1u << 29) - 1u;

enum Purpose : uint32_t { P_SHIFT = 1, P_ROT = 2, P_REACT = 3, P_THERMO = 4, P_VIRT = 5, P_CAT = 6 };

enum ErrSlot { ERR_OVERFLOW = 0, ERR_SKIN = 1, ERR_TIMEOUT = 2, ERR_BOUNDS = 3, ERR_RATTLE = 4, ERR_COUNT = 8 };

// Per-replica constants, computed on the host once.
struct ReplicaDev {
    int L[3];
    int nz;                 // z layers of the shifted grid: L[2] + walls
    int walls, rho_wall, n_md, n_slabs;
    int n_part, part_off;   // solvent slots [part_off, part_off + n_part)
    int n_cells, cell_off;  // cells [cell_off, cell_off + n_cells), cell_off = CPT * tile_off
    int tile_off, n_tiles;
    int n_col, col_off, n_bond, bond_off;
    int bulk_on, has_g;
    int thr_off;
    int body;               // index of the replica's rigid bead body, -1: none
    int net;                // index of the replica's bead network (iterative RATTLE), -1: none
    double kT, tau, dt, hdt, ca, sa, omc;
    double g[3];
    double gnorm, cat_thr, skin;
    double slab_x0[4], slab_x1[4], slab_sd[4];
    int slab_lo[4], slab_hi[4];      // cx in slab k iff slab_lo <= cx < slab_hi
    int res_y[4];                    // species reservoirs: cy in [res_y[0], res_y[1]) -> A, [res_y[2], res_y[3]) -> B
    double cc_eps, cc_sigma, cc_rc;
    float tau_f, dt_f, hdt_f, ca_f, sa_f, omc_f;
    float g_f[3];
    float gnorm_f, skin_f;
    float slab_sd_f[4];
    unsigned long long seed;
};

struct BondDev { int a, b; double d; };

// A bead network of one replica (the Janus particle under iterative RATTLE):
// beads [bead_off, bead_off + nb) of the network arrays, links [link_off,
// link_off + nl) grouped by colour (colour c: links cs[c] .. cs[c + 1] of the
// colour starts at color_off), the beads' WCA sigma and cut-off^2, and the
// RATTLE tolerance and sweep bound.
struct NetDev {
    int nb, bead_off, nl, link_off, ncol, color_off, max_sweeps, pad;
    double sigma, rc2, tol;
};

// The replica constants the mixed per-particle code reads (flight, cell key,
// minimum image, near test), as a value the compiler keeps in registers: a
// reference into shared memory would be reloaded after every shared store.
struct HotM {
    int L[3];
    int nz, walls, has_g;
    float tau_f;
    float g_f[3];
};
__device__ __forceinline__ HotM hot_m(const ReplicaDev &rp)
{
    HotM h;
    for (int k = 0; k < 3; ++k) { h.L[k] = rp.L[k]; h.g_f[k] = rp.g_f[k]; }
    h.nz = rp.nz; h.walls = rp.walls; h.has_g = rp.has_g; h.tau_f = rp.tau_f;
    return h;
}

// A rigid bead body (the Janus particle): FP64 state, constants, and the
// body-frame lookup grid whose cell lists every bead that a particle in the
// cell can reach, in ascending bead order.
struct BodyDev {
    double X[3], V[3], q[4], l[3];   // centre of mass (unwrapped), its velocity,
                                     // orientation (w, x, y, z), body-frame angular momentum
    double M, I[3];                  // mass, principal moments
    double sigma, rc2, reach;        // bead WCA sigma, cut-off^2, max|b| + cut-off
    float sigma_f, rc2_f;
    float glo, ginv;                 // grid cell of body-frame u: floor((u - glo) ginv) per axis
    int gn;                          // grid cells per axis
    int nb;                          // beads [bead_off, bead_off + nb)
    int bead_off;
    int gstart_off;                  // gn^3 + 1 list offsets at grid_start + gstart_off
    int glist_off;                   // list entries at grid_list + glist_off
    int pad;
};

// Device-resident interval control: the collision index of the next fused
// interval and the launch counter of the cell pass (ticket parity and
// look-back tag).  Kernels launched with step == STEP_DEVICE read the step
// here; the cell pass advances both, so a captured CUDA graph of intervals
// replays without any argument update.
struct Ctl {
    uint32_t step;
    uint32_t epoch;
};
constexpr uint32_t STEP_DEVICE = 0xFFFFFFFFu;

// Grid-wide scratch of the wide MD kernel: force accumulators of three
// consecutive rounds and the grid barrier.
struct MdWideGlobal {
    unsigned long long acc[3][MAXC * 3];
    unsigned int count, gen;
};

// All device pointers of a system (passed by value to every kernel).
//
// Two layouts hold the solvent.  The flat one (rec[]) keeps every replica's
// records in slots [part_off, part_off + n_part), sorted by the cells of a
// collision after a sorting pass; the granular calls, the state transfers and
// the observables work on it, through index buckets (bucket[]: slot numbers
// per cell).  The fused run keeps the records themselves in per-cell rows
// (brec[]: row `cell` holds that cell's records at [cell * cap, cell * cap +
// count)), so that a collision reads each cell's particles contiguously and
// writes each particle's record straight into the row of its next cell; the
// particles near a colloid wait in near_rec for the MD kernel, which then bins
// them into the rows.  bucket[b] and brec[b] share memory (one layout is in
// use at a time).
struct Dev {
    const ReplicaDev *rep;
    const int *tile_rep;         // tile -> replica
    void *rec[2];                // flat solvent records, double buffered
    int *count[2];               // particles per cell, double buffered
    int *bucket[2];              // flat layout: [cell * cap + rank] -> storage slot
    void *brec[2];               // fused run: [cell * cap + rank] -> record (same memory as bucket[b])
    int2 *ovf[2];                // entries past cap: (cell, slot) (flat layout) or (cell, index into orec)
    void *orec[2];               // fused run: records of the overflow entries
    unsigned int *ovf_n;         // [2]: entries appended to ovf[b] (reset by the pass that consumes b)
    void *near_rec;              // records of the near particles, per replica [part_off, part_off + near_count)
    int *near_list;              // per replica: flat slot of each near particle (granular interval)
    int *near_count;             // [n_rep]
    unsigned long long *tile_state;  // decoupled look-back, one word per tile
    unsigned int *ticket;        // [4]: tile tickets, finished CTAs (per launch parity)
    unsigned int *err;           // [ERR_COUNT]
    double *obs_part;            // [n_tiles][8]
    double *obs_out;             // [n_rep][8]
    const unsigned long long *bulk_thr;   // per replica [cap + 1]: accept iff draw < thr[N_B]
    double *colX, *colV;         // fp64 path: [n_col_total * 3], unwrapped
    int *colXi, *colCi;          // mixed path: unwrapped / wrapped integer cell [3n]
    float *colXf, *colVf;        // mixed path: FP32 offset in the cell, velocity [3n]
    const double *colM, *colSig, *colEpsA, *colEpsB, *colRc2, *colRc;
    const float *colSig_f, *colEpsA_f, *colEpsB_f, *colRc2_f, *colRc_f;
    const float *colRb_f;        // r_c + |g| tau^2 / 2 + skin (near-list radius without |v| tau)
    const float *colInvM_f;      // 1 / mass
    const int *colCat;
    const BondDev *bonds;
    void *md_work;               // near-particle working state
    void *md_col_save;           // per replica: colloid state between the calls of a sub-stepped interval
    MdWideGlobal *md_wide;       // wide MD kernel scratch
    Ctl *ctl;                    // interval control (step, cell-pass launch counter)
    unsigned int *maxcnt;        // largest cell count seen (bucket-width tuner)
    NetDev *net;                 // bead networks
    double *net_x, *net_v;       // [3 * bead] network bead positions (unwrapped), velocities
    const double *net_m, *net_eps;   // [bead], [2 * bead] (eps_A, eps_B)
    const int *net_cat;          // [bead]
    const int *net_la, *net_lb;  // [link] bead indices within the network, grouped by colour
    const double *net_d;         // [link] lengths
    const int *net_cs;           // colour starts per network
    BodyDev *body;               // rigid bead bodies
    const double *bead_b;        // [3 * bead] body-frame bead positions
    const double *bead_eps;      // [2 * bead] eps_A, eps_B
    const float *bead_eps_f;
    const int *bead_cat;
    const int *grid_start;       // lookup-grid list offsets
    const unsigned short *grid_list;
    int cap;
    int ovf_cap;                 // entries each overflow list holds
    int lb_limit;                // polls before a look-back wait gives up (ERR_TIMEOUT)
    int lb_stall;                // test hook: the look-back treats every predecessor as not ready
    const int *cell_rank;        // Hilbert order: place of cell key k of a replica at cell_off + k (NULL: linear)
    const int *cell_key;         //   and the key of the cell at place cell_off + p
    int many_col;                // 1: some replica has >= CP_NEAR_CAND_MIN colloids
    int n_rep;
    int n_tiles;
    int n_total;
};

// Where the cells live: the row (and tile place) of the cell with key k of
// a replica whose cells start at cell_off -- k itself in linear order, its
// compact Hilbert rank in Hilbert order -- and the key of the cell at a
// place.  A cell's draws and geometry always use its key.
__device__ __forceinline__ int bin_cell(const Dev &d, int cell_off, int key)
{
    return cell_off + (d.cell_rank ? __ldg(d.cell_rank + cell_off + key) : key);
}
__device__ __forceinline__ int cell_key_at(const Dev &d, int cell_off, int place)
{
    return d.cell_key ? __ldg(d.cell_key + cell_off + place) : place;
}

__device__ __forceinline__ uint32_t resolve_step(const Dev &d, uint32_t step)
{
    return step == STEP_DEVICE ? *(volatile const uint32_t *)&d.ctl->step : step;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of the
// multiply-xor bijection with a Weyl key schedule.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     unsigned long long seed)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// 24-bit uniform in [0,1), exact in FP32 and FP64.
__device__ __forceinline__ double u24d(uint32_t b) { return (double)(b >> 8) * 0x1p-24; }
__device__ __forceinline__ float u24f(uint32_t b) { return (float)(b >> 8) * 0x1p-24f; }

// Random grid shift of one collision (§1.4): s uniform in [0,1)^3.
__device__ __forceinline__ void grid_shift(unsigned long long seed, uint32_t step, double s[3])
{
    U4 w = philox(0u, step, P_SHIFT, 0u, seed);
    s[0] = u24d(w.x); s[1] = u24d(w.y); s[2] = u24d(w.z);
}
// The same shift in FP32 (exact: 24-bit uniforms).
__device__ __forceinline__ void grid_shift(unsigned long long seed, uint32_t step, float s[3])
{
    U4 w = philox(0u, step, P_SHIFT, 0u, seed);
    s[0] = u24f(w.x); s[1] = u24f(w.y); s[2] = u24f(w.z);
}

// x as R with one rounding, for |x| <= 2^48: hi 2^24 + lo with both parts
// exact in FP32 and FP64, summed by one fma (64-bit integer conversions take
// several times as long on this GPU).
__device__ __forceinline__ float exact_to_R(long long x, float)
{
    return fmaf((float)(int)(x >> 24), 0x1p24f, (float)(int)(x & 0xFFFFFF));
}
__device__ __forceinline__ double exact_to_R(long long x, double)
{
    return fma((double)(int)(x >> 24), 0x1p24, (double)(int)(x & 0xFFFFFF));
}

// One Marsaglia (1972) attempt for the rotation axis: two candidate pairs
// from the four words of a draw; true and n set when one is accepted.  The
// acceptance test is exact integer arithmetic.
template <typename R>
__device__ __forceinline__ bool axis_attempt(const U4 &w, R n[3])
{
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int pair = 0; pair < 2; ++pair) {
        const int A = 2 * (int)(ws[2 * pair] >> 8) + 1 - (1 << 24);
        const int B = 2 * (int)(ws[2 * pair + 1] >> 8) + 1 - (1 << 24);
        const long long S = (long long)A * A + (long long)B * B;
        if (S < (1ll << 48)) {
            // 1 - s and 1 - 2s are formed as exact integers before the one
            // rounding to R: no cancellation near the poles in FP32, and in
            // FP64 the same values as (1 - s), (1 - 2 s) computed directly.
            const R a = (R)A * (R)0x1p-24;
            const R b = (R)B * (R)0x1p-24;
            const R q = sqrt(exact_to_R((1ll << 48) - S, R(0)) * (R)0x1p-48);
            n[0] = R(2) * a * q;
            n[1] = R(2) * b * q;
            n[2] = exact_to_R((1ll << 48) - 2 * S, R(0)) * (R)0x1p-48;
            return true;
        }
    }
    return false;
}

// Uniform point on the unit sphere (Marsaglia 1972) for the rotation axis of
// one cell; the acceptance test is exact integer arithmetic.
template <typename R>
__device__ __forceinline__ void rotation_axis(unsigned long long seed, uint32_t step, uint32_t cell, R n[3])
{
    for (uint32_t attempt = 0; attempt < 16u; ++attempt)
        if (axis_attempt(philox(cell, step, P_ROT, attempt, seed), n)) return;
    n[0] = R(0); n[1] = R(0); n[2] = R(1);
}
// The same, given the first attempt's draw w0 = philox(cell, step, P_ROT, 0).
template <typename R>
__device__ __forceinline__ void rotation_axis_from(unsigned long long seed, uint32_t step, uint32_t cell, const U4 &w0,
                                                   R n[3])
{
    if (axis_attempt(w0, n)) return;
    for (uint32_t attempt = 1; attempt < 16u; ++attempt)
        if (axis_attempt(philox(cell, step, P_ROT, attempt, seed), n)) return;
    n[0] = R(0); n[1] = R(0); n[2] = R(1);
}

// Box-Muller pair from two words, u1 in (0,1], u2 in [0,1).
__device__ __forceinline__ void box_muller(uint32_t b0, uint32_t b1, double &g0, double &g1)
{
    double u1 = (double)((b0 >> 8) + 1u) * 0x1p-24;
    double u2 = (double)(b1 >> 8) * 0x1p-24;
    double r = sqrt(-2.0 * log(u1));
    double ph = 6.283185307179586 * u2;
    double sn, cs;
    sincos(ph, &sn, &cs);
    g0 = r * cs;
    g1 = r * sn;
}
__device__ __forceinline__ void box_muller(uint32_t b0, uint32_t b1, float &g0, float &g1)
{
    float u1 = (float)((b0 >> 8) + 1u) * 0x1p-24f;
    float u2 = (float)(b1 >> 8) * 0x1p-24f;
    float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    g0 = r * cs;
    g1 = r * sn;
}

// ---------------------------------------------------------------------------
// Records.
// ---------------------------------------------------------------------------
struct __align__(16) RecM {
    uint32_t cw;        // cx | cy << 10 | cz << 20
    float o[3];         // offset in the cell
    float v[3];
    uint32_t fid;       // id | flags
};
struct __align__(16) RecD {
    double x[3];
    uint32_t fid;
    uint32_t u0;
    double v[3];
    double u1;
};
static_assert(sizeof(RecM) == 32, "mixed record is one 32-byte sector");
static_assert(sizeof(RecD) == 64, "fp64 record is two 32-byte sectors");

// A mixed record is one 32-byte sector, moved by one 256-bit access (every
// record array is 32-byte aligned): one request per record instead of two
// half-sector ones.
__device__ __forceinline__ RecM load_rec(const RecM *p)
{
    unsigned a[8];
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7])
                 : "l"(p));
    RecM r;
    r.cw = a[0]; r.o[0] = __uint_as_float(a[1]); r.o[1] = __uint_as_float(a[2]); r.o[2] = __uint_as_float(a[3]);
    r.v[0] = __uint_as_float(a[4]); r.v[1] = __uint_as_float(a[5]); r.v[2] = __uint_as_float(a[6]); r.fid = a[7];
    return r;
}
__device__ __forceinline__ void store_rec(RecM *p, const RecM &r)
{
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(r.cw), "r"(__float_as_uint(r.o[0])),
                 "r"(__float_as_uint(r.o[1])), "r"(__float_as_uint(r.o[2])), "r"(__float_as_uint(r.v[0])),
                 "r"(__float_as_uint(r.v[1])), "r"(__float_as_uint(r.v[2])), "r"(r.fid)
                 : "memory");
}
__device__ __forceinline__ RecD load_rec(const RecD *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
    RecD r;
    r.x[0] = a.x; r.x[1] = a.y; r.x[2] = b.x;
    unsigned long long w = (unsigned long long)__double_as_longlong(b.y);
    r.fid = (uint32_t)w; r.u0 = (uint32_t)(w >> 32);
    r.v[0] = c.x; r.v[1] = c.y; r.v[2] = d.x; r.u1 = d.y;
    return r;
}
__device__ __forceinline__ void store_rec(RecD *p, const RecD &r)
{
    double2 *q = reinterpret_cast<double2 *>(p);
    unsigned long long w = (unsigned long long)r.fid | ((unsigned long long)r.u0 << 32);
    q[0] = make_double2(r.x[0], r.x[1]);
    q[1] = make_double2(r.x[2], __longlong_as_double((long long)w));
    q[2] = make_double2(r.v[0], r.v[1]);
    q[3] = make_double2(r.v[2], 0.0);
}

__device__ __forceinline__ int cw_get(uint32_t cw, int d) { return (int)((cw >> (10 * d)) & 1023u); }
__device__ __forceinline__ uint32_t cw_make(int cx, int cy, int cz)
{
    return (uint32_t)cx | ((uint32_t)cy << 10) | ((uint32_t)cz << 20);
}
__device__ __forceinline__ int imod(int a, int L) { int m = a % L; return m < 0 ? m + L : m; }
// a mod L for a within one box of [0, L) (the usual case: two selects); any
// other a takes the integer division.
__device__ __forceinline__ int wrap_cell(int a, int L)
{
    a = a >= L ? a - L : a;
    a = a < 0 ? a + L : a;
    if ((unsigned)a >= (unsigned)L) a = imod(a, L);
    return a;
}

// ---------------------------------------------------------------------------
// Free flight over time t (§1.1 streaming; §1.4 constant acceleration).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fly_d(const ReplicaDev &rp, double x[3], double v[3], double t)
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        x[d] = fma(v[d], t, x[d]);
        if (rp.has_g) {
            x[d] = x[d] + 0.5 * rp.g[d] * t * t;
            v[d] = v[d] + rp.g[d] * t;
        }
    }
}

__device__ __forceinline__ void wrap_periodic_d(const ReplicaDev &rp, double x[3])
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d == 2 && rp.walls) continue;
        double L = (double)rp.L[d];
        if (x[d] >= L) x[d] = x[d] - L;
        else if (x[d] < 0.0) { x[d] = x[d] + L; if (x[d] >= L) x[d] = 0.0; }
    }
}

// Flight over tau with stick walls at z = 0, L[2] (bounce-back: the whole
// velocity reverses at the wall) or periodic boundaries.
__device__ __forceinline__ void flight_d(const ReplicaDev &rp, double x[3], double v[3])
{
    if (!rp.walls) { fly_d(rp, x, v, rp.tau); wrap_periodic_d(rp, x); return; }
    double Lz = (double)rp.L[2];
    double zend = fma(v[2], rp.tau, x[2]);
    double th = -1.0, wall = 0.0;
    if (zend < 0.0) { th = -x[2] / v[2]; wall = 0.0; }
    else if (zend > Lz) { th = (Lz - x[2]) / v[2]; wall = Lz; }
    if (th < 0.0) {
        fly_d(rp, x, v, rp.tau);
    } else {
        fly_d(rp, x, v, th);
        x[2] = wall;
        v[0] = -v[0]; v[1] = -v[1]; v[2] = -v[2];
        fly_d(rp, x, v, rp.tau - th);
        if (x[2] < 0.0) x[2] = 0.0;
        if (x[2] > Lz) x[2] = Lz;
    }
    wrap_periodic_d(rp, x);
}

// Mixed precision: position = integer cell + FP32 offset.  Renormalise the
// offset to [0,1) and carry into the cell index (periodic axes wrap).
template <class P>
__device__ __forceinline__ void renorm_m(const P &rp, int c[3], float o[3])
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float fl = floorf(o[d]);
        c[d] += (int)fl;
        o[d] = o[d] - fl;
        if (o[d] >= 1.0f) { o[d] = 0.0f; c[d] += 1; }
        if (d == 2 && rp.walls) {
            if (c[2] < 0) { c[2] = 0; o[2] = 0.0f; }
            if (c[2] > rp.L[2] - 1) { c[2] = rp.L[2] - 1; o[2] = 1.0f; }
        } else {
            c[d] = wrap_cell(c[d], rp.L[d]);
        }
    }
}

template <class P>
__device__ __forceinline__ void fly_m(const P &rp, float o[3], float v[3], float t)
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        o[d] = fmaf(v[d], t, o[d]);
        if (rp.has_g) {
            o[d] = o[d] + 0.5f * rp.g_f[d] * t * t;
            v[d] = v[d] + rp.g_f[d] * t;
        }
    }
}

template <class P>
__device__ __forceinline__ void flight_m(const P &rp, int c[3], float o[3], float v[3])
{
    const float tau = rp.tau_f;
    if (rp.walls) {
        // distance to the wall the particle moves towards, from the nearby cell
        float th = -1.0f;
        int hit = 0;
        if (v[2] < 0.0f) {
            float dist = (float)c[2] + o[2];
            if (v[2] * tau < -dist) { th = dist / -v[2]; hit = 1; }
        } else if (v[2] > 0.0f) {
            float dist = (float)(rp.L[2] - 1 - c[2]) + (1.0f - o[2]);
            if (v[2] * tau > dist) { th = dist / v[2]; hit = 2; }
        }
        if (hit) {
            fly_m(rp, o, v, th);
            if (hit == 1) { c[2] = 0; o[2] = 0.0f; } else { c[2] = rp.L[2] - 1; o[2] = 1.0f; }
            v[0] = -v[0]; v[1] = -v[1]; v[2] = -v[2];
            fly_m(rp, o, v, tau - th);
            renorm_m(rp, c, o);
            return;
        }
    }
    fly_m(rp, o, v, tau);
    renorm_m(rp, c, o);
}

// ---------------------------------------------------------------------------
// Cell key on the grid shifted by s (x fastest); walls add one z layer.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_key_d(const ReplicaDev &rp, const double x[3], const double s[3])
{
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double f = floor(x[d] - s[d]);
        if (d == 2 && rp.walls) {
            long long k = (long long)f + 1;
            if (k < 0) k = 0;
            if (k > rp.nz - 1) k = rp.nz - 1;
            c[d] = (int)k;
        } else if (f >= -1.0 && f < (double)rp.L[d]) {
            c[d] = wrap_cell((int)f, rp.L[d]);
        } else {
            long long k = (long long)f % rp.L[d];
            if (k < 0) k += rp.L[d];
            c[d] = (int)k;
        }
    }
    return c[0] + rp.L[0] * (c[1] + rp.L[1] * c[2]);
}

template <class P>
__device__ __forceinline__ int cell_key_m(const P &rp, const int cc[3], const float o[3], const float s[3])
{
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int k = cc[d] + (int)floorf(o[d] - s[d]);   // exact: the sign of o - s is exact
        if (d == 2 && rp.walls) {
            k += 1;
            if (k < 0) k = 0;
            if (k > rp.nz - 1) k = rp.nz - 1;
        } else {
            k = wrap_cell(k, rp.L[d]);
        }
        c[d] = k;
    }
    return c[0] + rp.L[0] * (c[1] + rp.L[1] * c[2]);
}

// Minimum image along periodic axes, |d| < 1.5 L assumed.
template <typename R, class P>
__device__ __forceinline__ void min_image(const P &rp, R d[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (k == 2 && rp.walls) continue;
        R L = (R)rp.L[k];
        if (d[k] > R(0.5) * L) d[k] = d[k] - L;
        else if (d[k] < -R(0.5) * L) d[k] = d[k] + L;
    }
}

__device__ __forceinline__ void wrapped_colloid(const ReplicaDev &rp, const double *X, double out[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double L = (double)rp.L[k];
        out[k] = X[k] - L * floor(X[k] / L);
    }
}

// ---------------------------------------------------------------------------
// Cell rows: place r of global cell g is element g * cap + r.  A cell's
// records are contiguous, so the consecutive particles a warp stages (a few
// cells' worth) are a few contiguous runs: each load instruction touches few
// lines.  (Measured: a plane-major order within a tile, place r of a tile's
// cells contiguous, was 5 % slower for the uncoalesced loads it makes.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long row_index(const Dev &d, long long g, int r)
{
    return g * d.cap + r;
}

// ---------------------------------------------------------------------------
// Bins: one particle into its cell.  The first bucket_cap entries of a cell go
// to its bucket row; the rest are appended to the buffer's overflow list,
// which the cell pass reads for the cells that need it.  A full overflow list
// raises ERR_OVERFLOW (the entry is dropped; the step is then invalid).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bin_store(const Dev &d, int buf, int gcell, int r, int slot)
{
    if (r < d.cap) {
        d.bucket[buf][row_index(d, gcell, r)] = slot;
    } else {
        const unsigned k = atomicAdd(&d.ovf_n[buf], 1u);
        if (k < (unsigned)d.ovf_cap) d.ovf[buf][k] = make_int2(gcell, slot);
        else atomicMax(&d.err[ERR_OVERFLOW], (unsigned int)(r + 1));
    }
}
__device__ __forceinline__ void bin_particle(const Dev &d, int buf, int gcell, int slot)
{
    bin_store(d, buf, gcell, atomicAdd(&d.count[buf][gcell], 1), slot);
}

// Fused run: the record of a particle that takes place r of cell gcell (its
// count before this particle) into the cell's row, or past cap into the
// overflow records.  A full overflow list raises ERR_OVERFLOW.
template <class Rec>
__device__ __forceinline__ void bin_record_at(const Dev &d, int buf, int gcell, int r, const Rec &rec)
{
    if (r < d.cap) {
        store_rec(reinterpret_cast<Rec *>(d.brec[buf]) + row_index(d, gcell, r), rec);
    } else {
        const unsigned k = atomicAdd(&d.ovf_n[buf], 1u);
        if (k < (unsigned)d.ovf_cap) {
            store_rec(reinterpret_cast<Rec *>(d.orec[buf]) + k, rec);
            d.ovf[buf][k] = make_int2(gcell, (int)k);
        } else {
            atomicMax(&d.err[ERR_OVERFLOW], (unsigned int)(r + 1));
        }
    }
}
template <class Rec>
__device__ __forceinline__ void bin_record(const Dev &d, int buf, int gcell, const Rec &rec)
{
    bin_record_at(d, buf, gcell, atomicAdd(&d.count[buf][gcell], 1), rec);
}

// The record of near particle k of a replica (its copy in the near area).
template <class Rec>
__device__ __forceinline__ Rec load_near(const Dev &d, const ReplicaDev &rp, int k)
{
    return load_rec(reinterpret_cast<const Rec *>(d.near_rec) + rp.part_off + k);
}

// A near particle after its interval: binned into the rows of the collision
// ahead (fused run: do_bin) or written back to its flat slot (granular call).
template <class Rec>
__device__ __forceinline__ void put_near(const Dev &d, int rbuf, int bbuf, int do_bin, int gcell, int slot,
                                         const Rec &rec)
{
    if (do_bin) bin_record(d, bbuf, gcell, rec);
    else store_rec(reinterpret_cast<Rec *>(d.rec[rbuf]) + slot, rec);
}

// Near-colloid test of §1.4's Verlet-list radius: may this particle come
// within a colloid's cut-off during the interval?
__device__ __forceinline__ bool near_test_d(const Dev &d, const ReplicaDev &rp, const double x[3], const double v[3])
{
    double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int j = 0; j < rp.n_col; ++j) {
        const double *X = d.colX + 3 * (rp.col_off + j);
        double Xw[3];
        wrapped_colloid(rp, X, Xw);
        double dd[3] = {x[0] - Xw[0], x[1] - Xw[1], x[2] - Xw[2]};
        min_image(rp, dd);
        double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
        double R = d.colRc[rp.col_off + j] + speed * rp.tau + 0.5 * rp.gnorm * rp.tau * rp.tau + rp.skin;
        if (r2 < R * R) return true;
    }
    return false;
}

// Mixed path: colloids as wrapped integer cell Ci + FP32 offset Cf (stride 3),
// so the test needs no FP64 arithmetic.
template <class P>
__device__ __forceinline__ bool near_test_m(const P &rp, int nc, const int *Ci, const float *Cf,
                                            const float *Rb, const int c[3], const float o[3], const float v[3])
{
    const float st = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * rp.tau_f;
    for (int j = 0; j < nc; ++j) {
        float dd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) dd[k] = (float)(c[k] - Ci[3 * j + k]) + (o[k] - Cf[3 * j + k]);
        min_image(rp, dd);
        const float r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
        const float R = Rb[j] + st;
        if (r2 < R * R) return true;
    }
    return false;
}

// A tagged A particle that has left every catalytic range becomes B with
// probability cat_prob (§1.5); an A particle inside a range is tagged.
__device__ __forceinline__ uint32_t catalysis(const ReplicaDev &rp, uint32_t fid, bool inside, uint32_t step, int s)
{
    if (fid & F_B) return fid;
    if (inside) return fid | F_TAG;
    if (!(fid & F_TAG)) return fid;
    bool go = true;
    if (rp.cat_thr < 4294967296.0) {
        U4 w = philox(fid & ID_MASK, step, P_CAT, (uint32_t)s, rp.seed);
        go = (double)w.x < rp.cat_thr;
    }
    fid &= ~F_TAG;
    if (go) fid |= F_B;
    return fid;
}

// Mixed-path MD arithmetic shared by both MD kernels (so that they agree bit
// for bit).  Divisions on the sub-step's critical path use the hardware
// reciprocal (MUFU, within 2 ulp) rather than an IEEE division, which takes
// about twice as long on this GPU.
__device__ __forceinline__ float fdiv_m(float a, float b) { return __fdividef(a, b); }

// WCA force magnitude over distance, F(r) / r = 24 eps s^6 (2 s^6 - 1) / r^2
// with s^2 = sigma^2 / r^2 (§1.4), for r^2 inside the cut-off.
__device__ __forceinline__ float wca_fr_m(float eps, float sig, float r2)
{
    const float ir2 = fdiv_m(1.0f, r2);
    const float s2 = sig * sig * ir2;
    const float s6 = s2 * s2 * s2;
    return 24.0f * eps * s6 * (2.0f * s6 - 1.0f) * ir2;
}

// x 2^-40 of a 64-bit fixed-point force total as FP32, by two 32-bit
// conversions (within one unit in the last place of the correctly rounded
// value; a 64-bit conversion has several times the latency).
__device__ __forceinline__ float fixed40_to_float(long long x)
{
    const int hi = (int)(x >> 32);
    const unsigned lo = (unsigned)x;
    return fmaf((float)hi, 0x1p-8f, (float)lo * 0x1p-40f);
}

// Acquire / release accesses for the look-back scan.
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Tile base by decoupled look-back (Merrill & Garland 2016), run by one full
// warp: publishes the tile's aggregate (unless the caller already did, by
// tile_publish), inspects 32 predecessor tiles, then 128 at a time, summing aggregates
// back to the nearest inclusive prefix, publishes the tile's inclusive prefix
// and returns its exclusive prefix (in every lane).
// Tiles are taken in ticket order by resident CTAs, each finishing its tiles
// in that order, so every predecessor is held by a CTA that will publish it
// without waiting on this tile.  Words
// carry a 16-bit tag of the launch (never 0, the initial state), a 2-bit flag
// (1 aggregate, 2 inclusive prefix) and a 46-bit value.  A wait that runs out
// (d.lb_limit polls) sets ERR_TIMEOUT and returns a base that puts every write
// of the tile out of bounds.  d.lb_stall (a test hook) makes every predecessor
// read as not ready, a flag that nothing sets, so every wait runs out.
// ---------------------------------------------------------------------------
constexpr unsigned long long LB_VALUE_MASK = (1ull << 46) - 1ull;
constexpr int LB_SPIN_LIMIT = 1 << 22;   // default of Dev::lb_limit
constexpr int LB_W = 4;   // 32-tile windows the look-back inspects per round trip

__device__ __forceinline__ void tile_publish(const Dev &d, uint32_t epoch, int tile, int total)
{
    const unsigned long long ep = (unsigned long long)(epoch % 65535u) + 1ull;
    st_release(&d.tile_state[tile], (ep << 48) | (1ull << 46) | (unsigned long long)total);
}

__device__ __forceinline__ int tile_lookback(const Dev &d, uint32_t epoch, int tile, int total, int lane,
                                             bool publish = true)
{
    const unsigned long long ep = (unsigned long long)(epoch % 65535u) + 1ull;
    if (publish && lane == 0) tile_publish(d, epoch, tile, total);
    unsigned long long prefix = 0;
    int t = tile - 1;
    int spins = 0;
    bool ok = true;
    int nw = 1;   // windows per round: one first, LB_W once a scan has to go further back
    while (t >= 0) {
        // nw windows of 32 predecessors per round trip: position q = 32 u +
        // lane is tile t - q (windows beyond nw read as not ready)
        unsigned long long flag[LB_W], val[LB_W];
#pragma unroll
        for (int u = 0; u < LB_W; ++u) {
            const int idx = t - lane - 32 * u;
            flag[u] = u < nw ? 2ull : 0ull;   // before tile 0: inclusive prefix 0
            val[u] = 0ull;
            if (u < nw && idx >= 0) {
                const unsigned long long w = ld_acquire(&d.tile_state[idx]);
                flag[u] = ((w >> 48) == ep && !d.lb_stall) ? ((w >> 46) & 3ull) : 0ull;
                val[u] = w & LB_VALUE_MASK;
            }
        }
        // the nearest inclusive prefix, and every position up to it ready
        int first = -1;
        bool ready_all = true;
#pragma unroll
        for (int u = 0; u < LB_W; ++u) {
            if (u >= nw) break;
            const unsigned incl = __ballot_sync(0xffffffffu, flag[u] == 2ull);
            const unsigned ready = __ballot_sync(0xffffffffu, flag[u] != 0ull);
            if (first < 0) {
                if (incl) {
                    const int f = __ffs(incl) - 1;
                    const unsigned need = (f == 31) ? 0xffffffffu : ((2u << f) - 1u);
                    ready_all = ready_all && (ready & need) == need;
                    first = 32 * u + f;
                } else {
                    ready_all = ready_all && ready == 0xffffffffu;
                }
            }
        }
        if (!ready_all) {
            if (++spins > d.lb_limit) { ok = false; break; }
            __nanosleep(32);
            continue;
        }
        unsigned long long part = 0;
#pragma unroll
        for (int u = 0; u < LB_W; ++u)
            if (u < nw && (first < 0 || 32 * u + lane <= first)) part += val[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        prefix += __shfl_sync(0xffffffffu, part, 0);
        if (first >= 0) break;
        t -= 32 * nw;
        nw = LB_W;
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) prefix = 0x3FFFFFFFull;   // pushes every write of this tile out of bounds
    if (lane == 0) {
        if (!ok) atomicOr(&d.err[ERR_TIMEOUT], 1u);
        st_release(&d.tile_state[tile], (ep << 48) | (2ull << 46) | ((prefix + (unsigned long long)total) & LB_VALUE_MASK));
    }
    return (int)(prefix > 0x3FFFFFFFull ? 0x3FFFFFFF : prefix);
}

}  // namespace rmpcd
