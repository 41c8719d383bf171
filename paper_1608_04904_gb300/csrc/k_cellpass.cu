// k_cellpass.cu -- the per-cell pass of one collision (§1.4 of the RMPCDMD
// paper, arXiv:1608.04904): gather by cell, SRD / MPC-AT / virtual-particle
// collision, bulk B -> A reaction, and (fused run) free flight + binning of
// every particle for the next collision.
//
// The work is cut into tiles of CPT consecutive cells of one replica.  As many
// CTAs as fit on the GPU run persistently, each taking tiles in ticket order.
// A CTA stages a tile's particles in shared memory (in batches of whole cells
// when they exceed the staging area) in the order they arrive.  The result of
// a cell must not depend on that order:
//   FP64: the particles of each cell are ranked by id, the canonical order in
//     which the cell's velocities are summed (the order of the definition),
//     its reaction partner counted and (flat layout) its records written;
//   mixed: the cell's velocity sum is taken in units of 2^-24 as an integer
//     sum (exact in any order) and the reaction partner is found by comparing
//     ids, so the fused pass needs no ranks; MPC-AT cells (per-particle
//     draws), observable passes and the flat layout's write order still rank.
// Stages run with all threads of the CTA: one thread per particle for the
// gather, rotation, write and binning, one thread per cell for the cell sums
// and the per-cell draws.
//
// Two layouts (see Dev):
//   fused run (FUSED): a cell's records are read contiguously from its row;
//     each far particle's record is written into the row of the cell it will
//     occupy at the next collision (an atomic count gives its place), near
//     particles into the near area.  One read and one write of each record,
//     no index traffic, no global prefix: tiles are independent.
//   flat layout: records come from flat slots through index buckets and are
//     written to flat slots in canonical order; a tile's first slot is the
//     exclusive prefix of all earlier tiles' particle counts, found by a
//     single-pass decoupled look-back (Merrill & Garland 2016).
#include <algorithm>

#include "rmpcd_kernels.cuh"

namespace rmpcd {

template <bool MIXED> struct Traits;
template <> struct Traits<true> {
    using Rec = RecM;
    using R = float;
    static constexpr int K = CP_STAGE_M;        // staged particles per thread
    static constexpr int TP = K * CP_THREADS;
};
template <> struct Traits<false> {
    using Rec = RecD;
    using R = double;
    static constexpr int K = CP_STAGE_D;
    // 1408 64-byte records: a whole tile (1280 particles at density 10, the
    // Poisson tail included) in one batch, with two CTAs per SM
    static constexpr int TP = 1408;
    static_assert(TP <= K * CP_THREADS, "each thread stages at most K particles");
    static_assert(TP <= CP_MAX_CELL, "reaction thresholds cover every cell count");
};
static_assert(Traits<true>::TP <= CP_MAX_CELL, "reaction thresholds cover every cell count");

// --- per-record helpers ----------------------------------------------------
__device__ __forceinline__ void rec_flight(const HotM &rp, RecM &r)
{
    int c[3] = {cw_get(r.cw, 0), cw_get(r.cw, 1), cw_get(r.cw, 2)};
    flight_m(rp, c, r.o, r.v);
    r.cw = cw_make(c[0], c[1], c[2]);
}
__device__ __forceinline__ void rec_flight(const ReplicaDev &rp, RecD &r) { flight_d(rp, r.x, r.v); }

// s: the shift in FP64; sf: the same shift in FP32 (exact: 24-bit uniforms)
__device__ __forceinline__ int rec_key(const HotM &rp, const RecM &r, const double *, const float *sf)
{
    int c[3] = {cw_get(r.cw, 0), cw_get(r.cw, 1), cw_get(r.cw, 2)};
    return cell_key_m(rp, c, r.o, sf);
}
__device__ __forceinline__ int rec_key(const ReplicaDev &rp, const RecD &r, const double *s, const float *)
{
    return cell_key_d(rp, r.x, s);
}

// Colloid frames of the tile's replica, staged in shared memory (mixed path).
struct NearFrames {
    int Ci[3 * MAXC];
    float Cf[3 * MAXC];
    float Rb[MAXC];
};

// The near test of the mixed path over the colloids of a bit mask.
__device__ __forceinline__ bool near_test_mask(const HotM &rp, unsigned long long mask, const NearFrames &nf,
                                               const int c[3], const float o[3], const float v[3])
{
    const float st = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * rp.tau_f;
    for (; mask; mask &= mask - 1ull) {
        const int j = __ffsll((long long)mask) - 1;
        float dd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) dd[k] = (float)(c[k] - nf.Ci[3 * j + k]) + (o[k] - nf.Cf[3 * j + k]);
        min_image(rp, dd);
        const float r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
        const float R = nf.Rb[j] + st;
        if (r2 < R * R) return true;
    }
    return false;
}

__device__ __forceinline__ bool rec_near(const Dev &, const HotM &rp, int nc, const NearFrames &nf, const RecM &r)
{
    int c[3] = {cw_get(r.cw, 0), cw_get(r.cw, 1), cw_get(r.cw, 2)};
    return near_test_m(rp, nc, nf.Ci, nf.Cf, nf.Rb, c, r.o, r.v);
}
__device__ __forceinline__ bool rec_near(const Dev &d, const ReplicaDev &rp, int, const NearFrames &, const RecD &r)
{
    return near_test_d(d, rp, r.x, r.v);
}
// The many-colloid variant (mixed path): the batch's candidate colloids, or
// every colloid where the cell has no speed bound (all).
__device__ __forceinline__ bool rec_near_cand(const HotM &rp, int nc, const NearFrames &nf, const RecM &r,
                                              unsigned long long mask, bool all)
{
    int c[3] = {cw_get(r.cw, 0), cw_get(r.cw, 1), cw_get(r.cw, 2)};
    if (all) return near_test_m(rp, nc, nf.Ci, nf.Cf, nf.Rb, c, r.o, r.v);
    return near_test_mask(rp, mask, nf, c, r.o, r.v);
}
__device__ __forceinline__ bool rec_near_cand(const ReplicaDev &, int, const NearFrames &, const RecD &,
                                              unsigned long long, bool)
{
    return false;   // not used: the candidate path is the mixed path's
}

// What the per-particle loops read of the replica: a register copy for the
// mixed path, the shared-memory struct for the fp64 path.
template <bool MIXED> struct HotPick;
template <> struct HotPick<true> {
    static __device__ __forceinline__ const HotM &get(const ReplicaDev &, const HotM &h) { return h; }
};
template <> struct HotPick<false> {
    static __device__ __forceinline__ const ReplicaDev &get(const ReplicaDev &r, const HotM &) { return r; }
};

__device__ __forceinline__ float slab_sd(const ReplicaDev &rp, int k, float) { return rp.slab_sd_f[k]; }
__device__ __forceinline__ double slab_sd(const ReplicaDev &rp, int k, double) { return rp.slab_sd[k]; }
__device__ __forceinline__ float r_ca(const ReplicaDev &rp, float) { return rp.ca_f; }
__device__ __forceinline__ double r_ca(const ReplicaDev &rp, double) { return rp.ca; }
__device__ __forceinline__ float r_sa(const ReplicaDev &rp, float) { return rp.sa_f; }
__device__ __forceinline__ double r_sa(const ReplicaDev &rp, double) { return rp.sa; }
__device__ __forceinline__ float r_omc(const ReplicaDev &rp, float) { return rp.omc_f; }
__device__ __forceinline__ double r_omc(const ReplicaDev &rp, double) { return rp.omc; }

// 16-byte asynchronous copy global -> shared, cached in L2 only (every
// record is read once per pass).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
template <class Rec>
__device__ __forceinline__ void cp_async_rec(Rec *dst, const Rec *src)
{
#pragma unroll
    for (int q = 0; q < (int)(sizeof(Rec) / 16); ++q)
        cp_async16(reinterpret_cast<char *>(dst) + 16 * q, reinterpret_cast<const char *>(src) + 16 * q);
}

// v * 2^24 rounded to an integer, for any v: an integer part and a fraction,
// each converted exactly (adding an integer commutes with the rounding).
__device__ __forceinline__ long long fixed24(float v)
{
    if (fabsf(v) < 128.0f) return (long long)__float2int_rn(v * 0x1p24f);
    const float t = truncf(v);
    return ((long long)__float2int_rz(t) << 24) + (long long)__float2int_rn((v - t) * 0x1p24f);
}

// Staging place of the i-th particle of a cell of n in canonical order
// (clamped to the cell: a state with colliding ids leaves gaps in perm).
__device__ __forceinline__ int canon(const unsigned short *pm, int i, int n)
{
    const int q = pm[i];
    return q < n ? q : n - 1;
}

// Per-tile state shared by the threads of one CTA.
template <bool MIXED>
struct TileShared {
    using R = typename Traits<MIXED>::R;
    ReplicaDev rp;
    NearFrames nf;
    int tile, next_tile, r, base;
    uint32_t epoch, step;     // this launch's counter and collision index (from the control block)
    int cnt[CPT], ls[CPT + 1], wt[CPT / 32];
    int __align__(16) cnt_next[CPT];   // the next tile's counts (asynchronous copy during this tile)
    double sh[3], shn[3];     // fp64 path
    float shf[3], shnf[3];
    __align__(16) R vcm[CPT][4];   // [3]: padding (a cell's row is one 16-byte load on the mixed path)
    __align__(16) R ax[CPT][4];
    int react[CPT];
    unsigned char mode[CPT];    // bits 0-1: 0 untouched, 1 SRD rotation, 2 MPC-AT; 4: reservoir A, 8: reservoir B
    unsigned char mnear[CPT];   // 0: no particle of the cell can come near a colloid
    float vbc[CPT];   // bound on the cell's post-collision speeds (< 0: none, MPC-AT)
    unsigned long long cand;   // colloids that can reach the batch (many-colloid replicas)
    double red[CP_WARPS][8];
};

// Anderson thermostat (MPC-AT, §1.4) of one cell of n particles, the i-th in
// canonical order at v[pm[i]]: v_i <- v_cm + xi_i - <xi>, xi ~ N(0, kT_slab),
// with rho_wall - n virtual partners in v_cm when virt.  The per-cell momentum
// sums are FP64 on both paths; the Gaussian draws are in the path's precision R.
template <typename R, class Rec>
__device__ __forceinline__ void mpcat_cell(const ReplicaDev &rp, uint32_t step, uint32_t lc, int slab, int n,
                                           bool virt, Rec *v, const unsigned short *pm)
{
    double sum[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) sum[k] = sum[k] + (double)v[canon(pm, i, n)].v[k];
    double vcm[3];
    if (virt) {
        const int nv = rp.rho_wall - n;
        U4 w = philox(lc, step, P_VIRT, 0u, rp.seed);
        R g0, g1, g2, g3;
        box_muller(w.x, w.y, g0, g1);
        box_muller(w.z, w.w, g2, g3);
        const double sd = sqrt((double)nv * rp.kT);
        const double gg[3] = {(double)g0, (double)g1, (double)g2};
        for (int k = 0; k < 3; ++k) vcm[k] = (sum[k] + sd * gg[k]) / (double)(n + nv);
    } else {
        for (int k = 0; k < 3; ++k) vcm[k] = sum[k] / (double)n;
    }
    const R sd = slab_sd(rp, slab, R(0));
    double xs[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        U4 w = philox(lc, step, P_THERMO, (uint32_t)i, rp.seed);
        R g0, g1, g2, g3;
        box_muller(w.x, w.y, g0, g1);
        box_muller(w.z, w.w, g2, g3);
        const R gg[3] = {g0, g1, g2};
        for (int k = 0; k < 3; ++k) {
            const R xi = sd * gg[k];
            v[canon(pm, i, n)].v[k] = xi;
            xs[k] = xs[k] + (double)xi;
        }
    }
    for (int k = 0; k < 3; ++k) xs[k] = xs[k] / (double)n;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) v[canon(pm, i, n)].v[k] = (R)(vcm[k] + ((double)v[canon(pm, i, n)].v[k] - xs[k]));
}

// Stage D, one thread per cell, particles summed in canonical order (the
// order of the FP64 definition, and on the mixed path what makes reruns
// bit-identical whatever order the atomics delivered the particles in): the
// i-th particle of the cell at staging index lo + perm[lo + i].
template <bool MIXED, bool MANY, bool FUSED>
__device__ __forceinline__ void cells_D(const Dev &d, const CellPassArgs &a, TileShared<MIXED> &T, int gt,
                                        int cb, int ce, int pofs, typename Traits<MIXED>::Rec *srec,
                                        const unsigned short *perm)
{
    using R = typename Traits<MIXED>::R;
    const ReplicaDev &rp = T.rp;
    const int lc0 = T.tile * CPT - rp.cell_off;
    const int opts = a.opts;
    const bool want_near = FUSED && MIXED && (opts & CP_NEXT) && rp.n_col > 0;
    for (int c = cb + gt; c < ce; c += CP_THREADS) {
        const int n = T.cnt[c];
        const int lo = T.ls[c] - pofs;
        const unsigned short *pm = perm + lo;
        typename Traits<MIXED>::Rec *cr = srec + lo;
        const int lc = cell_key_at(d, rp.cell_off, lc0 + c);   // the cell's key (its place in Hilbert order)
        T.mode[c] = 0;
        T.react[c] = -1;
        T.mnear[c] = MIXED ? 0 : 1;
        const int cx = lc % rp.L[0];
        const int cz = lc / (rp.L[0] * rp.L[1]);
        // a wall cell short of rho_wall collides with virtual partners, a
        // single real particle included (its v_cm then differs from v)
        const bool virt = rp.walls && (cz == 0 || cz == rp.nz - 1) && n > 0 && n < rp.rho_wall;
        const bool coll = (opts & CP_COLLIDE) && (n >= 2 || virt);
        int slab = -1;
        if (coll)
            for (int k = 0; k < rp.n_slabs; ++k)
                if (cx >= rp.slab_lo[k] && cx < rp.slab_hi[k]) { slab = k; break; }
        const bool nearq = want_near && n > 0;
        // the cell's velocity sum: for the SRD collision and for the near
        // bound (stage D leaves the velocities unchanged outside MPC-AT
        // slabs, where the bound is not taken).  FP64: in canonical order.
        // Mixed: each component rounded to a multiple of 2^-24 and summed as
        // a 64-bit integer -- exact, so the same in any order -- then rounded
        // once to FP32 (|v| < 128 takes one conversion; wider values or
        // non-finite ones take the split conversion for the whole cell).
        R sum[3] = {R(0), R(0), R(0)};
        if (slab < 0 && (coll || nearq)) {
            if constexpr (MIXED) {
                long long fx[3] = {0ll, 0ll, 0ll};
                bool wide = false;
#pragma unroll 2
                for (int i = 0; i < n; ++i) {
                    const float4 q = *reinterpret_cast<const float4 *>(cr[i].v);   // v and fid: one load
                    const float vi[3] = {q.x, q.y, q.z};
                    for (int k = 0; k < 3; ++k) {
                        const float t = vi[k] * 0x1p24f;
                        wide |= !(fabsf(t) < 0x1p31f);
                        fx[k] += (long long)__float2int_rn(t);
                    }
                }
                if (wide) {
                    // a speed of 128 or more (or not finite): the split conversion
                    fx[0] = fx[1] = fx[2] = 0ll;
                    for (int i = 0; i < n; ++i)
                        for (int k = 0; k < 3; ++k) fx[k] += fixed24(cr[i].v[k]);
                }
                for (int k = 0; k < 3; ++k) sum[k] = exact_to_R(fx[k], R(0)) * (R)0x1p-24;
            } else {
                for (int i = 0; i < n; ++i) {
                    const int q = canon(pm, i, n);
                    for (int k = 0; k < 3; ++k) sum[k] = sum[k] + cr[q].v[k];
                }
            }
        }
        int nbB = -1;   // B count, when the near bound's loop has taken it
        unsigned char res = 0;   // species reservoir of the cell's y column (chemotactic set-up)
        if ((opts & CP_REACT) && (rp.res_y[0] < rp.res_y[1] || rp.res_y[2] < rp.res_y[3])) {
            const int cy = (lc / rp.L[0]) % rp.L[1];
            if (cy >= rp.res_y[0] && cy < rp.res_y[1]) res = 4;
            else if (cy >= rp.res_y[2] && cy < rp.res_y[3]) res = 8;
            T.mode[c] = res;
        }
        if (coll) {
            if (slab >= 0) {
                mpcat_cell<R>(rp, a.step, (uint32_t)lc, slab, n, virt, cr, pm);
                T.mode[c] = 2 | res;
            } else {
                R vcm[3];
                if (virt) {
                    // virtual particles fill the wall cell up to rho_wall (§1.4)
                    const int nv = rp.rho_wall - n;
                    U4 w = philox((uint32_t)lc, a.step, P_VIRT, 0u, rp.seed);
                    R g0, g1, g2, g3;
                    box_muller(w.x, w.y, g0, g1);
                    box_muller(w.z, w.w, g2, g3);
                    const R sd = sqrt((R)nv * (R)rp.kT);
                    const R gg[3] = {g0, g1, g2};
                    for (int k = 0; k < 3; ++k) vcm[k] = (sum[k] + sd * gg[k]) / (R)(n + nv);
                } else {
                    for (int k = 0; k < 3; ++k) vcm[k] = sum[k] / (R)n;
                }
                R ax[3];
                rotation_axis<R>(rp.seed, a.step, (uint32_t)lc, ax);
                for (int k = 0; k < 3; ++k) { T.vcm[c][k] = vcm[k]; T.ax[c][k] = ax[k]; }
                T.mode[c] = 1 | res;
            }
        }
        if (nearq) {
            // can a particle of the cell come near a colloid in the next
            // interval?  Its post-collision speed is at most |v_cm| + max
            // |v - v_cm| (the rotation keeps |v - v_cm|) and it lies within
            // sqrt(3)/2 of the cell centre on this step's grid.  With many
            // colloids the test runs after the batch's candidates are known.
            // MPC-AT cells have their new velocities already: the largest
            // of their speeds is the bound.
            float vb;
            if (slab >= 0) {
                R w2 = R(0);
                for (int i = 0; i < n; ++i)
                    w2 = max(w2, cr[i].v[0] * cr[i].v[0] + cr[i].v[1] * cr[i].v[1] + cr[i].v[2] * cr[i].v[2]);
                vb = (float)sqrt(w2);
            } else {
                // the centre the rotation turns about: with virtual wall
                // partners the collision's v_cm, else the cell's own mean
                const R inv = R(1) / (R)n;
                R vc[3] = {sum[0] * inv, sum[1] * inv, sum[2] * inv};
                if (coll && virt)
                    for (int k = 0; k < 3; ++k) vc[k] = T.vcm[c][k];
                R u2 = R(0);
                int nb_ = 0;
                for (int i = 0; i < n; ++i) {   // order-free: a maximum and a count
                    R vi[3];
                    uint32_t fi;
                    if constexpr (MIXED) {
                        const float4 q = *reinterpret_cast<const float4 *>(cr[i].v);   // v and fid: one load
                        vi[0] = q.x; vi[1] = q.y; vi[2] = q.z;
                        fi = __float_as_uint(q.w);
                    } else {
                        vi[0] = cr[i].v[0]; vi[1] = cr[i].v[1]; vi[2] = cr[i].v[2];
                        fi = cr[i].fid;
                    }
                    const R a0 = vi[0] - vc[0], a1 = vi[1] - vc[1], a2 = vi[2] - vc[2];
                    u2 = max(u2, a0 * a0 + a1 * a1 + a2 * a2);
                    nb_ += (fi & F_B) ? 1 : 0;
                }
                nbB = nb_;
                vb = (float)(sqrt(vc[0] * vc[0] + vc[1] * vc[1] + vc[2] * vc[2]) + sqrt(u2));
            }
            if (MANY) T.vbc[c] = vb;
            const int t = lc / rp.L[0];
            const int kc[3] = {lc % rp.L[0], t % rp.L[1], rp.walls ? t / rp.L[1] - 1 : t / rp.L[1]};
            int mn = 0;
            for (int j = 0; j < (MANY ? 0 : rp.n_col) && !mn; ++j) {
                float dd[3];
                for (int k = 0; k < 3; ++k)
                    dd[k] = (float)(kc[k] - T.nf.Ci[3 * j + k]) + ((0.5f + T.shf[k]) - T.nf.Cf[3 * j + k]);
                min_image(rp, dd);
                const float dist = sqrtf(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
                if (dist - 0.8661f < T.nf.Rb[j] + vb * rp.tau_f + 1e-3f) mn = 1;
            }
            T.mnear[c] = mn;
        }
        if ((opts & CP_REACT) && rp.bulk_on && n > 0) {
            if (nbB < 0) {
                nbB = 0;
                for (int i = 0; i < n; ++i) nbB += (cr[i].fid & F_B) ? 1 : 0;
            }
            if (nbB > 0) {
                U4 w = philox((uint32_t)lc, a.step, P_REACT, 0u, rp.seed);
                if ((unsigned long long)w.x < d.bulk_thr[rp.thr_off + nbB]) {
                    // the pick-th B particle of the cell in canonical order
                    const int pick = (int)(((unsigned long long)w.y * (unsigned long long)nbB) >> 32);
                    if constexpr (MIXED) {
                        // without ranks: the B particle with pick B particles of smaller id
                        for (int q = 0; q < n; ++q) {
                            if (!(cr[q].fid & F_B)) continue;
                            const uint32_t idq = cr[q].fid & ID_MASK;
                            int below = 0;
                            for (int k = 0; k < n; ++k)
                                below += ((cr[k].fid & F_B) && (cr[k].fid & ID_MASK) < idq) ? 1 : 0;
                            if (below == pick) { T.react[c] = lo + q; break; }
                        }
                    } else {
                        for (int i = 0, seen = 0; i < n; ++i) {
                            const int q = canon(pm, i, n);
                            if (cr[q].fid & F_B) {
                                if (seen == pick) { T.react[c] = lo + q; break; }
                                ++seen;
                            }
                        }
                    }
                }
            }
        }
    }
}

// Many-colloid replicas (mixed path), after stage D: warp 0 finds the
// colloids that any particle of the batch can reach during the next interval
// -- distance from the colloid to the box of the batch's cells on this
// step's grid below its near-list radius plus the batch's largest
// post-collision speed times tau -- and then every cell tests only those
// (cells without a speed bound, MPC-AT, keep every colloid).
template <bool MIXED>
__device__ void near_candidates(const Dev &d, TileShared<MIXED> &T, int gt, int cb, int ce)
{
    const ReplicaDev &rp = T.rp;
    const int lc0 = T.tile * CPT - rp.cell_off;
    if (gt < 32) {
        int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
        float vmax = 0.0f;
        for (int c = cb + gt; c < ce; c += 32) {
            const int lc = cell_key_at(d, rp.cell_off, lc0 + c);
            const int t = lc / rp.L[0];
            const int kc[3] = {lc % rp.L[0], t % rp.L[1], t / rp.L[1]};
            for (int k = 0; k < 3; ++k) { lo[k] = min(lo[k], kc[k]); hi[k] = max(hi[k], kc[k]); }
            if (T.cnt[c] > 0) vmax = fmaxf(vmax, T.vbc[c]);
        }
        for (int k = 0; k < 3; ++k) {
            lo[k] = __reduce_min_sync(0xffffffffu, lo[k]);
            hi[k] = __reduce_max_sync(0xffffffffu, hi[k]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        unsigned long long m = 0ull;
        for (int h = 0; h < 2; ++h) {
            const int j = gt + 32 * h;
            bool reach = false;
            if (j < rp.n_col) {
                float d2 = 0.0f;
                for (int k = 0; k < 3; ++k) {
                    const float L = (float)rp.L[k];
                    const float a = (float)lo[k] + T.shf[k], b = (float)hi[k] + 1.0f + T.shf[k];
                    const float X = (float)T.nf.Ci[3 * j + k] + T.nf.Cf[3 * j + k];
                    float dk = 0.0f;
                    if (b - a < L) {
                        dk = 1e30f;
                        for (int s = -1; s <= 1; ++s) {
                            const float y = X + (float)s * L;
                            dk = fminf(dk, fmaxf(0.0f, fmaxf(a - y, y - b)));
                        }
                    }
                    d2 += dk * dk;
                }
                reach = sqrtf(d2) < T.nf.Rb[j] + vmax * rp.tau_f + 1e-3f;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, reach);
            m |= (unsigned long long)bal << (32 * h);
        }
        if (gt == 0) T.cand = m;
    }
    __syncthreads();
    for (int c = cb + gt; c < ce; c += CP_THREADS) {
        if (T.cnt[c] == 0 || T.vbc[c] < 0.0f) continue;   // empty cell: no test
        const int lc = cell_key_at(d, rp.cell_off, lc0 + c);
        const int t = lc / rp.L[0];
        const int kc[3] = {lc % rp.L[0], t % rp.L[1], t / rp.L[1]};
        int mn = 0;
        for (unsigned long long m = T.cand; m && !mn; m &= m - 1ull) {
            const int j = __ffsll((long long)m) - 1;
            float dd[3];
            for (int k = 0; k < 3; ++k)
                dd[k] = (float)(kc[k] - T.nf.Ci[3 * j + k]) + ((0.5f + T.shf[k]) - T.nf.Cf[3 * j + k]);
            min_image(rp, dd);
            const float dist = sqrtf(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
            if (dist - 0.8661f < T.nf.Rb[j] + T.vbc[c] * rp.tau_f + 1e-3f) mn = 1;
        }
        T.mnear[c] = mn;
    }
}

// The stages of the cell pass for the cells [cb, ce) of the tile, run by the
// whole CTA (gt = thread index).  srec/ent/perm/cellof are the staging arrays
// (>= the batch); ovf: a cell of the tile holds more than cap particles.
template <bool MIXED, bool MANY, bool FUSED>
__device__ void cells_batch(const Dev &d, const CellPassArgs &a, TileShared<MIXED> &T, int gt, int cb, int ce,
                            typename Traits<MIXED>::Rec *srec, int *ent, unsigned short *perm,
                            unsigned char *cellof, double acc[8], bool &have_base, bool &pref, bool ovf)
{
    using Rec = typename Traits<MIXED>::Rec;
    using R = typename Traits<MIXED>::R;
    constexpr int G = CP_THREADS;
    const ReplicaDev &rp = T.rp;
    const int gc0 = T.tile * CPT;
    const int pofs = T.ls[cb];
    const int nb = T.ls[ce] - pofs;
    const int opts = a.opts;
    // register copies of what the per-particle loops read
    const HotM hm = hot_m(rp);
    const auto &hp = HotPick<MIXED>::get(rp, hm);
    const R ca = r_ca(rp, R(0)), sa = r_sa(rp, R(0)), omc = r_omc(rp, R(0));
    const int n_col = rp.n_col;
    const float shnf[3] = {T.shnf[0], T.shnf[1], T.shnf[2]};

    // Every thread owns at most K particles of a batch (j = gt + u G); the
    // global loads and atomics of a stage are issued for all of them before
    // any result is used, so a thread waits for one memory round trip per
    // stage.
    constexpr int K = Traits<MIXED>::K;

    // A: the cell of every staged particle
    for (int c = cb + gt; c < ce; c += G) {
        const int lo = T.ls[c] - pofs, n = T.cnt[c];
        for (int i = 0; i < n; ++i) cellof[lo + i] = (unsigned char)(c - cb);
    }
    __syncthreads();
    if (pref) {
        // the next tile's counts, copied now (no register waits on them)
        // and read when this tile is done; stage B's wait covers the copy
        const int nt = T.next_tile;
        if (gt < CPT / 4 && nt < d.n_tiles) cp_async16(&T.cnt_next[4 * gt], d.count[a.cur] + (long long)nt * CPT + 4 * gt);
        pref = false;
    }
    // B: every particle's record into the staging area, in arrival order
    if constexpr (FUSED) {
        // the first cap of a cell from its row, contiguous in memory (16-byte
        // asynchronous copies issued by every thread: measured faster than
        // one bulk copy per cell issued by one warp)
        const Rec *rows = reinterpret_cast<const Rec *>(d.brec[a.cur]);
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int j = gt + u * G;
            if (j < nb) {
                const int c = cb + cellof[j];
                const int r = j + pofs - T.ls[c];
                if (r < d.cap) cp_async_rec(srec + j, rows + row_index(d, gc0 + c, r));
            }
        }
        if (ovf) {
            // the rest from the overflow records of the tile's cells (any
            // order: the rank below orders them); T.react is the per-cell
            // cursor, stage D rewrites it
            for (int c = cb + gt; c < ce; c += G) T.react[c] = d.cap;
            __syncthreads();
            const int no = min((int)*(volatile const unsigned int *)&d.ovf_n[a.cur], d.ovf_cap);
            const Rec *orec = reinterpret_cast<const Rec *>(d.orec[a.cur]);
            for (int k = gt; k < no; k += G) {
                const int2 q = d.ovf[a.cur][k];
                const int c = q.x - gc0;
                if (c >= cb && c < ce && q.y >= 0 && q.y < d.ovf_cap) {
                    const int r = atomicAdd(&T.react[c], 1);
                    if (r < T.cnt[c]) cp_async_rec(srec + T.ls[c] - pofs + r, orec + q.y);
                }
            }
        }
    } else {
        // flat layout: slot numbers from the index buckets (past cap from the
        // overflow entries), then the records from those slots
        const int part_lo = rp.part_off, part_hi = rp.part_off + rp.n_part;
        int e[K];
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int j = gt + u * G;
            if (j < nb) {
                const int c = cb + cellof[j];
                const int r = j + pofs - T.ls[c];
                e[u] = r < d.cap ? d.bucket[a.cur][row_index(d, gc0 + c, r)] : -1;
            }
        }
#pragma unroll
        for (int u = 0; u < K; ++u)
            if (gt + u * G < nb) ent[gt + u * G] = e[u];
        if (ovf) {
            for (int c = cb + gt; c < ce; c += G) T.react[c] = d.cap;
            __syncthreads();
            const int no = min((int)*(volatile const unsigned int *)&d.ovf_n[a.cur], d.ovf_cap);
            for (int k = gt; k < no; k += G) {
                const int2 q = d.ovf[a.cur][k];
                const int c = q.x - gc0;
                if (c >= cb && c < ce) {
                    const int r = atomicAdd(&T.react[c], 1);
                    if (r < T.cnt[c]) ent[T.ls[c] - pofs + r] = q.y;
                }
            }
        }
        __syncthreads();
        const Rec *rin = reinterpret_cast<const Rec *>(d.rec[a.rin]);
        bool bad = false;
#pragma unroll
        for (int u = 0; u < K; ++u) {
            const int j = gt + u * G;
            if (j < nb) {
                const int s = ent[j];
                if (s >= part_lo && s < part_hi) {
                    cp_async_rec(srec + j, rin + s);
                } else {
                    bad = true;
                    srec[j] = Rec{};
                }
            }
        }
        if (bad) atomicOr(&d.err[ERR_BOUNDS], 1u);
    }
    cp_async_wait_all();
    __syncthreads();
    // the canonical place of every particle in its cell: its rank by id, read
    // from the staged records (ids are unique in a valid state; should two
    // collide -- a record left stale after an overflow, which the run has
    // latched --, two ranks coincide and the reads of perm below clamp to the
    // cell, so every access stays in the staging area).  Stage C may rewrite
    // a record meanwhile: only its flag bits change, not the id read here.
    // The mixed fused pass ranks only for MPC-AT replicas and observable
    // passes (the flat layout ranks for its write order).
    const bool need_rank = !MIXED || !FUSED || rp.n_slabs > 0 || (opts & CP_OBS);
    int rk[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const int j = gt + u * G;
        if (need_rank && j < nb) {
            const int c = cb + cellof[j];
            const int lo = T.ls[c] - pofs, n = T.cnt[c];
            const uint32_t id = srec[j].fid & ID_MASK;
            int rank = 0;
            for (int k = 0; k < n; ++k) rank += (srec[lo + k].fid & ID_MASK) < id ? 1 : 0;
            rk[u] = rank;
            perm[lo + rank] = (unsigned short)(j - lo);
        }
    }
    if constexpr (!FUSED) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < K; ++u)
            if (gt + u * G < nb) ent[gt + u * G] = rk[u];   // the canonical place within the cell
    }
    // C: fly the records the MD kernel did not move, with the velocities of
    // the interval.  Stage E may fly them instead (before it rotates the
    // velocities) unless the flight changes velocities that stage D sums
    // (walls, body force) or stage D replaces velocities before E runs
    // (MPC-AT slabs).
    const bool c_stage = (opts & CP_FLIGHT) && (rp.walls || rp.has_g || rp.n_slabs > 0);
    const bool fly_in_E = (opts & CP_FLIGHT) && !c_stage;
    if (c_stage) {
#pragma unroll 1
        for (int p = gt; p < nb; p += G) {
            Rec rec = srec[p];
            if (!(rec.fid & F_PROP)) rec_flight(hp, rec);
            rec.fid &= ~F_PROP;
            srec[p] = rec;
        }
    }
    __syncthreads();
    // D: per-cell work
    cells_D<MIXED, MANY, FUSED>(d, a, T, gt, cb, ce, pofs, srec, perm);
    __syncthreads();
    if constexpr (MANY) {
        if (opts & CP_NEXT) {
            near_candidates(d, T, gt, cb, ce);
            __syncthreads();
        }
    }
    if (!FUSED && !have_base && (opts & CP_WRITE)) {
        // stages A-D do not need the tile base; the flat write does.  The
        // aggregate went out in the prologue; warp 0 scans back now.
        if (gt < 32) {
            const int base = tile_lookback(d, T.epoch, T.tile, T.ls[CPT], gt, false);
            if (gt == 0) T.base = base;
        }
        __syncthreads();
        have_base = true;
    }
    // E: apply and write (flat layout: at the canonical slot; fused run:
    // classify for the next collision -- the next cell of a far particle goes
    // to ent[p], -2 marks a near particle)
    if constexpr (MIXED && FUSED) {
        // the mixed fused pass: the cell word unpacked once per particle (the
        // flight, the near test and the next key take the coordinates) and
        // packed again only when the flight moved it; a cell's centre and
        // axis are one 16-byte load each
#pragma unroll 1
        for (int p = gt; p < nb; p += G) {
            const int c = cb + cellof[p];
            RecM rec = srec[p];
            int cc[3] = {cw_get(rec.cw, 0), cw_get(rec.cw, 1), cw_get(rec.cw, 2)};
            if (fly_in_E && !(rec.fid & F_PROP)) {
                flight_m(hp, cc, rec.o, rec.v);
                rec.cw = cw_make(cc[0], cc[1], cc[2]);
            }
            rec.fid &= ~F_PROP;
            const unsigned mode = T.mode[c];
            if ((mode & 3) == 1) {
                const float4 vq = *reinterpret_cast<const float4 *>(T.vcm[c]);
                const float4 nq = *reinterpret_cast<const float4 *>(T.ax[c]);
                const float vc[3] = {vq.x, vq.y, vq.z}, nh[3] = {nq.x, nq.y, nq.z};
                const float u0 = rec.v[0] - vc[0], u1 = rec.v[1] - vc[1], u2 = rec.v[2] - vc[2];
                const float dot = nh[0] * u0 + nh[1] * u1 + nh[2] * u2;
                const float x0 = nh[1] * u2 - nh[2] * u1;
                const float x1 = nh[2] * u0 - nh[0] * u2;
                const float x2 = nh[0] * u1 - nh[1] * u0;
                const float od = omc * dot;
                rec.v[0] = vc[0] + (ca * u0 + sa * x0 + od * nh[0]);
                rec.v[1] = vc[1] + (ca * u1 + sa * x1 + od * nh[1]);
                rec.v[2] = vc[2] + (ca * u2 + sa * x2 + od * nh[2]);
            }
            if (T.react[c] == p) rec.fid &= ~(F_B | F_TAG);
            if (mode & 4) rec.fid &= ~(F_B | F_TAG);
            if (mode & 8) rec.fid = (rec.fid & ~F_TAG) | F_B;
            srec[p] = rec;
            int nkey = -1;
            if (opts & CP_NEXT) {
                bool near;
                if constexpr (MANY)
                    near = T.mnear[c] && (T.vbc[c] < 0.0f
                                              ? near_test_m(hp, n_col, T.nf.Ci, T.nf.Cf, T.nf.Rb, cc, rec.o, rec.v)
                                              : near_test_mask(hp, T.cand, T.nf, cc, rec.o, rec.v));
                else
                    near = n_col > 0 && T.mnear[c] && near_test_m(hp, n_col, T.nf.Ci, T.nf.Cf, T.nf.Rb, cc, rec.o, rec.v);
                if (near) {
                    nkey = -2;
                } else {
                    int fc[3] = {cc[0], cc[1], cc[2]};
                    float fo[3] = {rec.o[0], rec.o[1], rec.o[2]}, fv[3] = {rec.v[0], rec.v[1], rec.v[2]};
                    flight_m(hp, fc, fo, fv);
                    nkey = bin_cell(d, rp.cell_off, cell_key_m(hp, fc, fo, shnf));
                }
            }
            ent[p] = nkey;
        }
    } else {
#pragma unroll 1
    for (int p = gt; p < nb; p += G) {
        const int c = cb + cellof[p];
        Rec rec = srec[p];
        if (fly_in_E && !(rec.fid & F_PROP)) rec_flight(hp, rec);
        rec.fid &= ~F_PROP;
        const unsigned mode = T.mode[c];
        if ((mode & 3) == 1) {
            const R *vc = T.vcm[c];
            const R *nh = T.ax[c];
            const R u0 = rec.v[0] - vc[0], u1 = rec.v[1] - vc[1], u2 = rec.v[2] - vc[2];
            // Rodrigues: R u = u cos a + (n x u) sin a + n (n.u)(1 - cos a)
            const R dot = nh[0] * u0 + nh[1] * u1 + nh[2] * u2;
            const R x0 = nh[1] * u2 - nh[2] * u1;
            const R x1 = nh[2] * u0 - nh[0] * u2;
            const R x2 = nh[0] * u1 - nh[1] * u0;
            const R od = omc * dot;
            rec.v[0] = vc[0] + (ca * u0 + sa * x0 + od * nh[0]);
            rec.v[1] = vc[1] + (ca * u1 + sa * x1 + od * nh[1]);
            rec.v[2] = vc[2] + (ca * u2 + sa * x2 + od * nh[2]);
        }
        if (T.react[c] == p) rec.fid &= ~(F_B | F_TAG);
        // species reservoirs (§1.5 chemotactic_cell): after the bulk
        // reaction, the cells of the reservoir y columns are made pure
        if (mode & 4) rec.fid &= ~(F_B | F_TAG);
        if (mode & 8) rec.fid = (rec.fid & ~F_TAG) | F_B;
        if constexpr (FUSED) {
            srec[p] = rec;
            int nkey = -1;
            if (opts & CP_NEXT) {
                bool near;
                if constexpr (MANY) near = T.mnear[c] && rec_near_cand(hp, n_col, T.nf, rec, T.cand, T.vbc[c] < 0.0f);
                else near = n_col > 0 && T.mnear[c] && rec_near(d, hp, n_col, T.nf, rec);
                if (near) {
                    nkey = -2;
                } else {
                    Rec fl = rec;
                    rec_flight(hp, fl);
                    nkey = bin_cell(d, rp.cell_off, rec_key(hp, fl, T.shn, shnf));
                }
            }
            ent[p] = nkey;
        } else {
            if (opts & CP_WRITE) {
                const int gslot = T.base + T.ls[c] + ent[p];
                if (gslot >= rp.part_off && gslot < rp.part_off + rp.n_part)
                    store_rec(reinterpret_cast<Rec *>(d.rec[a.rout]) + gslot, rec);
                else
                    atomicOr(&d.err[ERR_BOUNDS], 1u);
            }
            if (opts & CP_OBS) srec[p] = rec;
        }
    }
    }
    if constexpr (FUSED) {
        // bin for the next collision: all count atomics, then the record
        // writes; the near particles join the near area with one atomic per
        // warp, in flight together with the count atomics
        if (opts & CP_NEXT) {
            int mine = 0;
            const bool appends = n_col > 0;   // uniform: replicas without colloids skip the near area
            if (appends)
#pragma unroll
                for (int u = 0; u < K; ++u) {
                    const int p = gt + u * G;
                    mine += (p < nb && ent[p] == -2) ? 1 : 0;
                }
            int incl = mine;
            if (appends)
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((gt & 31) >= o) incl += y;
                }
            const int wtot = appends ? __shfl_sync(0xffffffffu, incl, 31) : 0;
            int nbase = 0;
            if ((gt & 31) == 31 && wtot > 0) nbase = atomicAdd(&d.near_count[T.r], wtot);
            // the lanes that bin into one cell take their places with one
            // atomic (the group's size), issued for every u before any result
            // is used; then each lane's place is the leader's base plus its
            // rank in the group
            int pos[K];
            unsigned grp[K];
#pragma unroll
            for (int u = 0; u < K; ++u) {
                const int p = gt + u * G;
                const int key = p < nb ? ent[p] : -1;
                grp[u] = __match_any_sync(0xffffffffu, key);
                const int leader = __ffs(grp[u]) - 1;
                pos[u] = (key >= 0 && (gt & 31) == leader) ? atomicAdd(&d.count[a.nxt][key], __popc(grp[u])) : -1;
            }
#pragma unroll
            for (int u = 0; u < K; ++u) {
                const int p = gt + u * G;
                const int key = p < nb ? ent[p] : -1;
                const int leader = __ffs(grp[u]) - 1;
                const int base = __shfl_sync(0xffffffffu, pos[u], leader);
                pos[u] = key >= 0 ? base + __popc(grp[u] & ((1u << (gt & 31)) - 1u)) : -1;
            }
            if (wtot > 0) {
                int k = __shfl_sync(0xffffffffu, nbase, 31) + incl - mine;
                Rec *near_rec = reinterpret_cast<Rec *>(d.near_rec) + rp.part_off;
#pragma unroll
                for (int u = 0; u < K; ++u) {
                    const int p = gt + u * G;
                    if (p < nb && ent[p] == -2) {
                        if (k < rp.n_part) store_rec(near_rec + k, srec[p]);
                        else atomicOr(&d.err[ERR_BOUNDS], 1u);
                        ++k;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < K; ++u) {
                if (pos[u] < 0) continue;
                const int p = gt + u * G;
                bin_record_at(d, a.nxt, ent[p], pos[u], srec[p]);
            }
        }
    }
    __syncthreads();
    // F: observables of the post-collision state (§1.4 temperature)
    if (opts & CP_OBS) {
        for (int c = cb + gt; c < ce; c += G) {
            const int n = T.cnt[c];
            const int lo = T.ls[c] - pofs;
            const unsigned short *pm = perm + lo;
            const Rec *cr = srec + lo;
            // the conservation diagnostics: per-cell momentum and energy sums
            // in FP64 on both paths (a pass with observables is not a timed one)
            double sum[3] = {0.0, 0.0, 0.0};
            double ke2 = 0.0;
            int nbB = 0;
            for (int i = 0; i < n; ++i) {
                const Rec &ri = cr[canon(pm, i, n)];
                for (int k = 0; k < 3; ++k) {
                    const double vk = (double)ri.v[k];
                    sum[k] = sum[k] + vk;
                    ke2 = ke2 + vk * vk;
                }
                nbB += (ri.fid & F_B) ? 1 : 0;
            }
            if (n >= 2) {
                const double vcm[3] = {sum[0] / (double)n, sum[1] / (double)n, sum[2] / (double)n};
                double ke = 0.0;
                for (int i = 0; i < n; ++i)
                    for (int k = 0; k < 3; ++k) {
                        const double u = (double)cr[canon(pm, i, n)].v[k] - vcm[k];
                        ke = ke + u * u;
                    }
                acc[0] += ke / (double)(n - 1);
                acc[1] += 1.0;
            }
            acc[2] += sum[0]; acc[3] += sum[1]; acc[4] += sum[2];
            acc[5] += 0.5 * ke2;
            acc[6] += (double)nbB;
            acc[7] += (double)n;
        }
        __syncthreads();
    }
}

// A run of cells from cb on whose particles fit `cap` staging slots (at
// least one cell; a single cell holds at most cap particles).
__device__ __forceinline__ int batch_end(const int *ls, int cb, int cend, int cap)
{
    if (ls[cend] - ls[cb] <= cap) return cend;   // the usual case: the rest fits
    int ce = cb + 1;
    while (ce < cend && ls[ce + 1] - ls[cb] <= cap) ++ce;
    return ce;
}

// Dynamic shared memory of the staging area: records, ids / ranks, canonical
// order, cell of each staged particle.
template <bool MIXED>
constexpr size_t stage_bytes()
{
    return (size_t)Traits<MIXED>::TP *
           (sizeof(typename Traits<MIXED>::Rec) + sizeof(int) + sizeof(unsigned short) + 1);
}

// MANY: the system has a replica with at least CP_NEAR_CAND_MIN colloids
// (mixed path only): near tests through per-batch candidate colloids.
// FUSED: the fused run's layout (record rows in, record rows and near area
// out); else the flat layout.
template <bool MIXED, bool MANY, bool FUSED>
__global__ void __launch_bounds__(CP_THREADS, MIXED ? 3 : 2) k_cellpass(Dev d, CellPassArgs a0)
{
    using Rec = typename Traits<MIXED>::Rec;
    constexpr int TP = Traits<MIXED>::TP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Rec *srec = reinterpret_cast<Rec *>(smem_raw);
    int *ent = reinterpret_cast<int *>(srec + TP);
    unsigned short *perm = reinterpret_cast<unsigned short *>(ent + TP);
    unsigned char *cellof = reinterpret_cast<unsigned char *>(perm + TP);
    __shared__ TileShared<MIXED> T;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        // the launch counter and the step, read before the first ticket is
        // taken; the last CTA to finish advances them, after every CTA has read
        const uint32_t epoch = *(volatile uint32_t *)&d.ctl->epoch;
        const uint32_t step = resolve_step(d, a0.step);
        __threadfence();
        T.tile = (int)atomicAdd(&d.ticket[epoch & 1u], 1u);
        T.epoch = epoch;
        T.step = step;
        if (blockIdx.x == 0) d.ticket[(epoch + 1u) & 1u] = 0u;
    }
    __syncthreads();
    CellPassArgs a = a0;
    a.step = T.step;
    // Persistent CTA: tiles in ticket order.  The next ticket is taken when a
    // tile starts and that tile's counts are read during the current one, so
    // the chain ticket -> counts is off the critical path; the replica's
    // constants are reloaded only when the replica changes.
    int cur_r = -1;
    if (tid < CPT && T.tile < d.n_tiles) T.cnt_next[tid] = d.count[a.cur][T.tile * CPT + tid];
    for (;;) {
        const int tile = T.tile;
        if (tile >= d.n_tiles) break;
        if (tid == 0) T.r = d.tile_rep[tile];
        __syncthreads();
        const ReplicaDev &rp = T.rp;
        if (T.r != cur_r) {
            cur_r = T.r;
            const int *src = reinterpret_cast<const int *>(d.rep + cur_r);
            int *dst = reinterpret_cast<int *>(&T.rp);
            for (int i = tid; i < (int)(sizeof(ReplicaDev) / sizeof(int)); i += CP_THREADS) dst[i] = src[i];
            __syncthreads();
            if (tid == 0) {
                grid_shift(rp.seed, a.step, T.shf);
                if (!MIXED) grid_shift(rp.seed, a.step, T.sh);
            } else if (tid == 32) {
                grid_shift(rp.seed, a.step + 1u, T.shnf);
                if (!MIXED) grid_shift(rp.seed, a.step + 1u, T.shn);
            }
            if (MIXED && FUSED && (a.opts & CP_NEXT)) {
                for (int i = tid; i < 3 * rp.n_col; i += CP_THREADS) {
                    T.nf.Ci[i] = d.colCi[3 * rp.col_off + i];
                    T.nf.Cf[i] = d.colXf[3 * rp.col_off + i];
                }
                for (int j = tid; j < rp.n_col; j += CP_THREADS) T.nf.Rb[j] = d.colRb_f[rp.col_off + j];
            }
        }
        // the next ticket, taken now so that its round trip overlaps the
        // count scan (tickets stay in order per CTA)
        unsigned nt_next = 0u;
        if (tid == 0) nt_next = atomicAdd(&d.ticket[T.epoch & 1u], 1u);
        const int gc0 = tile * CPT;
        // counts of the tile's cells (consumed: reset for reuse two passes later)
        int x = 0;
        bool big = false;   // a cell of the tile holds more than cap
        if (tid < CPT) {
            int n = T.cnt_next[tid];
            d.count[a.cur][gc0 + tid] = 0;
            const int mraw = __reduce_max_sync(0xffffffffu, n);
            if (lane == 0 && mraw > 0) atomicMax(d.maxcnt, (unsigned int)mraw);   // for the bucket-width tuner
            if (n > TP) {
                // more than a cell can stage: the step is invalid
                atomicMax(&d.err[ERR_OVERFLOW], (unsigned int)n);
                n = TP;
            }
            big = n > d.cap;
            T.cnt[tid] = n;
            x = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) T.wt[wid] = x;
        }
        const bool tile_ovf = __syncthreads_or(big);
        if (tid < CPT) {
            int pre = 0;
            for (int w = 0; w < wid; ++w) pre += T.wt[w];
            T.ls[tid + 1] = x + pre;
        }
        if (tid == 0) T.ls[0] = 0;
        __syncthreads();

        // flat write: tile base by decoupled look-back (warp 0); the tile's
        // aggregate goes out now, the scan over predecessors waits until the
        // first batch needs the base (stage E)
        if (tid == 0) {
            if (!FUSED && (a.opts & CP_WRITE)) tile_publish(d, T.epoch, tile, T.ls[CPT]);
            T.next_tile = (int)nt_next;
        }

        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // T sum, cells, px, py, pz, ke, nB, n
        bool have_base = false, pref = true;
        for (int cb = 0; cb < CPT;) {
            const int ce = batch_end(T.ls, cb, CPT, TP);
            cells_batch<MIXED, MANY, FUSED>(d, a, T, tid, cb, ce, srec, ent, perm, cellof, acc, have_base, pref,
                                            tile_ovf);
            cb = ce;
        }

        if (a.opts & CP_OBS) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                double v = acc[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) T.red[wid][k] = v;
            }
            __syncthreads();
            if (tid < 8) {
                double v = 0.0;
                for (int w = 0; w < CP_WARPS; ++w) v += T.red[w][tid];
                d.obs_part[(long long)tile * 8 + tid] = v;
            }
        }
        __syncthreads();
        if (tid == 0) T.tile = T.next_tile;
        __syncthreads();
    }
    // the last CTA to finish advances the interval control
    if (tid == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&d.ticket[2 + (T.epoch & 1u)], 1u);
        if (done == gridDim.x - 1) {
            d.ticket[2 + (T.epoch & 1u)] = 0u;
            d.ovf_n[a0.cur] = 0u;   // every CTA has read the consumed overflow list
            __threadfence();
            d.ctl->epoch = T.epoch + 1u;
            if (a0.opts & CP_ADVANCE) d.ctl->step = T.step + 1u;
        }
    }
}

size_t cellpass_smem(bool mixed) { return mixed ? stage_bytes<true>() : stage_bytes<false>(); }

// Co-resident CTAs of the persistent cell pass on the current device.
template <bool MIXED, bool MANY, bool FUSED>
static int cellpass_grid()
{
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int &g = cached[dev & 63];
    if (g == 0) {
        const size_t sm = stage_bytes<MIXED>();
        int per_sm = 0, n_sm = 0;
        cudaFuncSetAttribute(k_cellpass<MIXED, MANY, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cellpass<MIXED, MANY, FUSED>, CP_THREADS, sm);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        g = std::max(1, per_sm) * std::max(1, n_sm);
    }
    return g;
}

template <bool MIXED, bool MANY, bool FUSED>
static void launch_cp(const Dev &d, const CellPassArgs &a, cudaStream_t s)
{
    const size_t sm = stage_bytes<MIXED>();
    const int grid = std::min(d.n_tiles, cellpass_grid<MIXED, MANY, FUSED>());
    k_cellpass<MIXED, MANY, FUSED><<<grid, CP_THREADS, sm, s>>>(d, a);
}

// The fused run's pass reads and writes record rows (CP_NEXT, never
// CP_WRITE); every other pass works on the flat layout (never CP_NEXT).
void launch_cellpass(bool mixed, const Dev &d, const CellPassArgs &a, cudaStream_t s)
{
    if (d.n_tiles == 0) return;
    if (a.opts & CP_NEXT) {
        if (!mixed) launch_cp<false, false, true>(d, a, s);
        else if (d.many_col) launch_cp<true, true, true>(d, a, s);
        else launch_cp<true, false, true>(d, a, s);
    } else {
        if (!mixed) launch_cp<false, false, false>(d, a, s);
        else launch_cp<true, false, false>(d, a, s);
    }
}

}  // namespace rmpcd
