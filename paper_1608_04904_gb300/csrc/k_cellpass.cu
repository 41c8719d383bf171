// k_cellpass.cu -- the per-cell pass of one collision (§1.4 of the RMPCDMD
// paper, arXiv:1608.04904): sorted gather, SRD / MPC-AT / virtual-particle
// collision, bulk B -> A reaction, and (fused) free flight + binning of every
// particle for the next collision.
//
// One CTA owns a tile of CPT consecutive cells of one replica.  Its particles
// are the bucket entries of those cells; within a cell they are put back in
// increasing storage slot order, which makes the sort stable and the result
// independent of the atomic order in which the buckets were filled.  The
// tile's first output slot is the exclusive prefix of all earlier tiles'
// particle counts, found by a single-pass decoupled look-back (Merrill &
// Garland 2016) over tiles taken in ticket order.
//
// Per particle this reads its bucket entry (4 B) and its record (32 B mixed /
// 64 B fp64) and writes its record and its next bucket entry: one pass over
// the solvent per collision.
#include "rmpcd_kernels.cuh"

namespace rmpcd {

template <bool MIXED> struct Traits;
template <> struct Traits<true> {
    using Rec = RecM;
    using R = float;
    static constexpr int TP = TP_M;
};
template <> struct Traits<false> {
    using Rec = RecD;
    using R = double;
    static constexpr int TP = TP_D;
};

// --- per-record helpers ----------------------------------------------------
__device__ __forceinline__ void rec_flight(const ReplicaDev &rp, RecM &r)
{
    int c[3] = {cw_get(r.cw, 0), cw_get(r.cw, 1), cw_get(r.cw, 2)};
    flight_m(rp, c, r.o, r.v);
    r.cw = cw_make(c[0], c[1], c[2]);
}
__device__ __forceinline__ void rec_flight(const ReplicaDev &rp, RecD &r) { flight_d(rp, r.x, r.v); }

// s: the shift in FP64; sf: the same shift in FP32 (exact: 24-bit uniforms)
__device__ __forceinline__ int rec_key(const ReplicaDev &rp, const RecM &r, const double *, const float *sf)
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

__device__ __forceinline__ bool rec_near(const Dev &d, const ReplicaDev &rp, const NearFrames &nf, const RecM &r)
{
    int c[3] = {cw_get(r.cw, 0), cw_get(r.cw, 1), cw_get(r.cw, 2)};
    return near_test_m(rp, rp.n_col, nf.Ci, nf.Cf, nf.Rb, c, r.o, r.v);
}
__device__ __forceinline__ bool rec_near(const Dev &d, const ReplicaDev &rp, const NearFrames &, const RecD &r)
{
    return near_test_d(d, rp, r.x, r.v);
}

__device__ __forceinline__ float slab_sd(const ReplicaDev &rp, int k, float) { return rp.slab_sd_f[k]; }
__device__ __forceinline__ double slab_sd(const ReplicaDev &rp, int k, double) { return rp.slab_sd[k]; }
__device__ __forceinline__ float r_ca(const ReplicaDev &rp, float) { return rp.ca_f; }
__device__ __forceinline__ double r_ca(const ReplicaDev &rp, double) { return rp.ca; }
__device__ __forceinline__ float r_sa(const ReplicaDev &rp, float) { return rp.sa_f; }
__device__ __forceinline__ double r_sa(const ReplicaDev &rp, double) { return rp.sa; }
__device__ __forceinline__ float r_omc(const ReplicaDev &rp, float) { return rp.omc_f; }
__device__ __forceinline__ double r_omc(const ReplicaDev &rp, double) { return rp.omc; }

constexpr unsigned long long LB_VALUE_MASK = (1ull << 46) - 1ull;
constexpr int LB_SPIN_LIMIT = 1 << 22;

template <bool MIXED>
__global__ void __launch_bounds__(CP_THREADS) k_cellpass(Dev d, CellPassArgs a)
{
    using T = Traits<MIXED>;
    using Rec = typename T::Rec;
    using R = typename T::R;
    constexpr int TP = T::TP;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    Rec *srec = reinterpret_cast<Rec *>(smem_raw);
    int *ent = reinterpret_cast<int *>(srec + TP);
    int *srt = ent + TP;
    unsigned char *cellof = reinterpret_cast<unsigned char *>(srt + TP);

    __shared__ ReplicaDev s_rp;
    __shared__ int s_tile, s_r, s_ce, s_base;
    __shared__ int s_cnt[CPT], s_ls[CPT + 1], s_wt[2];
    __shared__ double s_sh[3], s_shn[3];
    __shared__ float s_shnf[3];
    __shared__ R s_vcm[CPT][3], s_ax[CPT][3];
    __shared__ int s_mode[CPT], s_react[CPT];
    __shared__ double s_red[CP_THREADS / 32][8];
    __shared__ NearFrames s_nf;

    const int tid = threadIdx.x;
    if (tid == 0) {
        s_tile = (int)atomicAdd(&d.ticket[a.epoch & 1u], 1u);
        if (blockIdx.x == 0) d.ticket[(a.epoch + 1u) & 1u] = 0u;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= d.n_tiles) return;
    if (tid == 0) {
        s_r = d.tile_rep[tile];
        s_rp = d.rep[s_r];
    }
    __syncthreads();
    const ReplicaDev &rp = s_rp;
    const int r = s_r;
    if (MIXED && (a.opts & CP_NEXT)) {
        for (int i = tid; i < 3 * rp.n_col; i += CP_THREADS) {
            s_nf.Ci[i] = d.colCi[3 * rp.col_off + i];
            s_nf.Cf[i] = d.colXf[3 * rp.col_off + i];
        }
        for (int j = tid; j < rp.n_col; j += CP_THREADS) s_nf.Rb[j] = d.colRb_f[rp.col_off + j];
    }
    const int gc0 = tile * CPT;            // global index of the tile's first cell
    const int lc0 = gc0 - rp.cell_off;     // replica-local index of that cell

    // counts of the tile's cells (consumed: reset for reuse two passes later)
    if (tid < CPT) {
        int n = d.count[a.cur][gc0 + tid];
        d.count[a.cur][gc0 + tid] = 0;
        if (n > d.cap) {
            atomicMax(&d.err[ERR_OVERFLOW], (unsigned int)n);
            n = d.cap;
        }
        s_cnt[tid] = n;
        int x = n;
        const int lane = tid & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wt[tid >> 5] = x;
        s_ls[tid + 1] = x;   // inclusive within the warp for now
    }
    if (tid == 0) {
        s_ls[0] = 0;
        double s[3];
        grid_shift(rp.seed, a.step, s);
        s_sh[0] = s[0]; s_sh[1] = s[1]; s_sh[2] = s[2];
        grid_shift(rp.seed, a.step + 1u, s);
        s_shn[0] = s[0]; s_shn[1] = s[1]; s_shn[2] = s[2];
        s_shnf[0] = (float)s[0]; s_shnf[1] = (float)s[1]; s_shnf[2] = (float)s[2];
    }
    __syncthreads();
    if (tid >= 32 && tid < CPT) s_ls[tid + 1] += s_wt[0];
    __syncthreads();

    // tile base by decoupled look-back: warp 0 inspects 32 predecessor tiles
    // at a time, sums aggregates back to the nearest inclusive prefix
    if (tid < 32) {
        const int lane = tid;
        // 16-bit tag of this launch, never 0 (the initial state)
        const unsigned long long ep = (unsigned long long)(a.epoch % 65535u) + 1ull;
        const unsigned long long total = (unsigned long long)s_ls[CPT];
        if (lane == 0) st_release(&d.tile_state[tile], (ep << 48) | (1ull << 46) | total);
        unsigned long long prefix = 0;
        int t = tile - 1;
        int spins = 0;
        bool ok = true;
        while (t >= 0) {
            const int idx = t - lane;
            unsigned long long flag = 2ull, val = 0ull;   // before tile 0: inclusive prefix 0
            if (idx >= 0) {
                const unsigned long long w = ld_acquire(&d.tile_state[idx]);
                flag = ((w >> 48) == ep) ? ((w >> 46) & 3ull) : 0ull;
                val = w & LB_VALUE_MASK;
            }
            const unsigned incl = __ballot_sync(0xffffffffu, flag == 2ull);
            const unsigned ready = __ballot_sync(0xffffffffu, flag != 0ull);
            const int first = incl ? __ffs(incl) - 1 : 31;
            const unsigned need = (first == 31) ? 0xffffffffu : ((2u << first) - 1u);
            if ((ready & need) != need) {
                if (++spins > LB_SPIN_LIMIT) { ok = false; break; }
                __nanosleep(32);
                continue;
            }
            unsigned long long part = (lane <= first) ? val : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
            prefix += __shfl_sync(0xffffffffu, part, 0);
            if (incl) break;
            t -= 32;
        }
        if (lane == 0) {
            if (!ok) {
                atomicOr(&d.err[ERR_TIMEOUT], 1u);
                prefix = 0x3FFFFFFFull;   // pushes every write of this tile out of bounds
            }
            st_release(&d.tile_state[tile], (ep << 48) | (2ull << 46) | ((prefix + total) & LB_VALUE_MASK));
            s_base = (int)(prefix > 0x3FFFFFFFull ? 0x3FFFFFFF : prefix);
        }
    }
    __syncthreads();
    const int base = s_base;
    const int part_lo = rp.part_off, part_hi = rp.part_off + rp.n_part;
    const int opts = a.opts;
    const Rec *rin = reinterpret_cast<const Rec *>(d.rec[a.rin]);
    Rec *rout = reinterpret_cast<Rec *>(d.rec[a.rout]);

    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // T sum, cells, px, py, pz, ke, nB, n

    int cb = 0;
    while (cb < CPT) {
        if (tid == 0) {
            int ce = cb + 1;
            while (ce < CPT && s_ls[ce + 1] - s_ls[cb] <= TP) ++ce;
            s_ce = ce;
        }
        __syncthreads();
        const int ce = s_ce;
        const int pofs = s_ls[cb];
        const int nb = s_ls[ce] - pofs;

        // A: bucket entries of the batch's cells
        for (int j = tid; j < nb; j += CP_THREADS) {
            const int jj = j + pofs;
            int lo = cb, hi = ce - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (s_ls[mid] <= jj) lo = mid; else hi = mid - 1;
            }
            ent[j] = d.bucket[a.cur][(long long)(gc0 + lo) * d.cap + (jj - s_ls[lo])];
            cellof[j] = (unsigned char)lo;
        }
        __syncthreads();
        // B: stable order inside each cell = increasing previous slot
        for (int j = tid; j < nb; j += CP_THREADS) {
            const int c = cellof[j];
            const int lo = s_ls[c] - pofs, n = s_cnt[c];
            const int e = ent[j];
            int rank = 0;
            for (int k = 0; k < n; ++k) rank += (ent[lo + k] < e) ? 1 : 0;
            srt[lo + rank] = e;
        }
        __syncthreads();
        // C: gather (and fly the records the MD kernel did not move)
        for (int p = tid; p < nb; p += CP_THREADS) {
            const int slot = srt[p];
            Rec rec;
            if (slot >= part_lo && slot < part_hi) {
                rec = load_rec(rin + slot);
            } else {
                atomicOr(&d.err[ERR_BOUNDS], 1u);
                rec = Rec{};
            }
            if ((opts & CP_FLIGHT) && !(rec.fid & F_PROP)) rec_flight(rp, rec);
            rec.fid &= ~F_PROP;
            srec[p] = rec;
        }
        __syncthreads();
        // D: per-cell work
        for (int c = cb + tid; c < ce; c += CP_THREADS) {
            const int n = s_cnt[c];
            const int lo = s_ls[c] - pofs;
            const int lc = lc0 + c;
            s_mode[c] = 0;
            s_react[c] = -1;
            if ((opts & CP_COLLIDE) && n >= 2) {
                R sum[3] = {R(0), R(0), R(0)};
                for (int i = 0; i < n; ++i)
                    for (int k = 0; k < 3; ++k) sum[k] = sum[k] + srec[lo + i].v[k];
                const int cx = lc % rp.L[0];
                const int cz = lc / (rp.L[0] * rp.L[1]);
                R vcm[3];
                const bool wall_cell = rp.walls && (cz == 0 || cz == rp.nz - 1);
                if (wall_cell && n < rp.rho_wall) {
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
                int slab = -1;
                for (int k = 0; k < rp.n_slabs; ++k)
                    if ((double)cx >= rp.slab_x0[k] && (double)cx < rp.slab_x1[k]) { slab = k; break; }
                if (slab >= 0) {
                    // Anderson thermostat (MPC-AT): fresh relative velocities
                    const R sd = slab_sd(rp, slab, R(0));
                    R xs[3] = {R(0), R(0), R(0)};
                    for (int i = 0; i < n; ++i) {
                        U4 w = philox((uint32_t)lc, a.step, P_THERMO, (uint32_t)i, rp.seed);
                        R g0, g1, g2, g3;
                        box_muller(w.x, w.y, g0, g1);
                        box_muller(w.z, w.w, g2, g3);
                        const R gg[3] = {g0, g1, g2};
                        for (int k = 0; k < 3; ++k) {
                            const R xi = sd * gg[k];
                            srec[lo + i].v[k] = xi;
                            xs[k] = xs[k] + xi;
                        }
                    }
                    for (int k = 0; k < 3; ++k) xs[k] = xs[k] / (R)n;
                    for (int i = 0; i < n; ++i)
                        for (int k = 0; k < 3; ++k) srec[lo + i].v[k] = vcm[k] + (srec[lo + i].v[k] - xs[k]);
                    s_mode[c] = 2;
                } else {
                    R ax[3];
                    rotation_axis<R>(rp.seed, a.step, (uint32_t)lc, ax);
                    for (int k = 0; k < 3; ++k) { s_vcm[c][k] = vcm[k]; s_ax[c][k] = ax[k]; }
                    s_mode[c] = 1;
                }
            }
            if ((opts & CP_REACT) && rp.bulk_on && n > 0) {
                int nbB = 0;
                for (int i = 0; i < n; ++i) nbB += (srec[lo + i].fid & F_B) ? 1 : 0;
                if (nbB > 0) {
                    U4 w = philox((uint32_t)lc, a.step, P_REACT, 0u, rp.seed);
                    if ((double)w.x < d.bulk_thr[rp.thr_off + nbB]) {
                        const int pick = (int)(((unsigned long long)w.y * (unsigned long long)nbB) >> 32);
                        for (int i = 0, seen = 0; i < n; ++i) {
                            if (srec[lo + i].fid & F_B) {
                                if (seen == pick) { s_react[c] = lo + i; break; }
                                ++seen;
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        // E: apply, write, classify / bin for the next collision
        for (int p = tid; p < nb; p += CP_THREADS) {
            const int c = cellof[p];
            Rec rec = srec[p];
            if (s_mode[c] == 1) {
                const R ca = r_ca(rp, R(0)), sa = r_sa(rp, R(0)), omc = r_omc(rp, R(0));
                const R *vc = s_vcm[c];
                const R *nh = s_ax[c];
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
            if (s_react[c] == p) rec.fid &= ~(F_B | F_TAG);
            const int gslot = base + pofs + p;
            const bool inb = gslot >= part_lo && gslot < part_hi;
            if (!inb) atomicOr(&d.err[ERR_BOUNDS], 1u);
            if ((opts & CP_WRITE) && inb) store_rec(rout + gslot, rec);
            srec[p] = rec;
            if ((opts & CP_NEXT) && inb) {
                if (rp.n_col > 0 && rec_near(d, rp, s_nf, rec)) {
                    const int k = atomicAdd(&d.near_count[r], 1);
                    if (k < rp.n_part) d.near_list[rp.part_off + k] = gslot;
                    else atomicOr(&d.err[ERR_BOUNDS], 1u);
                } else {
                    Rec fl = rec;
                    rec_flight(rp, fl);
                    const int key = rec_key(rp, fl, s_shn, s_shnf);
                    bin_particle(d, a.nxt, rp.cell_off + key, gslot);
                }
            }
        }
        __syncthreads();
        // F: observables of the post-collision state (§1.4 temperature)
        if (opts & CP_OBS) {
            for (int c = cb + tid; c < ce; c += CP_THREADS) {
                const int n = s_cnt[c];
                const int lo = s_ls[c] - pofs;
                // within a cell in the path's precision, across cells in FP64
                R sum[3] = {R(0), R(0), R(0)};
                R ke2 = R(0);
                int nbB = 0;
                for (int i = 0; i < n; ++i) {
                    for (int k = 0; k < 3; ++k) {
                        const R vk = srec[lo + i].v[k];
                        sum[k] = sum[k] + vk;
                        ke2 = ke2 + vk * vk;
                    }
                    nbB += (srec[lo + i].fid & F_B) ? 1 : 0;
                }
                if (n >= 2) {
                    R vcm[3] = {sum[0] / (R)n, sum[1] / (R)n, sum[2] / (R)n};
                    R ke = R(0);
                    for (int i = 0; i < n; ++i)
                        for (int k = 0; k < 3; ++k) {
                            const R u = srec[lo + i].v[k] - vcm[k];
                            ke = ke + u * u;
                        }
                    acc[0] += (double)(ke / (R)(n - 1));
                    acc[1] += 1.0;
                }
                acc[2] += (double)sum[0]; acc[3] += (double)sum[1]; acc[4] += (double)sum[2];
                acc[5] += 0.5 * (double)ke2;
                acc[6] += (double)nbB;
                acc[7] += (double)n;
            }
            __syncthreads();
        }
        cb = ce;
    }

    if (opts & CP_OBS) {
        const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            double x = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) s_red[wid][k] = x;
        }
        __syncthreads();
        if (tid < 8) {
            double x = 0.0;
            for (int w = 0; w < CP_THREADS / 32; ++w) x += s_red[w][tid];
            d.obs_part[(long long)tile * 8 + tid] = x;
        }
    }
}

size_t cellpass_smem(bool mixed)
{
    if (mixed) return (size_t)TP_M * (sizeof(RecM) + 2 * sizeof(int) + 1);
    return (size_t)TP_D * (sizeof(RecD) + 2 * sizeof(int) + 1);
}

void launch_cellpass(bool mixed, const Dev &d, const CellPassArgs &a, cudaStream_t s)
{
    if (d.n_tiles == 0) return;
    const size_t sm = cellpass_smem(mixed);
    if (mixed) {
        cudaFuncSetAttribute(k_cellpass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_cellpass<true><<<d.n_tiles, CP_THREADS, sm, s>>>(d, a);
    } else {
        cudaFuncSetAttribute(k_cellpass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_cellpass<false><<<d.n_tiles, CP_THREADS, sm, s>>>(d, a);
    }
}

}  // namespace rmpcd
