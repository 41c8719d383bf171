// k_particles.cu -- particle-parallel kernels: state conversion, the granular
// interval flight and binning (§1.1 streaming, §1.4 grid shift and sort), and
// the final reduction of the observables (§1.4 temperature estimator).
#include <algorithm>

#include "rmpcd_kernels.cuh"

namespace rmpcd {

// Replica of a global storage slot (replicas are contiguous and in order).
__device__ __forceinline__ int replica_of(const Dev &d, int slot)
{
    int lo = 0, hi = d.n_rep - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (d.rep[mid].part_off <= slot) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// State conversion: canonical FP64 arrays <-> records.
// ---------------------------------------------------------------------------
__global__ void k_set_state_m(Dev d, int r, int n, const double *x, const double *v, const uint8_t *fl, int rbuf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ReplicaDev rp = d.rep[r];
    RecM rec;
    int c[3];
    for (int k = 0; k < 3; ++k) {
        double xk = x[3 * i + k];
        int ck = (int)floor(xk);
        if (ck < 0) ck = 0;
        if (ck > rp.L[k] - 1) ck = rp.L[k] - 1;
        c[k] = ck;
        rec.o[k] = (float)(xk - (double)ck);
        rec.v[k] = (float)v[3 * i + k];
    }
    rec.cw = cw_make(c[0], c[1], c[2]);
    uint8_t f = fl ? fl[i] : 0;
    rec.fid = (uint32_t)i | ((f & 1) ? F_B : 0u) | ((f & 2) ? F_TAG : 0u);
    store_rec(reinterpret_cast<RecM *>(d.rec[rbuf]) + rp.part_off + i, rec);
}

__global__ void k_set_state_d(Dev d, int r, int n, const double *x, const double *v, const uint8_t *fl, int rbuf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int off = d.rep[r].part_off;
    RecD rec;
    for (int k = 0; k < 3; ++k) { rec.x[k] = x[3 * i + k]; rec.v[k] = v[3 * i + k]; }
    uint8_t f = fl ? fl[i] : 0;
    rec.fid = (uint32_t)i | ((f & 1) ? F_B : 0u) | ((f & 2) ? F_TAG : 0u);
    rec.u0 = 0u;
    rec.u1 = 0.0;
    store_rec(reinterpret_cast<RecD *>(d.rec[rbuf]) + off + i, rec);
}

__global__ void k_get_state_m(Dev d, int r, int n, int rbuf, double *x, double *v, uint8_t *fl, uint32_t *id,
                              int32_t *cell, int has_sort, uint32_t sort_step)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ReplicaDev rp = d.rep[r];
    RecM rec = load_rec(reinterpret_cast<const RecM *>(d.rec[rbuf]) + rp.part_off + i);
    int c[3] = {cw_get(rec.cw, 0), cw_get(rec.cw, 1), cw_get(rec.cw, 2)};
    for (int k = 0; k < 3; ++k) {
        if (x) x[3 * i + k] = (double)c[k] + (double)rec.o[k];
        if (v) v[3 * i + k] = (double)rec.v[k];
    }
    if (fl) fl[i] = (uint8_t)(((rec.fid & F_B) ? 1 : 0) | ((rec.fid & F_TAG) ? 2 : 0));
    if (id) id[i] = rec.fid & ID_MASK;
    if (cell) {
        if (has_sort) {
            double s[3];
            grid_shift(rp.seed, sort_step, s);
            float sf[3] = {(float)s[0], (float)s[1], (float)s[2]};
            cell[i] = cell_key_m(rp, c, rec.o, sf);
        } else {
            cell[i] = -1;
        }
    }
}

__global__ void k_get_state_d(Dev d, int r, int n, int rbuf, double *x, double *v, uint8_t *fl, uint32_t *id,
                              int32_t *cell, int has_sort, uint32_t sort_step)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ReplicaDev rp = d.rep[r];
    RecD rec = load_rec(reinterpret_cast<const RecD *>(d.rec[rbuf]) + rp.part_off + i);
    for (int k = 0; k < 3; ++k) {
        if (x) x[3 * i + k] = rec.x[k];
        if (v) v[3 * i + k] = rec.v[k];
    }
    if (fl) fl[i] = (uint8_t)(((rec.fid & F_B) ? 1 : 0) | ((rec.fid & F_TAG) ? 2 : 0));
    if (id) id[i] = rec.fid & ID_MASK;
    if (cell) {
        if (has_sort) {
            double s[3];
            grid_shift(rp.seed, sort_step, s);
            cell[i] = cell_key_d(rp, rec.x, s);
        } else {
            cell[i] = -1;
        }
    }
}

// ---------------------------------------------------------------------------
// Particle pass over every flat slot.
//   PM_STREAM: near-colloid particles join the near list (slot) and the near
//              area (record), the others fly over tau and are stored
//              (granular interval motion).
//   PM_BIN:    bin the stored positions on the grid of collision `step`
//              (index buckets of the flat layout).
//   PM_PRIME:  first interval of a fused run: a far particle's record, unmoved,
//              goes into the row of the cell of its flown position; near
//              particles go to the near area for the MD kernel.
// ---------------------------------------------------------------------------
// Near particle: its slot into the near list, its record into the near area.
template <class Rec>
__device__ __forceinline__ void add_near(const Dev &d, int r, const ReplicaDev &rp, int slot, const Rec &rec)
{
    const int k = atomicAdd(&d.near_count[r], 1);
    if (k < rp.n_part) {
        d.near_list[rp.part_off + k] = slot;
        store_rec(reinterpret_cast<Rec *>(d.near_rec) + rp.part_off + k, rec);
    } else {
        atomicOr(&d.err[ERR_BOUNDS], 1u);
    }
}

template <bool MIXED>
__global__ void k_particles(Dev d, int mode, uint32_t step, int rbuf, int bbuf)
{
    step = resolve_step(d, step);   // STEP_DEVICE: the step of the control block
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n_total) return;
    const int r = replica_of(d, i);
    const ReplicaDev &rp = d.rep[r];
    double s[3];
    if (mode != PM_STREAM) grid_shift(rp.seed, step, s);
    if (MIXED) {
        RecM *recs = reinterpret_cast<RecM *>(d.rec[rbuf]);
        RecM rec = load_rec(recs + i);
        int c[3] = {cw_get(rec.cw, 0), cw_get(rec.cw, 1), cw_get(rec.cw, 2)};
        if (mode == PM_BIN) {
            float sf[3] = {(float)s[0], (float)s[1], (float)s[2]};
            bin_particle(d, bbuf, bin_cell(d, rp.cell_off, cell_key_m(rp, c, rec.o, sf)), i);
            return;
        }
        if (rp.n_col > 0 && near_test_m(rp, rp.n_col, d.colCi + 3 * rp.col_off, d.colXf + 3 * rp.col_off,
                                        d.colRb_f + rp.col_off, c, rec.o, rec.v)) {
            add_near(d, r, rp, i, rec);
            return;
        }
        float o[3] = {rec.o[0], rec.o[1], rec.o[2]};
        float v[3] = {rec.v[0], rec.v[1], rec.v[2]};
        flight_m(rp, c, o, v);
        if (mode == PM_STREAM) {
            rec.cw = cw_make(c[0], c[1], c[2]);
            for (int k = 0; k < 3; ++k) { rec.o[k] = o[k]; rec.v[k] = v[k]; }
            store_rec(recs + i, rec);
        } else {
            float sf[3] = {(float)s[0], (float)s[1], (float)s[2]};
            bin_record(d, bbuf, bin_cell(d, rp.cell_off, cell_key_m(rp, c, o, sf)), rec);
        }
    } else {
        RecD *recs = reinterpret_cast<RecD *>(d.rec[rbuf]);
        RecD rec = load_rec(recs + i);
        if (mode == PM_BIN) {
            bin_particle(d, bbuf, bin_cell(d, rp.cell_off, cell_key_d(rp, rec.x, s)), i);
            return;
        }
        if (rp.n_col > 0 && near_test_d(d, rp, rec.x, rec.v)) {
            add_near(d, r, rp, i, rec);
            return;
        }
        double x[3] = {rec.x[0], rec.x[1], rec.x[2]};
        double v[3] = {rec.v[0], rec.v[1], rec.v[2]};
        flight_d(rp, x, v);
        if (mode == PM_STREAM) {
            for (int k = 0; k < 3; ++k) { rec.x[k] = x[k]; rec.v[k] = v[k]; }
            store_rec(recs + i, rec);
        } else {
            bin_record(d, bbuf, bin_cell(d, rp.cell_off, cell_key_d(rp, x, s)), rec);
        }
    }
}

// ---------------------------------------------------------------------------
// Flatten a fused run's state: every record of the rows of buffer b, of its
// overflow records and of the near area goes to the next free flat slot of its
// replica (in no particular order; a sorting pass follows).  fill[r] counts the
// records placed; it must end at n_part.
// ---------------------------------------------------------------------------
template <class Rec>
__device__ __forceinline__ void flat_put(const Dev &d, int r, int fbuf, int *fill, const Rec &rec)
{
    const ReplicaDev &rp = d.rep[r];
    const int k = atomicAdd(&fill[r], 1);
    if (k < rp.n_part) store_rec(reinterpret_cast<Rec *>(d.rec[fbuf]) + rp.part_off + k, rec);
    else atomicOr(&d.err[ERR_BOUNDS], 1u);
}

// One thread per cell; the 32 cells of a warp lie in one tile, so in one
// replica: the warp takes its slots with one atomic (a per-particle atomic on
// the replica's single counter serialises on that address).
template <class Rec>
__global__ void k_flatten_rows(Dev d, int b, int fbuf, int *fill)
{
    static_assert(CPT % 32 == 0, "a warp's cells share a tile");
    const long long nc = (long long)d.n_tiles * CPT;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); g0 < nc; g0 += stride) {
        const long long g = g0 + lane;   // g0 is a multiple of 32 and nc of CPT: every lane is in range
        const int n = max(0, min(d.count[b][g], d.cap));
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (tot == 0) continue;
        const int r = d.tile_rep[g0 / CPT];
        int base = 0;
        if (lane == 31) base = atomicAdd(&fill[r], tot);
        base = __shfl_sync(0xffffffffu, base, 31);
        const ReplicaDev &rp = d.rep[r];
        const Rec *rows = reinterpret_cast<const Rec *>(d.brec[b]);
        Rec *out = reinterpret_cast<Rec *>(d.rec[fbuf]) + rp.part_off;
        const int k0 = base + incl - n;
        for (int i = 0; i < n; ++i) {
            const int k = k0 + i;
            if (k < rp.n_part) store_rec(out + k, load_rec(rows + row_index(d, g, i)));
            else atomicOr(&d.err[ERR_BOUNDS], 1u);
        }
    }
}

template <class Rec>
__global__ void k_flatten_ovf(Dev d, int b, int fbuf, int *fill)
{
    const int no = min((int)d.ovf_n[b], d.ovf_cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < no; k += gridDim.x * blockDim.x) {
        const int2 q = d.ovf[b][k];
        const long long nc = (long long)d.n_tiles * CPT;
        if (q.x < 0 || q.x >= nc || q.y < 0 || q.y >= d.ovf_cap) { atomicOr(&d.err[ERR_BOUNDS], 1u); continue; }
        flat_put(d, d.tile_rep[q.x / CPT], fbuf, fill, load_rec(reinterpret_cast<const Rec *>(d.orec[b]) + q.y));
    }
}

template <class Rec>
__global__ void k_flatten_near(Dev d, int fbuf, int *fill)
{
    const int r = blockIdx.y;
    const ReplicaDev &rp = d.rep[r];
    const int nn = min(d.near_count[r], rp.n_part);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += gridDim.x * blockDim.x)
        flat_put(d, r, fbuf, fill, load_near<Rec>(d, rp, k));
}

__global__ void k_flatten_check(Dev d, const int *fill)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < d.n_rep; r += gridDim.x * blockDim.x)
        if (fill[r] != d.rep[r].n_part) atomicOr(&d.err[ERR_BOUNDS], 1u);
}

void launch_flatten(bool mixed, const Dev &d, int b, int fbuf, int *fill, cudaStream_t s)
{
    const long long nc = (long long)d.n_tiles * CPT;
    const int nb = (int)std::max<long long>(1, std::min<long long>((nc + 255) / 256, 8192));
    const dim3 gn(64, (unsigned)std::max(1, d.n_rep));
    if (mixed) {
        k_flatten_rows<RecM><<<nb, 256, 0, s>>>(d, b, fbuf, fill);
        k_flatten_ovf<RecM><<<64, 256, 0, s>>>(d, b, fbuf, fill);
        k_flatten_near<RecM><<<gn, 256, 0, s>>>(d, fbuf, fill);
    } else {
        k_flatten_rows<RecD><<<nb, 256, 0, s>>>(d, b, fbuf, fill);
        k_flatten_ovf<RecD><<<64, 256, 0, s>>>(d, b, fbuf, fill);
        k_flatten_near<RecD><<<gn, 256, 0, s>>>(d, fbuf, fill);
    }
    k_flatten_check<<<1, 256, 0, s>>>(d, fill);
}

// Per replica: sum the per-tile partial observables in tile order.
__global__ void k_obs_reduce(Dev d)
{
    const int r = blockIdx.x;
    const ReplicaDev &rp = d.rep[r];
    __shared__ double part[256][8];
    const int tid = threadIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // thread t sums tiles t, t + 256, ... in order; then a fixed tree
    for (int t = tid; t < rp.n_tiles; t += 256)
        for (int k = 0; k < 8; ++k) acc[k] += d.obs_part[(long long)(rp.tile_off + t) * 8 + k];
    for (int k = 0; k < 8; ++k) part[tid][k] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w)
            for (int k = 0; k < 8; ++k) part[tid][k] += part[tid + w][k];
        __syncthreads();
    }
    if (tid < 8) d.obs_out[r * 8 + tid] = part[0][tid];
}

// Slab profile of one replica along one axis (the flow profile of the
// Poiseuille set-up and the slab temperatures of the thermal-gradient set-up,
// §"Applications of RMPCDMD"; the histogram routine of the `common` module).
// Bin b = floor(x_axis * n_bins / L_axis), clamped to [0, n_bins).  Per bin:
// count, B count, sum v_k in units of 2^-32 and sum v_k^2 in units of 2^-24,
// each term rounded to nearest-even before the integer sum, so the result is
// exact and independent of the summation order.  Integer sums wrap modulo
// 2^64; only the final value must fit (|sum v_k| < 2^31, sum v_k^2 < 2^39).
template <bool MIXED>
__global__ void __launch_bounds__(256) k_profile(Dev d, int r, int rbuf, int axis, int n_bins, unsigned long long *acc)
{
    __shared__ unsigned long long sh[PROF_MAX_BINS * PROF_FIELDS];
    for (int k = threadIdx.x; k < n_bins * PROF_FIELDS; k += blockDim.x) sh[k] = 0ull;
    __syncthreads();
    const ReplicaDev &rp = d.rep[r];
    const double nb = (double)n_bins, len = (double)rp.L[axis];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rp.n_part; i += gridDim.x * blockDim.x) {
        double x, v[3];
        uint32_t fid;
        if (MIXED) {
            RecM rec = load_rec(reinterpret_cast<const RecM *>(d.rec[rbuf]) + rp.part_off + i);
            x = (double)cw_get(rec.cw, axis) + (double)rec.o[axis];
            for (int k = 0; k < 3; ++k) v[k] = (double)rec.v[k];
            fid = rec.fid;
        } else {
            RecD rec = load_rec(reinterpret_cast<const RecD *>(d.rec[rbuf]) + rp.part_off + i);
            x = rec.x[axis];
            for (int k = 0; k < 3; ++k) v[k] = rec.v[k];
            fid = rec.fid;
        }
        int b = (int)floor(x * nb / len);
        b = b < 0 ? 0 : (b > n_bins - 1 ? n_bins - 1 : b);
        unsigned long long *s = sh + PROF_FIELDS * b;
        atomicAdd(s, 1ull);
        if (fid & F_B) atomicAdd(s + 1, 1ull);
        for (int k = 0; k < 3; ++k) {
            atomicAdd(s + 2 + k, (unsigned long long)__double2ll_rn(v[k] * 0x1p32));
            atomicAdd(s + 5 + k, (unsigned long long)__double2ll_rn(v[k] * v[k] * 0x1p24));
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_bins * PROF_FIELDS; k += blockDim.x)
        if (sh[k]) atomicAdd(acc + k, sh[k]);
}

__global__ void k_set_step(Dev d, uint32_t step) { d.ctl->step = step; }

// Largest count of count buffer b (bucket-width tuner).
__global__ void k_count_max(Dev d, int b)
{
    const long long nc = (long long)d.n_tiles * CPT;
    unsigned int m = 0u;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x)
        m = max(m, (unsigned int)d.count[b][c]);
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m > 0u) atomicMax(d.maxcnt, m);
}

void launch_count_max(const Dev &d, int b, cudaStream_t s)
{
    const long long nc = (long long)d.n_tiles * CPT;
    const int nb = (int)std::min<long long>((nc + 255) / 256, 4096);
    if (nb > 0) k_count_max<<<nb, 256, 0, s>>>(d, b);
}

void launch_set_step(const Dev &d, uint32_t step, cudaStream_t s) { k_set_step<<<1, 1, 0, s>>>(d, step); }

void launch_set_state(bool mixed, const Dev &d, int replica, int n, const double *x, const double *v,
                      const uint8_t *flags, int rbuf, cudaStream_t s)
{
    if (n <= 0) return;
    int nb = (n + 255) / 256;
    if (mixed) k_set_state_m<<<nb, 256, 0, s>>>(d, replica, n, x, v, flags, rbuf);
    else k_set_state_d<<<nb, 256, 0, s>>>(d, replica, n, x, v, flags, rbuf);
}

void launch_get_state(bool mixed, const Dev &d, int replica, int n, int rbuf, double *x, double *v, uint8_t *flags,
                      uint32_t *id, int32_t *cell, int has_sort, uint32_t sort_step, cudaStream_t s)
{
    if (n <= 0) return;
    int nb = (n + 255) / 256;
    if (mixed) k_get_state_m<<<nb, 256, 0, s>>>(d, replica, n, rbuf, x, v, flags, id, cell, has_sort, sort_step);
    else k_get_state_d<<<nb, 256, 0, s>>>(d, replica, n, rbuf, x, v, flags, id, cell, has_sort, sort_step);
}

void launch_particles(bool mixed, const Dev &d, int mode, uint32_t step, int rbuf, int bbuf, cudaStream_t s)
{
    if (d.n_total <= 0) return;
    int nb = (d.n_total + 255) / 256;
    if (mixed) k_particles<true><<<nb, 256, 0, s>>>(d, mode, step, rbuf, bbuf);
    else k_particles<false><<<nb, 256, 0, s>>>(d, mode, step, rbuf, bbuf);
}

void launch_profile(bool mixed, const Dev &d, int replica, int n, int rbuf, int axis, int n_bins,
                    unsigned long long *acc, cudaStream_t s)
{
    if (n <= 0) return;
    // one pass over the replica; a few CTAs per SM so each bin's shared
    // partials are merged into the global sums only once per CTA
    int nb = (n + 255) / 256;
    if (nb > 4 * 152) nb = 4 * 152;
    if (mixed) k_profile<true><<<nb, 256, 0, s>>>(d, replica, rbuf, axis, n_bins, acc);
    else k_profile<false><<<nb, 256, 0, s>>>(d, replica, rbuf, axis, n_bins, acc);
}

void launch_obs_reduce(const Dev &d, cudaStream_t s)
{
    if (d.n_rep <= 0) return;
    k_obs_reduce<<<d.n_rep, 256, 0, s>>>(d);
}

}  // namespace rmpcd
