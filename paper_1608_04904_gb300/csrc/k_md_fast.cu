// k_md_fast.cu -- near-colloid MD for replicas with few colloids (at most
// MD_FAST_NC: the sphere-dimer motor or a single sphere) and no
// colloid-colloid potential: §1.1 velocity Verlet, §1.4 WCA forces and exact
// RATTLE, §1.5 catalytic A -> B.
//
// Every thread of every CTA of the replica's cluster keeps the complete state
// of the (at most MD_FAST_NC) colloids in registers and integrates it itself:
// all threads compute identical colloid trajectories from the identical force
// totals, so no thread waits for another to update the colloids, and the
// colloid update needs no data exchange.  The colloid forces are 64-bit fixed-point
// sums: per thread, per warp (shuffles), then one atomic add per warp and
// component into a triple-buffered accumulator in the shared memory of CTA 0
// of the cluster.  One barrier (the cluster barrier, or the CTA barrier for a
// lone CTA) per sub-step separates the additions from the reads.
//
// The colloid arithmetic is the same, operation by operation, as the general
// MD kernel's (FP64 for the fp64 path, integer cell + FP32 for the mixed path),
// so both kernels give bit-identical results.
#include <cooperative_groups.h>
#include <type_traits>

#include "rmpcd_kernels.cuh"

namespace cg = cooperative_groups;

namespace rmpcd {

constexpr int NC = MD_FAST_NC;

// One warp per SM sub-partition; the CTA is small because every thread repeats
// the colloid update.
template <int CS> struct FGeom {
    static constexpr int NT = 128;
};
constexpr int PPT = 4;   // near particles a thread keeps in registers

struct __align__(16) FWorkM {
    int c[3];
    uint32_t fid;
    float o[3];
    int slot;
    float v[3];
    float p0;
    float f[3];
    float p1;
};
struct __align__(16) FWorkD {
    double x[3];
    double v[3];
    double f[3];
    uint32_t fid;
    int slot;
};

struct FShared {
    unsigned long long tot[3][NC * 3];   // cluster totals (used in CTA 0)
    float sigf[NC], epsAf[NC], epsBf[NC], rc2f[NC];
    double sig[NC], epsA[NC], epsB[NC], rc2[NC];
    int cat[NC];
    int nn;
};

// --- complete colloid state in every thread ----------------------------------
// mixed: unwrapped integer cell, wrapped cell, FP32 offset in [0,1), FP32
// velocity and force (the same representation as the general MD kernel)
struct ColRM {
    int Xi[NC][3], Ci[NC][3], Xoi[NC][3], X0i[NC][3];
    float Xf[NC][3], Xof[NC][3], X0f[NC][3], V[NC][3], F[NC][3], invM[NC];
};
// fp64: unwrapped positions (same operations as the FP64 oracle)
struct ColRD {
    double X[NC][3], V[NC][3], F[NC][3], Xold[NC][3], X0[NC][3], Xw[NC][3], M[NC];
};

__device__ __forceinline__ void carry(const ReplicaDev &rp, ColRM &C, int j, int t)
{
    const float fl = floorf(C.Xf[j][t]);
    int k = (int)fl;
    float f = C.Xf[j][t] - fl;
    if (f >= 1.0f) { f = 0.0f; k += 1; }
    C.Xf[j][t] = f;
    C.Xi[j][t] += k;
    int ci = C.Ci[j][t] + k;
    if (ci >= rp.L[t] || ci < 0) ci = imod(ci, rp.L[t]);
    C.Ci[j][t] = ci;
}

__device__ __forceinline__ void kick_drift(const ReplicaDev &rp, ColRM &C, int nc)
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            C.V[j][t] = fmaf(rp.hdt_f, C.F[j][t] * C.invM[j], C.V[j][t]);
            C.Xoi[j][t] = C.Xi[j][t];
            C.Xof[j][t] = C.Xf[j][t];
            C.Xf[j][t] = fmaf(rp.dt_f, C.V[j][t], C.Xf[j][t]);
            carry(rp, C, j, t);
        }
    }
}

// Exact RATTLE position stage (Andersen 1983) for each bond.  With at most
// two colloids every bond joins colloids 0 and 1; the order of its ends does
// not matter (swapping them negates the bond vector exactly), and fixed
// indices keep the colloid arrays in registers.
__device__ __forceinline__ void rattle_pos(const ReplicaDev &rp, ColRM &C, const BondDev *bond, int nbond)
{
    const float idt = 1.0f / rp.dt_f;
    for (int k = 0; k < nbond; ++k) {
        constexpr int a = 0, b = 1;
        const float dd = (float)bond[k].d;
        float ro[3], rn[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            ro[t] = (float)(C.Xoi[a][t] - C.Xoi[b][t]) + (C.Xof[a][t] - C.Xof[b][t]);
            rn[t] = (float)(C.Xi[a][t] - C.Xi[b][t]) + (C.Xf[a][t] - C.Xf[b][t]);
        }
        const float inv = C.invM[a] + C.invM[b];
        const float oo = ro[0] * ro[0] + ro[1] * ro[1] + ro[2] * ro[2];
        const float on = rn[0] * ro[0] + rn[1] * ro[1] + rn[2] * ro[2];
        const float nn = rn[0] * rn[0] + rn[1] * rn[1] + rn[2] * rn[2];
        const float qa = inv * inv * oo;
        const float qb = 2.0f * inv * on;
        const float qc = nn - dd * dd;
        float disc = qb * qb - 4.0f * qa * qc;
        if (disc < 0.0f) disc = 0.0f;
        const float q = -0.5f * (qb + copysignf(sqrtf(disc), qb));
        const float gmul = qc / q;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const float ca = gmul * ro[t] * C.invM[a];
            const float cb = gmul * ro[t] * C.invM[b];
            C.Xf[a][t] += ca;
            C.Xf[b][t] -= cb;
            C.V[a][t] += ca * idt;
            C.V[b][t] -= cb * idt;
            carry(rp, C, a, t);
            carry(rp, C, b, t);
        }
    }
}

__device__ __forceinline__ void kick_rattle_vel(const ReplicaDev &rp, ColRM &C, int nc, const BondDev *bond, int nbond)
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
#pragma unroll
        for (int t = 0; t < 3; ++t) C.V[j][t] = fmaf(rp.hdt_f, C.F[j][t] * C.invM[j], C.V[j][t]);
    }
    for (int k = 0; k < nbond; ++k) {
        constexpr int a = 0, b = 1;
        float r[3], dv[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            r[t] = (float)(C.Xi[a][t] - C.Xi[b][t]) + (C.Xf[a][t] - C.Xf[b][t]);
            dv[t] = C.V[a][t] - C.V[b][t];
        }
        const float inv = C.invM[a] + C.invM[b];
        const float rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const float rv = dv[0] * r[0] + dv[1] * r[1] + dv[2] * r[2];
        const float kk = rv / (rr * inv);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            C.V[a][t] -= kk * r[t] * C.invM[a];
            C.V[b][t] += kk * r[t] * C.invM[b];
        }
    }
}

__device__ __forceinline__ void kick_drift(const ReplicaDev &rp, ColRD &C, int nc)
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            C.V[j][t] = fma(rp.hdt, C.F[j][t] / C.M[j], C.V[j][t]);
            C.Xold[j][t] = C.X[j][t];
            C.X[j][t] = fma(rp.dt, C.V[j][t], C.X[j][t]);
        }
    }
}

__device__ __forceinline__ void rattle_pos(const ReplicaDev &rp, ColRD &C, const BondDev *bond, int nbond)
{
    const double dt = rp.dt;
    for (int k = 0; k < nbond; ++k) {
        constexpr int a = 0, b = 1;
        const double dd = bond[k].d;
        double ro[3], rn[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            ro[t] = C.Xold[a][t] - C.Xold[b][t];
            rn[t] = C.X[a][t] - C.X[b][t];
        }
        const double inv = 1.0 / C.M[a] + 1.0 / C.M[b];
        const double oo = ro[0] * ro[0] + ro[1] * ro[1] + ro[2] * ro[2];
        const double on = rn[0] * ro[0] + rn[1] * ro[1] + rn[2] * ro[2];
        const double nn = rn[0] * rn[0] + rn[1] * rn[1] + rn[2] * rn[2];
        const double qa = inv * inv * oo;
        const double qb = 2.0 * inv * on;
        const double qc = nn - dd * dd;
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc < 0.0) disc = 0.0;
        const double q = -0.5 * (qb + copysign(sqrt(disc), qb));
        const double gmul = qc / q;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const double ca = gmul * ro[t] / C.M[a];
            const double cb = gmul * ro[t] / C.M[b];
            C.X[a][t] = C.X[a][t] + ca;
            C.X[b][t] = C.X[b][t] - cb;
            C.V[a][t] = C.V[a][t] + ca / dt;
            C.V[b][t] = C.V[b][t] - cb / dt;
        }
    }
}

__device__ __forceinline__ void kick_rattle_vel(const ReplicaDev &rp, ColRD &C, int nc, const BondDev *bond, int nbond)
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
#pragma unroll
        for (int t = 0; t < 3; ++t) C.V[j][t] = fma(rp.hdt, C.F[j][t] / C.M[j], C.V[j][t]);
    }
    for (int k = 0; k < nbond; ++k) {
        constexpr int a = 0, b = 1;
        double r[3], dv[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            r[t] = C.X[a][t] - C.X[b][t];
            dv[t] = C.V[a][t] - C.V[b][t];
        }
        const double inv = 1.0 / C.M[a] + 1.0 / C.M[b];
        const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double rv = dv[0] * r[0] + dv[1] * r[1] + dv[2] * r[2];
        const double kk = rv / (rr * inv);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            C.V[a][t] = C.V[a][t] - kk * r[t] / C.M[a];
            C.V[b][t] = C.V[b][t] + kk * r[t] / C.M[b];
        }
    }
}

__device__ __forceinline__ void frames(const ReplicaDev &, ColRM &, int) {}
__device__ __forceinline__ void frames(const ReplicaDev &rp, ColRD &C, int nc)
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double L = (double)rp.L[k];
            C.Xw[j][k] = C.X[j][k] - L * floor(C.X[j][k] / L);
        }
    }
}

__device__ __forceinline__ void set_forces(ColRM &C, const long long *tot, int nc)
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
#pragma unroll
        for (int t = 0; t < 3; ++t) C.F[j][t] = __ll2float_rn(tot[3 * j + t]) * 0x1p-40f;
    }
}
__device__ __forceinline__ void set_forces(ColRD &C, const long long *tot, int nc)
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
#pragma unroll
        for (int t = 0; t < 3; ++t) C.F[j][t] = (double)tot[3 * j + t] * 0x1p-40;
    }
}

// --- particle side ----------------------------------------------------------
// WCA force on one solvent particle (§1.4); the reaction on colloid j goes to
// acc in fixed point.
__device__ __forceinline__ void pforce(const ReplicaDev &rp, const FShared &S, const ColRM &C, int nc, FWorkM &w,
                                       long long acc[NC][3])
{
    w.f[0] = w.f[1] = w.f[2] = 0.0f;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
        float d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = (float)(w.c[k] - C.Ci[j][k]) + (w.o[k] - C.Xf[j][k]);
        min_image(rp, d);
        const float eps = (w.fid & F_B) ? S.epsBf[j] : S.epsAf[j];
        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < S.rc2f[j]) {
            const float ir2 = 1.0f / r2;
            const float s2 = S.sigf[j] * S.sigf[j] * ir2;
            const float s6 = s2 * s2 * s2;
            const float fr = 24.0f * eps * s6 * (2.0f * s6 - 1.0f) * ir2;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float fk = fr * d[k];
                w.f[k] = w.f[k] + fk;
                acc[j][k] -= __float2ll_rn(fk * 0x1p40f);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) w.f[k] = w.f[k] + rp.g_f[k];
}

__device__ __forceinline__ void pforce(const ReplicaDev &rp, const FShared &S, const ColRD &C, int nc, FWorkD &w,
                                       long long acc[NC][3])
{
    w.f[0] = w.f[1] = w.f[2] = 0.0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
        double d[3] = {w.x[0] - C.Xw[j][0], w.x[1] - C.Xw[j][1], w.x[2] - C.Xw[j][2]};
        min_image(rp, d);
        const double eps = (w.fid & F_B) ? S.epsB[j] : S.epsA[j];
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < S.rc2[j]) {
            const double ir2 = 1.0 / r2;
            const double s2 = S.sig[j] * S.sig[j] * ir2;
            const double s6 = s2 * s2 * s2;
            const double fr = 24.0 * eps * s6 * (2.0 * s6 - 1.0) * ir2;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double fk = fr * d[k];
                w.f[k] = w.f[k] + fk;
                acc[j][k] -= __double2ll_rn(fk * 0x1p40);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) w.f[k] = w.f[k] + rp.g[k];
}

__device__ __forceinline__ bool pinside(const ReplicaDev &rp, const FShared &S, const ColRM &C, int nc,
                                        const FWorkM &w)
{
    bool in = false;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
        if (!S.cat[j]) continue;
        float d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = (float)(w.c[k] - C.Ci[j][k]) + (w.o[k] - C.Xf[j][k]);
        min_image(rp, d);
        in = in || (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < S.rc2f[j]);
    }
    return in;
}
__device__ __forceinline__ bool pinside(const ReplicaDev &rp, const FShared &S, const ColRD &C, int nc,
                                        const FWorkD &w)
{
    bool in = false;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
        if (!S.cat[j]) continue;
        double d[3] = {w.x[0] - C.Xw[j][0], w.x[1] - C.Xw[j][1], w.x[2] - C.Xw[j][2]};
        min_image(rp, d);
        in = in || (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < S.rc2[j]);
    }
    return in;
}

// A tagged A particle that has left every catalytic range becomes B with
// probability cat_prob (§1.5); an A particle inside a range is tagged.
__device__ __forceinline__ uint32_t fcatalysis(const ReplicaDev &rp, uint32_t fid, bool inside, uint32_t step, int s)
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

__device__ __forceinline__ void pkick_drift(const ReplicaDev &rp, FWorkM &w, bool second)
{
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        if (second) w.v[t] = fmaf(rp.hdt_f, w.f[t], w.v[t]);
        w.v[t] = fmaf(rp.hdt_f, w.f[t], w.v[t]);
        w.o[t] = fmaf(rp.dt_f, w.v[t], w.o[t]);
    }
}
__device__ __forceinline__ void pkick_drift(const ReplicaDev &rp, FWorkD &w, bool second)
{
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        if (second) w.v[t] = fma(rp.hdt, w.f[t], w.v[t]);
        w.v[t] = fma(rp.hdt, w.f[t], w.v[t]);
        w.x[t] = fma(rp.dt, w.v[t], w.x[t]);
    }
}

// Exact warp sum of a 64-bit fixed-point value by three 32-bit reductions:
// x = hi 2^32 + mid 2^16 + lo with mid, lo in [0, 2^16).  Per-lane |x| < 2^58
// keeps the sum of the hi parts inside 32 bits.
__device__ __forceinline__ long long warp_sum64(long long x)
{
    const int hi = (int)(x >> 32);
    const unsigned mid = (unsigned)((unsigned long long)x >> 16) & 0xFFFFu;
    const unsigned lo = (unsigned)x & 0xFFFFu;
    const int H = __reduce_add_sync(0xffffffffu, hi);
    const unsigned M = __reduce_add_sync(0xffffffffu, mid);
    const unsigned Lo = __reduce_add_sync(0xffffffffu, lo);
    return ((long long)H << 32) + ((long long)M << 16) + (long long)Lo;
}

// Warp sums of the fixed-point partials added into the round's buffer of the
// cluster accumulator (CTA 0's shared memory).
template <int CS>
__device__ __forceinline__ void contribute(cg::cluster_group &cl, FShared &S, long long acc[NC][3], int nc, int buf,
                                           int lane)
{
    unsigned long long mine = 0ull;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const long long x = warp_sum64(acc[j][k]);
            if (lane == 3 * j + k) mine = (unsigned long long)x;
        }
    }
    if (lane < 3 * nc && mine != 0ull) {
        unsigned long long *dst = &S.tot[buf][lane];
        if (CS > 1) dst = cl.map_shared_rank(dst, 0);
        atomicAdd(dst, mine);
    }
}

// Every thread reads the round's totals (broadcast reads of CTA 0's buffer).
template <int CS>
__device__ __forceinline__ void read_totals(cg::cluster_group &cl, FShared &S, int buf, int nc, long long *tot)
{
    unsigned long long *src = &S.tot[buf][0];
    if (CS > 1) src = cl.map_shared_rank(src, 0);
#pragma unroll
    for (int i = 0; i < 3 * NC; ++i)
        tot[i] = i < 3 * nc ? (long long)((volatile unsigned long long *)src)[i] : 0ll;
}

template <int CS>
__device__ __forceinline__ void round_barrier(cg::cluster_group &cl)
{
    if (CS > 1) cl.sync();
    else __syncthreads();
}


__device__ __forceinline__ void zero_acc(long long acc[NC][3])
{
#pragma unroll
    for (int j = 0; j < NC; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[j][k] = 0;
}

template <bool MIXED, typename ColR, typename W>
__device__ __forceinline__ void load_particle(const Dev &d, const ReplicaDev &rp, const FShared &S, const ColR &C, int nc,
                                              int slot, int rbuf, W &w, long long acc[NC][3])
{
    w.slot = slot;
    if constexpr (MIXED) {
        RecM rec = load_rec(reinterpret_cast<const RecM *>(d.rec[rbuf]) + slot);
        for (int q = 0; q < 3; ++q) { w.c[q] = cw_get(rec.cw, q); w.o[q] = rec.o[q]; w.v[q] = rec.v[q]; }
        w.fid = rec.fid;
    } else {
        RecD rec = load_rec(reinterpret_cast<const RecD *>(d.rec[rbuf]) + slot);
        for (int q = 0; q < 3; ++q) { w.x[q] = rec.x[q]; w.v[q] = rec.v[q]; }
        w.fid = rec.fid;
    }
    pforce(rp, S, C, nc, w, acc);
}

template <typename ColR, typename W>
__device__ __forceinline__ void substep_particle(const ReplicaDev &rp, const FShared &S, const ColR &C, int nc, W &w,
                                                 long long acc[NC][3], uint32_t step, int s)
{
    pkick_drift(rp, w, s > 0);
    pforce(rp, S, C, nc, w, acc);
    w.fid = fcatalysis(rp, w.fid, pinside(rp, S, C, nc, w), step, s);
}

__device__ __forceinline__ void finish_particle(const Dev &d, const ReplicaDev &rp, FWorkM &w, const double sh[3],
                                                int rbuf, int bbuf, int do_bin)
{
    for (int q = 0; q < 3; ++q) w.v[q] = fmaf(rp.hdt_f, w.f[q], w.v[q]);
    renorm_m(rp, w.c, w.o);
    RecM rec;
    rec.cw = cw_make(w.c[0], w.c[1], w.c[2]);
    for (int q = 0; q < 3; ++q) { rec.o[q] = w.o[q]; rec.v[q] = w.v[q]; }
    rec.fid = do_bin ? (w.fid | F_PROP) : (w.fid & ~F_PROP);
    store_rec(reinterpret_cast<RecM *>(d.rec[rbuf]) + w.slot, rec);
    if (do_bin) {
        float sf[3] = {(float)sh[0], (float)sh[1], (float)sh[2]};
        bin_particle(d, bbuf, rp.cell_off + cell_key_m(rp, w.c, w.o, sf), w.slot);
    }
}

__device__ __forceinline__ void finish_particle(const Dev &d, const ReplicaDev &rp, FWorkD &w, const double sh[3],
                                                int rbuf, int bbuf, int do_bin)
{
    for (int q = 0; q < 3; ++q) w.v[q] = fma(rp.hdt, w.f[q], w.v[q]);
    wrap_periodic_d(rp, w.x);
    RecD rec;
    for (int q = 0; q < 3; ++q) { rec.x[q] = w.x[q]; rec.v[q] = w.v[q]; }
    rec.fid = do_bin ? (w.fid | F_PROP) : (w.fid & ~F_PROP);
    rec.u0 = 0u;
    rec.u1 = 0.0;
    store_rec(reinterpret_cast<RecD *>(d.rec[rbuf]) + w.slot, rec);
    if (do_bin) bin_particle(d, bbuf, rp.cell_off + cell_key_d(rp, w.x, sh), w.slot);
}

template <bool MIXED, int CS>
__global__ void __launch_bounds__(FGeom<CS>::NT, 1) k_md_fast(Dev d, uint32_t step, int rbuf, int bbuf, int do_bin)
{
    using W = typename std::conditional<MIXED, FWorkM, FWorkD>::type;
    using ColR = typename std::conditional<MIXED, ColRM, ColRD>::type;
    constexpr int NT = FGeom<CS>::NT;
    __shared__ FShared S;
    __shared__ ReplicaDev s_rp;
    __shared__ BondDev s_bond[MAXB];
    cg::cluster_group cl = cg::this_cluster();
    const int r = blockIdx.x / CS;
    const int tid = threadIdx.x, lane = tid & 31;
    const int rank = CS == 1 ? 0 : (int)cl.block_rank();
    if (tid == 0) s_rp = d.rep[r];
    __syncthreads();
    const ReplicaDev &rp = s_rp;
    if (rp.n_col == 0) return;   // uniform over the cluster
    const int nc = rp.n_col, nbond = rp.n_bond;
    if (tid == 0) S.nn = min(d.near_count[r], rp.n_part);
    if (tid < nc) {
        const int g = rp.col_off + tid;
        S.sig[tid] = d.colSig[g]; S.epsA[tid] = d.colEpsA[g]; S.epsB[tid] = d.colEpsB[g]; S.rc2[tid] = d.colRc2[g];
        S.sigf[tid] = d.colSig_f[g]; S.epsAf[tid] = d.colEpsA_f[g]; S.epsBf[tid] = d.colEpsB_f[g];
        S.rc2f[tid] = d.colRc2_f[g];
        S.cat[tid] = d.colCat[g];
    }
    if (tid < nbond) s_bond[tid] = d.bonds[rp.bond_off + tid];
    if (tid < 3 * 3 * NC) (&S.tot[0][0])[tid] = 0ull;

    // the complete colloid state, in every thread
    ColR C;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const int g = rp.col_off + (j < nc ? j : 0);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if constexpr (MIXED) {
                C.Xi[j][t] = d.colXi[3 * g + t];
                C.Xf[j][t] = d.colXf[3 * g + t];
                C.Ci[j][t] = d.colCi[3 * g + t];
                C.V[j][t] = d.colVf[3 * g + t];
                C.Xoi[j][t] = C.Xi[j][t]; C.Xof[j][t] = C.Xf[j][t];
                C.X0i[j][t] = C.Xi[j][t]; C.X0f[j][t] = C.Xf[j][t];
                C.F[j][t] = 0.0f;
            } else {
                C.X[j][t] = d.colX[3 * g + t];
                C.V[j][t] = d.colV[3 * g + t];
                C.Xold[j][t] = C.X[j][t]; C.X0[j][t] = C.X[j][t];
                C.F[j][t] = 0.0;
            }
        }
        if constexpr (MIXED) C.invM[j] = d.colInvM_f[g];
        else C.M[j] = d.colM[g];
    }
    frames(rp, C, nc);
    __syncthreads();
    // every CTA has read near_count before CTA 0 may reset it
    if (CS > 1) cl.sync();

    const int nn = S.nn;
    const int *list = d.near_list + rp.part_off;
    W *work = reinterpret_cast<W *>(d.md_work) + rp.part_off;
    const int first = rank * NT + tid;
    const int stride = CS * NT;
    const int over = first + PPT * stride;   // beyond the registers: global memory
    long long acc[NC][3];
    long long tot[3 * NC];
    W reg[PPT];
    // round 0: forces at the start of the interval
    zero_acc(acc);
#pragma unroll
    for (int p = 0; p < PPT; ++p)
        if (first + p * stride < nn) load_particle<MIXED>(d, rp, S, C, nc, list[first + p * stride], rbuf, reg[p], acc);
    for (int k = over; k < nn; k += stride) {
        W w;
        load_particle<MIXED>(d, rp, S, C, nc, list[k], rbuf, w, acc);
        work[k] = w;
    }
    contribute<CS>(cl, S, acc, nc, 0, lane);
    round_barrier<CS>(cl);
    read_totals<CS>(cl, S, 0, nc, tot);
    set_forces(C, tot, nc);

    for (int s = 0; s < rp.n_md; ++s) {
        const int buf = (s + 1) % 3;
        // CTA 0 clears the buffer of round s + 2 (last read before this barrier)
        if (rank == 0 && tid < 3 * nc) S.tot[(s + 2) % 3][tid] = 0ull;
        // colloids: first half kick, drift, RATTLE position stage
        kick_drift(rp, C, nc);
        rattle_pos(rp, C, s_bond, nbond);
        frames(rp, C, nc);
        // solvent: second half kick of the previous sub-step, first half
        // kick and drift of this one, new forces, catalytic conversion
        zero_acc(acc);
#pragma unroll
        for (int p = 0; p < PPT; ++p)
            if (first + p * stride < nn) substep_particle(rp, S, C, nc, reg[p], acc, step, s);
        for (int k = over; k < nn; k += stride) {
            W w = work[k];
            substep_particle(rp, S, C, nc, w, acc, step, s);
            work[k] = w;
        }
        contribute<CS>(cl, S, acc, nc, buf, lane);
        round_barrier<CS>(cl);
        read_totals<CS>(cl, S, buf, nc, tot);
        set_forces(C, tot, nc);
        // colloids: second half kick, RATTLE velocity stage
        kick_rattle_vel(rp, C, nc, s_bond, nbond);
    }

    // last half kick, wrap, write back (and bin for the collision of `step`)
    double sh[3];
    grid_shift(rp.seed, step, sh);
#pragma unroll
    for (int p = 0; p < PPT; ++p)
        if (first + p * stride < nn) finish_particle(d, rp, reg[p], sh, rbuf, bbuf, do_bin);
    for (int k = over; k < nn; k += stride) {
        W w = work[k];
        finish_particle(d, rp, w, sh, rbuf, bbuf, do_bin);
    }
    // CTA 0, thread 0: colloids back to memory, skin check, near list reset
    if (rank == 0 && tid == 0) {
        bool bad = false;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (j >= nc) continue;
            const int g = rp.col_off + j;
            if constexpr (MIXED) {
                float e[3];
                for (int t = 0; t < 3; ++t) {
                    d.colXi[3 * g + t] = C.Xi[j][t];
                    d.colXf[3 * g + t] = C.Xf[j][t];
                    d.colVf[3 * g + t] = C.V[j][t];
                    d.colCi[3 * g + t] = C.Ci[j][t];
                    e[t] = (float)(C.Xi[j][t] - C.X0i[j][t]) + (C.Xf[j][t] - C.X0f[j][t]);
                }
                const float dd = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
                if (!(dd <= rp.skin_f * rp.skin_f)) bad = true;
            } else {
                double dd = 0.0;
                for (int t = 0; t < 3; ++t) {
                    d.colX[3 * g + t] = C.X[j][t];
                    d.colV[3 * g + t] = C.V[j][t];
                    const double e = C.X[j][t] - C.X0[j][t];
                    dd = dd + e * e;
                }
                if (!(dd <= rp.skin * rp.skin)) bad = true;
            }
        }
        if (bad) atomicAdd(&d.err[ERR_SKIN], 1u);
        d.near_count[r] = 0;
    }
    if (CS > 1) cl.sync();   // CTA 0's accumulator outlives every remote access
}

template <bool MIXED, int CS>
static void launch_fast_cs(const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, cudaStream_t s)
{
    if (CS > 8) cudaFuncSetAttribute(k_md_fast<MIXED, CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(d.n_rep * CS), 1, 1);
    cfg.blockDim = dim3(FGeom<CS>::NT, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_md_fast<MIXED, CS>, d, step, rbuf, bbuf, do_bin);
}

void launch_md_fast(bool mixed, const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, int cs, cudaStream_t s)
{
    if (d.n_rep <= 0) return;
    switch (cs) {
    case 1: mixed ? launch_fast_cs<true, 1>(d, step, rbuf, bbuf, do_bin, s) : launch_fast_cs<false, 1>(d, step, rbuf, bbuf, do_bin, s); break;
    case 2: mixed ? launch_fast_cs<true, 2>(d, step, rbuf, bbuf, do_bin, s) : launch_fast_cs<false, 2>(d, step, rbuf, bbuf, do_bin, s); break;
    case 4: mixed ? launch_fast_cs<true, 4>(d, step, rbuf, bbuf, do_bin, s) : launch_fast_cs<false, 4>(d, step, rbuf, bbuf, do_bin, s); break;
    case 8: mixed ? launch_fast_cs<true, 8>(d, step, rbuf, bbuf, do_bin, s) : launch_fast_cs<false, 8>(d, step, rbuf, bbuf, do_bin, s); break;
    default: mixed ? launch_fast_cs<true, 16>(d, step, rbuf, bbuf, do_bin, s) : launch_fast_cs<false, 16>(d, step, rbuf, bbuf, do_bin, s); break;
    }
}

// Largest cluster size the device can schedule for the few-colloid kernel.
int md_fast_max_cluster(bool mixed)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(FGeom<16>::NT, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e;
    if (mixed) {
        cudaFuncSetAttribute(k_md_fast<true, 16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        e = cudaOccupancyMaxActiveClusters(&n, k_md_fast<true, 16>, &cfg);
    } else {
        cudaFuncSetAttribute(k_md_fast<false, 16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        e = cudaOccupancyMaxActiveClusters(&n, k_md_fast<false, 16>, &cfg);
    }
    cudaGetLastError();
    return (e == cudaSuccess && n > 0) ? 16 : 8;
}

}  // namespace rmpcd
