// k_md_fast.cu -- near-colloid MD for replicas with few colloids (at most
// MD_FAST_NC: the sphere-dimer motor or a single sphere) and no
// colloid-colloid potential: §1.1 velocity Verlet, §1.4 WCA forces and exact
// RATTLE, §1.5 catalytic A -> B.
//
// A thread-block cluster of CS CTAs integrates one replica.  The near
// solvent sits in registers, spread over all threads of the cluster; warp 0
// of every CTA holds the colloid state lane-parallel (lane 3 j + t holds
// axis t of colloid j) and integrates it from the force totals.  One round
// per force evaluation:
//   every warp: the colloid positions from shared memory, the force on each
//               of its particles (the WCA part only inside the cut-off),
//               warp sums of the reaction forces to shared memory;
//   CTA barrier;
//   warp 0:     the CTA's partials to every CTA of the cluster (st.async,
//               counted on each CTA's mbarrier);
//   every warp: its particles' catalytic test and move to the next round;
//   warp 0:     waits for the round's partials, sums them, runs the colloid
//               second half kick + RATTLE velocity stage, first half kick +
//               drift + RATTLE position stage, and writes the new positions
//               to shared memory;
//   CTA barrier.
// Forces on the colloids are 64-bit fixed-point sums (2^-40), exact and
// independent of the order of the near list and of the cluster size.
//
// The colloid arithmetic is the same, operation by operation, as the general
// MD kernel's (FP64 for the fp64 path, integer cell + FP32 for the mixed path),
// so both kernels give bit-identical results.
#include <cooperative_groups.h>
#include <type_traits>

#include "rmpcd_kernels.cuh"
#include "rmpcd_fixed.cuh"

namespace cg = cooperative_groups;

namespace rmpcd {

constexpr int NC = MD_FAST_NC;
constexpr int MDF_NT = 256;             // threads per CTA
constexpr int MDF_NW = MDF_NT / 32;
constexpr int MDF_PPT = 2;              // near particles a thread keeps in registers
constexpr int MDF_SPIN_LIMIT = 1 << 22; // polls of one exchange before giving up (ERR_TIMEOUT)
static_assert(NC == 2, "the lane layout below assumes at most two colloids (lanes 0..5)");

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
    unsigned long long part[2][16][8];   // [round parity][source CTA][colloid * 3 + axis]
    unsigned long long mbar[2];          // one per parity: completes when the round's partials arrived
    long long wpart[2][MDF_NW][8];       // [round parity][warp][colloid * 3 + axis]
    float sigf[NC], epsAf[NC], epsBf[NC], rc2f[NC];
    double sig[NC], epsA[NC], epsB[NC], rc2[NC];
    int cat[NC];
    int nn;
    int dead;                            // an exchange timed out: stop waiting
    int pCi[NC][3];                      // colloid positions of the round (warp 0 writes them):
    float pXf[NC][3];                    //   mixed, cell + offset
    double pXw[NC][3];                   //   FP64, wrapped
};

// --- colloid state ------------------------------------------------------------
// Mixed path (warp 0 integrates the colloids): lane l < 3 nc owns colloid
// j = l / 3, axis t = l % 3 (lanes beyond: a copy of component 0) and does the
// per-component work; every lane keeps a copy of all positions (refreshed by
// one shuffle round after each move) for the dot products of RATTLE, which
// each lane evaluates itself.  The operations and their order are those of
// the general MD kernel, so both kernels give bit-identical results.
struct ColL {
    int Xi, Ci;                 // own component: unwrapped and wrapped cell
    float Xf, V, invM;          //   offset in [0,1), velocity, 1 / mass
    int Xa[NC][3];              // all components: unwrapped cells
    float Xfa[NC][3];           //   and offsets
    float invMa[NC];
};
// FP64 path: lane l < 3 nc holds colloid j = l / 3, axis t = l % 3; the bond
// of a dimer always joins colloids 0 and 1, so the other end of a lane's
// component is lane l +- 3.  Lanes >= 3 nc carry copies that are never stored.
struct LaneD {   // unwrapped FP64 position
    double X, V, F, Xold, X0, Xw, M;
};

// (float)i for |i| < 2^22, exactly, on the integer and FP32 pipes: the bits
// of 1.5 2^23 + i, minus 1.5 2^23.  Cell differences here are below 2^11.
__device__ __forceinline__ float small_i2f(int i)
{
    return __int_as_float(0x4B400000 + i) - 12582912.0f;
}

// Sum over lanes 0..2, in lane order (every lane gets the result): the
// component sum of a 3-vector held by axis lanes (FP64 path).
__device__ __forceinline__ double sum3(double a)
{
    return (__shfl_sync(0xffffffffu, a, 0) + __shfl_sync(0xffffffffu, a, 1)) + __shfl_sync(0xffffffffu, a, 2);
}

// Carry of the FP32 offset into the integer cell: f = x - floor(x) (signed
// zero included), k = floor(x), with no branch (branches here split the
// colloid update into serial blocks).  The wrapped cell moves one box length up or down
// by selects; a colloid that crossed more than a box length in one sub-step
// is left out of [0, L) here and put back at the end of the update.
__device__ __forceinline__ void carry(const ReplicaDev &rp, int &Xi, int &Ci, float &Xf, int t)
{
    const float x = Xf;
    const float fl = floorf(x);
    int k = (int)fl;
    float f = x - fl;
    const bool one = f >= 1.0f;
    f = one ? 0.0f : f;
    k += one ? 1 : 0;
    Xf = f;
    Xi += k;
    const int L = rp.L[t];
    int ci = Ci + k;
    ci = ci < 0 ? ci + L : ci;
    ci = ci >= L ? ci - L : ci;
    Ci = ci;
}

__device__ __forceinline__ void set_force(LaneD &C, long long tot) { C.F = (double)tot * 0x1p-40; }

__device__ __forceinline__ void kick_drift(const ReplicaDev &rp, LaneD &C, int)
{
    C.V = fma(rp.hdt, C.F / C.M, C.V);
    C.Xold = C.X;
    C.X = fma(rp.dt, C.V, C.X);
}

// Own-component value of a 3-vector held in every lane.
__device__ __forceinline__ float pick3(const float a[3], int t) { return t == 0 ? a[0] : (t == 1 ? a[1] : a[2]); }

// Every lane: all positions from their owner lanes.
__device__ __forceinline__ void share_positions(ColL &C)
{
#pragma unroll
    for (int j = 0; j < NC; ++j)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            C.Xa[j][t] = __shfl_sync(0xffffffffu, C.Xi, 3 * j + t);
            C.Xfa[j][t] = __shfl_sync(0xffffffffu, C.Xf, 3 * j + t);
        }
}

// Second half kick and RATTLE velocity stage of the bond 0-1 (Andersen
// 1983).  F: this lane's component of the force.
__device__ __forceinline__ void col_kick_rattle_vel(const ReplicaDev &rp, ColL &C, float F, int cj, int ct, int nbond)
{
    C.V = fmaf(rp.hdt_f, F * C.invM, C.V);
    if (nbond == 0) return;
    float Va[NC][3];
#pragma unroll
    for (int j = 0; j < NC; ++j)
#pragma unroll
        for (int t = 0; t < 3; ++t) Va[j][t] = __shfl_sync(0xffffffffu, C.V, 3 * j + t);
    float r[3], dv[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        r[t] = small_i2f(C.Xa[0][t] - C.Xa[1][t]) + (C.Xfa[0][t] - C.Xfa[1][t]);
        dv[t] = Va[0][t] - Va[1][t];
    }
    const float ia = C.invMa[0], ib = C.invMa[1];
    const float inv = ia + ib;
    const float rr = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
    const float rv = (dv[0] * r[0] + dv[1] * r[1]) + dv[2] * r[2];
    const float kk = fdiv_m(rv, rr * inv);
    const float ro = pick3(r, ct);
    if (cj == 0) C.V -= kk * ro * ia;
    else C.V += kk * ro * ib;
}

// First half kick, drift and exact RATTLE position stage (bond length dd);
// ends with every lane holding the new positions.
__device__ __forceinline__ void col_kick_drift_rattle(const ReplicaDev &rp, ColL &C, float F, int cj, int ct,
                                                      int nbond, float dd, float idt)
{
    C.V = fmaf(rp.hdt_f, F * C.invM, C.V);
    C.Xf = fmaf(rp.dt_f, C.V, C.Xf);
    carry(rp, C.Xi, C.Ci, C.Xf, ct);
    if (nbond > 0) {
        int Xn[NC][3];
        float Xfn[NC][3];
#pragma unroll
        for (int j = 0; j < NC; ++j)
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                Xn[j][t] = __shfl_sync(0xffffffffu, C.Xi, 3 * j + t);
                Xfn[j][t] = __shfl_sync(0xffffffffu, C.Xf, 3 * j + t);
            }
        // old positions: the copy from the end of the previous move
        float ro[3], rn[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            ro[t] = small_i2f(C.Xa[0][t] - C.Xa[1][t]) + (C.Xfa[0][t] - C.Xfa[1][t]);
            rn[t] = small_i2f(Xn[0][t] - Xn[1][t]) + (Xfn[0][t] - Xfn[1][t]);
        }
        const float ia = C.invMa[0], ib = C.invMa[1];
        const float inv = ia + ib;
        const float oo = (ro[0] * ro[0] + ro[1] * ro[1]) + ro[2] * ro[2];
        const float on = (rn[0] * ro[0] + rn[1] * ro[1]) + rn[2] * ro[2];
        const float nn = (rn[0] * rn[0] + rn[1] * rn[1]) + rn[2] * rn[2];
        const float qa = inv * inv * oo;
        const float qb = 2.0f * inv * on;
        const float qc = nn - dd * dd;
        float disc = qb * qb - 4.0f * qa * qc;
        if (disc < 0.0f) disc = 0.0f;
        const float q = -0.5f * (qb + copysignf(sqrtf(disc), qb));
        const float gmul = fdiv_m(qc, q);
        const float rot = pick3(ro, ct);
        if (cj == 0) {
            const float ca = gmul * rot * ia;
            C.Xf += ca;
            C.V += ca * idt;
        } else {
            const float cb = gmul * rot * ib;
            C.Xf -= cb;
            C.V -= cb * idt;
        }
        carry(rp, C.Xi, C.Ci, C.Xf, ct);
    }
    // a colloid that crossed more than a box length in one sub-step
    if ((unsigned)C.Ci >= (unsigned)rp.L[ct]) C.Ci = imod(C.Ci, rp.L[ct]);
    share_positions(C);
}

// FP64 path, lane-parallel: exact RATTLE position stage for the bond 0-1.
// a_end: this lane belongs to colloid 0 (the bond's first end).
__device__ __forceinline__ void rattle_pos(const ReplicaDev &rp, LaneD &C, int, double dd, double, bool a_end,
                                           int other)
{
    const double oXold = __shfl_sync(0xffffffffu, C.Xold, other), oX = __shfl_sync(0xffffffffu, C.X, other);
    const double oM = __shfl_sync(0xffffffffu, C.M, other);
    const double ro = a_end ? C.Xold - oXold : oXold - C.Xold;
    const double rn = a_end ? C.X - oX : oX - C.X;
    const double Ma = a_end ? C.M : oM, Mb = a_end ? oM : C.M;
    const double inv = 1.0 / Ma + 1.0 / Mb;
    const double oo = sum3(ro * ro), on = sum3(rn * ro), nn = sum3(rn * rn);
    const double qa = inv * inv * oo;
    const double qb = 2.0 * inv * on;
    const double qc = nn - dd * dd;
    double disc = qb * qb - 4.0 * qa * qc;
    if (disc < 0.0) disc = 0.0;
    const double q = -0.5 * (qb + copysign(sqrt(disc), qb));
    const double gmul = qc / q;
    if (a_end) {
        const double ca = gmul * ro / Ma;
        C.X = C.X + ca;
        C.V = C.V + ca / rp.dt;
    } else {
        const double cb = gmul * ro / Mb;
        C.X = C.X - cb;
        C.V = C.V - cb / rp.dt;
    }
}

// FP64 path: second half kick and RATTLE velocity stage.
__device__ __forceinline__ void kick_rattle_vel(const ReplicaDev &rp, LaneD &C, int nbond, bool a_end, int other)
{
    C.V = fma(rp.hdt, C.F / C.M, C.V);
    if (nbond == 0) return;
    const double oX = __shfl_sync(0xffffffffu, C.X, other), oV = __shfl_sync(0xffffffffu, C.V, other);
    const double oM = __shfl_sync(0xffffffffu, C.M, other);
    const double r = a_end ? C.X - oX : oX - C.X;
    const double dv = a_end ? C.V - oV : oV - C.V;
    const double Ma = a_end ? C.M : oM, Mb = a_end ? oM : C.M;
    const double inv = 1.0 / Ma + 1.0 / Mb;
    const double rr = sum3(r * r), rv = sum3(dv * r);
    const double kk = rv / (rr * inv);
    if (a_end) C.V = C.V - kk * r / Ma;
    else C.V = C.V + kk * r / Mb;
}

__device__ __forceinline__ void frames(const ReplicaDev &rp, LaneD &C, int t)
{
    const double L = (double)rp.L[t];
    C.Xw = C.X - L * floor(C.X / L);
}

// --- colloid positions seen by the particles (FP64 path) --------------------------
struct ColPM {
    int Ci[NC][3];
    float Xf[NC][3];
};
struct ColPD {
    double Xw[NC][3];
};
__device__ __forceinline__ void read_positions(const FShared &S, ColPM &P)
{
#pragma unroll
    for (int j = 0; j < NC; ++j)
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            P.Ci[j][t] = S.pCi[j][t];
            P.Xf[j][t] = S.pXf[j][t];
        }
}
__device__ __forceinline__ void read_positions(const FShared &S, ColPD &P)
{
#pragma unroll
    for (int j = 0; j < NC; ++j)
#pragma unroll
        for (int t = 0; t < 3; ++t) P.Xw[j][t] = S.pXw[j][t];
}
// Warp 0: the colloid positions of the next round for every warp of the CTA.
__device__ __forceinline__ void write_positions(FShared &S, const ColL &C, int lane, int nc)
{
    if (lane < 3 * nc) {
        S.pCi[lane / 3][lane % 3] = C.Ci;
        S.pXf[lane / 3][lane % 3] = C.Xf;
    }
}
__device__ __forceinline__ void write_positions_d(FShared &S, const LaneD &C, int lane)
{
    if (lane < 3 * NC) S.pXw[lane / 3][lane % 3] = C.Xw;
}

// --- particle side ----------------------------------------------------------

// WCA force on one solvent particle (§1.4); the reaction on colloid j goes to
// acc in fixed point.  inside: the particle is within the cut-off of a
// catalytic colloid (§1.5).  Both colloids are evaluated without branches so
// that their dependency chains overlap; a colloid out of range contributes
// nothing (selects, so the sums are the same as with a branch).
// Per-replica constants of the mixed particle force, held in registers for
// the whole interval (shared memory would be re-read after every barrier).
struct PConstM {
    float sig[NC], epsA[NC], epsB[NC], rc2[NC];
    bool cat[NC];
    float L[3], hL[3], g[3];
    bool wrap_z;   // z periodic (no walls)
    int nc;
};
__device__ __forceinline__ void load_pconst(const ReplicaDev &rp, const FShared &S, PConstM &K)
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        K.sig[j] = S.sigf[j];
        K.epsA[j] = S.epsAf[j];
        K.epsB[j] = S.epsBf[j];
        K.rc2[j] = S.rc2f[j];
        K.cat[j] = S.cat[j] != 0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        K.L[k] = (float)rp.L[k];
        K.hL[k] = 0.5f * K.L[k];
        K.g[k] = rp.g_f[k];
    }
    K.wrap_z = !rp.walls;
    K.nc = rp.n_col;
}

__device__ __forceinline__ void pforce(const ReplicaDev &, const PConstM &K, const ColPM &C, int, FWorkM &w,
                                       long long acc[NC][3], bool &inside)
{
    float d[NC][3], r2[NC];
    bool in[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float dk = (float)(w.c[k] - C.Ci[j][k]) + (w.o[k] - C.Xf[j][k]);
            // minimum image by selects (periodic axes)
            float m = dk > K.hL[k] ? dk - K.L[k] : dk;
            m = dk < -K.hL[k] ? dk + K.L[k] : m;
            d[j][k] = (k < 2 || K.wrap_z) ? m : dk;
        }
        r2[j] = d[j][0] * d[j][0] + d[j][1] * d[j][1] + d[j][2] * d[j][2];
        in[j] = j < K.nc && r2[j] < K.rc2[j];
    }
    inside = (in[0] && K.cat[0]) || (in[1] && K.cat[1]);
    // the WCA force only inside the cut-off: most near particles are outside
    // it, and a warp whose lanes all are skips the work (the near list comes
    // in cell order, so a warp's particles are neighbours)
    float f[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (in[j]) {
            const float eps = (w.fid & F_B) ? K.epsB[j] : K.epsA[j];
            const float fr = wca_fr_m(eps, K.sig[j], r2[j]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float fk = fr * d[j][k];
                f[k] = f[k] + fk;
                acc[j][k] -= fx40(fk);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) w.f[k] = f[k] + K.g[k];
}

__device__ __forceinline__ void pforce(const ReplicaDev &rp, const FShared &S, const ColPD &C, int nc, FWorkD &w,
                                       long long acc[NC][3], bool &inside)
{
    w.f[0] = w.f[1] = w.f[2] = 0.0;
    inside = false;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j >= nc) continue;
        double d[3] = {w.x[0] - C.Xw[j][0], w.x[1] - C.Xw[j][1], w.x[2] - C.Xw[j][2]};
        min_image(rp, d);
        const double eps = (w.fid & F_B) ? S.epsB[j] : S.epsA[j];
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < S.rc2[j]) {
            inside = inside || S.cat[j];
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

// Velocity-Verlet particle update between two force evaluations: the second
// half kick of the last sub-step (when there was one), the first half kick
// and the drift of the next.
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

// Near particle k of the replica: its record from the near area; its flat
// slot (the write-back target of a granular interval) from the near list.
template <bool MIXED, typename W>
__device__ __forceinline__ void load_particle(const Dev &d, const ReplicaDev &rp, int k, const int *list, int do_bin,
                                              W &w)
{
    w.slot = do_bin ? -1 : list[k];
    if constexpr (MIXED) {
        RecM rec = load_near<RecM>(d, rp, k);
        for (int q = 0; q < 3; ++q) { w.c[q] = cw_get(rec.cw, q); w.o[q] = rec.o[q]; w.v[q] = rec.v[q]; }
        w.fid = rec.fid;
    } else {
        RecD rec = load_near<RecD>(d, rp, k);
        for (int q = 0; q < 3; ++q) { w.x[q] = rec.x[q]; w.v[q] = rec.v[q]; }
        w.fid = rec.fid;
    }
}

// One round of one particle: the force at its current position (round > 0:
// then the catalytic test of sub-step round - 1), and, unless this was the
// last round, the move to its position of the next round.
template <typename KT, typename ColT, typename W>
__device__ __forceinline__ void round_particle(const ReplicaDev &rp, const KT &K, const ColT &P, int nc, W &w,
                                               long long acc[NC][3], uint32_t step, int round, int n_md)
{
    bool inside;
    pforce(rp, K, P, nc, w, acc, inside);
    if (round > 0) w.fid = fcatalysis(rp, w.fid, inside, step, round - 1);
    if (round < n_md) pkick_drift(rp, w, round > 0);
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
    const float sf[3] = {(float)sh[0], (float)sh[1], (float)sh[2]};
    put_near(d, rbuf, bbuf, do_bin, do_bin ? bin_cell(d, rp.cell_off, cell_key_m(rp, w.c, w.o, sf)) : 0, w.slot, rec);
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
    put_near(d, rbuf, bbuf, do_bin, do_bin ? bin_cell(d, rp.cell_off, cell_key_d(rp, w.x, sh)) : 0, w.slot, rec);
}

// --- the cluster exchange of the force partials -------------------------------
// Warp 0 of every CTA writes the CTA's six fixed-point partials into slot
// [rank] of every CTA's buffer for the round's parity with st.async; the bytes
// are counted on that CTA's mbarrier for the parity, whose single arrival is
// the expect-tx thread 0 posts at the start of the round.  Warp 0 waits for
// the phase and sums the slots in rank order.  Round r + 2 reuses the buffer
// and the barrier of round r: a CTA sends round r + 2 only after its warp 0
// read round r, and after every CTA sent round r + 1, which each does after
// its own warp 0 read round r; thread 0 posts round r + 2's expect-tx after
// it saw round r's phase complete.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_async_v2(uint32_t a, unsigned long long x, unsigned long long y, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.u64 [%0], {%1, %2}, [%3];" ::"r"(a),
                 "l"(x), "l"(y), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t a, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, unsigned bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(a),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t a, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0u;
}

constexpr unsigned MDF_TX_BYTES = 6 * 8;   // partials one CTA sends to one CTA per round

// Remote addresses of warp 0's st.async items, computed once per launch:
// item = lane + 32 k goes to CTA item / 3 and carries pair item % 3 of the
// six partials, into slot [rank] of that CTA's buffer for each parity.
template <int CS>
struct SendPlan {
    static constexpr int K = (3 * CS + 31) / 32;
    uint32_t dst[2][K], bar[2][K];
};
template <int CS>
__device__ __forceinline__ void plan_sends(FShared &S, int rank, int lane, SendPlan<CS> &P)
{
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const uint32_t src = smem_addr(&S.part[b][rank][0]), bar = smem_addr(&S.mbar[b]);
#pragma unroll
        for (int k = 0; k < SendPlan<CS>::K; ++k) {
            const int item = lane + 32 * k;
            const int q = item < 3 * CS ? item / 3 : 0;
            P.dst[b][k] = cluster_addr(src + 16u * (uint32_t)(item % 3), q);
            P.bar[b][k] = cluster_addr(bar, q);
        }
    }
}

// Warp 0 of a CTA: its CTA's partials (lane l < 6 holds component l) to every
// CTA of the cluster, as three 16-byte st.async per destination spread over
// the lanes.  The expected byte count of the round was posted at its start.
template <int CS>
__device__ __forceinline__ void send_partials(const SendPlan<CS> &P, int b, int lane, long long mine)
{
#pragma unroll
    for (int k = 0; k < SendPlan<CS>::K; ++k) {
        const int item = lane + 32 * k;
        const int pi = item % 3;
        const long long x = __shfl_sync(0xffffffffu, mine, 2 * pi);
        const long long y = __shfl_sync(0xffffffffu, mine, 2 * pi + 1);
        if (item < 3 * CS)
            st_async_v2(b ? P.dst[1][k] : P.dst[0][k], (unsigned long long)x, (unsigned long long)y,
                        b ? P.bar[1][k] : P.bar[0][k]);
    }
}

// Warp 0 waits for the partials of round `round` (parity b) from every CTA
// of the cluster and sums them in rank order (lane l < 6: component l).
// Without a cluster the CTA's own sum `tot` is the total.
template <int CS>
__device__ __forceinline__ long long exchange_partials(const Dev &d, FShared &S, int b, int round, int lane,
                                                       long long tot)
{
    if constexpr (CS > 1) {
        const uint32_t bar = smem_addr(&S.mbar[b]);
        const unsigned parity = (unsigned)(round >> 1) & 1u;
        if (!S.dead) {
            int spins = 0;
            while (!mbar_try_wait_cluster(bar, parity)) {
                if (++spins > MDF_SPIN_LIMIT) {
                    if (lane == 0) {
                        atomicOr(&d.err[ERR_TIMEOUT], 1u);
                        S.dead = 1;
                    }
                    break;
                }
            }
            __syncwarp();
        }
        tot = 0;
        if (lane < 3 * NC)
#pragma unroll
            for (int q = 0; q < CS; ++q) tot += (long long)S.part[b][q][lane];
    }
    return tot;
}

template <bool MIXED, int CS>
__global__ void __launch_bounds__(MDF_NT, 1) k_md_fast(Dev d, uint32_t step, int rbuf, int bbuf, int do_bin)
{
    step = resolve_step(d, step);   // STEP_DEVICE: the step of the control block
    using W = typename std::conditional<MIXED, FWorkM, FWorkD>::type;
    using R = typename std::conditional<MIXED, float, double>::type;
    __shared__ FShared S;
    __shared__ ReplicaDev s_rp;
    cg::cluster_group cl = cg::this_cluster();
    const int r = blockIdx.x / CS;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int rank = CS == 1 ? 0 : (int)cl.block_rank();
    if (tid == 0) s_rp = d.rep[r];
    __syncthreads();
    const ReplicaDev &rp = s_rp;
    if (rp.n_col == 0 || rp.body >= 0 || rp.net >= 0) return;   // uniform over the cluster (bodies, networks: own kernels)
    const int nc = rp.n_col, nbond = rp.n_bond, n_md = rp.n_md;
    if (tid == 0) {
        S.nn = min(d.near_count[r], rp.n_part);
        S.dead = 0;
        if (CS > 1) {
            mbar_init(smem_addr(&S.mbar[0]), 1u);
            mbar_init(smem_addr(&S.mbar[1]), 1u);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    if (tid < nc) {
        const int g = rp.col_off + tid;
        S.sig[tid] = d.colSig[g]; S.epsA[tid] = d.colEpsA[g]; S.epsB[tid] = d.colEpsB[g]; S.rc2[tid] = d.colRc2[g];
        S.sigf[tid] = d.colSig_f[g];
        S.epsAf[tid] = d.colEpsA_f[g]; S.epsBf[tid] = d.colEpsB_f[g];
        S.rc2f[tid] = d.colRc2_f[g];
        S.cat[tid] = d.colCat[g];
    }

    const R bond_d = nbond > 0 ? (R)d.bonds[rp.bond_off].d : R(0);
    const R idt = R(1) / (MIXED ? (R)rp.dt_f : (R)rp.dt);
    // colloid state: lane l < 3 nc owns component l (lanes beyond: a copy of
    // component 0); mixed, every lane also keeps all positions
    ColL CM;
    LaneD CD;
    const int cl_l = lane < 3 * nc ? lane : 0;
    const int cj = cl_l / 3, ct = cl_l % 3;
    const bool a_end = cj == 0;
    const int other = nc == 2 ? (cj == 0 ? cl_l + 3 : cl_l - 3) : cl_l;
    if constexpr (MIXED) {
        const int g = rp.col_off + cj;
        CM.Xi = d.colXi[3 * g + ct];
        CM.Xf = d.colXf[3 * g + ct];
        CM.Ci = d.colCi[3 * g + ct];
        CM.V = d.colVf[3 * g + ct];
        CM.invM = d.colInvM_f[g];
#pragma unroll
        for (int j = 0; j < NC; ++j) CM.invMa[j] = d.colInvM_f[rp.col_off + (j < nc ? j : 0)];
        share_positions(CM);
    } else {
        const int g = rp.col_off + cj;
        CD.X = d.colX[3 * g + ct];
        CD.V = d.colV[3 * g + ct];
        CD.Xold = CD.X; CD.X0 = CD.X;
        CD.F = 0.0;
        CD.M = d.colM[g];
        frames(rp, CD, ct);
    }
    if (wid == 0) {
        if constexpr (MIXED) write_positions(S, CM, lane, nc);
        else write_positions_d(S, CD, lane);
    }
    __syncthreads();
    // every CTA has read near_count and set up its barriers before any
    // remote access and before CTA 0 resets the count
    if (CS > 1) cl.sync();

    const int nn = S.nn;
    SendPlan<CS> plan;
    if constexpr (CS > 1) plan_sends<CS>(S, rank, lane, plan);
    PConstM K;
    load_pconst(rp, S, K);
    const int *list = d.near_list + rp.part_off;
    W *work = reinterpret_cast<W *>(d.md_work) + rp.part_off;
    const int first = rank * MDF_NT + tid;
    const int stride = CS * MDF_NT;
    const int over = first + MDF_PPT * stride;   // beyond the registers: global memory
    W reg[MDF_PPT];
#pragma unroll
    for (int p = 0; p < MDF_PPT; ++p)
        if (first + p * stride < nn) load_particle<MIXED>(d, rp, first + p * stride, list, do_bin, reg[p]);
    for (int k = over; k < nn; k += stride) {
        W w;
        load_particle<MIXED>(d, rp, k, list, do_bin, w);
        work[k] = w;
    }

    long long acc[NC][3];
    bool ins[MDF_PPT];
    using ColP = typename std::conditional<MIXED, ColPM, ColPD>::type;
    // round 0: forces at the start of the interval; round k (1 <= k <= n_md):
    // forces at the end of sub-step k - 1.  Per round: every warp computes
    // its particles' forces and the warp sums of the reactions; after a CTA
    // barrier warp 0 sends the CTA's partials, waits for every CTA's, and
    // integrates the colloids, while the other warps move their particles;
    // a second CTA barrier publishes the new colloid positions.
    for (int round = 0; round <= n_md; ++round) {
        const int b = round & 1;
        // the byte count this round's barrier expects (its previous phase, two
        // rounds ago, has completed: warp 0 waited for it)
        if constexpr (CS > 1)
            if (tid == 0 && !S.dead) mbar_expect_tx(smem_addr(&S.mbar[b]), (unsigned)(CS * MDF_TX_BYTES));
        ColP P;
        read_positions(S, P);
#pragma unroll
        for (int j = 0; j < NC; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[j][k] = 0;
        // forces on the register particles; the particles beyond the
        // registers also take their whole round here (one pass over memory)
        if constexpr (MIXED) {
#pragma unroll
            for (int p = 0; p < MDF_PPT; ++p)
                if (first + p * stride < nn) pforce(rp, K, P, nc, reg[p], acc, ins[p]);
            for (int k = over; k < nn; k += stride) {
                W w = work[k];
                round_particle(rp, K, P, nc, w, acc, step, round, n_md);
                work[k] = w;
            }
        } else {
#pragma unroll
            for (int p = 0; p < MDF_PPT; ++p)
                if (first + p * stride < nn) pforce(rp, S, P, nc, reg[p], acc, ins[p]);
            for (int k = over; k < nn; k += stride) {
                W w = work[k];
                round_particle(rp, S, P, nc, w, acc, step, round, n_md);
                work[k] = w;
            }
        }
        long long ws = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const long long x = warp_sum64(acc[j][k]);
                if (lane == 3 * j + k) ws = x;
            }
        if (lane < 3 * NC) S.wpart[b][wid][lane] = ws;
        __syncthreads();
        long long tot = 0;
        if (wid == 0) {
            // the CTA's partials (lane l < 6: component l, warps in order)
            if (lane < 3 * NC)
#pragma unroll
                for (int w = 0; w < MDF_NW; ++w) tot += S.wpart[b][w][lane];
            if constexpr (CS > 1) send_partials<CS>(plan, b, lane, tot);
        }
        // the register particles' catalytic test of sub-step round - 1 and
        // their move to the next round need only their own force: done while
        // the partials travel
#pragma unroll
        for (int p = 0; p < MDF_PPT; ++p)
            if (first + p * stride < nn) {
                if (round > 0) reg[p].fid = fcatalysis(rp, reg[p].fid, ins[p], step, round - 1);
                if (round < n_md) pkick_drift(rp, reg[p], round > 0);
            }
        if (wid == 0) {
            tot = exchange_partials<CS>(d, S, b, round, lane, tot);
            // the colloids: force of this round, end of sub-step round - 1
            // (second half kick, RATTLE velocity stage), start of sub-step
            // round (first half kick, drift, RATTLE position stage)
            if constexpr (MIXED) {
                const float F = fixed40_to_float(tot);   // lane l < 6: component l
                if (round > 0) col_kick_rattle_vel(rp, CM, F, cj, ct, nbond);
                if (round < n_md) {
                    col_kick_drift_rattle(rp, CM, F, cj, ct, nbond, bond_d, idt);
                    write_positions(S, CM, lane, nc);
                }
            } else {
                set_force(CD, __shfl_sync(0xffffffffu, tot, cl_l));
                if (round > 0) kick_rattle_vel(rp, CD, nbond, a_end, other);
                if (round < n_md) {
                    kick_drift(rp, CD, ct);
                    if (nbond > 0) rattle_pos(rp, CD, ct, bond_d, idt, a_end, other);
                    frames(rp, CD, ct);
                    write_positions_d(S, CD, lane);
                }
            }
        }
        __syncthreads();
    }

    // last half kick, wrap, write back (and bin for the collision of `step`)
    double sh[3];
    grid_shift(rp.seed, step, sh);
#pragma unroll
    for (int p = 0; p < MDF_PPT; ++p)
        if (first + p * stride < nn) finish_particle(d, rp, reg[p], sh, rbuf, bbuf, do_bin);
    for (int k = over; k < nn; k += stride) {
        W w = work[k];
        finish_particle(d, rp, w, sh, rbuf, bbuf, do_bin);
    }
    // CTA 0, warp 0: colloids back to memory, skin check, near list reset
    if (rank == 0 && wid == 0) {
        if constexpr (MIXED) {
            // displacement over the interval, against the stored start
            const int g = rp.col_off + cj;
            const float e = (float)(CM.Xi - d.colXi[3 * g + ct]) + (CM.Xf - d.colXf[3 * g + ct]);
            const float e0 = __shfl_sync(0xffffffffu, e, 3 * cj), e1 = __shfl_sync(0xffffffffu, e, 3 * cj + 1);
            const float e2 = __shfl_sync(0xffffffffu, e, 3 * cj + 2);
            __syncwarp();   // every lane has read the start before it is overwritten
            if (lane < 3 * nc) {
                d.colXi[3 * g + ct] = CM.Xi;
                d.colXf[3 * g + ct] = CM.Xf;
                d.colVf[3 * g + ct] = CM.V;
                d.colCi[3 * g + ct] = CM.Ci;
            }
            if (lane < 3 * nc && ct == 0) {
                const float dd = e0 * e0 + e1 * e1 + e2 * e2;
                if (!(dd <= rp.skin_f * rp.skin_f)) atomicAdd(&d.err[ERR_SKIN], 1u);
            }
        } else {
            const int g = rp.col_off + cj;
            const double e = CD.X - CD.X0;
            const double e0 = __shfl_sync(0xffffffffu, e, 3 * cj), e1 = __shfl_sync(0xffffffffu, e, 3 * cj + 1);
            const double e2 = __shfl_sync(0xffffffffu, e, 3 * cj + 2);
            if (lane < 3 * nc) {
                d.colX[3 * g + ct] = CD.X;
                d.colV[3 * g + ct] = CD.V;
            }
            bool bad = false;
            if (lane < 3 * nc && ct == 0) {
                double dd = 0.0;
                dd = dd + e0 * e0;
                dd = dd + e1 * e1;
                dd = dd + e2 * e2;
                bad = !(dd <= rp.skin * rp.skin);
            }
            if (bad) atomicAdd(&d.err[ERR_SKIN], 1u);
        }
        if (lane == 0) d.near_count[r] = 0;
    }
    if (CS > 1) cl.sync();   // no CTA leaves while another may still write its shared memory
}

template <bool MIXED, int CS>
static void launch_fast_cs(const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, cudaStream_t s)
{
    if (CS > 8) cudaFuncSetAttribute(k_md_fast<MIXED, CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(d.n_rep * CS), 1, 1);
    cfg.blockDim = dim3(MDF_NT, 1, 1);
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
    cfg.blockDim = dim3(MDF_NT, 1, 1);
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
