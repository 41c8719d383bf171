// k_md.cu -- near-colloid molecular dynamics of one collision interval
// (§1.1 velocity Verlet; §1.4 WCA colloid-solvent potential, Verlet-list
// radius, exact RATTLE for the dimer; §1.5 catalytic A -> B on leaving the
// catalytic sphere) for the solvent particles in the near list.
//
// One thread-block cluster of MD_CS CTAs per replica runs all n_md
// sub-steps.  The near solvent is spread over the cluster's threads; the few
// colloids are integrated redundantly (identically) by thread 0 of every CTA
// in FP64.  Colloid forces are summed as 64-bit fixed point (2^-40
// resolution): per thread over its particles, per warp by shuffles, per CTA
// in shared memory, and across the cluster through distributed shared memory
// in rank order, so the sum is exact and does not depend on the order of the
// near list.  Per sub-step the cluster synchronises once and each CTA twice.
//
// The mixed path does no FP64 arithmetic per particle: every colloid position
// is split once per sub-step into an integer cell and an FP32 offset, so the
// particle-colloid separation is an integer difference plus FP32 offsets.
#include <cooperative_groups.h>
#include <type_traits>
#include <vector>

#include "rmpcd_kernels.cuh"
#include "rmpcd_fixed.cuh"

namespace cg = cooperative_groups;

namespace rmpcd {

constexpr int NCR = 4;          // colloids whose force partials live in registers
constexpr int MD_MAXW = 32;     // most warps of one MD CTA

// Threads per CTA of an MD cluster of CS CTAs: a lone CTA takes 1024.
template <int CS> struct MDGeom {
    static constexpr int NT = CS == 1 ? 1024 : 512;
    static constexpr int NW = NT / 32;
};

struct __align__(16) WorkM {
    int c[3];
    uint32_t fid;
    float o[3];
    int slot;
    float v[3];
    float p0;
    float f[3];
    float p1;
};
struct __align__(16) WorkD {
    double x[3];
    double v[3];
    double f[3];
    uint32_t fid;
    int slot;
};

// FP64 colloid state (fp64 path): unwrapped positions, wrapped copies.
struct ColD {
    double X[MAXC][3], V[MAXC][3], Xw[MAXC][3], F[MAXC][3], X0[MAXC][3], Xold[MAXC][3];
};
// Mixed colloid state: unwrapped integer cell + FP32 offset in [0,1), FP32
// velocity and force; Ci is the wrapped integer cell.
struct ColM {
    int Xi[MAXC][3], Xoi[MAXC][3], X0i[MAXC][3], Ci[MAXC][3];
    float Xf[MAXC][3], Xof[MAXC][3], X0f[MAXC][3], V[MAXC][3], F[MAXC][3];
    float invM[MAXC];
};

template <bool MIXED>
struct MDShared {
    typename std::conditional<MIXED, ColM, ColD>::type C;
    double M[MAXC], sig[MAXC], epsA[MAXC], epsB[MAXC], rc2[MAXC];
    float sigf[MAXC], epsAf[MAXC], epsBf[MAXC], rc2f[MAXC];
    int cat[MAXC];
    BondDev bond[MAXB];
    unsigned long long Fq[MAXC * 3];                 // this CTA's partial (atomic path)
    unsigned long long wpart[MD_MAXW][NCR * 3];      // per-warp partials (register path)
    unsigned long long part[2][8][MAXC * 3];         // partials of every CTA of the cluster
    long long Fsum[MAXC * 3];                        // cluster total
    int nc, nbond, nn;
};

// --- per-particle forces ----------------------------------------------------
// Force on one solvent particle from all colloids (WCA, §1.4).  The reaction
// on colloid j is -f_j, added in fixed point to acc (register path, j < NCR)
// or to the CTA's shared sums (atomic path).
template <bool REG>
__device__ __forceinline__ void force_d(const ReplicaDev &rp, MDShared<false> &S, const double x[3], uint32_t fid,
                                        double f[3], long long acc[NCR][3])
{
    f[0] = f[1] = f[2] = 0.0;
    for (int j = 0; j < S.nc; ++j) {
        double d[3] = {x[0] - S.C.Xw[j][0], x[1] - S.C.Xw[j][1], x[2] - S.C.Xw[j][2]};
        min_image(rp, d);
        const double eps = (fid & F_B) ? S.epsB[j] : S.epsA[j];
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < S.rc2[j]) {
            const double ir2 = 1.0 / r2;
            const double s2 = S.sig[j] * S.sig[j] * ir2;
            const double s6 = s2 * s2 * s2;
            const double fr = 24.0 * eps * s6 * (2.0 * s6 - 1.0) * ir2;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double fk = fr * d[k];
                f[k] = f[k] + fk;
                const long long q = __double2ll_rn(fk * 0x1p40);
                if (REG) {
#pragma unroll
                    for (int jj = 0; jj < NCR; ++jj)
                        if (jj == j) acc[jj][k] -= q;
                } else {
                    atomicAdd(&S.Fq[3 * j + k], (unsigned long long)(-q));
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = f[k] + rp.g[k];
}

// Mixed: separation from the wrapped colloid cell and offset, FP32 only.
template <class SH>
__device__ __forceinline__ void sep_m(const ReplicaDev &rp, const SH &S, int j, const int c[3],
                                      const float o[3], float d[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = (float)(c[k] - S.C.Ci[j][k]) + (o[k] - S.C.Xf[j][k]);
    min_image(rp, d);
}

template <bool REG>
__device__ __forceinline__ void force_m(const ReplicaDev &rp, MDShared<true> &S, const int c[3], const float o[3],
                                        uint32_t fid, float f[3], long long acc[NCR][3])
{
    f[0] = f[1] = f[2] = 0.0f;
    for (int j = 0; j < S.nc; ++j) {
        float d[3];
        sep_m(rp, S, j, c, o, d);
        const float eps = (fid & F_B) ? S.epsBf[j] : S.epsAf[j];
        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < S.rc2f[j]) {
            const float fr = wca_fr_m(eps, S.sigf[j], r2);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float fk = fr * d[k];
                f[k] = f[k] + fk;
                const long long q = fx40_any(fk);   // exact scaling, one rounding
                if (REG) {
#pragma unroll
                    for (int jj = 0; jj < NCR; ++jj)
                        if (jj == j) acc[jj][k] -= q;
                } else {
                    atomicAdd(&S.Fq[3 * j + k], (unsigned long long)(-q));
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = f[k] + rp.g_f[k];
}

__device__ __forceinline__ bool inside_cat_d(const ReplicaDev &rp, const MDShared<false> &S, const double x[3])
{
    for (int j = 0; j < S.nc; ++j) {
        if (!S.cat[j]) continue;
        double d[3] = {x[0] - S.C.Xw[j][0], x[1] - S.C.Xw[j][1], x[2] - S.C.Xw[j][2]};
        min_image(rp, d);
        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < S.rc2[j]) return true;
    }
    return false;
}

template <class SH>
__device__ __forceinline__ bool inside_cat_m(const ReplicaDev &rp, const SH &S, const int c[3],
                                             const float o[3])
{
    for (int j = 0; j < S.nc; ++j) {
        if (!S.cat[j]) continue;
        float d[3];
        sep_m(rp, S, j, c, o, d);
        if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < S.rc2f[j]) return true;
    }
    return false;
}

__device__ __forceinline__ bool bonded(const BondDev *bond, int nbond, int a, int b)
{
    for (int k = 0; k < nbond; ++k)
        if ((bond[k].a == a && bond[k].b == b) || (bond[k].a == b && bond[k].b == a)) return true;
    return false;
}

// ===========================================================================
// FP64 colloid integrator (fp64 path; same operation order as the FP64 oracle)
// ===========================================================================
// Colloid-colloid truncated LJ (energy shifted at cc_rc), bonded pairs excluded.
__device__ void colloid_colloid(const ReplicaDev &rp, MDShared<false> &S, long long *Fq)
{
    if (!(rp.cc_rc > 0.0)) return;
    for (int a = 0; a < S.nc; ++a)
        for (int b = a + 1; b < S.nc; ++b) {
            if (bonded(S.bond, S.nbond, a, b)) continue;
            double d[3] = {S.C.Xw[a][0] - S.C.Xw[b][0], S.C.Xw[a][1] - S.C.Xw[b][1], S.C.Xw[a][2] - S.C.Xw[b][2]};
            min_image(rp, d);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rp.cc_rc * rp.cc_rc)) continue;
            const double ir2 = 1.0 / r2;
            const double s2 = rp.cc_sigma * rp.cc_sigma * ir2;
            const double s6 = s2 * s2 * s2;
            const double fr = 24.0 * rp.cc_eps * s6 * (2.0 * s6 - 1.0) * ir2;
            for (int k = 0; k < 3; ++k) {
                const long long q = __double2ll_rn(fr * d[k] * 0x1p40);
                Fq[3 * a + k] += q;
                Fq[3 * b + k] -= q;
            }
        }
}

// Exact RATTLE for single bonds (Andersen 1983): the position stage moves
// both bodies along the old bond vector onto |X_a - X_b| = d (root of smaller
// magnitude of the quadratic) and corrects their velocities accordingly.
__device__ void rattle_pos(MDShared<false> &S, double dt)
{
    ColD &C = S.C;
    for (int k = 0; k < S.nbond; ++k) {
        const int a = S.bond[k].a, b = S.bond[k].b;
        const double dd = S.bond[k].d;
        double ro[3], rn[3];
        for (int t = 0; t < 3; ++t) {
            ro[t] = C.Xold[a][t] - C.Xold[b][t];
            rn[t] = C.X[a][t] - C.X[b][t];
        }
        const double inv = 1.0 / S.M[a] + 1.0 / S.M[b];
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
        for (int t = 0; t < 3; ++t) {
            const double ca = gmul * ro[t] / S.M[a];
            const double cb = gmul * ro[t] / S.M[b];
            C.X[a][t] = C.X[a][t] + ca;
            C.X[b][t] = C.X[b][t] - cb;
            C.V[a][t] = C.V[a][t] + ca / dt;
            C.V[b][t] = C.V[b][t] - cb / dt;
        }
    }
}

// Velocity stage: remove the relative velocity along each bond.
__device__ void rattle_vel(MDShared<false> &S)
{
    ColD &C = S.C;
    for (int k = 0; k < S.nbond; ++k) {
        const int a = S.bond[k].a, b = S.bond[k].b;
        double r[3], dv[3];
        for (int t = 0; t < 3; ++t) {
            r[t] = C.X[a][t] - C.X[b][t];
            dv[t] = C.V[a][t] - C.V[b][t];
        }
        const double inv = 1.0 / S.M[a] + 1.0 / S.M[b];
        const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double rv = dv[0] * r[0] + dv[1] * r[1] + dv[2] * r[2];
        const double kk = rv / (rr * inv);
        for (int t = 0; t < 3; ++t) {
            C.V[a][t] = C.V[a][t] - kk * r[t] / S.M[a];
            C.V[b][t] = C.V[b][t] + kk * r[t] / S.M[b];
        }
    }
}

__device__ void col_load(const Dev &d, const ReplicaDev &rp, MDShared<false> &S, int j)
{
    const int g = rp.col_off + j;
    for (int k = 0; k < 3; ++k) {
        S.C.X[j][k] = d.colX[3 * g + k];
        S.C.V[j][k] = d.colV[3 * g + k];
        S.C.X0[j][k] = S.C.X[j][k];
    }
}

__device__ void col_frames(const ReplicaDev &rp, MDShared<false> &S)
{
    for (int j = 0; j < S.nc; ++j) wrapped_colloid(rp, S.C.X[j], S.C.Xw[j]);
}

template <int CS>
__device__ void col_gather(const ReplicaDev &rp, MDShared<false> &S, int par)
{
    long long *Fq = S.Fsum;
    for (int i = 0; i < 3 * S.nc; ++i) Fq[i] = (long long)S.part[par][0][i];
    for (int q = 1; q < CS; ++q)
        for (int i = 0; i < 3 * S.nc; ++i) Fq[i] += (long long)S.part[par][q][i];
    colloid_colloid(rp, S, Fq);
    for (int j = 0; j < S.nc; ++j)
        for (int k = 0; k < 3; ++k) S.C.F[j][k] = (double)Fq[3 * j + k] * 0x1p-40;
}

__device__ void col_kick_drift(const ReplicaDev &rp, MDShared<false> &S)
{
    const double dt = rp.dt, hdt = rp.hdt;
    for (int j = 0; j < S.nc; ++j)
        for (int t = 0; t < 3; ++t) {
            S.C.V[j][t] = fma(hdt, S.C.F[j][t] / S.M[j], S.C.V[j][t]);
            S.C.Xold[j][t] = S.C.X[j][t];
            S.C.X[j][t] = fma(dt, S.C.V[j][t], S.C.X[j][t]);
        }
    rattle_pos(S, dt);
}

__device__ void col_kick(const ReplicaDev &rp, MDShared<false> &S)
{
    for (int j = 0; j < S.nc; ++j)
        for (int t = 0; t < 3; ++t) S.C.V[j][t] = fma(rp.hdt, S.C.F[j][t] / S.M[j], S.C.V[j][t]);
    rattle_vel(S);
}

__device__ void col_store(const Dev &d, const ReplicaDev &rp, MDShared<false> &S)
{
    bool bad = false;
    for (int j = 0; j < S.nc; ++j) {
        const int g = rp.col_off + j;
        double dd = 0.0;
        for (int t = 0; t < 3; ++t) {
            const double e = S.C.X[j][t] - S.C.X0[j][t];
            dd = dd + e * e;
            d.colX[3 * g + t] = S.C.X[j][t];
            d.colV[3 * g + t] = S.C.V[j][t];
        }
        if (!(dd <= rp.skin * rp.skin)) bad = true;
    }
    if (bad) atomicAdd(&d.err[ERR_SKIN], 1u);
}

// ===========================================================================
// Mixed colloid integrator: integer cell + FP32 offset, FP32 arithmetic, run
// by warp 0 with one lane per colloid component (lane l: colloid l / 3, axis
// l % 3) and three lanes per bond for RATTLE.
// ===========================================================================
__device__ __forceinline__ void col_carry(const ReplicaDev &rp, ColM &C, int j, int t)
{
    const float fl = floorf(C.Xf[j][t]);
    int c = (int)fl;
    float f = C.Xf[j][t] - fl;
    if (f >= 1.0f) { f = 0.0f; c += 1; }
    C.Xf[j][t] = f;
    C.Xi[j][t] += c;
    int ci = C.Ci[j][t] + c;
    const int L = rp.L[t];
    if (ci >= L || ci < 0) ci = imod(ci, L);
    C.Ci[j][t] = ci;
}

// Sum over lanes 0..2 of warp 0, in lane order (all lanes get the result).
__device__ __forceinline__ float sum3(float a)
{
    return (__shfl_sync(0xffffffffu, a, 0) + __shfl_sync(0xffffffffu, a, 1)) + __shfl_sync(0xffffffffu, a, 2);
}

__device__ __forceinline__ float col_sep1(const ColM &C, int a, int b, int t)
{
    return (float)(C.Xi[a][t] - C.Xi[b][t]) + (C.Xf[a][t] - C.Xf[b][t]);
}

// RATTLE position stage for every bond (warp 0; lanes 0..2 = axes).
template <class SH>
__device__ void rattle_pos_w(const ReplicaDev &rp, SH &S, int lane)
{
    ColM &C = S.C;
    const float idt = 1.0f / rp.dt_f;
    for (int k = 0; k < S.nbond; ++k) {
        const int a = S.bond[k].a, b = S.bond[k].b;
        const float dd = (float)S.bond[k].d;
        const int t = lane < 3 ? lane : 0;
        const float ro = (float)(C.Xoi[a][t] - C.Xoi[b][t]) + (C.Xof[a][t] - C.Xof[b][t]);
        const float rn = col_sep1(C, a, b, t);
        const float inv = C.invM[a] + C.invM[b];
        const float oo = sum3(ro * ro), on = sum3(rn * ro), nn = sum3(rn * rn);
        const float qa = inv * inv * oo;
        const float qb = 2.0f * inv * on;
        const float qc = nn - dd * dd;
        float disc = qb * qb - 4.0f * qa * qc;
        if (disc < 0.0f) disc = 0.0f;
        const float q = -0.5f * (qb + copysignf(sqrtf(disc), qb));
        const float gmul = fdiv_m(qc, q);
        __syncwarp();
        if (lane < 3) {
            const float ca = gmul * ro * C.invM[a];
            const float cb = gmul * ro * C.invM[b];
            C.Xf[a][t] += ca;
            C.Xf[b][t] -= cb;
            C.V[a][t] += ca * idt;
            C.V[b][t] -= cb * idt;
            col_carry(rp, C, a, t);
            col_carry(rp, C, b, t);
        }
        __syncwarp();
    }
}

// RATTLE velocity stage (warp 0).
template <class SH>
__device__ void rattle_vel_w(SH &S, int lane)
{
    ColM &C = S.C;
    for (int k = 0; k < S.nbond; ++k) {
        const int a = S.bond[k].a, b = S.bond[k].b;
        const int t = lane < 3 ? lane : 0;
        const float r = col_sep1(C, a, b, t);
        const float dv = C.V[a][t] - C.V[b][t];
        const float inv = C.invM[a] + C.invM[b];
        const float rr = sum3(r * r), rv = sum3(dv * r);
        const float kk = fdiv_m(rv, rr * inv);
        __syncwarp();
        if (lane < 3) {
            C.V[a][t] -= kk * r * C.invM[a];
            C.V[b][t] += kk * r * C.invM[b];
        }
        __syncwarp();
    }
}

// One colloid-colloid pair (mixed path): the fixed-point LJ force on a
// (b receives -q); false when the pair is beyond the cut-off.
template <class SH>
__device__ __forceinline__ bool cc_pair_m(const ReplicaDev &rp, const SH &S, int a, int b, long long q[3])
{
    const float rc = (float)rp.cc_rc, sg = (float)rp.cc_sigma, ep = (float)rp.cc_eps;
    float d[3];
    for (int t = 0; t < 3; ++t) d[t] = (float)(S.C.Ci[a][t] - S.C.Ci[b][t]) + (S.C.Xf[a][t] - S.C.Xf[b][t]);
    min_image(rp, d);
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < rc * rc)) return false;
    const float ir2 = 1.0f / r2;
    const float s2 = sg * sg * ir2;
    const float s6 = s2 * s2 * s2;
    const float fr = 24.0f * ep * s6 * (2.0f * s6 - 1.0f) * ir2;
    for (int k = 0; k < 3; ++k) q[k] = fx40_any(fr * d[k]);
    return true;
}

__device__ void colloid_colloid(const ReplicaDev &rp, MDShared<true> &S, long long *Fq)
{
    if (!(rp.cc_rc > 0.0)) return;
    for (int a = 0; a < S.nc; ++a)
        for (int b = a + 1; b < S.nc; ++b) {
            if (bonded(S.bond, S.nbond, a, b)) continue;
            long long q[3];
            if (!cc_pair_m(rp, S, a, b, q)) continue;
            for (int k = 0; k < 3; ++k) {
                Fq[3 * a + k] += q[k];
                Fq[3 * b + k] -= q[k];
            }
        }
}

template <class SH>
__device__ void col_load(const Dev &d, const ReplicaDev &rp, SH &S, int j)
{
    const int g = rp.col_off + j;
    for (int k = 0; k < 3; ++k) {
        S.C.Xi[j][k] = d.colXi[3 * g + k];
        S.C.Xf[j][k] = d.colXf[3 * g + k];
        S.C.Ci[j][k] = d.colCi[3 * g + k];
        S.C.V[j][k] = d.colVf[3 * g + k];
        S.C.X0i[j][k] = S.C.Xi[j][k];
        S.C.X0f[j][k] = S.C.Xf[j][k];
    }
    S.C.invM[j] = d.colInvM_f[g];
}

// Warp 0: sum the force partials (per warp of a lone CTA when FROM_WARPS,
// else per CTA of the cluster), add colloid-colloid forces, convert to FP32.
template <int CS, bool FROM_WARPS>
__device__ void col_gather_w(const ReplicaDev &rp, MDShared<true> &S, int par, int lane)
{
    constexpr int NW = MDGeom<CS>::NW;
    for (int l = lane; l < 3 * S.nc; l += 32) {
        long long x = 0;
        if (FROM_WARPS) {
            for (int w = 0; w < NW; ++w) x += (long long)S.wpart[w][l];
        } else {
            for (int q = 0; q < CS; ++q) x += (long long)S.part[par][q][l];
        }
        S.Fsum[l] = x;
    }
    __syncwarp();
    if (rp.cc_rc > 0.0) {
        if (lane == 0) colloid_colloid(rp, S, S.Fsum);
        __syncwarp();
    }
    for (int l = lane; l < 3 * S.nc; l += 32) S.C.F[l / 3][l % 3] = fixed40_to_float(S.Fsum[l]);
    __syncwarp();
}

// Warp 0: first half kick, drift, carry, RATTLE position stage.
template <class SH>
__device__ void col_kick_drift_w(const ReplicaDev &rp, SH &S, int lane)
{
    for (int l = lane; l < 3 * S.nc; l += 32) {
        const int j = l / 3, t = l % 3;
        ColM &C = S.C;
        C.V[j][t] = fmaf(rp.hdt_f, C.F[j][t] * C.invM[j], C.V[j][t]);
        C.Xoi[j][t] = C.Xi[j][t];
        C.Xof[j][t] = C.Xf[j][t];
        C.Xf[j][t] = fmaf(rp.dt_f, C.V[j][t], C.Xf[j][t]);
        col_carry(rp, C, j, t);
    }
    __syncwarp();
    rattle_pos_w(rp, S, lane);
}

// Warp 0: second half kick, RATTLE velocity stage.
template <class SH>
__device__ void col_kick_w(const ReplicaDev &rp, SH &S, int lane)
{
    for (int l = lane; l < 3 * S.nc; l += 32) {
        const int j = l / 3, t = l % 3;
        S.C.V[j][t] = fmaf(rp.hdt_f, S.C.F[j][t] * S.C.invM[j], S.C.V[j][t]);
    }
    __syncwarp();
    rattle_vel_w(S, lane);
}

template <class SH>
__device__ void col_store(const Dev &d, const ReplicaDev &rp, SH &S)
{
    bool bad = false;
    const float skin = rp.skin_f;
    for (int j = 0; j < S.nc; ++j) {
        const int g = rp.col_off + j;
        float e[3];
        for (int t = 0; t < 3; ++t) e[t] = (float)(S.C.Xi[j][t] - S.C.X0i[j][t]) + (S.C.Xf[j][t] - S.C.X0f[j][t]);
        const float dd = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        for (int t = 0; t < 3; ++t) {
            d.colXi[3 * g + t] = S.C.Xi[j][t];
            d.colXf[3 * g + t] = S.C.Xf[j][t];
            d.colVf[3 * g + t] = S.C.V[j][t];
            d.colCi[3 * g + t] = S.C.Ci[j][t];
        }
        if (!(dd <= skin * skin)) bad = true;
    }
    if (bad) atomicAdd(&d.err[ERR_SKIN], 1u);
}

// ===========================================================================
// Reduction of the colloid forces over the CTA and the cluster
// ===========================================================================
// Each warp reduces its lanes' fixed-point partials (exact integer sums).
template <bool MIXED, bool REG>
__device__ __forceinline__ void warp_partials(MDShared<MIXED> &S, long long acc[NCR][3])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (REG) {
        const int nc = S.nc;
#pragma unroll
        for (int j = 0; j < NCR; ++j) {
            if (j >= nc) break;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                long long x = acc[j][k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0) S.wpart[wid][3 * j + k] = (unsigned long long)x;
            }
        }
    }
}

// After the CTA barrier: this CTA's total goes to slot `rank` of every CTA of
// the cluster (buffer = sub-step parity).
template <bool MIXED, bool REG, int CS>
__device__ __forceinline__ void publish_cluster(cg::cluster_group &cl, MDShared<MIXED> &S, int par)
{
    constexpr int NT = MDGeom<CS>::NT, NW = MDGeom<CS>::NW;
    const int tid = threadIdx.x;
    const int rank = (int)cl.block_rank();
    for (int i = tid; i < 3 * S.nc; i += NT) {
        long long x = 0;
        if (REG) {
            for (int w = 0; w < NW; ++w) x += (long long)S.wpart[w][i];
        } else {
            x = (long long)S.Fq[i];
        }
        for (int q = 0; q < CS; ++q) *cl.map_shared_rank(&S.part[par][rank][i], q) = (unsigned long long)x;
    }
}

// Copy the colloid state of replica r between shared memory and its save
// slot (the sub-stepped interval of rmpcd_md_substep), by all threads.
template <bool MIXED>
__device__ void col_state_copy(const Dev &d, MDShared<MIXED> &S, int r, bool save)
{
    using CT = typename std::conditional<MIXED, ColM, ColD>::type;
    static_assert(sizeof(CT) % 4 == 0, "word copy");
    unsigned *g = reinterpret_cast<unsigned *>(reinterpret_cast<unsigned char *>(d.md_col_save) + (size_t)r * sizeof(CT));
    unsigned *s = reinterpret_cast<unsigned *>(&S.C);
    for (int i = threadIdx.x; i < (int)(sizeof(CT) / 4); i += blockDim.x) {
        if (save) g[i] = s[i];
        else s[i] = g[i];
    }
}

// Sub-steps [s0, s1) of the interval (s1 < 0: to the end).  s0 = 0 starts
// the interval from the near area; s0 > 0 continues from the near working set
// in md_work and the colloid state saved by the previous call.  An interval
// that ends before its last sub-step saves the colloid state (and stores its
// positions and velocities for inspection) and keeps the near particles.
template <bool MIXED, bool REG, int CS>
__device__ void md_body(const Dev &d, MDShared<MIXED> &S, const ReplicaDev &rp, cg::cluster_group &cl,
                        uint32_t step, int rbuf, int bbuf, int do_bin, int r, int s0, int s1)
{
    const int s_end = s1 < 0 ? rp.n_md : min(s1, rp.n_md);
    using W = typename std::conditional<MIXED, WorkM, WorkD>::type;
    constexpr int NT = MDGeom<CS>::NT;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int rank = CS == 1 ? 0 : (int)cl.block_rank();
    const int nn = S.nn;
    const int *list = d.near_list + rp.part_off;
    W *work = reinterpret_cast<W *>(d.md_work) + rp.part_off;
    const int first = rank * NT + tid;
    const int stride = CS * NT;
    long long acc[NCR][3];
    auto zero_acc = [&]() {
#pragma unroll
        for (int j = 0; j < NCR; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[j][k] = 0;
    };
    // fixed-point sums of this CTA (and the cluster), then warp 0 / thread 0
    // turns them into colloid forces
    auto reduce_forces = [&](int par) {
        warp_partials<MIXED, REG>(S, acc);
        __syncthreads();
        if (CS == 1 && REG) {
            // a lone CTA sums the per-warp partials directly
            if (!MIXED && tid < 3 * S.nc) {
                long long x = 0;
                for (int w = 0; w < MDGeom<CS>::NW; ++w) x += (long long)S.wpart[w][tid];
                S.part[par][0][tid] = (unsigned long long)x;
            }
            if (!MIXED) __syncthreads();
        } else if (CS == 1) {
            if (tid < 3 * S.nc) S.part[par][0][tid] = S.Fq[tid];
            __syncthreads();
        } else {
            publish_cluster<MIXED, REG, CS>(cl, S, par);
            cl.sync();
        }
    };
    auto zero_fq = [&]() {
        if (!REG)
            for (int i = tid; i < 3 * S.nc; i += NT) S.Fq[i] = 0ull;
    };

    // forces at the start of the interval
    if (s0 == 0) {
    zero_acc();
    zero_fq();
    __syncthreads();
    for (int k = first; k < nn; k += stride) {
        W w;
        w.slot = do_bin ? -1 : list[k];   // flat slot: the write-back target of a granular interval
        if constexpr (MIXED) {
            RecM rec = load_near<RecM>(d, rp, k);
            for (int t = 0; t < 3; ++t) { w.c[t] = cw_get(rec.cw, t); w.o[t] = rec.o[t]; w.v[t] = rec.v[t]; }
            w.fid = rec.fid;
            force_m<REG>(rp, S, w.c, w.o, w.fid, w.f, acc);
        } else {
            RecD rec = load_near<RecD>(d, rp, k);
            for (int t = 0; t < 3; ++t) { w.x[t] = rec.x[t]; w.v[t] = rec.v[t]; }
            w.fid = rec.fid;
            force_d<REG>(rp, S, w.x, w.fid, w.f, acc);
        }
        work[k] = w;
    }
    reduce_forces(0);
    if constexpr (MIXED) {
        if (wid == 0) col_gather_w<CS, (CS == 1 && REG)>(rp, S, 0, lane);
    } else {
        if (tid == 0) col_gather<CS>(rp, S, 0);
    }
    }   // s0 == 0

    const double dt = rp.dt, hdt = rp.hdt;
    for (int s = s0; s < s_end; ++s) {
        const int par = (s + 1) & 1;
        // colloids: first half kick, drift, RATTLE position stage
        if constexpr (MIXED) {
            if (wid == 0) col_kick_drift_w(rp, S, lane);
        } else {
            if (tid == 0) {
                col_kick_drift(rp, S);
                col_frames(rp, S);
            }
        }
        zero_acc();
        zero_fq();
        __syncthreads();
        // solvent: second half kick of the previous sub-step, first half kick
        // and drift of this one, new forces, catalytic conversion
        for (int k = first; k < nn; k += stride) {
            W w = work[k];
            if constexpr (MIXED) {
                const float hdtf = rp.hdt_f, dtf = rp.dt_f;
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    if (s > 0) w.v[t] = fmaf(hdtf, w.f[t], w.v[t]);
                    w.v[t] = fmaf(hdtf, w.f[t], w.v[t]);
                    w.o[t] = fmaf(dtf, w.v[t], w.o[t]);
                }
                force_m<REG>(rp, S, w.c, w.o, w.fid, w.f, acc);
                w.fid = catalysis(rp, w.fid, inside_cat_m(rp, S, w.c, w.o), step, s);
            } else {
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    if (s > 0) w.v[t] = fma(hdt, w.f[t], w.v[t]);
                    w.v[t] = fma(hdt, w.f[t], w.v[t]);
                    w.x[t] = fma(dt, w.v[t], w.x[t]);
                }
                force_d<REG>(rp, S, w.x, w.fid, w.f, acc);
                w.fid = catalysis(rp, w.fid, inside_cat_d(rp, S, w.x), step, s);
            }
            work[k] = w;
        }
        reduce_forces(par);
        // colloids: new forces, second half kick, RATTLE velocity stage
        if constexpr (MIXED) {
            if (wid == 0) {
                col_gather_w<CS, (CS == 1 && REG)>(rp, S, par, lane);
                col_kick_w(rp, S, lane);
            }
        } else {
            if (tid == 0) {
                col_gather<CS>(rp, S, par);
                col_kick(rp, S);
            }
        }
    }

    if (s_end < rp.n_md) {
        // a sub-stepped interval continues later: save the colloids, keep
        // the near particles in md_work and the near count
        __syncthreads();
        if (rank == 0) {
            if (tid == 0) {
                if constexpr (!MIXED) col_frames(rp, S);
                col_store(d, rp, S);
            }
            __syncthreads();
            col_state_copy<MIXED>(d, S, r, true);
        }
        if (CS > 1) cl.sync();
        return;
    }
    // last half kick, wrap, write back (and bin for the collision of `step`)
    double sh[3];
    grid_shift(rp.seed, step, sh);
    for (int k = first; k < nn; k += stride) {
        W w = work[k];
        if constexpr (MIXED) {
            for (int t = 0; t < 3; ++t) w.v[t] = fmaf(rp.hdt_f, w.f[t], w.v[t]);
            renorm_m(rp, w.c, w.o);
            RecM rec;
            rec.cw = cw_make(w.c[0], w.c[1], w.c[2]);
            for (int t = 0; t < 3; ++t) { rec.o[t] = w.o[t]; rec.v[t] = w.v[t]; }
            rec.fid = do_bin ? (w.fid | F_PROP) : (w.fid & ~F_PROP);
            const float sf[3] = {(float)sh[0], (float)sh[1], (float)sh[2]};
            put_near(d, rbuf, bbuf, do_bin, do_bin ? bin_cell(d, rp.cell_off, cell_key_m(rp, w.c, w.o, sf)) : 0, w.slot, rec);
        } else {
            for (int t = 0; t < 3; ++t) w.v[t] = fma(hdt, w.f[t], w.v[t]);
            wrap_periodic_d(rp, w.x);
            RecD rec;
            for (int t = 0; t < 3; ++t) { rec.x[t] = w.x[t]; rec.v[t] = w.v[t]; }
            rec.fid = do_bin ? (w.fid | F_PROP) : (w.fid & ~F_PROP);
            rec.u0 = 0u;
            rec.u1 = 0.0;
            put_near(d, rbuf, bbuf, do_bin, do_bin ? bin_cell(d, rp.cell_off, cell_key_d(rp, w.x, sh)) : 0, w.slot, rec);
        }
    }
    __syncwarp();
    if (tid == 0 && rank == 0) {
        if constexpr (!MIXED) col_frames(rp, S);
        col_store(d, rp, S);
        // every CTA read near_count before the first barrier of the cluster
        d.near_count[r] = 0;
    }
    if (CS > 1) cl.sync();   // no CTA leaves while a peer may still write to its shared memory
}

template <bool MIXED, int CS>
__global__ void __launch_bounds__(MDGeom<CS>::NT, 1) k_md(Dev d, uint32_t step, int rbuf, int bbuf, int do_bin,
                                                          int s0, int s1)
{
    step = resolve_step(d, step);   // STEP_DEVICE: the step of the control block
    __shared__ MDShared<MIXED> S;
    __shared__ ReplicaDev s_rp;
    cg::cluster_group cl = cg::this_cluster();
    const int r = blockIdx.x / CS;
    const int tid = threadIdx.x;
    if (tid == 0) s_rp = d.rep[r];
    __syncthreads();
    const ReplicaDev &rp = s_rp;
    if (rp.n_col == 0 || rp.body >= 0 || rp.net >= 0) return;   // uniform over the cluster (bodies, networks: own kernels)
    if (tid == 0) {
        S.nc = rp.n_col;
        S.nbond = rp.n_bond;
        S.nn = min(d.near_count[r], rp.n_part);
    }
    if (tid < rp.n_col) {
        const int j = tid, g = rp.col_off + tid;
        col_load(d, rp, S, j);
        S.M[j] = d.colM[g];
        S.sig[j] = d.colSig[g]; S.epsA[j] = d.colEpsA[g]; S.epsB[j] = d.colEpsB[g]; S.rc2[j] = d.colRc2[g];
        S.sigf[j] = d.colSig_f[g]; S.epsAf[j] = d.colEpsA_f[g]; S.epsBf[j] = d.colEpsB_f[g];
        S.rc2f[j] = d.colRc2_f[g];
        S.cat[j] = d.colCat[g];
    }
    if (tid < rp.n_bond) S.bond[tid] = d.bonds[rp.bond_off + tid];
    __syncthreads();
    if (s0 > 0) {
        // a continued interval: the colloid state of the previous call
        col_state_copy<MIXED>(d, S, r, false);
        __syncthreads();
    }
    if constexpr (!MIXED) {
        if (tid == 0) col_frames(rp, S);
        __syncthreads();
    }
    // all CTAs of the cluster must have read near_count before rank 0 resets it
    if (CS > 1) cl.sync();
    if (s0 >= rp.n_md) return;   // this replica's interval has fewer sub-steps
    if (rp.n_col <= NCR) md_body<MIXED, true, CS>(d, S, rp, cl, step, rbuf, bbuf, do_bin, r, s0, s1);
    else md_body<MIXED, false, CS>(d, S, rp, cl, step, rbuf, bbuf, do_bin, r, s0, s1);
}

// ===========================================================================
// Wide MD kernel (mixed path): one replica with many colloids, whose near
// solvent is too large for one thread-block cluster.  A cooperative grid of
// CTAs covers all SMs; every CTA keeps an identical copy of the colloids in
// shared memory and integrates it with the general kernel's warp-0 code, from
// force totals gathered once per sub-step through device memory and one
// grid-wide barrier.  Each near particle keeps the (at most MDW_KC) colloids it
// can reach during the interval, found once at the start with the near-list
// radius plus a margin, so a force evaluation visits a few colloids instead
// of all; a particle with more candidates scans every colloid.  Colloid pairs
// within reach of the LJ cut-off (distance plus two skins) are listed once.
// The forces are the same exact fixed-point sums as in the general kernel, so
// both give bit-identical results.
// ===========================================================================
constexpr int MDW_NT = 256;
constexpr int MDW_PPT = 2;             // near particles a thread keeps in registers
constexpr int MDW_KC = 4;              // candidate colloids per particle
constexpr int MDW_MAXP = 1024;         // listed colloid pairs
constexpr float MDW_MARGIN = 1.5f;     // added to the near radius for the candidate test
constexpr int MDW_SPIN_LIMIT = 1 << 24;

struct WideShared {
    ColM C;
    float sigf[MAXC], epsAf[MAXC], epsBf[MAXC], rc2f[MAXC], Rbf[MAXC];
    int cat[MAXC];
    BondDev bond[MAXB];
    unsigned long long Fq[MAXC * 3];   // this CTA's fixed-point partials
    long long Fsum[MAXC * 3];          // the grid total
    short pa[MDW_MAXP], pb[MDW_MAXP];
    int npairs, all_pairs;
    int nc, nbond, nn;
    unsigned gen;                      // grid barrier generation seen by this CTA
    int dead;                          // a grid barrier timed out: stop waiting
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier over co-resident CTAs: thread 0 of each CTA arrives on a
// counter; the last one resets it and advances the generation the others
// wait for (bounded: ERR_TIMEOUT, after which this CTA stops waiting).
__device__ __forceinline__ void wide_barrier(const Dev &d, WideShared &S)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        MdWideGlobal *g = d.md_wide;
        const unsigned gen = S.gen;
        __threadfence();
        if (atomicAdd(&g->count, 1u) == gridDim.x - 1u) {
            g->count = 0u;
            __threadfence();
            st_release_u32(&g->gen, gen + 1u);
        } else if (!S.dead) {
            int spins = 0;
            while (ld_acquire_u32(&g->gen) == gen) {
                if (++spins > MDW_SPIN_LIMIT) {
                    atomicOr(&d.err[ERR_TIMEOUT], 1u);
                    S.dead = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        S.gen = gen + 1u;
    }
    __syncthreads();
}

// Candidate colloids of a particle, packed 8 bits each into w.p0; the count
// (or MDW_KC + 1: scan every colloid) into w.p1.
__device__ __forceinline__ void wide_candidates(const ReplicaDev &rp, const WideShared &S, WorkM &w)
{
    const float st = sqrtf(w.v[0] * w.v[0] + w.v[1] * w.v[1] + w.v[2] * w.v[2]) * rp.tau_f;
    unsigned packed = 0u;
    int k = 0;
    for (int j = 0; j < S.nc; ++j) {
        float d[3];
        sep_m(rp, S, j, w.c, w.o, d);
        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const float R = S.Rbf[j] + st + MDW_MARGIN;
        if (r2 < R * R) {
            if (k < MDW_KC) packed |= (unsigned)j << (8 * k);
            ++k;
        }
    }
    w.p0 = __uint_as_float(packed);
    w.p1 = __int_as_float(k > MDW_KC ? MDW_KC + 1 : k);
}

// The general kernel's force on one particle (atomic path), over the
// particle's candidates in increasing colloid order; inside: within the
// cut-off of a catalytic colloid.
__device__ __forceinline__ void force_wide(const ReplicaDev &rp, WideShared &S, WorkM &w, bool &inside)
{
    w.f[0] = w.f[1] = w.f[2] = 0.0f;
    inside = false;
    const int ncand = __float_as_int(w.p1);
    const unsigned packed = __float_as_uint(w.p0);
    const int jn = ncand > MDW_KC ? S.nc : ncand;
    for (int q = 0; q < jn; ++q) {
        const int j = ncand > MDW_KC ? q : (int)((packed >> (8 * q)) & 0xFFu);
        float d[3];
        sep_m(rp, S, j, w.c, w.o, d);
        const float eps = (w.fid & F_B) ? S.epsBf[j] : S.epsAf[j];
        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < S.rc2f[j]) {
            inside = inside || S.cat[j];
            const float fr = wca_fr_m(eps, S.sigf[j], r2);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float fk = fr * d[k];
                w.f[k] = w.f[k] + fk;
                sub_fixed_agg(S.Fq, 3 * j + k, fx40_any(fk));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) w.f[k] = w.f[k] + rp.g_f[k];
}

// One sub-step of a particle after the colloids moved: kicks, drift, force,
// catalysis (s < 0: only the force, at the start of the interval).
__device__ __forceinline__ void wide_particle(const ReplicaDev &rp, WideShared &S, WorkM &w, uint32_t step, int s)
{
    if (s >= 0) {
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (s > 0) w.v[t] = fmaf(rp.hdt_f, w.f[t], w.v[t]);
            w.v[t] = fmaf(rp.hdt_f, w.f[t], w.v[t]);
            w.o[t] = fmaf(rp.dt_f, w.v[t], w.o[t]);
        }
    }
    bool inside;
    force_wide(rp, S, w, inside);
    if (s >= 0) w.fid = catalysis(rp, w.fid, inside, step, s);
}

// After a CTA barrier: this CTA's partials into the grid accumulator of round
// `round` (three buffers: round r is zeroed by CTA 0 after the barrier of
// round r - 1), the grid barrier, then warp 0 forms the colloid forces.
__device__ __forceinline__ void wide_reduce(const Dev &d, const ReplicaDev &rp, WideShared &S, int round)
{
    MdWideGlobal *g = d.md_wide;
    const int tid = threadIdx.x, lane = tid & 31;
    const int b = round % 3;
    __syncthreads();
    for (int i = tid; i < 3 * S.nc; i += MDW_NT)
        if (S.Fq[i] != 0ull) atomicAdd(&g->acc[b][i], S.Fq[i]);
    wide_barrier(d, S);
    if (tid < 32) {
        for (int l = lane; l < 3 * S.nc; l += 32) S.Fsum[l] = (long long)__ldcg(&g->acc[b][l]);
        __syncwarp();
        if (rp.cc_rc > 0.0) {
            const int np = S.all_pairs ? S.nc * S.nc : S.npairs;
            for (int p = lane; p < np; p += 32) {
                int a, c;
                if (S.all_pairs) {
                    a = p / S.nc;
                    c = p % S.nc;
                    if (c <= a || bonded(S.bond, S.nbond, a, c)) continue;
                } else {
                    a = S.pa[p];
                    c = S.pb[p];
                }
                long long q[3];
                if (!cc_pair_m(rp, S, a, c, q)) continue;
                for (int k = 0; k < 3; ++k) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&S.Fsum[3 * a + k]), (unsigned long long)q[k]);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&S.Fsum[3 * c + k]), (unsigned long long)(-q[k]));
                }
            }
            __syncwarp();
        }
        for (int l = lane; l < 3 * S.nc; l += 32) S.C.F[l / 3][l % 3] = fixed40_to_float(S.Fsum[l]);
        __syncwarp();
    }
    if (blockIdx.x == 0)
        for (int i = tid; i < 3 * S.nc; i += MDW_NT) g->acc[(round + 2) % 3][i] = 0ull;
}

__global__ void __launch_bounds__(MDW_NT) k_md_wide(Dev d, int r, uint32_t step, int rbuf, int bbuf, int do_bin)
{
    step = resolve_step(d, step);   // STEP_DEVICE: the step of the control block
    __shared__ WideShared S;
    __shared__ ReplicaDev s_rp;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        s_rp = d.rep[r];
        S.gen = ld_acquire_u32(&d.md_wide->gen);
        S.dead = 0;
        S.npairs = 0;
        S.all_pairs = 0;
    }
    __syncthreads();
    const ReplicaDev &rp = s_rp;
    if (rp.n_col == 0) return;   // uniform over the grid
    if (tid == 0) {
        S.nc = rp.n_col;
        S.nbond = rp.n_bond;
        S.nn = min(d.near_count[r], rp.n_part);
    }
    for (int j = tid; j < rp.n_col; j += MDW_NT) {
        const int g = rp.col_off + j;
        col_load(d, rp, S, j);
        S.sigf[j] = d.colSig_f[g]; S.epsAf[j] = d.colEpsA_f[g]; S.epsBf[j] = d.colEpsB_f[g];
        S.rc2f[j] = d.colRc2_f[g];
        S.Rbf[j] = d.colRb_f[g];
        S.cat[j] = d.colCat[g];
    }
    if (tid < rp.n_bond) S.bond[tid] = d.bonds[rp.bond_off + tid];
    for (int i = tid; i < 3 * rp.n_col; i += MDW_NT) S.Fq[i] = 0ull;
    __syncthreads();
    if (rp.cc_rc > 0.0) {
        // colloid pairs that can come within the cut-off this interval: each
        // colloid moves at most `skin` (a violation is reported)
        const float reach = (float)rp.cc_rc + 2.0f * rp.skin_f + 1e-3f;
        for (int p = tid; p < S.nc * S.nc; p += MDW_NT) {
            const int a = p / S.nc, c = p % S.nc;
            if (c <= a || bonded(S.bond, S.nbond, a, c)) continue;
            float dd[3];
            for (int t = 0; t < 3; ++t) dd[t] = (float)(S.C.Ci[a][t] - S.C.Ci[c][t]) + (S.C.Xf[a][t] - S.C.Xf[c][t]);
            min_image(rp, dd);
            if (dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2] < reach * reach) {
                const int k = atomicAdd(&S.npairs, 1);
                if (k < MDW_MAXP) { S.pa[k] = (short)a; S.pb[k] = (short)c; }
                else S.all_pairs = 1;
            }
        }
    }
    __syncthreads();

    const int nn = S.nn;
    const int *list = d.near_list + rp.part_off;
    WorkM *work = reinterpret_cast<WorkM *>(d.md_work) + rp.part_off;
    const int first = blockIdx.x * MDW_NT + tid;
    const int stride = gridDim.x * MDW_NT;
    const int over = first + MDW_PPT * stride;
    WorkM reg[MDW_PPT];
    auto load_w = [&](int k, WorkM &w) {
        w.slot = do_bin ? -1 : list[k];   // flat slot: the write-back target of a granular interval
        const RecM rec = load_near<RecM>(d, rp, k);
        for (int t = 0; t < 3; ++t) { w.c[t] = cw_get(rec.cw, t); w.o[t] = rec.o[t]; w.v[t] = rec.v[t]; }
        w.fid = rec.fid;
        wide_candidates(rp, S, w);
    };
    // forces at the start of the interval
#pragma unroll
    for (int p = 0; p < MDW_PPT; ++p)
        if (first + p * stride < nn) {
            load_w(first + p * stride, reg[p]);
            wide_particle(rp, S, reg[p], step, -1);
        }
    for (int k = over; k < nn; k += stride) {
        WorkM w;
        load_w(k, w);
        wide_particle(rp, S, w, step, -1);
        work[k] = w;
    }
    wide_reduce(d, rp, S, 0);
    __syncthreads();

    for (int s = 0; s < rp.n_md; ++s) {
        // colloids: first half kick, drift, RATTLE position stage
        if (wid == 0) col_kick_drift_w(rp, S, lane);
        for (int i = tid; i < 3 * S.nc; i += MDW_NT) S.Fq[i] = 0ull;
        __syncthreads();
        // solvent: second half kick of the previous sub-step, first half kick
        // and drift of this one, new forces, catalytic conversion
#pragma unroll
        for (int p = 0; p < MDW_PPT; ++p)
            if (first + p * stride < nn) wide_particle(rp, S, reg[p], step, s);
        for (int k = over; k < nn; k += stride) {
            WorkM w = work[k];
            wide_particle(rp, S, w, step, s);
            work[k] = w;
        }
        wide_reduce(d, rp, S, s + 1);
        // colloids: second half kick, RATTLE velocity stage
        if (wid == 0) col_kick_w(rp, S, lane);
        __syncthreads();
    }

    // last half kick, wrap, write back (and bin for the collision of `step`)
    double sh[3];
    grid_shift(rp.seed, step, sh);
    const float sf[3] = {(float)sh[0], (float)sh[1], (float)sh[2]};
    auto finish = [&](WorkM &w) {
        for (int t = 0; t < 3; ++t) w.v[t] = fmaf(rp.hdt_f, w.f[t], w.v[t]);
        renorm_m(rp, w.c, w.o);
        RecM rec;
        rec.cw = cw_make(w.c[0], w.c[1], w.c[2]);
        for (int t = 0; t < 3; ++t) { rec.o[t] = w.o[t]; rec.v[t] = w.v[t]; }
        rec.fid = do_bin ? (w.fid | F_PROP) : (w.fid & ~F_PROP);
        put_near(d, rbuf, bbuf, do_bin, do_bin ? bin_cell(d, rp.cell_off, cell_key_m(rp, w.c, w.o, sf)) : 0, w.slot, rec);
    };
#pragma unroll
    for (int p = 0; p < MDW_PPT; ++p)
        if (first + p * stride < nn) finish(reg[p]);
    for (int k = over; k < nn; k += stride) {
        WorkM w = work[k];
        finish(w);
    }
    if (blockIdx.x == 0 && tid == 0) {
        col_store(d, rp, S);
        d.near_count[r] = 0;   // every CTA read it before the first grid barrier
    }
}

// Co-resident CTAs the wide kernel can launch on this device (0: unsupported).
int md_wide_grid()
{
    int dev = 0, sms = 0, per = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_md_wide, MDW_NT, 0) != cudaSuccess) per = 0;
    cudaGetLastError();
    return coop ? sms * per : 0;
}

void launch_md_wide(const Dev &d, const std::vector<int> &reps, int grid, uint32_t step, int rbuf, int bbuf,
                    int do_bin, cudaStream_t s)
{
    for (int r : reps) {
        cudaMemsetAsync(d.md_wide->acc, 0, sizeof(d.md_wide->acc), s);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid, 1, 1);
        cfg.blockDim = dim3(MDW_NT, 1, 1);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_md_wide, d, r, step, rbuf, bbuf, do_bin);
    }
}

template <bool MIXED, int CS>
static void launch_md_cs(const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, int s0, int s1, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(d.n_rep * CS), 1, 1);
    cfg.blockDim = dim3(MDGeom<CS>::NT, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_md<MIXED, CS>, d, step, rbuf, bbuf, do_bin, s0, s1);
}

const int MD_CLUSTER_SIZES[4] = {1, 2, 4, 8};

void launch_md(bool mixed, const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, int cs, cudaStream_t s)
{
    launch_md_range(mixed, d, step, rbuf, bbuf, do_bin, cs, 0, -1, s);
}

void launch_md_range(bool mixed, const Dev &d, uint32_t step, int rbuf, int bbuf, int do_bin, int cs, int s0, int s1,
                     cudaStream_t s)
{
    if (d.n_rep <= 0) return;
    switch (cs) {
    case 1: mixed ? launch_md_cs<true, 1>(d, step, rbuf, bbuf, do_bin, s0, s1, s) : launch_md_cs<false, 1>(d, step, rbuf, bbuf, do_bin, s0, s1, s); break;
    case 2: mixed ? launch_md_cs<true, 2>(d, step, rbuf, bbuf, do_bin, s0, s1, s) : launch_md_cs<false, 2>(d, step, rbuf, bbuf, do_bin, s0, s1, s); break;
    case 4: mixed ? launch_md_cs<true, 4>(d, step, rbuf, bbuf, do_bin, s0, s1, s) : launch_md_cs<false, 4>(d, step, rbuf, bbuf, do_bin, s0, s1, s); break;
    default: mixed ? launch_md_cs<true, 8>(d, step, rbuf, bbuf, do_bin, s0, s1, s) : launch_md_cs<false, 8>(d, step, rbuf, bbuf, do_bin, s0, s1, s); break;
    }
}

size_t md_col_state_bytes(bool mixed) { return mixed ? sizeof(ColM) : sizeof(ColD); }

}  // namespace rmpcd
