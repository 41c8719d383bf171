// k_md_body.cu -- near-field MD of one collision interval for the replicas
// whose colloid is a rigid bead body: the Janus particle of §1.5, a network
// of WCA beads (§1.4) that moves as one rigid body.
//
// Per sub-step dt (§1.1 velocity Verlet):
//   body:    V += dt/2 F/M, l += dt/2 R^T T, X += dt V, free rotation by the
//            symmetric principal-axis splitting R_1(dt/2) R_2(dt/2) R_3(dt)
//            R_2(dt/2) R_1(dt/2) (Dullweber, Leimkuhler & McLachlan, J. Chem.
//            Phys. 107, 5840 (1997)), each turn R_k(h) by the angle phi with
//            tan(phi/2) = h l_k / (2 I_k): q <- q (1, tan(phi/2) e_k), l turned
//            by -phi about e_k; q normalised after the five turns;
//   solvent: v += dt/2 f, x += dt v;
//   forces:  WCA between each near particle and the beads it reaches; the
//            pair force f on the particle puts -f and the torque -(R b_j) x f
//            on the body;
//   kicks:   V += dt/2 F/M, l += dt/2 R^T T, v += dt/2 f;
//   §1.5:    an A particle inside a catalytic bead's range is tagged, a tagged
//            one that has left every such range becomes B.
//
// One CTA of MDB_NT threads per replica runs all n_md sub-steps; two CTAs
// share an SM, so one replica's serial body update overlaps the other's
// force pass.  Thread 0 integrates the body in FP64 on both paths: FP32
// rounding of the orientation accumulates over the sub-steps into bead
// positions that the steep bead potential turns into force errors well above
// the mixed path's tolerance.  FP64 division is slow on this GPU, so the
// mixed path's integrator has none on its sub-step chain (reciprocals of M
// and I_k precomputed, Newton reciprocal and inverse square root from an
// FP32 seed); the FP64 path keeps the FP64 definition's divisions.  After
// every turn the bead offsets R b_j are recomputed (FP64, rounded to FP32 on
// the mixed path) in shared memory.  On the mixed path the centre moves
// first, and the turn and the bead offsets (warp 0) run beside the first
// phase of the particles' sub-step, whose reach test needs the centre only.
// A particle finds the
// beads it can reach through a lookup grid in the body frame, built on the
// host once per body: the grid cell of the particle's body-frame position
// lists, in ascending order, every bead whose cut-off plus a margin reaches
// the cell, so the FP64 path adds the same pair forces in the same order as
// a scan over all beads.  Body force and torque are summed as 64-bit fixed
// point (2^-40) -- per pair on the FP64 path, per particle (its FP32 sums over
// its beads) on the mixed path --: per thread, per warp by shuffles, then over
// the warps, so the totals do not depend on the order of the near list.
#include <type_traits>

#include "rmpcd_kernels.cuh"
#include "rmpcd_fixed.cuh"

namespace rmpcd {

constexpr int MDB_NT = 512;
constexpr int MDB_NW = MDB_NT / 32;

// Mixed path work record: cell word, id|flags, FP32 offset and the
// half-step velocity v + dt/2 f of the leapfrog form of velocity Verlet (the
// same update; the record needs no force and the slot is re-read from the
// near list at the end).
struct __align__(16) BWorkM {
    uint32_t cw;
    uint32_t fid;
    float o[3];
    float v[3];
};
static_assert(sizeof(BWorkM) == 32, "mixed MD work record is two 16-byte words");
struct __align__(16) BWorkD {
    double x[3];
    double v[3];
    double f[3];
    uint32_t fid;
    int slot;
};

// Body state and per-sub-step frames; bead arrays follow in dynamic shared
// memory (see bead_layout).
struct BodyShared {
    // FP64 path
    double X[3], V[3], q[4], l[3], X0[3];
    double R[3][3];
    double Xw[3];
    double F[3], tb[3];
    double M, I[3], sigma, rc2;
    // mixed path integrator constants: 1/M, 0.5 h_s / I_k of the five turns
    double invM, ct[5];
    // both: rotation in FP32 (lookup grid, mixed forces), wrapped centre cell
    float Rf[3][3];
    float Cf[3];
    int Ci[3];
    float sigma_f, rc2_f, glo, ginv;
    float reach2_f;                  // beyond this squared distance from the centre no bead is in range
    int gn, nb, nn;
    const int *gstart;
    const unsigned short *glist;
    const unsigned short *gs16, *gl16;   // the lookup grid copied to shared memory (gsm: in use)
    int gsm;
    int nreach;                      // mixed sub-step: near particles listed in reach of a bead
    unsigned long long wpart[MDB_NW][6];
};

// Dynamic shared memory: FP64 path b[3nb], rb[3nb], Xb[3nb], eps[2nb] (double),
// cat[nb]; mixed path b[3nb] (double), rb[3nb], eps[2nb] (float), cat[nb].
struct BeadSmem {
    double *b, *rb, *Xb, *eps;
    float *rbf, *epsf;
    int *cat;
};

template <bool MIXED>
__host__ __device__ inline size_t bead_smem_bytes(int nb)
{
    return MIXED ? (size_t)nb * (3 * sizeof(double) + 5 * sizeof(float) + sizeof(int))
                 : (size_t)nb * (11 * sizeof(double) + sizeof(int));
}

template <bool MIXED>
__device__ inline BeadSmem bead_layout(unsigned char *p, int nb)
{
    BeadSmem B{};
    if (MIXED) {
        B.b = reinterpret_cast<double *>(p);
        p += sizeof(double) * 3 * nb;
        B.rbf = reinterpret_cast<float *>(p);
        p += sizeof(float) * 3 * nb;
        B.epsf = reinterpret_cast<float *>(p);
        p += sizeof(float) * 2 * nb;
    } else {
        B.b = reinterpret_cast<double *>(p);
        p += sizeof(double) * 3 * nb;
        B.rb = reinterpret_cast<double *>(p);
        p += sizeof(double) * 3 * nb;
        B.Xb = reinterpret_cast<double *>(p);
        p += sizeof(double) * 3 * nb;
        B.eps = reinterpret_cast<double *>(p);
        p += sizeof(double) * 2 * nb;
    }
    B.cat = reinterpret_cast<int *>(p);
    return B;
}

// --- body integrator (thread 0, FP64) ----------------------------------------
__device__ void body_frames(const ReplicaDev &rp, BodyShared &S)
{
    const double w = S.q[0], x = S.q[1], y = S.q[2], z = S.q[3];
    S.R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    S.R[0][1] = 2.0 * (x * y - w * z);
    S.R[0][2] = 2.0 * (x * z + w * y);
    S.R[1][0] = 2.0 * (x * y + w * z);
    S.R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    S.R[1][2] = 2.0 * (y * z - w * x);
    S.R[2][0] = 2.0 * (x * z - w * y);
    S.R[2][1] = 2.0 * (y * z + w * x);
    S.R[2][2] = 1.0 - 2.0 * (x * x + y * y);
    wrapped_colloid(rp, S.X, S.Xw);
    for (int k = 0; k < 3; ++k) {
        for (int t = 0; t < 3; ++t) S.Rf[k][t] = (float)S.R[k][t];
        const double fl = floor(S.Xw[k]);
        int c = (int)fl;
        float o = (float)(S.Xw[k] - fl);
        if (o >= 1.0f) { o = 0.0f; c += 1; }
        if (c >= rp.L[k]) c -= rp.L[k];
        S.Ci[k] = c;
        S.Cf[k] = o;
    }
}

__device__ void body_kick(BodyShared &S, double hdt)
{
    for (int t = 0; t < 3; ++t) {
        S.V[t] = fma(hdt, S.F[t] / S.M, S.V[t]);
        S.l[t] = fma(hdt, S.tb[t], S.l[t]);
    }
}

__device__ void body_kick_drift_rotate(BodyShared &S, double dt, double hdt)
{
    for (int t = 0; t < 3; ++t) {
        S.V[t] = fma(hdt, S.F[t] / S.M, S.V[t]);
        S.l[t] = fma(hdt, S.tb[t], S.l[t]);
        S.X[t] = fma(dt, S.V[t], S.X[t]);
    }
    double q[4] = {S.q[0], S.q[1], S.q[2], S.q[3]};
    double l[3] = {S.l[0], S.l[1], S.l[2]};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int k = (s == 2) ? 2 : (s == 1 || s == 3) ? 1 : 0;
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        const double h = (s == 2) ? dt : 0.5 * dt;
        const double t = 0.5 * (h * l[k] / S.I[k]);
        const double tt = t * t;
        const double inv = 1.0 / (1.0 + tt);
        const double c = (1.0 - tt) * inv;
        const double sn = (2.0 * t) * inv;
        const double la = c * l[a] + sn * l[b];
        const double lb = c * l[b] - sn * l[a];
        l[a] = la;
        l[b] = lb;
        const double w = q[0], v0 = q[1 + k], va = q[1 + a], vb = q[1 + b];
        q[0] = w - t * v0;
        q[1 + k] = v0 + t * w;
        q[1 + a] = va + t * vb;
        q[1 + b] = vb - t * va;
    }
    const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) S.q[i] = q[i] / nq;
    for (int i = 0; i < 3; ++i) S.l[i] = l[i];
}

// --- mixed path: the same integrator without divisions on the chain ---------
// FP64 reciprocal of x in [1, 2): FP32 seed and two Newton steps (error far
// below one FP64 ulp before the last rounding).
__device__ __forceinline__ double rcp_nr(double x)
{
    double y = (double)__frcp_rn((float)x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// 1/sqrt(x) for x near 1: FP32 seed and two Newton steps.
__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y = (double)rsqrtf((float)x);
    y = y * (1.5 - 0.5 * x * y * y);
    return y * (1.5 - 0.5 * x * y * y);
}

__device__ void body_kick_fast(BodyShared &S, double hdt)
{
    for (int t = 0; t < 3; ++t) {
        S.V[t] = fma(hdt, S.F[t] * S.invM, S.V[t]);
        S.l[t] = fma(hdt, S.tb[t], S.l[t]);
    }
}

// The sub-step's first half kick and drift of the centre, and the half kick
// of l; then (body_rotate_fast) the free rotation.  The particles' reach test
// needs the centre only, so the rotation runs beside it.
__device__ void body_kick_drift_fast(BodyShared &S, double dt, double hdt)
{
    for (int t = 0; t < 3; ++t) {
        S.V[t] = fma(hdt, S.F[t] * S.invM, S.V[t]);
        S.l[t] = fma(hdt, S.tb[t], S.l[t]);
        S.X[t] = fma(dt, S.V[t], S.X[t]);
    }
}

__device__ void body_rotate_fast(BodyShared &S, double dt)
{
    double q[4] = {S.q[0], S.q[1], S.q[2], S.q[3]};
    double l[3] = {S.l[0], S.l[1], S.l[2]};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int k = (s == 2) ? 2 : (s == 1 || s == 3) ? 1 : 0;
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        const double t = S.ct[s] * l[k];
        const double tt = t * t;
        const double inv = rcp_nr(1.0 + tt);
        const double c = (1.0 - tt) * inv;
        const double sn = (2.0 * t) * inv;
        const double la = c * l[a] + sn * l[b];
        const double lb = c * l[b] - sn * l[a];
        l[a] = la;
        l[b] = lb;
        const double w = q[0], v0 = q[1 + k], va = q[1 + a], vb = q[1 + b];
        q[0] = w - t * v0;
        q[1 + k] = v0 + t * w;
        q[1 + a] = va + t * vb;
        q[1 + b] = vb - t * va;
    }
    const double g = rsqrt_nr(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) S.q[i] = q[i] * g;
    for (int i = 0; i < 3; ++i) S.l[i] = l[i];
}

// Frame of the mixed path: R (body_rotation_frame_fast), the wrapped
// centre's cell and FP32 offset (body_centre_frame_fast).
__device__ void body_rotation_frame_fast(BodyShared &S)
{
    const double w = S.q[0], x = S.q[1], y = S.q[2], z = S.q[3];
    S.R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    S.R[0][1] = 2.0 * (x * y - w * z);
    S.R[0][2] = 2.0 * (x * z + w * y);
    S.R[1][0] = 2.0 * (x * y + w * z);
    S.R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    S.R[1][2] = 2.0 * (y * z - w * x);
    S.R[2][0] = 2.0 * (x * z - w * y);
    S.R[2][1] = 2.0 * (y * z + w * x);
    S.R[2][2] = 1.0 - 2.0 * (x * x + y * y);
    for (int k = 0; k < 3; ++k)
        for (int t = 0; t < 3; ++t) S.Rf[k][t] = (float)S.R[k][t];
}
__device__ void body_centre_frame_fast(const ReplicaDev &rp, BodyShared &S)
{
    for (int k = 0; k < 3; ++k) {
        const double fl = floor(S.X[k]);
        int c = (int)fl;
        float o = (float)(S.X[k] - fl);
        if (o >= 1.0f) { o = 0.0f; c += 1; }
        S.Ci[k] = imod(c, rp.L[k]);
        S.Cf[k] = o;
    }
}
__device__ void body_frames_fast(const ReplicaDev &rp, BodyShared &S)
{
    body_rotation_frame_fast(S);
    body_centre_frame_fast(rp, S);
}

// Fixed-point totals of the warps -> F and the body-frame torque R^T T.
__device__ void body_totals(BodyShared &S)
{
    long long Q[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < MDB_NW; ++w)
        for (int i = 0; i < 6; ++i) Q[i] += (long long)S.wpart[w][i];
    double T[3];
    for (int k = 0; k < 3; ++k) {
        S.F[k] = (double)Q[k] * 0x1p-40;
        T[k] = (double)Q[3 + k] * 0x1p-40;
    }
    for (int k = 0; k < 3; ++k) S.tb[k] = S.R[0][k] * T[0] + S.R[1][k] * T[1] + S.R[2][k] * T[2];
}

// Bead offsets R b_j (and FP64 positions Xw + R b_j) for the current frame.
template <bool MIXED>
__device__ void bead_frames(BodyShared &S, const BeadSmem &B, int first = threadIdx.x, int stride = MDB_NT)
{
    for (int j = first; j < S.nb; j += stride) {
        if (MIXED) {
            const double b0 = B.b[3 * j], b1 = B.b[3 * j + 1], b2 = B.b[3 * j + 2];
#pragma unroll
            for (int t = 0; t < 3; ++t) B.rbf[3 * j + t] = (float)(S.R[t][0] * b0 + S.R[t][1] * b1 + S.R[t][2] * b2);
        } else {
            const double b0 = B.b[3 * j], b1 = B.b[3 * j + 1], b2 = B.b[3 * j + 2];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const double r = S.R[t][0] * b0 + S.R[t][1] * b1 + S.R[t][2] * b2;
                B.rb[3 * j + t] = r;
                B.Xb[3 * j + t] = S.Xw[t] + r;
            }
        }
    }
}

// Lookup-grid range of a body-frame position u: [beg, end) in the list.  A
// particle farther from the centre than the reach (max |b| + cut-off, plus a
// margin far above the FP32 rounding of dc) has no bead in range and skips
// the lookup.
__device__ __forceinline__ void grid_range(const BodyShared &S, const float dc[3], int &beg, int &end)
{
    beg = end = 0;
    if (!(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2] < S.reach2_f)) return;
    int id[3];
    bool in = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float u = S.Rf[0][k] * dc[0] + S.Rf[1][k] * dc[1] + S.Rf[2][k] * dc[2];
        const float g = (u - S.glo) * S.ginv;
        in = in && g >= 0.0f && g < (float)S.gn;
        id[k] = (int)g;
    }
    if (in) {
        const int cell = id[0] + S.gn * (id[1] + S.gn * id[2]);
        if (S.gsm) {
            beg = S.gs16[cell];
            end = S.gs16[cell + 1];
        } else {
            beg = __ldg(S.gstart + cell);
            end = __ldg(S.gstart + cell + 1);
        }
    }
}

// A particle's pair-force sum f and torque sum tq (about the body centre)
// into the body's fixed-point totals, with the opposite sign.
__device__ __forceinline__ void sub_fixed6(long long acc[6], const float f[3], const float tq[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        acc[k] -= fx40_any(f[k]);
        acc[3 + k] -= fx40_any(tq[k]);
    }
}

// Mixed: force on one particle (cell c, offset o) from the beads it reaches.
// The particle's pair forces and their torques (R b_j) x f are summed in
// FP32 in bead order and enter the body's fixed-point totals once per
// particle: order-free over particles, like the per-pair sums of the FP64
// path, with six conversions per particle instead of six per pair.
__device__ __forceinline__ bool body_force_m(const ReplicaDev &rp, const BodyShared &S, const BeadSmem &B,
                                             const int c[3], const float o[3], uint32_t fid, float f[3],
                                             long long acc[6])
{
    float dc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dc[k] = (float)(c[k] - S.Ci[k]) + (o[k] - S.Cf[k]);
    min_image(rp, dc);
    int beg, end;
    grid_range(S, dc, beg, end);
    f[0] = f[1] = f[2] = 0.0f;
    float tq[3] = {0.0f, 0.0f, 0.0f};
    bool inside = false, touch = false;
    const int isb = (fid & F_B) ? 1 : 0;
    const unsigned short *gl = S.gsm ? S.gl16 : S.glist;
    int jn = beg < end ? gl[beg] : 0;
    for (int e = beg; e < end; ++e) {
        const int j = jn;
        if (e + 1 < end) jn = gl[e + 1];   // next index in flight during this pair
        const float rb[3] = {B.rbf[3 * j], B.rbf[3 * j + 1], B.rbf[3 * j + 2]};
        const float d[3] = {dc[0] - rb[0], dc[1] - rb[1], dc[2] - rb[2]};
        const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < S.rc2_f) {
            const float fr = wca_fr_m(B.epsf[2 * j + isb], S.sigma_f, r2);
            const float fk[3] = {fr * d[0], fr * d[1], fr * d[2]};
#pragma unroll
            for (int k = 0; k < 3; ++k) f[k] = f[k] + fk[k];
            tq[0] = tq[0] + (rb[1] * fk[2] - rb[2] * fk[1]);
            tq[1] = tq[1] + (rb[2] * fk[0] - rb[0] * fk[2]);
            tq[2] = tq[2] + (rb[0] * fk[1] - rb[1] * fk[0]);
            touch = true;
            inside = inside || B.cat[j] != 0;
        }
    }
    if (touch) sub_fixed6(acc, f, tq);
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = f[k] + rp.g_f[k];
    return inside;
}

// FP64: the same sums as the FP64 definition (ascending bead order).
__device__ __forceinline__ bool body_force_d(const ReplicaDev &rp, const BodyShared &S, const BeadSmem &B,
                                             const double x[3], uint32_t fid, double f[3], long long acc[6])
{
    double dcd[3] = {x[0] - S.Xw[0], x[1] - S.Xw[1], x[2] - S.Xw[2]};
    min_image(rp, dcd);
    const float dc[3] = {(float)dcd[0], (float)dcd[1], (float)dcd[2]};
    int beg, end;
    grid_range(S, dc, beg, end);
    f[0] = f[1] = f[2] = 0.0;
    bool inside = false;
    const int isb = (fid & F_B) ? 1 : 0;
    const unsigned short *gl = S.gsm ? S.gl16 : S.glist;
    int jn = beg < end ? gl[beg] : 0;
    for (int e = beg; e < end; ++e) {
        const int j = jn;
        if (e + 1 < end) jn = gl[e + 1];
        double d[3] = {x[0] - B.Xb[3 * j], x[1] - B.Xb[3 * j + 1], x[2] - B.Xb[3 * j + 2]};
        min_image(rp, d);
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < S.rc2) {
            const double eps = B.eps[2 * j + isb];
            const double ir2 = 1.0 / r2;
            const double s2 = S.sigma * S.sigma * ir2;
            const double s6 = s2 * s2 * s2;
            const double fr = 24.0 * eps * s6 * (2.0 * s6 - 1.0) * ir2;
            const double fk[3] = {fr * d[0], fr * d[1], fr * d[2]};
            const double *r = B.rb + 3 * j;
            const double cr[3] = {r[1] * fk[2] - r[2] * fk[1], r[2] * fk[0] - r[0] * fk[2], r[0] * fk[1] - r[1] * fk[0]};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                f[k] = f[k] + fk[k];
                acc[k] -= __double2ll_rn(fk[k] * 0x1p40);
                acc[3 + k] -= __double2ll_rn(cr[k] * 0x1p40);
            }
            inside = inside || B.cat[j] != 0;
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = f[k] + rp.g[k];
    return inside;
}

// Warp sums of the fixed-point partials into S.wpart[warp].
__device__ __forceinline__ void warp_partials6(BodyShared &S, const long long acc[6])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        long long x = acc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) S.wpart[wid][i] = (unsigned long long)x;
    }
}

// Mixed path, one sub-step of one near particle: drift by the half-step
// velocity, force, catalysis, then the kick to the next half step (or, at
// the last sub-step, to the full step).
__device__ __forceinline__ void substep_m(const ReplicaDev &rp, const BodyShared &S, const BeadSmem &B, BWorkM &w,
                                          long long acc[6], uint32_t step, int s, bool last)
{
#pragma unroll
    for (int t = 0; t < 3; ++t) w.o[t] = fmaf(rp.dt_f, w.v[t], w.o[t]);
    const int c[3] = {cw_get(w.cw, 0), cw_get(w.cw, 1), cw_get(w.cw, 2)};
    float f[3];
    const bool in = body_force_m(rp, S, B, c, w.o, w.fid, f, acc);
    w.fid = catalysis(rp, w.fid, in, step, s);
    const float h = last ? rp.hdt_f : rp.dt_f;
#pragma unroll
    for (int t = 0; t < 3; ++t) w.v[t] = fmaf(h, f[t], w.v[t]);
}

// Mixed path, first phase of one near particle's sub-step: true when the
// drifted particle may be in reach of a bead (the first test of grid_range),
// w unchanged; else the sub-step of substep_m completed here, with no bead in
// reach: body force g only, no catalytic range.
__device__ __forceinline__ bool substep_far_m(const ReplicaDev &rp, const BodyShared &S, BWorkM &w, uint32_t step,
                                              int s, bool last)
{
    float o[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) o[t] = fmaf(rp.dt_f, w.v[t], w.o[t]);
    const int c[3] = {cw_get(w.cw, 0), cw_get(w.cw, 1), cw_get(w.cw, 2)};
    float dc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) dc[k] = (float)(c[k] - S.Ci[k]) + (o[k] - S.Cf[k]);
    min_image(rp, dc);
    if (dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2] < S.reach2_f) return true;
    float f[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        w.o[t] = o[t];
        f[t] = f[t] + rp.g_f[t];
    }
    w.fid = catalysis(rp, w.fid, false, step, s);
    const float h = last ? rp.hdt_f : rp.dt_f;
#pragma unroll
    for (int t = 0; t < 3; ++t) w.v[t] = fmaf(h, f[t], w.v[t]);
    return false;
}

// Mixed path: write one particle back after the interval (and bin it for the
// collision of `step`).
__device__ __forceinline__ void finish_m(const Dev &d, const ReplicaDev &rp, int rbuf, int bbuf, int do_bin,
                                         const float sf[3], BWorkM &w, int slot)
{
    int c[3] = {cw_get(w.cw, 0), cw_get(w.cw, 1), cw_get(w.cw, 2)};
    renorm_m(rp, c, w.o);
    RecM rec;
    rec.cw = cw_make(c[0], c[1], c[2]);
    for (int t = 0; t < 3; ++t) { rec.o[t] = w.o[t]; rec.v[t] = w.v[t]; }
    rec.fid = do_bin ? (w.fid | F_PROP) : (w.fid & ~F_PROP);
    put_near(d, rbuf, bbuf, do_bin, do_bin ? bin_cell(d, rp.cell_off, cell_key_m(rp, c, w.o, sf)) : 0, slot, rec);
}

// gsm_bytes: room for the lookup grid at the start of the dynamic shared
// memory, ahead of the bead arrays (0: the grid is read from global memory).
template <bool MIXED>
__global__ void __launch_bounds__(MDB_NT, 2) k_md_body(Dev d, uint32_t step, int rbuf, int bbuf, int do_bin,
                                                       int gsm_bytes)
{
    step = resolve_step(d, step);   // STEP_DEVICE: the step of the control block
    using W = typename std::conditional<MIXED, BWorkM, BWorkD>::type;
    __shared__ BodyShared S;
    __shared__ ReplicaDev s_rp;
    extern __shared__ __align__(16) unsigned char bead_raw[];
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid == 0) s_rp = d.rep[r];
    __syncthreads();
    const ReplicaDev &rp = s_rp;
    if (rp.body < 0) return;   // uniform over the CTA
    const BodyDev &bd = d.body[rp.body];
    if (tid == 0) {
        for (int k = 0; k < 3; ++k) {
            S.X[k] = bd.X[k]; S.V[k] = bd.V[k]; S.l[k] = bd.l[k]; S.X0[k] = bd.X[k]; S.I[k] = bd.I[k];
        }
        for (int k = 0; k < 4; ++k) S.q[k] = bd.q[k];
        S.invM = 1.0 / bd.M;
        for (int s = 0; s < 5; ++s) {
            const int k = (s == 2) ? 2 : (s == 1 || s == 3) ? 1 : 0;
            S.ct[s] = 0.5 * ((s == 2) ? rp.dt : 0.5 * rp.dt) / bd.I[k];
        }
        S.M = bd.M; S.sigma = bd.sigma; S.rc2 = bd.rc2;
        S.sigma_f = bd.sigma_f; S.rc2_f = bd.rc2_f; S.glo = bd.glo; S.ginv = bd.ginv;
        S.gn = bd.gn; S.nb = bd.nb;
        S.reach2_f = (float)((bd.reach + 1e-3) * (bd.reach + 1e-3) * (1.0 + 1e-4));
        S.gstart = d.grid_start + bd.gstart_off;
        S.glist = d.grid_list + bd.glist_off;
        S.nn = min(d.near_count[r], rp.n_part);
        if (MIXED) body_frames_fast(rp, S);
        else body_frames(rp, S);
    }
    __syncthreads();
    const int nb = S.nb, nn = S.nn;
    const BeadSmem B = bead_layout<MIXED>(bead_raw + gsm_bytes, nb);
    {
        // the lookup grid into shared memory when it fits the room reserved
        const int ncell = S.gn * S.gn * S.gn + 1;
        const int nlist = __ldg(S.gstart + ncell - 1);
        const bool fits = gsm_bytes > 0 && 2 * (ncell + nlist) <= gsm_bytes;
        unsigned short *gs = reinterpret_cast<unsigned short *>(bead_raw);
        unsigned short *gl = gs + ncell;
        if (fits) {
            for (int i = tid; i < ncell; i += MDB_NT) gs[i] = (unsigned short)__ldg(S.gstart + i);
            for (int i = tid; i < nlist; i += MDB_NT) gl[i] = __ldg(S.glist + i);
        }
        if (tid == 0) {
            S.gsm = fits ? 1 : 0;
            S.gs16 = gs;
            S.gl16 = gl;
        }
    }
    for (int j = tid; j < nb; j += MDB_NT) {
        const int g = bd.bead_off + j;
        for (int t = 0; t < 3; ++t) B.b[3 * j + t] = d.bead_b[3 * g + t];
        if (MIXED) {
            B.epsf[2 * j] = d.bead_eps_f[2 * g];
            B.epsf[2 * j + 1] = d.bead_eps_f[2 * g + 1];
        } else {
            B.eps[2 * j] = d.bead_eps[2 * g];
            B.eps[2 * j + 1] = d.bead_eps[2 * g + 1];
        }
        B.cat[j] = d.bead_cat[g];
    }
    __syncthreads();
    bead_frames<MIXED>(S, B);
    __syncthreads();

    const int *list = d.near_list + rp.part_off;
    W *work = reinterpret_cast<W *>(d.md_work) + rp.part_off;
    long long acc[6];

    // forces at the start of the interval
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[i] = 0;
    for (int k = tid; k < nn; k += MDB_NT) {
        W w;
        const int slot = do_bin ? -1 : list[k];   // flat slot: the write-back target of a granular interval
        if constexpr (MIXED) {
            RecM rec = load_near<RecM>(d, rp, k);
            w.cw = rec.cw;
            w.fid = rec.fid;
            const int c[3] = {cw_get(rec.cw, 0), cw_get(rec.cw, 1), cw_get(rec.cw, 2)};
            float f[3];
            body_force_m(rp, S, B, c, rec.o, w.fid, f, acc);
            for (int t = 0; t < 3; ++t) { w.o[t] = rec.o[t]; w.v[t] = fmaf(rp.hdt_f, f[t], rec.v[t]); }
        } else {
            w.slot = slot;
            RecD rec = load_near<RecD>(d, rp, k);
            for (int t = 0; t < 3; ++t) { w.x[t] = rec.x[t]; w.v[t] = rec.v[t]; }
            w.fid = rec.fid;
            body_force_d(rp, S, B, w.x, w.fid, w.f, acc);
        }
        work[k] = w;
    }
    warp_partials6(S, acc);
    __syncthreads();
    if (tid == 0) body_totals(S);

    const double dt = rp.dt, hdt = rp.hdt;
    double sh[3];
    grid_shift(rp.seed, step, sh);
    const float sf[3] = {(float)sh[0], (float)sh[1], (float)sh[2]};
    for (int s = 0; s < rp.n_md; ++s) {
        if (tid == 0) {
            S.nreach = 0;
            if (MIXED) {
                // the centre now; the rotation beside the particles' first phase
                body_kick_drift_fast(S, dt, hdt);
                body_centre_frame_fast(rp, S);
            } else {
                body_kick_drift_rotate(S, dt, hdt);
                body_frames(rp, S);
            }
        }
        __syncthreads();
        if constexpr (!MIXED) {
            bead_frames<MIXED>(S, B);
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[i] = 0;
        if constexpr (MIXED) {
            // Two phases.  1: warps 1.. over the near particles; a particle
            // that no bead can reach (the test needs the body's centre only)
            // takes its whole sub-step here, one that may be in reach is
            // listed (one shared-memory atomic per warp); meanwhile warp 0
            // turns the body (thread 0) and recomputes the bead offsets.  2:
            // the threads take the listed particles densely, so the bead loops
            // run without the lanes of the particles out of reach.  The list
            // lives past the work records in md_work (64 bytes per solvent
            // slot for the mixed body path, the records take 32).
            const bool last = s + 1 == rp.n_md;
            const int lane = tid & 31, wid = tid >> 5;
            int *reach_list = reinterpret_cast<int *>(reinterpret_cast<BWorkM *>(d.md_work) + d.n_total) + rp.part_off;
            if (wid == 0) {
                // warp 0: the turn (thread 0), then the bead offsets of the new frame
                if (lane == 0) {
                    body_rotate_fast(S, dt);
                    body_rotation_frame_fast(S);
                }
                __syncwarp();
                bead_frames<MIXED>(S, B, lane, 32);
            }
            for (int kb = (wid - 1) * 32; wid > 0 && kb < nn; kb += (MDB_NW - 1) * 32) {
                const int k = kb + lane;
                bool reach = false;
                if (k < nn) {
                    BWorkM w = work[k];
                    reach = substep_far_m(rp, S, w, step, s, last);
                    if (!reach) {
                        if (!last) work[k] = w;
                        else finish_m(d, rp, rbuf, bbuf, do_bin, sf, w, do_bin ? -1 : list[k]);
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, reach);
                int base = 0;
                if (lane == 0 && m != 0u) base = atomicAdd(&S.nreach, __popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (reach) reach_list[base + __popc(m & ((1u << lane) - 1u))] = k;
            }
            __syncthreads();
            const int nr = S.nreach;
            int k_next = tid < nr ? reach_list[tid] : 0;   // each list entry is read one iteration ahead
            for (int i = tid; i < nr; i += MDB_NT) {
                const int k = k_next;
                if (i + MDB_NT < nr) k_next = reach_list[i + MDB_NT];
                BWorkM w = work[k];
                substep_m(rp, S, B, w, acc, step, s, last);
                if (!last) work[k] = w;
                else finish_m(d, rp, rbuf, bbuf, do_bin, sf, w, do_bin ? -1 : list[k]);
            }
        } else {
            for (int k = tid; k < nn; k += MDB_NT) {
                W w = work[k];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    if (s > 0) w.v[t] = fma(hdt, w.f[t], w.v[t]);
                    w.v[t] = fma(hdt, w.f[t], w.v[t]);
                    w.x[t] = fma(dt, w.v[t], w.x[t]);
                }
                const bool in = body_force_d(rp, S, B, w.x, w.fid, w.f, acc);
                w.fid = catalysis(rp, w.fid, in, step, s);
                work[k] = w;
            }
        }
        warp_partials6(S, acc);
        __syncthreads();
        if (tid == 0) {
            body_totals(S);
            if (MIXED) body_kick_fast(S, hdt);
            else body_kick(S, hdt);
        }
    }

    // FP64 path: last half kick, wrap, write back (and bin for the collision
    // of `step`); the mixed path did this in its last sub-step
    if constexpr (!MIXED) {
        for (int k = tid; k < nn; k += MDB_NT) {
            W w = work[k];
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
    if (tid == 0) {
        // body state, and its centre as the replica's near-list colloid
        BodyDev &bw = d.body[rp.body];
        const int g = rp.col_off;
        double dd = 0.0;
        for (int k = 0; k < 3; ++k) {
            bw.X[k] = S.X[k]; bw.V[k] = S.V[k]; bw.l[k] = S.l[k];
            const double e = S.X[k] - S.X0[k];
            dd = dd + e * e;
        }
        for (int k = 0; k < 4; ++k) bw.q[k] = S.q[k];
        const bool bad = !(dd <= rp.skin * rp.skin);
        if (MIXED) body_frames_fast(rp, S);
        else body_frames(rp, S);
        for (int k = 0; k < 3; ++k) {
            d.colX[3 * g + k] = S.X[k];
            d.colV[3 * g + k] = S.V[k];
            d.colXi[3 * g + k] = (int)floor(S.X[k]);
            d.colXf[3 * g + k] = S.Cf[k];
            d.colCi[3 * g + k] = S.Ci[k];
            d.colVf[3 * g + k] = (float)S.V[k];
        }
        if (bad) atomicAdd(&d.err[ERR_SKIN], 1u);
        d.near_count[r] = 0;
    }
}

size_t md_body_smem(bool mixed, int nb_max, int grid_bytes)
{
    return (size_t)grid_bytes + (mixed ? bead_smem_bytes<true>(nb_max) : bead_smem_bytes<false>(nb_max));
}

// Room for the lookup grid in shared memory: the largest body's grid (16-bit
// offsets and bead indices) when two CTAs still share an SM; else 0.
int md_body_grid_room(bool mixed, int nb_max, long long grid_entries_max)
{
    const long long bytes = ((2 * grid_entries_max + 15) / 16) * 16;
    const long long total = bytes + (long long)(mixed ? bead_smem_bytes<true>(nb_max) : bead_smem_bytes<false>(nb_max));
    return total <= 108 * 1024 ? (int)bytes : 0;
}

cudaError_t prepare_md_body(bool mixed, int nb_max, int grid_bytes)
{
    const int bytes = (int)md_body_smem(mixed, nb_max, grid_bytes);
    if (mixed) return cudaFuncSetAttribute(k_md_body<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return cudaFuncSetAttribute(k_md_body<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void launch_md_body(bool mixed, const Dev &d, int nb_max, int grid_bytes, uint32_t step, int rbuf, int bbuf,
                    int do_bin, cudaStream_t s)
{
    const size_t bytes = md_body_smem(mixed, nb_max, grid_bytes);
    if (mixed) k_md_body<true><<<d.n_rep, MDB_NT, bytes, s>>>(d, step, rbuf, bbuf, do_bin, grid_bytes);
    else k_md_body<false><<<d.n_rep, MDB_NT, bytes, s>>>(d, step, rbuf, bbuf, do_bin, grid_bytes);
}

}  // namespace rmpcd
