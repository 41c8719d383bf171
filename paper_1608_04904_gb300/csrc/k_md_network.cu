// k_md_network.cu -- near-field MD of one collision interval for the replicas
// whose colloid is a bead network held at fixed link lengths by iterative
// RATTLE: the Janus particle of §1.5 with the integrator §1.4 names for it
// (every bead a point mass; links between neighbouring beads).
//
// Per sub-step dt (§1.1 velocity Verlet), in the order of the FP64 definition:
//   beads:   v += dt/2 F/m, x += dt v; position stage of RATTLE;
//   solvent: v += dt/2 f, x += dt v;
//   forces:  WCA between every near particle and every bead it reaches; the
//            pair force on the particle puts its reaction on the bead
//            (64-bit fixed point, 2^-40, so the bead totals do not depend on
//            the order of the near list); catalytic tag / conversion (§1.5);
//   kicks:   beads v += dt/2 F/m, velocity stage of RATTLE; solvent
//            v += dt/2 f.
// RATTLE stages sweep the links until every link holds within tol: the
// position stage moves the two beads of a link along the link's vector at the
// sub-step's start until |x_a - x_b|^2 = d^2, the velocity stage removes their
// relative velocity along the current link vector.  The links arrive grouped
// by colour -- links of one colour share no bead --, so one thread per link
// corrects a whole colour at once and a colour-by-colour sweep gives exactly
// the sequential sweep over the links in that order.
//
// One CTA per replica with a network (FP64 path); the network's state, links
// and a candidate grid live in shared memory.  The candidate grid is rebuilt
// after every drift: cells of side h >= r_c + margin over the beads' bounding
// box, each cell holding a bit mask of the beads whose cut-off ball (plus the
// margin) touches it, so a particle visits, in ascending bead order, a set of
// beads that contains every bead within its cut-off -- the pair forces are
// added in the order of a scan over all beads.
#include <type_traits>

#include "rmpcd_kernels.cuh"

namespace rmpcd {

constexpr int MDN_NT = 512;
constexpr int MDN_G = 8;                     // candidate grid cells per axis (at most)
constexpr int MDN_CELLS = MDN_G * MDN_G * MDN_G;
constexpr double MDN_MARGIN = 0.01;          // added to the cut-off when marking cells

struct __align__(16) NWork {
    double x[3], v[3], f[3];
    uint32_t fid;
    int slot;
};
static_assert(sizeof(NWork) == 80, "network MD work record");

struct NetShared {
    double X0[3], X0w[3];      // centre of mass at the interval's start (unwrapped, wrapped)
    double lo[3], h;           // candidate grid: origin and cell side
    int gn[3];                 // cells per axis
    int nb, nl, ncol, words, nn, sweeps_bad;
    double sigma, rc2, tol;
    int max_sweeps;
};

// Dynamic shared layout of one network (nb beads, nl links, ncol colours).
struct NetSmem {
    double *x, *v, *xo, *F, *Xw, *m, *w, *eps;   // w = 1/m; eps: [2 nb] (A, B)
    long long *Fq;
    double *dl;
    int *la, *lb, *cs, *cat;
    unsigned *mask;                          // [MDN_CELLS * words]
};

// Bytes of the layout below: doubles x, v, xo, F, Xw (3 nb each), m, w (nb
// each), eps (2 nb), dl (nl); fixed-point sums (3 nb); ints la, lb (nl each), colour
// starts (ncol + 1), cat (nb); the candidate masks.
__host__ __device__ inline size_t net_smem_bytes(int nb, int nl, int ncol)
{
    const int words = (nb + 31) / 32;
    return sizeof(double) * (size_t)(19 * nb + nl) + sizeof(long long) * (size_t)(3 * nb) +
           sizeof(int) * (size_t)(2 * nl + ncol + 1 + nb) + sizeof(unsigned) * (size_t)MDN_CELLS * words;
}

__device__ NetSmem net_layout(unsigned char *raw, int nb, int nl, int ncol)
{
    NetSmem B;
    double *p = reinterpret_cast<double *>(raw);
    B.x = p; p += 3 * nb;
    B.v = p; p += 3 * nb;
    B.xo = p; p += 3 * nb;
    B.F = p; p += 3 * nb;
    B.Xw = p; p += 3 * nb;
    B.m = p; p += nb;
    B.w = p; p += nb;
    B.eps = p; p += 2 * nb;
    B.dl = p; p += nl;
    long long *q = reinterpret_cast<long long *>(p);
    B.Fq = q; q += 3 * nb;
    int *ip = reinterpret_cast<int *>(q);
    B.la = ip; ip += nl;
    B.lb = ip; ip += nl;
    B.cs = ip; ip += ncol + 1;
    B.cat = ip; ip += nb;
    B.mask = reinterpret_cast<unsigned *>(ip);
    return B;
}

// Wrapped position (X - L floor(X / L) per axis), as the colloid frames.
__device__ __forceinline__ void net_wrapped(const ReplicaDev &rp, const double *X, double *out)
{
    for (int k = 0; k < 3; ++k) {
        const double L = (double)rp.L[k];
        out[k] = X[k] - L * floor(X[k] / L);
    }
}

// Candidate grid over the beads' bounding box (thread 0 sizes it, the CTA
// fills it); positions relative to the centre of mass X0 of the interval.
__device__ void net_grid(NetShared &S, const NetSmem &B)
{
    const int tid = threadIdx.x;
    const double rcm = sqrt(S.rc2) + MDN_MARGIN;
    if (tid == 0) {
        double bmin[3] = {1e300, 1e300, 1e300}, bmax[3] = {-1e300, -1e300, -1e300};
        for (int j = 0; j < S.nb; ++j)
            for (int k = 0; k < 3; ++k) {
                const double r = B.x[3 * j + k] - S.X0[k];
                bmin[k] = fmin(bmin[k], r);
                bmax[k] = fmax(bmax[k], r);
            }
        double ext = 0.0;
        for (int k = 0; k < 3; ++k) {
            S.lo[k] = bmin[k] - rcm;
            ext = fmax(ext, bmax[k] - bmin[k] + 2.0 * rcm);
        }
        S.h = fmax(rcm, ext / (double)MDN_G) * (1.0 + 1e-9);
        for (int k = 0; k < 3; ++k)
            S.gn[k] = min(MDN_G, max(1, (int)ceil((bmax[k] - bmin[k] + 2.0 * rcm) / S.h)));
    }
    __syncthreads();
    const int ncell = S.gn[0] * S.gn[1] * S.gn[2];
    for (int i = tid; i < ncell * S.words; i += MDN_NT) B.mask[i] = 0u;
    __syncthreads();
    for (int j = tid; j < S.nb; j += MDN_NT) {
        int c0[3], c1[3];
        for (int k = 0; k < 3; ++k) {
            const double r = B.x[3 * j + k] - S.X0[k];
            c0[k] = max(0, (int)floor((r - rcm - S.lo[k]) / S.h));
            c1[k] = min(S.gn[k] - 1, (int)floor((r + rcm - S.lo[k]) / S.h));
        }
        for (int a = c0[0]; a <= c1[0]; ++a)
            for (int b = c0[1]; b <= c1[1]; ++b)
                for (int c = c0[2]; c <= c1[2]; ++c)
                    atomicOr(&B.mask[((c * S.gn[1] + b) * S.gn[0] + a) * S.words + (j >> 5)], 1u << (j & 31));
    }
    __syncthreads();
}

// Force on one near particle from the beads it can reach (ascending bead
// order, wrapped bead positions), reactions into the beads' fixed-point sums;
// returns 1 when it lies inside a catalytic bead's range.
__device__ int net_force(const ReplicaDev &rp, NetShared &S, const NetSmem &B, const double x[3], uint32_t fid,
                         double f[3])
{
    f[0] = f[1] = f[2] = 0.0;
    double rel[3] = {x[0] - S.X0w[0], x[1] - S.X0w[1], x[2] - S.X0w[2]};
    min_image(rp, rel);
    int cell[3];
    for (int k = 0; k < 3; ++k) {
        const double u = (rel[k] - S.lo[k]) / S.h;
        if (!(u >= 0.0) || u >= (double)S.gn[k]) return 0;   // beyond every bead's reach
        cell[k] = (int)u;
    }
    const unsigned *mk = B.mask + ((cell[2] * S.gn[1] + cell[1]) * S.gn[0] + cell[0]) * S.words;
    int inside = 0;
    for (int w = 0; w < S.words; ++w) {
        for (unsigned bits = mk[w]; bits; bits &= bits - 1u) {
            const int j = 32 * w + __ffs(bits) - 1;
            double d[3] = {x[0] - B.Xw[3 * j], x[1] - B.Xw[3 * j + 1], x[2] - B.Xw[3 * j + 2]};
            min_image(rp, d);
            const double eps = (fid & F_B) ? B.eps[2 * j + 1] : B.eps[2 * j];
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < S.rc2)) continue;
            const double ir2 = 1.0 / r2;
            const double s2 = S.sigma * S.sigma * ir2;
            const double s6 = s2 * s2 * s2;
            const double fr = 24.0 * eps * s6 * (2.0 * s6 - 1.0) * ir2;
            for (int k = 0; k < 3; ++k) {
                const double fk = fr * d[k];
                f[k] = f[k] + fk;
                atomicAdd(reinterpret_cast<unsigned long long *>(&B.Fq[3 * j + k]),
                          (unsigned long long)(-__double2ll_rn(fk * 0x1p40)));
            }
            if (B.cat[j]) inside = 1;
        }
    }
    return inside;
}

// Position stage: colour-parallel sweeps until every link holds.
__device__ void net_rattle_pos(NetShared &S, const NetSmem &B, double dt)
{
    const int tid = threadIdx.x;
    const double idt = 1.0 / dt;
    int sweep = 0;
    for (;;) {
        ++sweep;
        int moved = 0;
        for (int c = 0; c < S.ncol; ++c) {
            for (int k = B.cs[c] + tid; k < B.cs[c + 1]; k += MDN_NT) {
                const int a = B.la[k], b = B.lb[k];
                double s[3], ro[3];
                for (int t = 0; t < 3; ++t) {
                    s[t] = B.x[3 * a + t] - B.x[3 * b + t];
                    ro[t] = B.xo[3 * a + t] - B.xo[3 * b + t];
                }
                const double d2 = B.dl[k] * B.dl[k];
                const double diff = d2 - (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
                if (fabs(diff) <= 2.0 * S.tol * d2) continue;
                // inverse-mass form: one division per correction
                const double wa = B.w[a], wb = B.w[b];
                const double inv = wa + wb;
                const double sro = s[0] * ro[0] + s[1] * ro[1] + s[2] * ro[2];
                const double g = diff / (2.0 * sro * inv);
                const double ga = g * wa, gb = g * wb;
                for (int t = 0; t < 3; ++t) {
                    const double ca = ga * ro[t], cb = gb * ro[t];
                    B.x[3 * a + t] = B.x[3 * a + t] + ca;
                    B.x[3 * b + t] = B.x[3 * b + t] - cb;
                    B.v[3 * a + t] = B.v[3 * a + t] + ca * idt;
                    B.v[3 * b + t] = B.v[3 * b + t] - cb * idt;
                }
                moved = 1;
            }
            __syncthreads();
        }
        if (!__syncthreads_or(moved)) return;
        if (sweep >= S.max_sweeps) {
            if (tid == 0) S.sweeps_bad = 1;
            return;
        }
    }
}

// Velocity stage: colour-parallel sweeps until no link has a relative
// velocity along itself above tol d.
__device__ void net_rattle_vel(NetShared &S, const NetSmem &B)
{
    const int tid = threadIdx.x;
    int sweep = 0;
    for (;;) {
        ++sweep;
        int moved = 0;
        for (int c = 0; c < S.ncol; ++c) {
            for (int k = B.cs[c] + tid; k < B.cs[c + 1]; k += MDN_NT) {
                const int a = B.la[k], b = B.lb[k];
                double s[3], w[3];
                for (int t = 0; t < 3; ++t) {
                    s[t] = B.x[3 * a + t] - B.x[3 * b + t];
                    w[t] = B.v[3 * a + t] - B.v[3 * b + t];
                }
                const double rv = s[0] * w[0] + s[1] * w[1] + s[2] * w[2];
                if (fabs(rv) <= S.tol * B.dl[k]) continue;
                const double wa = B.w[a], wb = B.w[b];
                const double inv = wa + wb;
                const double ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
                const double kk = rv / (ss * inv);
                const double ka = kk * wa, kb = kk * wb;
                for (int t = 0; t < 3; ++t) {
                    B.v[3 * a + t] = B.v[3 * a + t] - ka * s[t];
                    B.v[3 * b + t] = B.v[3 * b + t] + kb * s[t];
                }
                moved = 1;
            }
            __syncthreads();
        }
        if (!__syncthreads_or(moved)) return;
        if (sweep >= S.max_sweeps) {
            if (tid == 0) S.sweeps_bad = 1;
            return;
        }
    }
}

// Centre of mass (sum in bead order) and reach (largest bead distance from it
// plus the cut-off), by one thread as the FP64 definition computes them.
__device__ void net_com_reach(const NetShared &S, const NetSmem &B, double X[3], double *reach)
{
    double s[3] = {0.0, 0.0, 0.0}, m = 0.0;
    for (int j = 0; j < S.nb; ++j) {
        m = m + B.m[j];
        for (int t = 0; t < 3; ++t) s[t] = s[t] + B.m[j] * B.x[3 * j + t];
    }
    for (int t = 0; t < 3; ++t) X[t] = s[t] / m;
    double rmax = 0.0;
    for (int j = 0; j < S.nb; ++j) {
        double e2 = 0.0;
        for (int t = 0; t < 3; ++t) { const double e = B.x[3 * j + t] - X[t]; e2 = e2 + e * e; }
        if (sqrt(e2) > rmax) rmax = sqrt(e2);
    }
    *reach = rmax + sqrt(S.rc2);
}

__global__ void __launch_bounds__(MDN_NT, 1) k_md_network(Dev d, uint32_t step, int rbuf, int bbuf, int do_bin)
{
    step = resolve_step(d, step);   // STEP_DEVICE: the step of the control block
    __shared__ NetShared S;
    __shared__ ReplicaDev s_rp;
    extern __shared__ __align__(16) unsigned char net_raw[];
    const int r = blockIdx.x;
    const int tid = threadIdx.x;
    if (tid == 0) s_rp = d.rep[r];
    __syncthreads();
    const ReplicaDev &rp = s_rp;
    if (rp.net < 0) return;   // uniform over the CTA
    const NetDev &nd = d.net[rp.net];
    if (tid == 0) {
        S.nb = nd.nb; S.nl = nd.nl; S.ncol = nd.ncol; S.words = (nd.nb + 31) / 32;
        S.sigma = nd.sigma; S.rc2 = nd.rc2; S.tol = nd.tol; S.max_sweeps = nd.max_sweeps;
        S.nn = min(d.near_count[r], rp.n_part);
        S.sweeps_bad = 0;
    }
    __syncthreads();
    const int nb = S.nb, nl = S.nl, ncol = S.ncol, nn = S.nn;
    const NetSmem B = net_layout(net_raw, nb, nl, ncol);
    for (int j = tid; j < nb; j += MDN_NT) {
        const int g = nd.bead_off + j;
        for (int t = 0; t < 3; ++t) { B.x[3 * j + t] = d.net_x[3 * g + t]; B.v[3 * j + t] = d.net_v[3 * g + t]; }
        B.m[j] = d.net_m[g];
        B.w[j] = 1.0 / B.m[j];   // the inverse masses of the RATTLE corrections
        B.eps[2 * j] = d.net_eps[2 * g];
        B.eps[2 * j + 1] = d.net_eps[2 * g + 1];
        B.cat[j] = d.net_cat[g];
    }
    for (int k = tid; k < nl; k += MDN_NT) {
        B.la[k] = d.net_la[nd.link_off + k];
        B.lb[k] = d.net_lb[nd.link_off + k];
        B.dl[k] = d.net_d[nd.link_off + k];
    }
    for (int c = tid; c <= ncol; c += MDN_NT) B.cs[c] = d.net_cs[nd.color_off + c];
    __syncthreads();
    if (tid == 0) {
        double reach;
        net_com_reach(S, B, S.X0, &reach);
        net_wrapped(rp, S.X0, S.X0w);
    }
    for (int j = tid; j < nb; j += MDN_NT) net_wrapped(rp, B.x + 3 * j, B.Xw + 3 * j);
    __syncthreads();
    net_grid(S, B);

    const int *list = d.near_list + rp.part_off;
    NWork *work = reinterpret_cast<NWork *>(d.md_work) + rp.part_off;
    const double dt = rp.dt, hdt = rp.hdt;

    // forces at the start of the interval
    for (int i = tid; i < 3 * nb; i += MDN_NT) B.Fq[i] = 0;
    __syncthreads();
    for (int k = tid; k < nn; k += MDN_NT) {
        NWork w;
        w.slot = do_bin ? -1 : list[k];   // flat slot: the write-back target of a granular interval
        const RecD rec = load_near<RecD>(d, rp, k);
        for (int t = 0; t < 3; ++t) { w.x[t] = rec.x[t]; w.v[t] = rec.v[t]; }
        w.fid = rec.fid;
        net_force(rp, S, B, w.x, w.fid, w.f);
        for (int t = 0; t < 3; ++t) w.f[t] = w.f[t] + rp.g[t];
        work[k] = w;
    }
    __syncthreads();
    for (int i = tid; i < 3 * nb; i += MDN_NT) B.F[i] = (double)B.Fq[i] * 0x1p-40;
    __syncthreads();

    for (int s = 0; s < rp.n_md; ++s) {
        // beads: half kick, drift, position stage
        for (int j = tid; j < nb; j += MDN_NT)
            for (int t = 0; t < 3; ++t) {
                B.v[3 * j + t] = fma(hdt, B.F[3 * j + t] / B.m[j], B.v[3 * j + t]);
                B.xo[3 * j + t] = B.x[3 * j + t];
                B.x[3 * j + t] = fma(dt, B.v[3 * j + t], B.x[3 * j + t]);
            }
        __syncthreads();
        net_rattle_pos(S, B, dt);
        for (int j = tid; j < nb; j += MDN_NT) net_wrapped(rp, B.x + 3 * j, B.Xw + 3 * j);
        for (int i = tid; i < 3 * nb; i += MDN_NT) B.Fq[i] = 0;
        __syncthreads();
        net_grid(S, B);
        // solvent: half kick, drift; new forces, catalytic conversion
        for (int k = tid; k < nn; k += MDN_NT) {
            NWork w = work[k];
            for (int t = 0; t < 3; ++t) {
                w.v[t] = fma(hdt, w.f[t], w.v[t]);
                w.x[t] = fma(dt, w.v[t], w.x[t]);
            }
            const int in = net_force(rp, S, B, w.x, w.fid, w.f);
            for (int t = 0; t < 3; ++t) w.f[t] = w.f[t] + rp.g[t];
            w.fid = catalysis(rp, w.fid, in != 0, step, s);
            work[k] = w;
        }
        __syncthreads();
        // beads: forces, half kick, velocity stage
        for (int j = tid; j < nb; j += MDN_NT)
            for (int t = 0; t < 3; ++t) {
                B.F[3 * j + t] = (double)B.Fq[3 * j + t] * 0x1p-40;
                B.v[3 * j + t] = fma(hdt, B.F[3 * j + t] / B.m[j], B.v[3 * j + t]);
            }
        __syncthreads();
        net_rattle_vel(S, B);
        // solvent: second half kick
        for (int k = tid; k < nn; k += MDN_NT) {
            NWork w = work[k];
            for (int t = 0; t < 3; ++t) w.v[t] = fma(hdt, w.f[t], w.v[t]);
            work[k] = w;
        }
    }
    __syncthreads();

    // wrap, write back (and bin for the collision of `step`)
    double sh[3];
    grid_shift(rp.seed, step, sh);
    for (int k = tid; k < nn; k += MDN_NT) {
        NWork w = work[k];
        wrap_periodic_d(rp, w.x);
        RecD rec;
        for (int t = 0; t < 3; ++t) { rec.x[t] = w.x[t]; rec.v[t] = w.v[t]; }
        rec.fid = do_bin ? (w.fid | F_PROP) : (w.fid & ~F_PROP);
        rec.u0 = 0u;
        rec.u1 = 0.0;
        put_near(d, rbuf, bbuf, do_bin, do_bin ? bin_cell(d, rp.cell_off, cell_key_d(rp, w.x, sh)) : 0, w.slot, rec);
    }
    // beads back to memory; centre and reach of the next interval's near test
    for (int j = tid; j < nb; j += MDN_NT) {
        const int g = nd.bead_off + j;
        for (int t = 0; t < 3; ++t) { d.net_x[3 * g + t] = B.x[3 * j + t]; d.net_v[3 * g + t] = B.v[3 * j + t]; }
    }
    if (tid == 0) {
        double X1[3], reach;
        net_com_reach(S, B, X1, &reach);
        double dd = 0.0;
        for (int t = 0; t < 3; ++t) { const double e = X1[t] - S.X0[t]; dd = dd + e * e; }
        if (!(dd <= rp.skin * rp.skin)) atomicAdd(&d.err[ERR_SKIN], 1u);
        if (S.sweeps_bad) atomicOr(&d.err[ERR_RATTLE], 1u);
        const int g = rp.col_off;
        for (int t = 0; t < 3; ++t) d.colX[3 * g + t] = X1[t];
        const_cast<double *>(d.colRc)[g] = reach;
        d.near_count[r] = 0;
    }
}

size_t md_network_smem(int nb, int nl, int ncol) { return net_smem_bytes(nb, nl, ncol); }

cudaError_t prepare_md_network(size_t smem)
{
    return cudaFuncSetAttribute(k_md_network, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

void launch_md_network(const Dev &d, size_t smem, uint32_t step, int rbuf, int bbuf, int do_bin, cudaStream_t s)
{
    if (d.n_rep <= 0) return;
    k_md_network<<<d.n_rep, MDN_NT, smem, s>>>(d, step, rbuf, bbuf, do_bin);
}

}  // namespace rmpcd
