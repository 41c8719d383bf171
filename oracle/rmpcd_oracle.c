/*
 * rmpcd_oracle.c -- plain, slow, FP64 CPU oracle of one MPCD collision interval.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py load this file's library.  The
 * product path (paper_1608_04904_gb300) never links, imports or calls it, and
 * the two share no code: this file has its own Philox, its own geometry and
 * its own arithmetic.
 *
 * What it computes follows de Buyl, Huang & Deprez, "RMPCDMD: Simulations of
 * colloids with coarse-grained hydrodynamics, chemical reactions and external
 * fields" (arXiv:1608.04904):
 *   - §1.1 (Introduction): solvent and colloids move by Newton's equations,
 *     integrated by velocity Verlet; no solvent-solvent potential.
 *   - §1.4 (Algorithms): original MPCD (SRD) collision rule, Anderson
 *     thermostat (MPC-AT), random grid shift every collision, constant body
 *     acceleration on the solvent, bounce-back walls with virtual particles,
 *     cut-off purely repulsive 12-6 LJ (WCA) potential, Verlet/cell lists
 *     sharing the MPCD sort, exact RATTLE for the dimer, counter-based RNG, and
 *     the cell-frame temperature estimator.
 *   - §1.5 (Applications): catalytic A->B conversion at one sphere of the dimer,
 *     and the composite Janus particle, whose bead network moves here as one
 *     rigid body (reading; see the rigid-body section), and, as the paper has
 *     it, as beads held by iterative RATTLE (the last section).
 *   - §1.1 / Appendix A: bulk RMPCD reaction B->A at a given rate.
 * Where the paper is silent this file takes a reading of it (the order of the
 * steps in an interval, the rotation sense, the reaction rule, the near/far
 * bound, ...); each function below states the reading it relies on.
 *
 * Conventions: cell side a = 1, solvent mass m = 1.  Everything is FP64.  The
 * file must be compiled with -ffp-contract=off so that every product and sum
 * is rounded where it is written; fused multiply-adds appear only as explicit
 * fma() calls.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Threads.  Loops whose iterations are independent (per particle or per    */
/* cell) may run on several OpenMP threads; colloid and body force totals    */
/* are exact 64-bit integer sums, so their reduction order does not matter.  */
/* Results are bit-identical for every thread count.  Default: 1 thread.     */
/* ------------------------------------------------------------------------ */
static int g_threads = 1;

int orc_set_threads(int n)
{
#ifdef _OPENMP
    g_threads = n > 0 ? n : omp_get_num_procs();
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

int orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Parameters of one system (one replica).                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t L[3];        /* box sides in cells                                  */
    int32_t walls;       /* 1: stick walls at z = 0 and z = L[2]               */
    int32_t rho_wall;    /* virtual-particle fill target per wall cell          */
    int32_t n_md;        /* velocity-Verlet sub-steps per collision interval    */
    int32_t n_slabs;     /* number of MPC-AT thermostat slabs (<= 4)            */
    int32_t bulk_mode;   /* 0: off, 1: one B->A per cell with p = 1-exp(-k N_B tau) */
    double kT;           /* solvent temperature (units of m = 1)                */
    double alpha;        /* SRD rotation angle, radians                         */
    double tau;          /* collision interval                                  */
    double g[3];         /* constant body acceleration on the solvent           */
    double bulk_rate;    /* k of the bulk B -> A reaction                       */
    double cat_prob;     /* A -> B probability on leaving a catalytic colloid   */
    double skin;         /* bound on colloid displacement per interval          */
    double slab_x0[4], slab_x1[4], slab_kT[4];
    double cc_eps, cc_sigma, cc_rc;  /* colloid-colloid LJ (cc_rc = 0: none)    */
    uint64_t seed;
} orc_params;

enum { P_SHIFT = 1, P_ROT = 2, P_REACT = 3, P_THERMO = 4, P_VIRT = 5, P_CAT = 6 };
enum { F_B = 1, F_TAG = 2 };  /* solvent flag bits: species B, catalytic tag */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  §1.4 names a         */
/* counter-based generator (Threefry-2x64 there); Philox4x32-10 is the same  */
/* family, one generator keyed by the seed and addressed by a counter.       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;   /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t index, uint32_t step, uint32_t purpose,
                 uint32_t sub, uint32_t out[4])
{
    uint32_t ctr[4] = {index, step, purpose, sub};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* 24-bit uniform in [0, 1): exactly representable in FP32 and FP64. */
static double u24(uint32_t b) { return (double)(b >> 8) * 0x1p-24; }

/* Box-Muller pair from two words: u1 in (0, 1], u2 in [0, 1). */
static void box_muller(uint32_t b0, uint32_t b1, double *g0, double *g1)
{
    double u1 = (double)((b0 >> 8) + 1u) * 0x1p-24;
    double u2 = (double)(b1 >> 8) * 0x1p-24;
    double r = sqrt(-2.0 * log(u1));
    double ph = 6.283185307179586 * u2;
    *g0 = r * cos(ph);
    *g1 = r * sin(ph);
}

/* ------------------------------------------------------------------------ */
/* Random grid shift (§1.4: the grid is shifted at random before every       */
/* collision).  Reading: s uniform in [0, a)^3, fresh for every collision.   */
/* ------------------------------------------------------------------------ */
void orc_grid_shift(uint64_t seed, uint32_t step, double s[3])
{
    uint32_t w[4];
    draw(seed, 0u, step, P_SHIFT, 0u, w);
    s[0] = u24(w[0]); s[1] = u24(w[1]); s[2] = u24(w[2]);
}

/* ------------------------------------------------------------------------ */
/* Random rotation axis of one cell: a point uniform on the unit sphere by   */
/* Marsaglia's (1972) method.  The acceptance test A^2 + B^2 < 2^48 is done  */
/* in integers so that it is exact; a and b are odd multiples of 2^-24.      */
/* ------------------------------------------------------------------------ */
void orc_rotation_axis(uint64_t seed, uint32_t step, uint32_t cell, double n[3])
{
    for (uint32_t attempt = 0; attempt < 16u; ++attempt) {
        uint32_t w[4];
        draw(seed, cell, step, P_ROT, attempt, w);
        for (int pair = 0; pair < 2; ++pair) {
            int64_t A = 2 * (int64_t)(w[2 * pair] >> 8) + 1 - (1 << 24);
            int64_t B = 2 * (int64_t)(w[2 * pair + 1] >> 8) + 1 - (1 << 24);
            int64_t S = A * A + B * B;
            if (S < ((int64_t)1 << 48)) {
                double a = (double)A * 0x1p-24;
                double b = (double)B * 0x1p-24;
                double s = (double)S * 0x1p-48;
                double q = sqrt(1.0 - s);
                n[0] = 2.0 * a * q;
                n[1] = 2.0 * b * q;
                n[2] = 1.0 - 2.0 * s;
                return;
            }
        }
    }
    n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;   /* reached with probability < 1e-21 */
}

/* ------------------------------------------------------------------------ */
/* Cells.  Periodic axes have L cells; with walls the z axis has L[2] + 1    */
/* layers because the shifted grid sticks out of [0, L[2]] on both sides.    */
/* ------------------------------------------------------------------------ */
int64_t orc_n_cells(const orc_params *p)
{
    return (int64_t)p->L[0] * p->L[1] * (p->L[2] + (p->walls ? 1 : 0));
}

/* Cell of every particle on the grid shifted by s (§1.4, grid shift; the
 * sort that follows is the one of the `particle_system` module, Table 1).
 * Key = cx + Lx * (cy + Ly * cz), x fastest. */
void orc_cell_keys(const orc_params *p, int64_t n, const double *x, const double s[3], int32_t *key)
{
    int64_t nz = p->L[2] + (p->walls ? 1 : 0);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        for (int d = 0; d < 3; ++d) {
            int64_t k = (int64_t)floor(x[3 * i + d] - s[d]);
            if (d == 2 && p->walls) {
                k += 1;
                if (k < 0) k = 0;
                if (k > nz - 1) k = nz - 1;
            } else {
                k %= p->L[d];
                if (k < 0) k += p->L[d];
            }
            c[d] = k;
        }
        key[i] = (int32_t)(c[0] + (int64_t)p->L[0] * (c[1] + (int64_t)p->L[1] * c[2]));
    }
}

/* Counting sort by key, particles of one cell in increasing id order:
 * perm[j] = old index of the particle that takes slot j.  The paper sorts the
 * particles by cell and leaves the order within a cell open; ordering by the
 * particle's id makes it canonical whatever order the particles arrive in.
 * Ids are unique within a system (NULL: the old index serves as the id).
 * count/start are per cell. */
void orc_counting_sort(int64_t n, const int32_t *key, const uint32_t *id, int64_t n_cells,
                       int64_t *perm, int64_t *count, int64_t *start)
{
    for (int64_t c = 0; c < n_cells; ++c) count[c] = 0;
    for (int64_t i = 0; i < n; ++i) count[key[i]]++;
    int64_t acc = 0;
    for (int64_t c = 0; c < n_cells; ++c) { start[c] = acc; acc += count[c]; }
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cells > 0 ? n_cells : 1));
    for (int64_t c = 0; c < n_cells; ++c) fill[c] = start[c];
    for (int64_t i = 0; i < n; ++i) perm[fill[key[i]]++] = i;
    free(fill);
    /* within each cell: insertion sort by id (cells hold a few particles) */
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t *p = perm + start[c];
        for (int64_t a = 1; a < count[c]; ++a) {
            int64_t q = p[a];
            uint64_t kq = id ? id[q] : (uint64_t)q;
            int64_t b = a - 1;
            while (b >= 0 && (id ? (uint64_t)id[p[b]] : (uint64_t)p[b]) > kq) { p[b + 1] = p[b]; --b; }
            p[b + 1] = q;
        }
    }
}

/* out[j] = in[perm[j]] for records of `width` bytes. */
void orc_gather(int64_t n, const int64_t *perm, const void *in, void *out, int64_t width)
{
    const char *src = (const char *)in;
    char *dst = (char *)out;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t j = 0; j < n; ++j)
        memcpy(dst + j * width, src + perm[j] * width, (size_t)width);
}

/* ------------------------------------------------------------------------ */
/* Collision step (§1.4).  Per cell of the shifted grid, in sorted order:    */
/*   SRD:  v_i <- v_cm + R(alpha, n)(v_i - v_cm)  (Malevanets & Kapral 1999) */
/*   MPC-AT in thermostat slabs: v_i <- v_cm + xi_i - <xi>, xi ~ N(0, kT_s)  */
/*   walls: wall cells with 0 < N < rho_wall get rho_wall - N virtual        */
/*   particles at rest on average, whose summed momentum is N(0, n_v kT).    */
/*   A wall cell holding a single particle collides too: with its virtual    */
/*   partners v_cm differs from v, so the rotation pulls it toward rest      */
/*   (the no-slip condition of Lamura et al. 2001).                          */
/* Other cells with fewer than two particles are left unchanged (a lone     */
/* particle is its own v_cm).  v is in sorted order; count/start come from   */
/* orc_counting_sort.                                                        */
/* ------------------------------------------------------------------------ */
static int slab_of(const orc_params *p, int64_t cx)
{
    for (int k = 0; k < p->n_slabs; ++k)
        if ((double)cx >= p->slab_x0[k] && (double)cx < p->slab_x1[k]) return k;
    return -1;
}

void orc_collide(const orc_params *p, uint32_t step, int64_t n_cells,
                 const int64_t *count, const int64_t *start, double *v)
{
    double ca = cos(p->alpha), sa = sin(p->alpha), omc = 1.0 - ca;
    int64_t nz = p->L[2] + (p->walls ? 1 : 0);
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 256)
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t N = count[c];
        int64_t cx = c % p->L[0];
        int64_t cz = c / ((int64_t)p->L[0] * p->L[1]);
        int wall_cell = p->walls && (cz == 0 || cz == nz - 1);
        int virt = wall_cell && N > 0 && N < p->rho_wall;
        if (N < 2 && !virt) continue;
        double *vc = v + 3 * start[c];
        double sum[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) sum[d] = sum[d] + vc[3 * i + d];
        double vcm[3];
        if (virt) {
            /* virtual particles fill the wall cell up to rho_wall (Lamura et al. 2001) */
            int64_t nv = p->rho_wall - N;
            uint32_t w[4];
            draw(p->seed, (uint32_t)c, step, P_VIRT, 0u, w);
            double gg[4];
            box_muller(w[0], w[1], &gg[0], &gg[1]);
            box_muller(w[2], w[3], &gg[2], &gg[3]);
            double sd = sqrt((double)nv * p->kT);
            for (int d = 0; d < 3; ++d) vcm[d] = (sum[d] + sd * gg[d]) / (double)(N + nv);
        } else {
            for (int d = 0; d < 3; ++d) vcm[d] = sum[d] / (double)N;
        }
        int slab = slab_of(p, cx);
        if (slab >= 0) {
            /* MPC-AT (Noguchi et al. 2007): fresh relative velocities at kT_slab */
            double sd = sqrt(p->slab_kT[slab]);
            double *xi = (double *)malloc(sizeof(double) * 3 * (size_t)N);
            double xs[3] = {0.0, 0.0, 0.0};
            for (int64_t i = 0; i < N; ++i) {
                uint32_t w[4];
                draw(p->seed, (uint32_t)c, step, P_THERMO, (uint32_t)i, w);
                double gg[4];
                box_muller(w[0], w[1], &gg[0], &gg[1]);
                box_muller(w[2], w[3], &gg[2], &gg[3]);
                for (int d = 0; d < 3; ++d) {
                    xi[3 * i + d] = sd * gg[d];
                    xs[d] = xs[d] + xi[3 * i + d];
                }
            }
            for (int d = 0; d < 3; ++d) xs[d] = xs[d] / (double)N;
            for (int64_t i = 0; i < N; ++i)
                for (int d = 0; d < 3; ++d) vc[3 * i + d] = vcm[d] + (xi[3 * i + d] - xs[d]);
            free(xi);
            continue;
        }
        double nh[3];
        orc_rotation_axis(p->seed, step, (uint32_t)c, nh);
        for (int64_t i = 0; i < N; ++i) {
            double u0 = vc[3 * i + 0] - vcm[0];
            double u1 = vc[3 * i + 1] - vcm[1];
            double u2 = vc[3 * i + 2] - vcm[2];
            /* Rodrigues: R u = u cos a + (n x u) sin a + n (n.u)(1 - cos a) */
            double dot = nh[0] * u0 + nh[1] * u1 + nh[2] * u2;
            double x0 = nh[1] * u2 - nh[2] * u1;
            double x1 = nh[2] * u0 - nh[0] * u2;
            double x2 = nh[0] * u1 - nh[1] * u0;
            double od = omc * dot;
            vc[3 * i + 0] = vcm[0] + (ca * u0 + sa * x0 + od * nh[0]);
            vc[3 * i + 1] = vcm[1] + (ca * u1 + sa * x1 + od * nh[1]);
            vc[3 * i + 2] = vcm[2] + (ca * u2 + sa * x2 + od * nh[2]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Bulk RMPCD reaction B -> A (§1.1, Rohlf et al. 2008; rate in Appendix A). */
/* Reading: per cell, with probability p = 1 - exp(-k N_B tau) one B, chosen */
/* uniformly among the cell's B particles in sorted order, becomes A.        */
/* The acceptance test is b0 < p * 2^32 and the choice floor(b1 * N_B / 2^32).*/
/* ------------------------------------------------------------------------ */
void orc_bulk_react(const orc_params *p, uint32_t step, int64_t n_cells,
                    const int64_t *count, const int64_t *start, uint8_t *flags)
{
    if (p->bulk_mode == 0) return;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 256)
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t N = count[c];
        uint8_t *fc = flags + start[c];
        int64_t nb = 0;
        for (int64_t i = 0; i < N; ++i) nb += (fc[i] & F_B) ? 1 : 0;
        if (nb == 0) continue;
        double prob = 1.0 - exp(-p->bulk_rate * (double)nb * p->tau);
        uint32_t w[4];
        draw(p->seed, (uint32_t)c, step, P_REACT, 0u, w);
        if (!((double)w[0] < prob * 4294967296.0)) continue;
        int64_t pick = (int64_t)(((uint64_t)w[1] * (uint64_t)nb) >> 32);
        for (int64_t i = 0, seen = 0; i < N; ++i) {
            if (fc[i] & F_B) {
                if (seen == pick) { fc[i] = (uint8_t)(fc[i] & ~(F_B | F_TAG)); break; }
                ++seen;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Free flight over one interval (§1.1 streaming; §1.4 body force and        */
/* bounce-back walls).  With walls (g_z must be 0) a particle that reaches   */
/* a wall reverses its whole velocity there and flies on for the rest of tau.*/
/* ------------------------------------------------------------------------ */
static void fly(const orc_params *p, double *x, double *v, double t)
{
    int hasg = (p->g[0] != 0.0 || p->g[1] != 0.0 || p->g[2] != 0.0);
    for (int d = 0; d < 3; ++d) {
        x[d] = fma(v[d], t, x[d]);
        if (hasg) {
            x[d] = x[d] + 0.5 * p->g[d] * t * t;
            v[d] = v[d] + p->g[d] * t;
        }
    }
}

static void wrap_periodic(const orc_params *p, double *x)
{
    for (int d = 0; d < 3; ++d) {
        if (d == 2 && p->walls) continue;
        double L = (double)p->L[d];
        if (x[d] >= L) x[d] = x[d] - L;
        else if (x[d] < 0.0) { x[d] = x[d] + L; if (x[d] >= L) x[d] = 0.0; }
    }
}

static void flight_one(const orc_params *p, double *x, double *v)
{
    if (!p->walls) { fly(p, x, v, p->tau); wrap_periodic(p, x); return; }
    double Lz = (double)p->L[2];
    double zend = fma(v[2], p->tau, x[2]);
    double th = -1.0;
    double wall = 0.0;
    if (zend < 0.0) { th = -x[2] / v[2]; wall = 0.0; }
    else if (zend > Lz) { th = (Lz - x[2]) / v[2]; wall = Lz; }
    if (th < 0.0) { fly(p, x, v, p->tau); }
    else {
        fly(p, x, v, th);
        x[2] = wall;
        for (int d = 0; d < 3; ++d) v[d] = -v[d];
        fly(p, x, v, p->tau - th);
        if (x[2] < 0.0) x[2] = 0.0;
        if (x[2] > Lz) x[2] = Lz;
    }
    wrap_periodic(p, x);
}

void orc_flight(const orc_params *p, int64_t n, double *x, double *v, const uint8_t *near)
{
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (near && near[i]) continue;
        flight_one(p, x + 3 * i, v + 3 * i);
    }
}

/* ------------------------------------------------------------------------ */
/* WCA pair force (§1.4): V(r) = 4 eps ((s/r)^12 - (s/r)^6 + 1/4), r < 2^(1/6)s.*/
/* Returns 1 and the force on the particle at +d (d = x_solvent - X_colloid) */
/* when r^2 < rc2, else 0.                                                   */
/* ------------------------------------------------------------------------ */
int orc_wca_force(const double d[3], double sigma, double eps, double rc2, double f[3], double *energy)
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < rc2)) { f[0] = f[1] = f[2] = 0.0; if (energy) *energy = 0.0; return 0; }
    double ir2 = 1.0 / r2;
    double s2 = sigma * sigma * ir2;
    double s6 = s2 * s2 * s2;
    double fr = 24.0 * eps * s6 * (2.0 * s6 - 1.0) * ir2;
    f[0] = fr * d[0]; f[1] = fr * d[1]; f[2] = fr * d[2];
    if (energy) *energy = 4.0 * eps * (s6 * (s6 - 1.0) + 0.25);
    return 1;
}

/* Truncated (not shifted in force) 12-6 LJ between colloids; energy shifted
 * to zero at cc_rc.  Reading for colloid-colloid interactions with a cut-off
 * beyond the WCA minimum. */
static int lj_cc_force(const double d[3], double sigma, double eps, double rc, double f[3])
{
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < rc * rc)) return 0;
    double ir2 = 1.0 / r2;
    double s2 = sigma * sigma * ir2;
    double s6 = s2 * s2 * s2;
    double fr = 24.0 * eps * s6 * (2.0 * s6 - 1.0) * ir2;
    f[0] = fr * d[0]; f[1] = fr * d[1]; f[2] = fr * d[2];
    return 1;
}

double orc_wca_rc2(double sigma) { return sigma * sigma * cbrt(2.0); }

/* Minimum image of a separation along the periodic axes (module `common`,
 * Table 1).  |d| < 1.5 L is assumed. */
static void min_image(const orc_params *p, double d[3])
{
    for (int k = 0; k < 3; ++k) {
        if (k == 2 && p->walls) continue;
        double L = (double)p->L[k];
        if (d[k] > 0.5 * L) d[k] = d[k] - L;
        else if (d[k] < -0.5 * L) d[k] = d[k] + L;
    }
}

static void wrapped(const orc_params *p, const double *X, double out[3])
{
    for (int k = 0; k < 3; ++k) {
        double L = (double)p->L[k];
        out[k] = X[k] - L * floor(X[k] / L);
    }
}

/* Colloid forces are summed in 64-bit fixed point with 2^-40 resolution, so
 * that the sum does not depend on the order of the terms (reading). */
#define FX_SCALE 0x1p40
#define FX_INV 0x1p-40

typedef struct {
    int nc;
    double *X, *V;            /* unwrapped colloid positions, velocities [nc*3] */
    const double *M, *sig, *epsA, *epsB, *rc2;
    const int32_t *cat;
    int n_bonds;
    const int32_t *ba, *bb;
    const double *bd;
} colloids_t;

/* Force on one solvent particle from all colloids; adds -f into Fq. */
static void solvent_force(const orc_params *p, const colloids_t *cs, const double Xw[][3],
                          const double *x, uint8_t fl, double f[3], int64_t *Fq)
{
    f[0] = f[1] = f[2] = 0.0;
    for (int j = 0; j < cs->nc; ++j) {
        double d[3] = {x[0] - Xw[j][0], x[1] - Xw[j][1], x[2] - Xw[j][2]};
        min_image(p, d);
        double fj[3];
        double eps = (fl & F_B) ? cs->epsB[j] : cs->epsA[j];
        if (orc_wca_force(d, cs->sig[j], eps, cs->rc2[j], fj, NULL)) {
            for (int k = 0; k < 3; ++k) {
                f[k] = f[k] + fj[k];
                Fq[3 * j + k] -= llrint(fj[k] * FX_SCALE);
            }
        }
    }
}

static int bonded(const colloids_t *cs, int a, int b)
{
    for (int k = 0; k < cs->n_bonds; ++k)
        if ((cs->ba[k] == a && cs->bb[k] == b) || (cs->ba[k] == b && cs->bb[k] == a)) return 1;
    return 0;
}

static void colloid_colloid(const orc_params *p, const colloids_t *cs, const double Xw[][3], int64_t *Fq)
{
    if (!(p->cc_rc > 0.0)) return;
    for (int a = 0; a < cs->nc; ++a)
        for (int b = a + 1; b < cs->nc; ++b) {
            if (bonded(cs, a, b)) continue;
            double d[3] = {Xw[a][0] - Xw[b][0], Xw[a][1] - Xw[b][1], Xw[a][2] - Xw[b][2]};
            min_image(p, d);
            double f[3];
            if (lj_cc_force(d, p->cc_sigma, p->cc_eps, p->cc_rc, f))
                for (int k = 0; k < 3; ++k) {
                    int64_t q = llrint(f[k] * FX_SCALE);
                    Fq[3 * a + k] += q;
                    Fq[3 * b + k] -= q;
                }
        }
}

/* RATTLE (Andersen 1983), exact for one bond between two bodies (§1.4 solves
 * the dimer motor's single bond exactly).  Position stage: move along the old bond
 * vector so that |X_a - X_b| = d; velocity stage: remove the relative
 * velocity along the bond. */
static void rattle_pos(colloids_t *cs, const double (*Xold)[3], double dt)
{
    for (int k = 0; k < cs->n_bonds; ++k) {
        int a = cs->ba[k], b = cs->bb[k];
        double d = cs->bd[k];
        double ro[3], rn[3];
        for (int t = 0; t < 3; ++t) {
            ro[t] = Xold[a][t] - Xold[b][t];
            rn[t] = cs->X[3 * a + t] - cs->X[3 * b + t];
        }
        double inv = 1.0 / cs->M[a] + 1.0 / cs->M[b];
        double oo = ro[0] * ro[0] + ro[1] * ro[1] + ro[2] * ro[2];
        double on = rn[0] * ro[0] + rn[1] * ro[1] + rn[2] * ro[2];
        double nn = rn[0] * rn[0] + rn[1] * rn[1] + rn[2] * rn[2];
        double qa = inv * inv * oo;
        double qb = 2.0 * inv * on;
        double qc = nn - d * d;
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc < 0.0) disc = 0.0;
        double q = -0.5 * (qb + copysign(sqrt(disc), qb));
        double gmul = qc / q;   /* root of smaller magnitude */
        for (int t = 0; t < 3; ++t) {
            double ca = gmul * ro[t] / cs->M[a];
            double cb = gmul * ro[t] / cs->M[b];
            cs->X[3 * a + t] = cs->X[3 * a + t] + ca;
            cs->X[3 * b + t] = cs->X[3 * b + t] - cb;
            cs->V[3 * a + t] = cs->V[3 * a + t] + ca / dt;
            cs->V[3 * b + t] = cs->V[3 * b + t] - cb / dt;
        }
    }
}

static void rattle_vel(colloids_t *cs)
{
    for (int k = 0; k < cs->n_bonds; ++k) {
        int a = cs->ba[k], b = cs->bb[k];
        double r[3], dv[3];
        for (int t = 0; t < 3; ++t) {
            r[t] = cs->X[3 * a + t] - cs->X[3 * b + t];
            dv[t] = cs->V[3 * a + t] - cs->V[3 * b + t];
        }
        double inv = 1.0 / cs->M[a] + 1.0 / cs->M[b];
        double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        double rv = dv[0] * r[0] + dv[1] * r[1] + dv[2] * r[2];
        double kk = rv / (rr * inv);
        for (int t = 0; t < 3; ++t) {
            cs->V[3 * a + t] = cs->V[3 * a + t] - kk * r[t] / cs->M[a];
            cs->V[3 * b + t] = cs->V[3 * b + t] + kk * r[t] / cs->M[b];
        }
    }
}

static int inside_catalytic(const orc_params *p, const colloids_t *cs, const double Xw[][3], const double *x)
{
    for (int j = 0; j < cs->nc; ++j) {
        if (!cs->cat[j]) continue;
        double d[3] = {x[0] - Xw[j][0], x[1] - Xw[j][1], x[2] - Xw[j][2]};
        min_image(p, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (r2 < cs->rc2[j]) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One collision interval of solvent + colloid motion (§1.1, §1.4).          */
/* Solvent particles that may come within a colloid's cut-off during the     */
/* interval ("near": start distance < r_c + |v| tau + |g| tau^2 / 2 + skin)  */
/* are integrated together with the colloids by n_md velocity-Verlet         */
/* sub-steps of dt = tau / n_md; the others feel no force all interval and   */
/* fly freely once over tau (the same motion, done once).  all_substep = 1   */
/* integrates every particle by sub-steps instead.  A tagged A particle that */
/* leaves every catalytic colloid's range becomes B with probability         */
/* cat_prob (§1.5).  Returns 0, or 1 if a colloid moved further than skin.   */
/* near_out (may be NULL) receives the near flag of every particle.          */
/* ------------------------------------------------------------------------ */
int orc_interval(const orc_params *p, uint32_t step, int64_t n, double *x, double *v,
                 uint8_t *flags, const uint32_t *id,
                 int nc, double *X, double *V, const double *M, const double *sig,
                 const double *epsA, const double *epsB, const int32_t *cat,
                 int n_bonds, const int32_t *ba, const int32_t *bb, const double *bd,
                 int all_substep, uint8_t *near_out)
{
    if (nc == 0) {
        orc_flight(p, n, x, v, NULL);
        if (near_out) memset(near_out, 0, (size_t)n);
        return 0;
    }
    double *rc2 = (double *)malloc(sizeof(double) * (size_t)nc);
    for (int j = 0; j < nc; ++j) rc2[j] = orc_wca_rc2(sig[j]);
    colloids_t cs = {nc, X, V, M, sig, epsA, epsB, rc2, cat, n_bonds, ba, bb, bd};
    double (*Xw)[3] = malloc(sizeof(double[3]) * (size_t)nc);
    double (*X0)[3] = malloc(sizeof(double[3]) * (size_t)nc);
    double (*Xold)[3] = malloc(sizeof(double[3]) * (size_t)nc);
    for (int j = 0; j < nc; ++j) {
        wrapped(p, X + 3 * j, Xw[j]);
        for (int t = 0; t < 3; ++t) X0[j][t] = X[3 * j + t];
    }
    double gnorm = sqrt(p->g[0] * p->g[0] + p->g[1] * p->g[1] + p->g[2] * p->g[2]);

    /* classification (Verlet-list radius r_c + skin, §1.4) */
    uint8_t *near = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t n_near = 0;
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(+ : n_near)
    for (int64_t i = 0; i < n; ++i) {
        if (all_substep) { near[i] = 1; ++n_near; continue; }
        double *vi = v + 3 * i;
        double speed = sqrt(vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
        for (int j = 0; j < nc; ++j) {
            double d[3] = {x[3 * i] - Xw[j][0], x[3 * i + 1] - Xw[j][1], x[3 * i + 2] - Xw[j][2]};
            min_image(p, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double R = sqrt(rc2[j]) + speed * p->tau + 0.5 * gnorm * p->tau * p->tau + p->skin;
            if (r2 < R * R) { near[i] = 1; ++n_near; break; }
        }
    }
    if (near_out) memcpy(near_out, near, (size_t)n);
    orc_flight(p, n, x, v, near);

    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_near > 0 ? n_near : 1));
    for (int64_t i = 0, k = 0; i < n; ++i) if (near[i]) list[k++] = i;
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)(n_near > 0 ? n_near : 1));
    int64_t *Fq = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)nc);
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)nc);

    double dt = p->tau / (double)p->n_md;
    double hdt = 0.5 * dt;

    /* forces at the start of the interval */
    memset(Fq, 0, sizeof(int64_t) * 3 * (size_t)nc);
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(+ : Fq[:3 * nc])
    for (int64_t k = 0; k < n_near; ++k) {
        int64_t i = list[k];
        solvent_force(p, &cs, (const double (*)[3])Xw, x + 3 * i, flags[i], f + 3 * k, Fq);
        for (int t = 0; t < 3; ++t) f[3 * k + t] = f[3 * k + t] + p->g[t];
    }
    colloid_colloid(p, &cs, (const double (*)[3])Xw, Fq);
    for (int j = 0; j < 3 * nc; ++j) F[j] = (double)Fq[j] * FX_INV;

    for (int s = 0; s < p->n_md; ++s) {
        /* first half kick and drift */
        for (int j = 0; j < nc; ++j)
            for (int t = 0; t < 3; ++t) {
                V[3 * j + t] = fma(hdt, F[3 * j + t] / M[j], V[3 * j + t]);
                Xold[j][t] = X[3 * j + t];
                X[3 * j + t] = fma(dt, V[3 * j + t], X[3 * j + t]);
            }
        rattle_pos(&cs, (const double (*)[3])Xold, dt);
        for (int j = 0; j < nc; ++j) wrapped(p, X + 3 * j, Xw[j]);
        for (int64_t k = 0; k < n_near; ++k) {
            int64_t i = list[k];
            for (int t = 0; t < 3; ++t) {
                v[3 * i + t] = fma(hdt, f[3 * k + t], v[3 * i + t]);
                x[3 * i + t] = fma(dt, v[3 * i + t], x[3 * i + t]);
            }
        }
        /* new forces, catalytic conversion, second half kick */
        memset(Fq, 0, sizeof(int64_t) * 3 * (size_t)nc);
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(+ : Fq[:3 * nc])
        for (int64_t k = 0; k < n_near; ++k) {
            int64_t i = list[k];
            solvent_force(p, &cs, (const double (*)[3])Xw, x + 3 * i, flags[i], f + 3 * k, Fq);
            for (int t = 0; t < 3; ++t) f[3 * k + t] = f[3 * k + t] + p->g[t];
            if (!(flags[i] & F_B)) {
                int in = inside_catalytic(p, &cs, (const double (*)[3])Xw, x + 3 * i);
                if (in) flags[i] |= F_TAG;
                else if (flags[i] & F_TAG) {
                    int go = 1;
                    if (p->cat_prob < 1.0) {
                        uint32_t w[4];
                        draw(p->seed, id[i], step, P_CAT, (uint32_t)s, w);
                        go = (double)w[0] < p->cat_prob * 4294967296.0;
                    }
                    flags[i] = (uint8_t)(flags[i] & ~F_TAG);
                    if (go) flags[i] |= F_B;
                }
            }
        }
        colloid_colloid(p, &cs, (const double (*)[3])Xw, Fq);
        for (int j = 0; j < 3 * nc; ++j) F[j] = (double)Fq[j] * FX_INV;
        for (int j = 0; j < nc; ++j)
            for (int t = 0; t < 3; ++t) V[3 * j + t] = fma(hdt, F[3 * j + t] / M[j], V[3 * j + t]);
        for (int64_t k = 0; k < n_near; ++k) {
            int64_t i = list[k];
            for (int t = 0; t < 3; ++t) v[3 * i + t] = fma(hdt, f[3 * k + t], v[3 * i + t]);
        }
        rattle_vel(&cs);
    }
    for (int64_t k = 0; k < n_near; ++k) wrap_periodic(p, x + 3 * list[k]);

    int status = 0;
    for (int j = 0; j < nc; ++j) {
        double dd = 0.0;
        for (int t = 0; t < 3; ++t) { double e = X[3 * j + t] - X0[j][t]; dd = dd + e * e; }
        if (!(dd <= p->skin * p->skin)) status = 1;   /* NaN counts as a violation */
    }
    free(rc2); free(Xw); free(X0); free(Xold); free(near); free(list); free(f); free(Fq); free(F);
    return status;
}

/* Total colloid force (fixed point, as above) and per-particle solvent force
 * for the given configuration; exported for the tests. */
void orc_forces(const orc_params *p, int64_t n, const double *x, const uint8_t *flags,
                int nc, const double *X, const double *sig, const double *epsA, const double *epsB,
                double *f, double *F)
{
    double *rc2 = (double *)malloc(sizeof(double) * (size_t)nc);
    double (*Xw)[3] = malloc(sizeof(double[3]) * (size_t)(nc > 0 ? nc : 1));
    int64_t *Fq = (int64_t *)calloc((size_t)(3 * nc > 0 ? 3 * nc : 1), sizeof(int64_t));
    for (int j = 0; j < nc; ++j) { rc2[j] = orc_wca_rc2(sig[j]); wrapped(p, X + 3 * j, Xw[j]); }
    colloids_t cs = {nc, (double *)X, NULL, NULL, sig, epsA, epsB, rc2, NULL, 0, NULL, NULL, NULL};
    for (int64_t i = 0; i < n; ++i)
        solvent_force(p, &cs, (const double (*)[3])Xw, x + 3 * i, flags[i], f + 3 * i, Fq);
    for (int j = 0; j < 3 * nc; ++j) F[j] = (double)Fq[j] * FX_INV;
    free(rc2); free(Xw); free(Fq);
}

/* ------------------------------------------------------------------------ */
/* Temperature estimator of §1.4: T = 1/(3 N_c) sum_xi 1/(N_xi - 1)          */
/*   sum_i m (v_i - v_xi)^2, over the cells with N_xi >= 2 (reading: the     */
/* 1/(N_xi - 1) factor is undefined for N_xi < 2).  v in sorted order.       */
/* ------------------------------------------------------------------------ */
double orc_temperature(int64_t n_cells, const int64_t *count, const int64_t *start, const double *v,
                       int64_t *n_used)
{
    double acc = 0.0;
    int64_t nc = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t N = count[c];
        if (N < 2) continue;
        const double *vc = v + 3 * start[c];
        double sum[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) sum[d] = sum[d] + vc[3 * i + d];
        double vcm[3] = {sum[0] / (double)N, sum[1] / (double)N, sum[2] / (double)N};
        double ke = 0.0;
        for (int64_t i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) { double u = vc[3 * i + d] - vcm[d]; ke = ke + u * u; }
        acc = acc + ke / (double)(N - 1);
        ++nc;
    }
    if (n_used) *n_used = nc;
    return nc > 0 ? acc / (3.0 * (double)nc) : 0.0;
}

/* Total colloid-solvent WCA energy (§1.4 potential) plus colloid-colloid LJ
 * energy (shifted to zero at cc_rc, bonded pairs excluded); for the
 * conservation checks. */
double orc_potential_energy(const orc_params *p, int64_t n, const double *x, const uint8_t *flags,
                            int nc, const double *X, const double *sig, const double *epsA,
                            const double *epsB, int n_bonds, const int32_t *ba, const int32_t *bb)
{
    double (*Xw)[3] = malloc(sizeof(double[3]) * (size_t)(nc > 0 ? nc : 1));
    for (int j = 0; j < nc; ++j) wrapped(p, X + 3 * j, Xw[j]);
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < nc; ++j) {
            double d[3] = {x[3 * i] - Xw[j][0], x[3 * i + 1] - Xw[j][1], x[3 * i + 2] - Xw[j][2]};
            min_image(p, d);
            double f[3], ej;
            double eps = (flags[i] & F_B) ? epsB[j] : epsA[j];
            if (orc_wca_force(d, sig[j], eps, orc_wca_rc2(sig[j]), f, &ej)) e = e + ej;
        }
    if (p->cc_rc > 0.0) {
        double sr = p->cc_sigma / p->cc_rc, sr6 = sr * sr * sr * sr * sr * sr;
        double eshift = 4.0 * p->cc_eps * (sr6 * sr6 - sr6);
        for (int a = 0; a < nc; ++a)
            for (int b = a + 1; b < nc; ++b) {
                int skip = 0;
                for (int k = 0; k < n_bonds; ++k)
                    if ((ba[k] == a && bb[k] == b) || (ba[k] == b && bb[k] == a)) skip = 1;
                if (skip) continue;
                double d[3] = {Xw[a][0] - Xw[b][0], Xw[a][1] - Xw[b][1], Xw[a][2] - Xw[b][2]};
                min_image(p, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 < p->cc_rc * p->cc_rc) {
                    double s2 = p->cc_sigma * p->cc_sigma / r2, s6 = s2 * s2 * s2;
                    e = e + 4.0 * p->cc_eps * (s6 * s6 - s6) - eshift;
                }
            }
    }
    free(Xw);
    return e;
}

/* ======================================================================== */
/* Rigid composite colloid: the Janus particle of §1.5, a sphere of WCA      */
/* beads (§1.4 holds its bead network together by an iterative RATTLE).      */
/* Reading: the network moves as one rigid body, which keeps every bead      */
/* distance exactly as the constraints do.                                   */
/*   state: centre of mass X (unwrapped), its velocity V, unit quaternion    */
/*   q = (w, x, y, z) taking the body frame to the space frame, and the      */
/*   angular momentum l in the body frame.                                   */
/*   geometry: n_b beads of mass m_b at fixed positions b_j, relative to X,  */
/*   in the body's principal frame; M = n_b m_b and the principal moments    */
/*   I_k = sum_j m_b (|b_j|^2 - b_jk^2).  All beads share sigma; each has    */
/*   its own eps_A, eps_B and catalytic flag.                                */
/*   forces: WCA between every solvent particle and every bead; the pair     */
/*   force f on the particle puts -f on the body and the torque              */
/*   -(R b_j) x f, both summed in 64-bit fixed point (2^-40) so the totals   */
/*   do not depend on the order of the pairs.                                */
/*   motion per sub-step dt: half kick of V (by F / M) and of l (by the      */
/*   body-frame torque R^T T), drift of X, free rotation by the symmetric    */
/*   splitting R_1(dt/2) R_2(dt/2) R_3(dt) R_2(dt/2) R_1(dt/2) of Dullweber, */
/*   Leimkuhler & McLachlan (J. Chem. Phys. 107, 5840 (1997)), new forces,   */
/*   second half kick.  R_k(h) turns the body about its principal axis k by  */
/*   the angle phi with tan(phi / 2) = h l_k / (2 I_k), the Cayley form of   */
/*   the exact angle h l_k / I_k (second order like the splitting itself,    */
/*   and built from +, -, *, / and sqrt only, so it is reproducible bit for  */
/*   bit): q <- q (1, tan(phi/2) e_k), normalised after the five turns, and  */
/*   l <- rotation of l by -phi about e_k.                                   */
/*   near radius: max_j |b_j| + r_c (the body's bounding sphere) in place of */
/*   a sphere's r_c; the skin bounds the displacement of X.                  */
/* ======================================================================== */
typedef struct {
    int nb;
    const double *b;          /* [nb*3] principal frame, relative to X        */
    const double *epsA, *epsB;
    const int32_t *cat;
    double sigma, rc2;
    double R[3][3];           /* body -> space                                */
    double Xw[3];             /* wrapped centre of mass                       */
    double *rb;               /* [nb*3] R b_j                                 */
    double *Xb;               /* [nb*3] Xw + R b_j                            */
} body_t;

/* Rotation matrix of a unit quaternion (w, x, y, z). */
void orc_quat_matrix(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

/* Mass and principal moments of a bead set (the diagonal of the inertia
 * tensor; the beads must be given in the principal frame). */
void orc_body_inertia(int nb, const double *b, double m_b, double *M, double I[3])
{
    I[0] = I[1] = I[2] = 0.0;
    for (int j = 0; j < nb; ++j) {
        const double *bj = b + 3 * j;
        I[0] = I[0] + m_b * (bj[1] * bj[1] + bj[2] * bj[2]);
        I[1] = I[1] + m_b * (bj[2] * bj[2] + bj[0] * bj[0]);
        I[2] = I[2] + m_b * (bj[0] * bj[0] + bj[1] * bj[1]);
    }
    *M = (double)nb * m_b;
}

/* Radius of the bounding sphere of the beads' interaction ranges. */
double orc_body_reach(int nb, const double *b, double sigma)
{
    double bmax = 0.0;
    for (int j = 0; j < nb; ++j) {
        const double *bj = b + 3 * j;
        double r = sqrt(bj[0] * bj[0] + bj[1] * bj[1] + bj[2] * bj[2]);
        if (r > bmax) bmax = r;
    }
    return bmax + sqrt(orc_wca_rc2(sigma));
}

/* Free rotation over one sub-step dt (the splitting above). */
void orc_body_rotate(const double I[3], double dt, double q[4], double l[3])
{
    static const int axis[5] = {0, 1, 2, 1, 0};
    double h[5];
    h[0] = 0.5 * dt; h[1] = 0.5 * dt; h[2] = dt; h[3] = 0.5 * dt; h[4] = 0.5 * dt;
    for (int s = 0; s < 5; ++s) {
        int k = axis[s], a = (k + 1) % 3, b = (k + 2) % 3;
        double t = 0.5 * (h[s] * l[k] / I[k]);      /* tan(phi / 2)              */
        double tt = t * t;
        double inv = 1.0 / (1.0 + tt);
        double c = (1.0 - tt) * inv;                 /* cos(phi)                  */
        double sn = (2.0 * t) * inv;                 /* sin(phi)                  */
        /* l turns by -phi about e_k */
        double la = c * l[a] + sn * l[b];
        double lb = c * l[b] - sn * l[a];
        l[a] = la;
        l[b] = lb;
        /* q <- q (1, t e_k) */
        double w = q[0], v[3] = {q[1], q[2], q[3]};
        q[0] = w - t * v[k];
        q[1 + k] = v[k] + t * w;
        q[1 + a] = v[a] + t * v[b];
        q[1 + b] = v[b] - t * v[a];
    }
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] = q[i] / nq;
}

/* Bead positions for the current X and q. */
static void body_frames(const orc_params *p, body_t *B, const double *X, const double q[4])
{
    orc_quat_matrix(q, B->R);
    wrapped(p, X, B->Xw);
    for (int j = 0; j < B->nb; ++j) {
        const double *bj = B->b + 3 * j;
        for (int t = 0; t < 3; ++t) {
            double r = B->R[t][0] * bj[0] + B->R[t][1] * bj[1] + B->R[t][2] * bj[2];
            B->rb[3 * j + t] = r;
            B->Xb[3 * j + t] = B->Xw[t] + r;
        }
    }
}

/* Force on one solvent particle from all beads (ascending bead order); adds
 * the reaction and its torque into Fq, Tq.  Returns 1 if the particle is
 * inside a catalytic bead's range. */
static int body_solvent_force(const orc_params *p, const body_t *B, const double *x, uint8_t fl,
                              double f[3], int64_t Fq[3], int64_t Tq[3], double *energy)
{
    int inside = 0;
    f[0] = f[1] = f[2] = 0.0;
    for (int j = 0; j < B->nb; ++j) {
        const double *Xb = B->Xb + 3 * j;
        double d[3] = {x[0] - Xb[0], x[1] - Xb[1], x[2] - Xb[2]};
        min_image(p, d);
        double fj[3], ej = 0.0;
        double eps = (fl & F_B) ? B->epsB[j] : B->epsA[j];
        if (orc_wca_force(d, B->sigma, eps, B->rc2, fj, energy ? &ej : NULL)) {
            const double *r = B->rb + 3 * j;
            double c[3] = {r[1] * fj[2] - r[2] * fj[1], r[2] * fj[0] - r[0] * fj[2], r[0] * fj[1] - r[1] * fj[0]};
            for (int k = 0; k < 3; ++k) {
                f[k] = f[k] + fj[k];
                Fq[k] -= llrint(fj[k] * FX_SCALE);
                Tq[k] -= llrint(c[k] * FX_SCALE);
            }
            if (energy) *energy = *energy + ej;
            if (B->cat[j]) inside = 1;
        }
    }
    return inside;
}

/* Body force F, space torque T and body-frame torque from fixed-point sums. */
static void body_totals(const body_t *B, const int64_t Fq[3], const int64_t Tq[3], double F[3], double tb[3])
{
    double T[3];
    for (int k = 0; k < 3; ++k) { F[k] = (double)Fq[k] * FX_INV; T[k] = (double)Tq[k] * FX_INV; }
    for (int k = 0; k < 3; ++k) tb[k] = B->R[0][k] * T[0] + B->R[1][k] * T[1] + B->R[2][k] * T[2];
}

/* Catalytic tag / conversion of one A particle (§1.5), as in orc_interval. */
static void catalytic_step(const orc_params *p, uint8_t *fl, uint32_t id, int in, uint32_t step, int s)
{
    if (*fl & F_B) return;
    if (in) { *fl |= F_TAG; return; }
    if (!(*fl & F_TAG)) return;
    int go = 1;
    if (p->cat_prob < 1.0) {
        uint32_t w[4];
        draw(p->seed, id, step, P_CAT, (uint32_t)s, w);
        go = (double)w[0] < p->cat_prob * 4294967296.0;
    }
    *fl = (uint8_t)(*fl & ~F_TAG);
    if (go) *fl |= F_B;
}

/* One collision interval of solvent + rigid body motion: as orc_interval,
 * with the body in place of the colloids.  X, V, q, l are updated in place.
 * Returns 0, or 1 if X moved further than skin. */
int orc_interval_body(const orc_params *p, uint32_t step, int64_t n, double *x, double *v,
                      uint8_t *flags, const uint32_t *id,
                      int nb, const double *b, const double *epsA, const double *epsB, const int32_t *cat,
                      double m_b, double sigma, double *X, double *V, double *q, double *l,
                      int all_substep, uint8_t *near_out)
{
    double M, I[3];
    orc_body_inertia(nb, b, m_b, &M, I);
    double reach = orc_body_reach(nb, b, sigma);
    body_t B = {nb, b, epsA, epsB, cat, sigma, orc_wca_rc2(sigma), {{0}}, {0}, NULL, NULL};
    B.rb = (double *)malloc(sizeof(double) * 3 * (size_t)(nb > 0 ? nb : 1));
    B.Xb = (double *)malloc(sizeof(double) * 3 * (size_t)(nb > 0 ? nb : 1));
    body_frames(p, &B, X, q);
    double X0[3] = {X[0], X[1], X[2]};
    double gnorm = sqrt(p->g[0] * p->g[0] + p->g[1] * p->g[1] + p->g[2] * p->g[2]);

    /* classification against the bounding sphere */
    uint8_t *near = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t n_near = 0;
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(+ : n_near)
    for (int64_t i = 0; i < n; ++i) {
        if (all_substep) { near[i] = 1; ++n_near; continue; }
        double *vi = v + 3 * i;
        double speed = sqrt(vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
        double d[3] = {x[3 * i] - B.Xw[0], x[3 * i + 1] - B.Xw[1], x[3 * i + 2] - B.Xw[2]};
        min_image(p, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double R = reach + speed * p->tau + 0.5 * gnorm * p->tau * p->tau + p->skin;
        if (r2 < R * R) { near[i] = 1; ++n_near; }
    }
    if (near_out) memcpy(near_out, near, (size_t)n);
    orc_flight(p, n, x, v, near);

    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_near > 0 ? n_near : 1));
    for (int64_t i = 0, k = 0; i < n; ++i) if (near[i]) list[k++] = i;
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)(n_near > 0 ? n_near : 1));
    double dt = p->tau / (double)p->n_md;
    double hdt = 0.5 * dt;
    int64_t Fq[3], Tq[3];
    double F[3], tb[3];

    /* forces at the start of the interval */
    memset(Fq, 0, sizeof Fq); memset(Tq, 0, sizeof Tq);
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(+ : Fq, Tq)
    for (int64_t k = 0; k < n_near; ++k) {
        int64_t i = list[k];
        body_solvent_force(p, &B, x + 3 * i, flags[i], f + 3 * k, Fq, Tq, NULL);
        for (int t = 0; t < 3; ++t) f[3 * k + t] = f[3 * k + t] + p->g[t];
    }
    body_totals(&B, Fq, Tq, F, tb);

    for (int s = 0; s < p->n_md; ++s) {
        /* body: half kick, drift, free rotation */
        for (int t = 0; t < 3; ++t) {
            V[t] = fma(hdt, F[t] / M, V[t]);
            l[t] = fma(hdt, tb[t], l[t]);
            X[t] = fma(dt, V[t], X[t]);
        }
        orc_body_rotate(I, dt, q, l);
        body_frames(p, &B, X, q);
        /* solvent: half kick, drift */
        for (int64_t k = 0; k < n_near; ++k) {
            int64_t i = list[k];
            for (int t = 0; t < 3; ++t) {
                v[3 * i + t] = fma(hdt, f[3 * k + t], v[3 * i + t]);
                x[3 * i + t] = fma(dt, v[3 * i + t], x[3 * i + t]);
            }
        }
        /* new forces, catalytic conversion, second half kicks */
        memset(Fq, 0, sizeof Fq); memset(Tq, 0, sizeof Tq);
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(+ : Fq, Tq)
        for (int64_t k = 0; k < n_near; ++k) {
            int64_t i = list[k];
            int in = body_solvent_force(p, &B, x + 3 * i, flags[i], f + 3 * k, Fq, Tq, NULL);
            for (int t = 0; t < 3; ++t) f[3 * k + t] = f[3 * k + t] + p->g[t];
            catalytic_step(p, flags + i, id[i], in, step, s);
        }
        body_totals(&B, Fq, Tq, F, tb);
        for (int t = 0; t < 3; ++t) {
            V[t] = fma(hdt, F[t] / M, V[t]);
            l[t] = fma(hdt, tb[t], l[t]);
        }
        for (int64_t k = 0; k < n_near; ++k) {
            int64_t i = list[k];
            for (int t = 0; t < 3; ++t) v[3 * i + t] = fma(hdt, f[3 * k + t], v[3 * i + t]);
        }
    }
    for (int64_t k = 0; k < n_near; ++k) wrap_periodic(p, x + 3 * list[k]);

    double dd = 0.0;
    for (int t = 0; t < 3; ++t) { double e = X[t] - X0[t]; dd = dd + e * e; }
    int status = (dd <= p->skin * p->skin) ? 0 : 1;   /* NaN counts as a violation */
    free(B.rb); free(B.Xb); free(near); free(list); free(f);
    return status;
}

/* Solvent forces f[n*3], body force F, space torque T and the WCA energy of
 * a configuration (for the tests). */
double orc_body_forces(const orc_params *p, int64_t n, const double *x, const uint8_t *flags,
                       int nb, const double *b, const double *epsA, const double *epsB, const int32_t *cat,
                       double sigma, const double *X, const double *q, double *f, double *F, double *T)
{
    body_t B = {nb, b, epsA, epsB, cat, sigma, orc_wca_rc2(sigma), {{0}}, {0}, NULL, NULL};
    B.rb = (double *)malloc(sizeof(double) * 3 * (size_t)(nb > 0 ? nb : 1));
    B.Xb = (double *)malloc(sizeof(double) * 3 * (size_t)(nb > 0 ? nb : 1));
    body_frames(p, &B, X, q);
    int64_t Fq[3] = {0, 0, 0}, Tq[3] = {0, 0, 0};
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i) body_solvent_force(p, &B, x + 3 * i, flags[i], f + 3 * i, Fq, Tq, &e);
    for (int k = 0; k < 3; ++k) { F[k] = (double)Fq[k] * FX_INV; T[k] = (double)Tq[k] * FX_INV; }
    free(B.rb); free(B.Xb);
    return e;
}

/* ------------------------------------------------------------------------ */
/* Iterative RATTLE for beads linked by fixed distances (§1.4 integrates the */
/* Janus particle's bead network with the iterative form of RATTLE; Andersen */
/* 1983).  Each link in turn is corrected, sweeping the list until every     */
/* link holds within the tolerance.  This models the Janus particle as the   */
/* paper does; the rigid body above is the other form the GPU path offers.   */
/* ------------------------------------------------------------------------ */

/* Position stage.  xold: bead positions at the start of the sub-step; x, v:
 * after the unconstrained drift, corrected in place -- link (a, b) moves its
 * beads along their bond vector at the start of the sub-step, by amounts
 * inverse to their masses, and the velocities by the same displacement over
 * dt.  Converged when |x_a - x_b|^2 is within 2 tol d^2 of d^2 for every
 * link.  Returns the number of sweeps, or -1 when max_sweeps ran out. */
int orc_rattle_pos_iter(int nl, const int32_t *la, const int32_t *lb, const double *dl, const double *m,
                        const double *xold, double *x, double *v, double dt, double tol, int max_sweeps)
{
    for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
        int moved = 0;
        for (int k = 0; k < nl; ++k) {
            const int a = la[k], b = lb[k];
            double s[3], ro[3];
            for (int t = 0; t < 3; ++t) {
                s[t] = x[3 * a + t] - x[3 * b + t];
                ro[t] = xold[3 * a + t] - xold[3 * b + t];
            }
            const double d2 = dl[k] * dl[k];
            const double diff = d2 - (s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
            if (fabs(diff) <= 2.0 * tol * d2) continue;
            /* inverse-mass form: bead a moves by g w_a along the old bond,
             * w = 1/m, and its velocity by that displacement times 1/dt */
            const double wa = 1.0 / m[a], wb = 1.0 / m[b], idt = 1.0 / dt;
            const double inv = wa + wb;
            const double sro = s[0] * ro[0] + s[1] * ro[1] + s[2] * ro[2];
            const double g = diff / (2.0 * sro * inv);
            const double ga = g * wa, gb = g * wb;
            for (int t = 0; t < 3; ++t) {
                const double ca = ga * ro[t], cb = gb * ro[t];
                x[3 * a + t] = x[3 * a + t] + ca;
                x[3 * b + t] = x[3 * b + t] - cb;
                v[3 * a + t] = v[3 * a + t] + ca * idt;
                v[3 * b + t] = v[3 * b + t] - cb * idt;
            }
            moved = 1;
        }
        if (!moved) return sweep;
    }
    return -1;
}

/* Velocity stage: each link in turn removes the beads' relative velocity
 * along its current bond vector, by amounts inverse to their masses, until
 * |(v_a - v_b) . (x_a - x_b)| <= tol d for every link.  Returns the number
 * of sweeps, or -1. */
int orc_rattle_vel_iter(int nl, const int32_t *la, const int32_t *lb, const double *dl, const double *m,
                        const double *x, double *v, double tol, int max_sweeps)
{
    for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
        int moved = 0;
        for (int k = 0; k < nl; ++k) {
            const int a = la[k], b = lb[k];
            double s[3], w[3];
            for (int t = 0; t < 3; ++t) {
                s[t] = x[3 * a + t] - x[3 * b + t];
                w[t] = v[3 * a + t] - v[3 * b + t];
            }
            const double rv = s[0] * w[0] + s[1] * w[1] + s[2] * w[2];
            if (fabs(rv) <= tol * dl[k]) continue;
            const double wa = 1.0 / m[a], wb = 1.0 / m[b];   /* inverse masses */
            const double inv = wa + wb;
            const double ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
            const double kk = rv / (ss * inv);
            const double ka = kk * wa, kb = kk * wb;
            for (int t = 0; t < 3; ++t) {
                v[3 * a + t] = v[3 * a + t] - ka * s[t];
                v[3 * b + t] = v[3 * b + t] + kb * s[t];
            }
            moved = 1;
        }
        if (!moved) return sweep;
    }
    return -1;
}

/* Velocity Verlet of a linked bead network under per-bead forces F (held
 * fixed over the step, NULL = none): half kick, drift, position stage, half
 * kick, velocity stage (§1.4).  Returns the larger sweep count of the two
 * stages, or -1. */
int orc_network_step(int nb, const double *m, int nl, const int32_t *la, const int32_t *lb, const double *dl,
                     const double *F, double *x, double *v, double dt, double tol, int max_sweeps)
{
    if (nb <= 0) return 0;
    double *xold = (double *)malloc(sizeof(double) * 3 * (size_t)nb);
    if (!xold) return -1;
    for (int i = 0; i < nb; ++i)
        for (int t = 0; t < 3; ++t) {
            if (F) v[3 * i + t] = v[3 * i + t] + 0.5 * dt * F[3 * i + t] / m[i];
            xold[3 * i + t] = x[3 * i + t];
            x[3 * i + t] = x[3 * i + t] + dt * v[3 * i + t];
        }
    const int sp = orc_rattle_pos_iter(nl, la, lb, dl, m, xold, x, v, dt, tol, max_sweeps);
    free(xold);
    if (F)
        for (int i = 0; i < nb; ++i)
            for (int t = 0; t < 3; ++t) v[3 * i + t] = v[3 * i + t] + 0.5 * dt * F[3 * i + t] / m[i];
    const int sv = orc_rattle_vel_iter(nl, la, lb, dl, m, x, v, tol, max_sweeps);
    if (sp < 0 || sv < 0) return -1;
    return sp > sv ? sp : sv;
}

/* Force on one solvent particle from every bead of a network (ascending bead
 * order, wrapped bead positions Xw); the reaction goes to the bead's
 * fixed-point sums Fq[3 nb].  Returns 1 if the particle is inside a
 * catalytic bead's range. */
static int network_solvent_force(const orc_params *p, int nb, const double *Xw, const double *epsA,
                                 const double *epsB, const int32_t *cat, double sigma, double rc2, const double *x,
                                 uint8_t fl, double f[3], int64_t *Fq, double *energy)
{
    int inside = 0;
    f[0] = f[1] = f[2] = 0.0;
    for (int j = 0; j < nb; ++j) {
        double d[3] = {x[0] - Xw[3 * j], x[1] - Xw[3 * j + 1], x[2] - Xw[3 * j + 2]};
        min_image(p, d);
        double fj[3], ej = 0.0;
        const double eps = (fl & F_B) ? epsB[j] : epsA[j];
        if (orc_wca_force(d, sigma, eps, rc2, fj, energy ? &ej : NULL)) {
            for (int k = 0; k < 3; ++k) {
                f[k] = f[k] + fj[k];
                Fq[3 * j + k] -= llrint(fj[k] * FX_SCALE);
            }
            if (energy) *energy = *energy + ej;
            if (cat[j]) inside = 1;
        }
    }
    return inside;
}

static void network_frames(const orc_params *p, int nb, const double *xb, double *Xw)
{
    for (int j = 0; j < nb; ++j) wrapped(p, xb + 3 * j, Xw + 3 * j);
}

static void network_com(int nb, const double *xb, const double *mb, double X[3], double *M)
{
    double s[3] = {0.0, 0.0, 0.0}, m = 0.0;
    for (int j = 0; j < nb; ++j) {
        m = m + mb[j];
        for (int t = 0; t < 3; ++t) s[t] = s[t] + mb[j] * xb[3 * j + t];
    }
    for (int t = 0; t < 3; ++t) X[t] = s[t] / m;
    *M = m;
}

/* One collision interval of solvent + a Janus particle made of beads held at
 * fixed distances by iterative RATTLE (§1.4, §1.5): as orc_interval_body, but
 * every bead is a point mass in the velocity-Verlet sub-steps, kicked by the
 * reactions of its own bead-solvent forces, with the position stage after
 * each drift and the velocity stage after each second half kick.  xb, vb
 * (bead positions, unwrapped, and velocities) are updated in place.  Near
 * particles: within the beads' bounding sphere about their centre of mass at
 * the start (largest bead distance + r_c) plus |v| tau + |g| tau^2 / 2 +
 * skin.  Returns 0; 1 if the centre of mass moved further than skin; 2 if a
 * RATTLE stage did not converge within max_sweeps. */
int orc_interval_network(const orc_params *p, uint32_t step, int64_t n, double *x, double *v, uint8_t *flags,
                         const uint32_t *id, int nb, double *xb, double *vb, const double *mb, const double *epsA,
                         const double *epsB, const int32_t *cat, double sigma, int nl, const int32_t *la,
                         const int32_t *lb, const double *dl, double tol, int max_sweeps, int all_substep,
                         uint8_t *near_out)
{
    const double rc2 = orc_wca_rc2(sigma);
    double X0[3], M;
    network_com(nb, xb, mb, X0, &M);
    double reach = 0.0;
    for (int j = 0; j < nb; ++j) {
        double e2 = 0.0;
        for (int t = 0; t < 3; ++t) { double e = xb[3 * j + t] - X0[t]; e2 = e2 + e * e; }
        if (sqrt(e2) > reach) reach = sqrt(e2);
    }
    reach = reach + sqrt(rc2);
    double X0w[3];
    wrapped(p, X0, X0w);
    const double gnorm = sqrt(p->g[0] * p->g[0] + p->g[1] * p->g[1] + p->g[2] * p->g[2]);
    const size_t nb3 = 3 * (size_t)(nb > 0 ? nb : 1);
    double *Xw = (double *)malloc(sizeof(double) * nb3);
    double *xold = (double *)malloc(sizeof(double) * nb3);
    double *Fb = (double *)malloc(sizeof(double) * nb3);
    int64_t *Fq = (int64_t *)malloc(sizeof(int64_t) * nb3);
    network_frames(p, nb, xb, Xw);

    uint8_t *near = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t n_near = 0;
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(+ : n_near)
    for (int64_t i = 0; i < n; ++i) {
        if (all_substep) { near[i] = 1; ++n_near; continue; }
        const double *vi = v + 3 * i;
        const double speed = sqrt(vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
        double d[3] = {x[3 * i] - X0w[0], x[3 * i + 1] - X0w[1], x[3 * i + 2] - X0w[2]};
        min_image(p, d);
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double R = reach + speed * p->tau + 0.5 * gnorm * p->tau * p->tau + p->skin;
        if (r2 < R * R) { near[i] = 1; ++n_near; }
    }
    if (near_out) memcpy(near_out, near, (size_t)n);
    orc_flight(p, n, x, v, near);

    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_near > 0 ? n_near : 1));
    for (int64_t i = 0, k = 0; i < n; ++i) if (near[i]) list[k++] = i;
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)(n_near > 0 ? n_near : 1));
    const double dt = p->tau / (double)p->n_md;
    const double hdt = 0.5 * dt;
    int status = 0;

    /* forces at the start of the interval */
    memset(Fq, 0, sizeof(int64_t) * nb3);
    for (int64_t k = 0; k < n_near; ++k) {
        const int64_t i = list[k];
        network_solvent_force(p, nb, Xw, epsA, epsB, cat, sigma, rc2, x + 3 * i, flags[i], f + 3 * k, Fq, NULL);
        for (int t = 0; t < 3; ++t) f[3 * k + t] = f[3 * k + t] + p->g[t];
    }
    for (size_t c = 0; c < 3 * (size_t)nb; ++c) Fb[c] = (double)Fq[c] * FX_INV;

    for (int s = 0; s < p->n_md; ++s) {
        /* beads: half kick, drift, position stage */
        for (int j = 0; j < nb; ++j)
            for (int t = 0; t < 3; ++t) {
                vb[3 * j + t] = fma(hdt, Fb[3 * j + t] / mb[j], vb[3 * j + t]);
                xold[3 * j + t] = xb[3 * j + t];
                xb[3 * j + t] = fma(dt, vb[3 * j + t], xb[3 * j + t]);
            }
        if (orc_rattle_pos_iter(nl, la, lb, dl, mb, xold, xb, vb, dt, tol, max_sweeps) < 0) status = 2;
        network_frames(p, nb, xb, Xw);
        /* solvent: half kick, drift */
        for (int64_t k = 0; k < n_near; ++k) {
            const int64_t i = list[k];
            for (int t = 0; t < 3; ++t) {
                v[3 * i + t] = fma(hdt, f[3 * k + t], v[3 * i + t]);
                x[3 * i + t] = fma(dt, v[3 * i + t], x[3 * i + t]);
            }
        }
        /* new forces, catalytic conversion, second half kicks, velocity stage */
        memset(Fq, 0, sizeof(int64_t) * nb3);
        for (int64_t k = 0; k < n_near; ++k) {
            const int64_t i = list[k];
            const int in = network_solvent_force(p, nb, Xw, epsA, epsB, cat, sigma, rc2, x + 3 * i, flags[i],
                                                 f + 3 * k, Fq, NULL);
            for (int t = 0; t < 3; ++t) f[3 * k + t] = f[3 * k + t] + p->g[t];
            catalytic_step(p, flags + i, id[i], in, step, s);
        }
        for (size_t c = 0; c < 3 * (size_t)nb; ++c) Fb[c] = (double)Fq[c] * FX_INV;
        for (int j = 0; j < nb; ++j)
            for (int t = 0; t < 3; ++t) vb[3 * j + t] = fma(hdt, Fb[3 * j + t] / mb[j], vb[3 * j + t]);
        if (orc_rattle_vel_iter(nl, la, lb, dl, mb, xb, vb, tol, max_sweeps) < 0) status = 2;
        for (int64_t k = 0; k < n_near; ++k) {
            const int64_t i = list[k];
            for (int t = 0; t < 3; ++t) v[3 * i + t] = fma(hdt, f[3 * k + t], v[3 * i + t]);
        }
    }
    for (int64_t k = 0; k < n_near; ++k) wrap_periodic(p, x + 3 * list[k]);

    double X1[3];
    network_com(nb, xb, mb, X1, &M);
    double dd = 0.0;
    for (int t = 0; t < 3; ++t) { const double e = X1[t] - X0[t]; dd = dd + e * e; }
    if (status == 0 && !(dd <= p->skin * p->skin)) status = 1;   /* NaN counts as a violation */
    free(Xw); free(xold); free(Fb); free(Fq); free(near); free(list); free(f);
    return status;
}

/* WCA energy between the solvent and a bead network (for the tests). */
double orc_network_energy(const orc_params *p, int64_t n, const double *x, const uint8_t *flags, int nb,
                          const double *xb, const double *epsA, const double *epsB, const int32_t *cat, double sigma)
{
    const size_t nb3 = 3 * (size_t)(nb > 0 ? nb : 1);
    double *Xw = (double *)malloc(sizeof(double) * nb3);
    int64_t *Fq = (int64_t *)calloc(nb3, sizeof(int64_t));
    network_frames(p, nb, xb, Xw);
    const double rc2 = orc_wca_rc2(sigma);
    double e = 0.0, f[3];
    for (int64_t i = 0; i < n; ++i)
        network_solvent_force(p, nb, Xw, epsA, epsB, cat, sigma, rc2, x + 3 * i, flags[i], f, Fq, &e);
    free(Xw); free(Fq);
    return e;
}

/* ------------------------------------------------------------------------ */
/* Hilbert order of the cells (§1.4: the paper sorts the solvent by compact  */
/* Hilbert indices).  Reading: the cells of an L0 x L1 x L2 box are ranked   */
/* by the index of the standard 3-D Hilbert curve through the smallest      */
/* enclosing cube of side 2^m -- the order compact indices preserve -- and  */
/* the rank is the cell's place in the sort.  The index follows Skilling's */
/* transform (AIP Conf. Proc. 707, 2004): undo the excess rotations level   */
/* by level, Gray-encode across the axes, then interleave the bits.         */
/* ------------------------------------------------------------------------ */
uint64_t orc_hilbert_index(int m, uint32_t x, uint32_t y, uint32_t z)
{
    uint32_t X[3] = {x, y, z};
    if (m <= 0) return 0;
    const uint32_t top = 1u << (m - 1);
    /* rotations and reflections, from the coarsest level down */
    for (uint32_t Q = top; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    /* Gray encoding across the axes */
    for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = top; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    /* interleave: bit b of the index triple (X0, X1, X2), most significant first */
    uint64_t h = 0;
    for (int b = m - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) h = (h << 1) | ((X[i] >> b) & 1u);
    return h;
}

static int cmp_u64_pair(const void *a, const void *b)
{
    const uint64_t *p = (const uint64_t *)a, *q = (const uint64_t *)b;
    return (p[0] > q[0]) - (p[0] < q[0]);
}

/* rank[c] for every cell c = x + L0 (y + L1 z) of the box: its place in the
 * Hilbert order.  Returns 0, or -1 if memory ran out. */
int orc_hilbert_rank(const int32_t L[3], int64_t *rank)
{
    int m = 0;
    const int32_t Lmax = L[0] > L[1] ? (L[0] > L[2] ? L[0] : L[2]) : (L[1] > L[2] ? L[1] : L[2]);
    while ((1 << m) < Lmax) ++m;
    const int64_t n = (int64_t)L[0] * L[1] * L[2];
    uint64_t *pairs = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)(n > 0 ? n : 1));
    if (!pairs) return -1;
    for (int64_t c = 0; c < n; ++c) {
        const uint32_t x = (uint32_t)(c % L[0]), y = (uint32_t)((c / L[0]) % L[1]), z = (uint32_t)(c / ((int64_t)L[0] * L[1]));
        pairs[2 * c] = orc_hilbert_index(m, x, y, z);
        pairs[2 * c + 1] = (uint64_t)c;
    }
    qsort(pairs, (size_t)n, 2 * sizeof(uint64_t), cmp_u64_pair);
    for (int64_t r = 0; r < n; ++r) rank[pairs[2 * r + 1]] = r;
    free(pairs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Species reservoirs (§1.5 chemotactic_cell: a Poiseuille flow with a       */
/* two-species gradient across it).  Reading: after each collision every     */
/* particle of a cell whose y column on the collision grid lies in [ya0,     */
/* ya1) becomes A, and in [yb0, yb1) becomes B (tags cleared); diffusion     */
/* between the two layers sets up the gradient.                              */
/* ------------------------------------------------------------------------ */
void orc_species_reservoirs(const orc_params *p, int64_t n_cells, const int64_t *count, const int64_t *start,
                            uint8_t *flags, int32_t ya0, int32_t ya1, int32_t yb0, int32_t yb1)
{
    for (int64_t c = 0; c < n_cells; ++c) {
        const int32_t cy = (int32_t)((c / p->L[0]) % p->L[1]);
        int to = -1;
        if (cy >= ya0 && cy < ya1) to = 0;
        else if (cy >= yb0 && cy < yb1) to = 1;
        if (to < 0) continue;
        for (int64_t k = start[c]; k < start[c] + count[c]; ++k)
            flags[k] = (uint8_t)(to ? F_B : 0);
    }
}

/* Colloid-colloid LJ forces F[nc*3] of a configuration (bonded pairs
 * excluded), as the interval sums them (for the tests). */
void orc_cc_forces(const orc_params *p, int nc, const double *X, int n_bonds, const int32_t *ba,
                   const int32_t *bb, double *F)
{
    double (*Xw)[3] = malloc(sizeof(double[3]) * (size_t)(nc > 0 ? nc : 1));
    int64_t *Fq = (int64_t *)calloc((size_t)(3 * nc > 0 ? 3 * nc : 1), sizeof(int64_t));
    for (int j = 0; j < nc; ++j) wrapped(p, X + 3 * j, Xw[j]);
    colloids_t cs = {nc, (double *)X, NULL, NULL, NULL, NULL, NULL, NULL, NULL, n_bonds, ba, bb, NULL};
    colloid_colloid(p, &cs, (const double (*)[3])Xw, Fq);
    for (int j = 0; j < 3 * nc; ++j) F[j] = (double)Fq[j] * FX_INV;
    free(Xw); free(Fq);
}
