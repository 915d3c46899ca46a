/*
 * FP64 CPU oracle for the DPD-CGMD multiscale model -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this library.  It shares no code with the CUDA path: it is a plain,
 * slow, literal restatement of what the paper's model computes.
 *
 *   Eq. 1  DPD pair forces  F = [a w - gamma w^2 (e.v) + sigma w zeta/sqrt(dt)] e,
 *          w = 1 - r/rc  (Groot-Warren discretisation of the sqrt(dt) noise term,
 *          fluctuation-dissipation w_D = w_R^2, sigma^2 = 2 gamma kT)
 *   Eq. 2  intra-platelet potential: LJ 12-6, Morse (the printed form), harmonic
 *          bonds U = k_b (r - r0)^2 and angles U = k_a (theta - theta0)^2 (no 1/2,
 *          as printed)
 *   Eq. 3  fluid-platelet interface: DPD with its own conservative amplitude
 *   Eq. 4  inter-platelet: Morse + f_A (1 - r/r0) receptor term
 *   Table 1  velocity-Verlet and the multi-level RESPA loop
 *   Sec. 4.2 observables (temperature, pressure, flow-speed profile, stress)
 *
 * The random number zeta_ij is Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11) with counter
 * (min id, max id, time index n, sub-index c) and key (seed lo, seed hi),
 * turned into a standard normal by the Box-Muller transform of its first
 * two words; symmetric in (i, j), so F^R is exactly antisymmetric.
 *
 * Pair forces are summed per particle over all partners j != i in ascending
 * id order (each pair force is computed twice, once per side), which keeps
 * every sum order-fixed and makes the code trivially correct to read.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LVL_FLUID 1u
#define LVL_IFACE 2u
#define LVL_PLT   4u

#define TAG_FLUID (-1)
#define TAG_WALL  (-2)
#define REC_BIT   (1 << 30)

typedef struct {
    double L[3];          /* fluid region [0,Lx) x [0,Ly) x [0,Lz) */
    int32_t walls;        /* 1: frozen walls outside y in [0,Ly], bounce-back */
    int32_t le;           /* 1: Lees-Edwards images in y (periodic y) */
    double le_rate;       /* shear rate gamma-dot */
    double le_offset;     /* current image x-offset delta in [0, Lx) */
    double g;             /* body force along +x on mobile particles */
    double rc, a_ff, a_fw, a_fp, gamma, sigma;
    double lj_eps, lj_sigma, lj_rc, lj_excl;
    double m_D, m_alpha, m_r0, m_rc, f_A;
    double k_b;
    uint32_t seed_lo, seed_hi;
    /* AI-MTS term selection (NULL: every term): with plt_k[P] set, a
     * platelet-level term counts only if the finer of its two platelets'
     * ratios, max(k_i, k_j), equals lvl_k */
    const int32_t *plt_k;
    int32_t lvl_k;
    /* Eq. 3 read with an LJ conservative term (the selectable variant): the
     * plasma-platelet conservative force is LJ(lj_eps, lj_sigma) cut at its
     * minimum 2^(1/6) lj_sigma (purely repulsive, shifted to zero there)
     * instead of a_fp (1 - r/rc); dissipative and random parts as Eq. 1 */
    int32_t iface_lj;
    /* zeta read as any variate of zero mean and unit variance (the
     * fluctuation-dissipation balance of Eq. 1 fixes only these two moments),
     * the selectable speed option: the uniform variate sqrt(3) (2u - 1), u the
     * midpoint of the 2^-24 bin given by the top 24 bits of the first word */
    int32_t uniform_noise;
    /* Eq. 2 angle term k_a (theta - theta0)^2 over triplets (i, j, k) of
     * particle rows, j the vertex (NULL / 0: none) */
    int32_t n_angles;
    const int32_t *angles;     /* [3 n_angles] */
    const double *theta0;      /* [n_angles] */
    double k_a;
} orc_params;

static int term_selected(const orc_params *p, int32_t ti, int32_t tj)
{
    if (!p->plt_k) return 1;
    int32_t ki = p->plt_k[ti & ~REC_BIT], kj = p->plt_k[tj & ~REC_BIT];
    return (ki > kj ? ki : kj) == p->lvl_k;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11) and the Gaussian                                    */
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
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Box-Muller on the top 24 bits of two words: u1 in (0,1], u2 in [0,1). */
double orc_gauss_from_bits(uint32_t r0, uint32_t r1)
{
    const double two_m24 = 1.0 / 16777216.0;
    double u1 = ((double)(r0 >> 8) + 1.0) * two_m24;
    double u2 = (double)(r1 >> 8) * two_m24;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Uniform variate of zero mean and unit variance on the top 24 bits of one word. */
double orc_uniform_from_bits(uint32_t r0)
{
    double u = ((double)(r0 >> 8) + 0.5) / 16777216.0;
    return sqrt(3.0) * (2.0 * u - 1.0);
}

double orc_zeta(const orc_params *p, int32_t id_i, int32_t id_j, uint32_t n_time, uint32_t c_sub)
{
    uint32_t a = (uint32_t)(id_i < id_j ? id_i : id_j);
    uint32_t b = (uint32_t)(id_i < id_j ? id_j : id_i);
    uint32_t ctr[4] = {a, b, n_time, c_sub};
    uint32_t key[2] = {p->seed_lo, p->seed_hi};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    if (p->uniform_noise) return orc_uniform_from_bits(r[0]);
    return orc_gauss_from_bits(r[0], r[1]);
}

/* ------------------------------------------------------------------------ */
/* geometry                                                                  */
/* ------------------------------------------------------------------------ */

/* Minimum-image separation r_ij = x_i - x_j (FP64) and the matching relative
 * velocity correction for Lees-Edwards images. */
static void min_image(const orc_params *p, double *dx, double *dy, double *dz, double *dvx)
{
    const double Lx = p->L[0], Ly = p->L[1], Lz = p->L[2];
    if (p->le) {
        if (*dy > 0.5 * Ly) {
            *dy -= Ly; *dx -= p->le_offset; *dvx -= p->le_rate * Ly;
        } else if (*dy < -0.5 * Ly) {
            *dy += Ly; *dx += p->le_offset; *dvx += p->le_rate * Ly;
        }
    } else if (!p->walls) {
        *dy -= Ly * nearbyint(*dy / Ly);
    }
    *dx -= Lx * nearbyint(*dx / Lx);
    *dz -= Lz * nearbyint(*dz / Lz);
}

/* ------------------------------------------------------------------------ */
/* pair classification                                                       */
/* ------------------------------------------------------------------------ */

enum { PK_NONE = 0, PK_DPD_FF, PK_DPD_FW, PK_DPD_FP, PK_PLT };

static int pair_kind(int32_t ti, int32_t tj)
{
    int fi = ti == TAG_FLUID, fj = tj == TAG_FLUID;
    int wi = ti == TAG_WALL, wj = tj == TAG_WALL;
    int pi = ti >= 0, pj = tj >= 0;
    if (fi && fj) return PK_DPD_FF;
    if ((fi && wj) || (wi && fj)) return PK_DPD_FW;
    if ((fi || wi) && pj) return PK_DPD_FP;
    if (pi && (fj || wj)) return PK_DPD_FP;
    if (pi && pj) return PK_PLT;
    return PK_NONE; /* wall-wall */
}

static unsigned kind_level(int k)
{
    switch (k) {
    case PK_DPD_FF: case PK_DPD_FW: return LVL_FLUID;
    case PK_DPD_FP: return LVL_IFACE;
    case PK_PLT: return LVL_PLT;
    default: return 0;
    }
}

/* ------------------------------------------------------------------------ */
/* pair forces: scalar f(r) such that F_ij = f * r_ij/r                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    double epot;        /* potential energy (each pair once) */
    double vir[9];      /* sum over pairs of r_a F_b, all forces */
    double vir_c[9];    /* same, conservative forces only */
} orc_acc;

/* Eq. 1: returns the three scalar parts (conservative, dissipative, random). */
static void dpd_parts(double a, double gamma, double sigma, double rc, double r,
                      double edotv, double zeta, double inv_sqrt_dt,
                      double *fc, double *fd, double *fr)
{
    double w = 1.0 - r / rc;
    *fc = a * w;
    *fd = -gamma * w * w * edotv;
    *fr = sigma * w * zeta * inv_sqrt_dt;
}

/* Eq. 2 LJ, shifted to zero at the cut-off: magnitude along e (positive = repulsive). */
static double lj_force(double eps, double sig, double r)
{
    double s6 = pow(sig / r, 6.0);
    return 24.0 * eps * (2.0 * s6 * s6 - s6) / r;
}
static double lj_energy(double eps, double sig, double r)
{
    double s6 = pow(sig / r, 6.0);
    return 4.0 * eps * (s6 * s6 - s6);
}

/* Eq. 2 Morse as printed: U = D[e^{alpha(1-r/r0)} - 2 e^{alpha(1-r/r0)/2}]. */
static double morse_force(double D, double alpha, double r0, double r)
{
    double t = alpha * (1.0 - r / r0);
    return D * alpha / r0 * (exp(t) - exp(0.5 * t));
}
static double morse_energy(double D, double alpha, double r0, double r)
{
    double t = alpha * (1.0 - r / r0);
    return D * (exp(t) - 2.0 * exp(0.5 * t));
}

static void acc_pair(orc_acc *acc, double dx, double dy, double dz,
                     double fx, double fy, double fz, double fcx, double fcy, double fcz,
                     double scale)
{
    double r[3] = {dx, dy, dz}, F[3] = {fx, fy, fz}, Fc[3] = {fcx, fcy, fcz};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            acc->vir[3 * a + b] += scale * r[a] * F[b];
            acc->vir_c[3 * a + b] += scale * r[a] * Fc[b];
        }
}

typedef struct {
    const orc_params *p;
    int32_t n;
    const double *x, *v, *X0;
    const int32_t *id, *tag;
    unsigned level_mask;
    uint32_t n_time_f, c_sub_f;   /* RNG time index of the fluid-level evaluation */
    uint32_t n_time_m, c_sub_m;   /* ... of the interface-level evaluation */
    double isdt_f, isdt_m;        /* 1/sqrt(dt) of those levels */
} pair_ctx;

/* Force on i from j (F_ij).  Returns 1 if the pair interacts.  Adds the
 * conservative part into *fcx.. for the virial and the potential into *u. */
static int pair_force(const pair_ctx *c, int32_t i, int32_t j, double *F, double *Fc, double *u,
                      double *rij)
{
    const orc_params *p = c->p;
    int32_t ti = c->tag[i], tj = c->tag[j];
    int kind = pair_kind(ti, tj);
    if (kind == PK_NONE) return 0;
    if (!(kind_level(kind) & c->level_mask)) return 0;
    double dx = c->x[3 * i] - c->x[3 * j];
    double dy = c->x[3 * i + 1] - c->x[3 * j + 1];
    double dz = c->x[3 * i + 2] - c->x[3 * j + 2];
    double dvx = c->v[3 * i] - c->v[3 * j];
    double dvy = c->v[3 * i + 1] - c->v[3 * j + 1];
    double dvz = c->v[3 * i + 2] - c->v[3 * j + 2];
    min_image(p, &dx, &dy, &dz, &dvx);
    double r2 = dx * dx + dy * dy + dz * dz;
    double r = sqrt(r2);
    rij[0] = dx; rij[1] = dy; rij[2] = dz;
    F[0] = F[1] = F[2] = 0.0;
    Fc[0] = Fc[1] = Fc[2] = 0.0;
    *u = 0.0;
    int hit = 0;
    if (kind == PK_DPD_FF || kind == PK_DPD_FW || kind == PK_DPD_FP) {
        if (r >= p->rc || r == 0.0) return 0;
        double a = kind == PK_DPD_FF ? p->a_ff : (kind == PK_DPD_FW ? p->a_fw : p->a_fp);
        int iface = kind == PK_DPD_FP;
        double ex = dx / r, ey = dy / r, ez = dz / r;
        double edotv = ex * dvx + ey * dvy + ez * dvz;
        double zeta = orc_zeta(p, c->id[i], c->id[j], iface ? c->n_time_m : c->n_time_f,
                               iface ? c->c_sub_m : c->c_sub_f);
        double fc, fd, fr;
        dpd_parts(a, p->gamma, p->sigma, p->rc, r, edotv, zeta, iface ? c->isdt_m : c->isdt_f,
                  &fc, &fd, &fr);
        double w = 1.0 - r / p->rc;
        *u = 0.5 * a * p->rc * w * w;
        if (iface && p->iface_lj) {
            const double rmin = pow(2.0, 1.0 / 6.0) * p->lj_sigma;
            fc = r < rmin ? lj_force(p->lj_eps, p->lj_sigma, r) : 0.0;
            *u = r < rmin ? lj_energy(p->lj_eps, p->lj_sigma, r) + p->lj_eps : 0.0;
        }
        double f = fc + fd + fr;
        F[0] = f * ex; F[1] = f * ey; F[2] = f * ez;
        Fc[0] = fc * ex; Fc[1] = fc * ey; Fc[2] = fc * ez;
        return 1;
    }
    /* platelet-platelet: LJ (Eq. 2) with the rest-distance exclusion, Morse +
     * receptor term between receptors of different platelets (Eq. 4) */
    if (!term_selected(p, ti, tj)) return 0;
    int32_t pi = ti & ~REC_BIT, pj = tj & ~REC_BIT;
    double fsum = 0.0, usum = 0.0;
    int lj_on = 1;
    if (pi == pj) {
        double ex0 = c->X0[3 * i] - c->X0[3 * j];
        double ey0 = c->X0[3 * i + 1] - c->X0[3 * j + 1];
        double ez0 = c->X0[3 * i + 2] - c->X0[3 * j + 2];
        double d0 = sqrt(ex0 * ex0 + ey0 * ey0 + ez0 * ez0);
        if (d0 < p->lj_excl) lj_on = 0;
    }
    if (lj_on && r < p->lj_rc && r > 0.0) {
        fsum += lj_force(p->lj_eps, p->lj_sigma, r);
        usum += lj_energy(p->lj_eps, p->lj_sigma, r) - lj_energy(p->lj_eps, p->lj_sigma, p->lj_rc);
        hit = 1;
    }
    if (pi != pj && (ti & REC_BIT) && (tj & REC_BIT) && r < p->m_rc && r > 0.0) {
        fsum += morse_force(p->m_D, p->m_alpha, p->m_r0, r);
        fsum += p->f_A * (1.0 - r / p->m_r0);
        usum += morse_energy(p->m_D, p->m_alpha, p->m_r0, r)
              - morse_energy(p->m_D, p->m_alpha, p->m_r0, p->m_rc);
        hit = 1;
    }
    if (!hit) return 0;
    F[0] = fsum * dx / r; F[1] = fsum * dy / r; F[2] = fsum * dz / r;
    Fc[0] = F[0]; Fc[1] = F[1]; Fc[2] = F[2];
    *u = usum;
    return 1;
}

/* Bond (Eq. 2): force on i from bond (i,j): -2 k_b (r - r0) e_ij. */
static void bond_force(const orc_params *p, const double *x, int32_t i, int32_t j, double r0,
                       double *F, double *u, double *rij)
{
    double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
    double dvx = 0.0;
    min_image(p, &dx, &dy, &dz, &dvx);
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double f = -2.0 * p->k_b * (r - r0);
    F[0] = f * dx / r; F[1] = f * dy / r; F[2] = f * dz / r;
    *u = p->k_b * (r - r0) * (r - r0);
    rij[0] = dx; rij[1] = dy; rij[2] = dz;
}

/* Angle (Eq. 2): U = k_a (theta - theta0)^2, theta the angle at vertex j
 * between r_ij = x_i - x_j and r_kj = x_k - x_j (minimum images).  With
 * c = cos theta, dc/dx_i = (e_kj - c e_ij) / |r_ij|, and theta = arccos c,
 * F_i = -dU/dx_i = 2 k_a (theta - theta0) / sin(theta) (e_kj - c e_ij) / |r_ij|,
 * F_k likewise with i and k exchanged, F_j = -F_i - F_k.  sin(theta) is held
 * at 1e-3 at least (the potential has a cone point at theta = pi, where the
 * direction of the force is undefined).  Returns the energy; rij, rkj get the
 * two arms (for the virial). */
static double angle_force(const orc_params *p, const double *x, int32_t i, int32_t j, int32_t k, double th0,
                          double *Fi, double *Fk, double *rij, double *rkj)
{
    double a[3], b[3], dv = 0.0;
    for (int d = 0; d < 3; ++d) { a[d] = x[3 * i + d] - x[3 * j + d]; b[d] = x[3 * k + d] - x[3 * j + d]; }
    min_image(p, &a[0], &a[1], &a[2], &dv);
    dv = 0.0;
    min_image(p, &b[0], &b[1], &b[2], &dv);
    double ra = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double rb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    double c = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (ra * rb);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c);
    double sn = sqrt(1.0 - c * c);
    if (sn < 1e-3) sn = 1e-3;
    double g = 2.0 * p->k_a * (th - th0) / sn;
    for (int d = 0; d < 3; ++d) {
        Fi[d] = g * (b[d] / rb - c * a[d] / ra) / ra;
        Fk[d] = g * (a[d] / ra - c * b[d] / rb) / rb;
        rij[d] = a[d];
        rkj[d] = b[d];
    }
    return p->k_a * (th - th0) * (th - th0);
}

/* Angle forces of every triplet selected for the platelet level, added to f
 * (3n); energy and virial into acc when given. */
static void add_angle_forces(const orc_params *p, const double *x, const int32_t *tag, double *f, orc_acc *acc)
{
    for (int32_t q = 0; q < p->n_angles; ++q) {
        int32_t i = p->angles[3 * q], j = p->angles[3 * q + 1], k = p->angles[3 * q + 2];
        if (!term_selected(p, tag[j], tag[j])) continue;
        double Fi[3], Fk[3], rij[3], rkj[3];
        double u = angle_force(p, x, i, j, k, p->theta0[q], Fi, Fk, rij, rkj);
        for (int d = 0; d < 3; ++d) {
            f[3 * i + d] += Fi[d];
            f[3 * k + d] += Fk[d];
            f[3 * j + d] -= Fi[d] + Fk[d];
        }
        if (acc) {
            acc->epot += u;
            acc_pair(acc, rij[0], rij[1], rij[2], Fi[0], Fi[1], Fi[2], Fi[0], Fi[1], Fi[2], 1.0);
            acc_pair(acc, rkj[0], rkj[1], rkj[2], Fk[0], Fk[1], Fk[2], Fk[0], Fk[1], Fk[2], 1.0);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* brute-force forces: every particle against every other                    */
/* ------------------------------------------------------------------------ */

/*
 * f[3n] <- sum of the forces of the levels in level_mask on every particle;
 * the fluid level includes the body force g x^ on non-wall particles.
 * acc (may be NULL) gets the potential energy and the pair virials.
 * bonds: nb pairs of particle indices (rows of x), r0: rest lengths.
 */
void orc_forces_brute(const orc_params *p, int32_t n, const double *x, const double *v,
                      const int32_t *id, const int32_t *tag, const double *X0,
                      int32_t nb, const int32_t *bonds, const double *r0,
                      uint32_t level_mask, uint32_t n_time_f, uint32_t c_sub_f, double dt_f,
                      uint32_t n_time_m, uint32_t c_sub_m, double dt_m,
                      double *f, double *acc_out)
{
    pair_ctx c = {p, n, x, v, X0, id, tag, level_mask, n_time_f, c_sub_f, n_time_m, c_sub_m,
                  1.0 / sqrt(dt_f), 1.0 / sqrt(dt_m)};
    orc_acc acc;
    memset(&acc, 0, sizeof acc);
#pragma omp parallel
    {
        orc_acc la;
        memset(&la, 0, sizeof la);
#pragma omp for schedule(dynamic, 64)
        for (int32_t i = 0; i < n; ++i) {
            double fi[3] = {0, 0, 0};
            for (int32_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double F[3], Fc[3], u, rij[3];
                if (!pair_force(&c, i, j, F, Fc, &u, rij)) continue;
                fi[0] += F[0]; fi[1] += F[1]; fi[2] += F[2];
                la.epot += 0.5 * u;
                acc_pair(&la, rij[0], rij[1], rij[2], F[0], F[1], F[2], Fc[0], Fc[1], Fc[2], 0.5);
            }
            if ((level_mask & LVL_FLUID) && tag[i] != TAG_WALL) fi[0] += p->g;
            f[3 * i] = fi[0]; f[3 * i + 1] = fi[1]; f[3 * i + 2] = fi[2];
        }
#pragma omp critical
        {
            acc.epot += la.epot;
            for (int k = 0; k < 9; ++k) { acc.vir[k] += la.vir[k]; acc.vir_c[k] += la.vir_c[k]; }
        }
    }
    if (level_mask & LVL_PLT) {
        for (int32_t b = 0; b < nb; ++b) {
            int32_t i = bonds[2 * b], j = bonds[2 * b + 1];
            double F[3], u, rij[3];
            if (!term_selected(p, tag[i], tag[j])) continue;
            bond_force(p, x, i, j, r0[b], F, &u, rij);
            for (int k = 0; k < 3; ++k) { f[3 * i + k] += F[k]; f[3 * j + k] -= F[k]; }
            acc.epot += u;
            acc_pair(&acc, rij[0], rij[1], rij[2], F[0], F[1], F[2], F[0], F[1], F[2], 1.0);
        }
        add_angle_forces(p, x, tag, f, &acc);
    }
    if (acc_out) {
        acc_out[0] = acc.epot;
        memcpy(acc_out + 1, acc.vir, 9 * sizeof(double));
        memcpy(acc_out + 10, acc.vir_c, 9 * sizeof(double));
    }
}

/*
 * Pair forces F_ij (Eq. 1-4, the levels in level_mask) for npair listed
 * pairs (pi[q], pj[q]) of particle rows: F[3 q ..] = force on pi[q] from
 * pj[q] (zero for a pair that does not interact).  Bonds and angles are not
 * pairs of this kind and are not included.
 */
void orc_pair_forces(const orc_params *p, int32_t n, const double *x, const double *v,
                     const int32_t *id, const int32_t *tag, const double *X0,
                     uint32_t level_mask, uint32_t n_time_f, uint32_t c_sub_f, double dt_f,
                     uint32_t n_time_m, uint32_t c_sub_m, double dt_m,
                     int64_t npair, const int32_t *pi, const int32_t *pj, double *F_out)
{
    pair_ctx c = {p, n, x, v, X0, id, tag, level_mask, n_time_f, c_sub_f, n_time_m, c_sub_m,
                  1.0 / sqrt(dt_f), 1.0 / sqrt(dt_m)};
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < npair; ++q) {
        double F[3] = {0, 0, 0}, Fc[3], u, rij[3];
        if (!pair_force(&c, pi[q], pj[q], F, Fc, &u, rij)) F[0] = F[1] = F[2] = 0.0;
        F_out[3 * q] = F[0]; F_out[3 * q + 1] = F[1]; F_out[3 * q + 2] = F[2];
    }
}

/* ------------------------------------------------------------------------ */
/* cell-list forces on selected particles (same definition, fewer pairs)     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nc[3];
    double lo[3], h[3];
    int32_t *head, *next;
} cells_t;

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void cells_build(const orc_params *p, int32_t n, const double *x, double cell, cells_t *cl)
{
    double lo[3] = {0.0, 0.0, 0.0}, hi[3] = {p->L[0], p->L[1], p->L[2]};
    if (p->walls) {
        /* walls extend the binned region in y; find the actual extent */
        double ymin = 0.0, ymax = p->L[1];
        for (int32_t i = 0; i < n; ++i) {
            if (x[3 * i + 1] < ymin) ymin = x[3 * i + 1];
            if (x[3 * i + 1] > ymax) ymax = x[3 * i + 1];
        }
        lo[1] = ymin - 1e-9; hi[1] = ymax + 1e-9;
    }
    for (int d = 0; d < 3; ++d) {
        cl->lo[d] = lo[d];
        cl->nc[d] = (int)floor((hi[d] - lo[d]) / cell);
        if (cl->nc[d] < 1) cl->nc[d] = 1;
        cl->h[d] = (hi[d] - lo[d]) / cl->nc[d];
    }
    size_t nct = (size_t)cl->nc[0] * cl->nc[1] * cl->nc[2];
    cl->head = (int32_t *)malloc(nct * sizeof(int32_t));
    cl->next = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    for (size_t c = 0; c < nct; ++c) cl->head[c] = -1;
    /* insert in descending index order so each cell lists ascending indices */
    for (int32_t i = n - 1; i >= 0; --i) {
        int ci[3];
        for (int d = 0; d < 3; ++d)
            ci[d] = clampi((int)floor((x[3 * i + d] - cl->lo[d]) / cl->h[d]), 0, cl->nc[d] - 1);
        size_t c = ((size_t)ci[2] * cl->nc[1] + ci[1]) * cl->nc[0] + ci[0];
        cl->next[i] = cl->head[c];
        cl->head[c] = i;
    }
}

static void cells_free(cells_t *cl) { free(cl->head); free(cl->next); }

/* Visit every particle j in cells within reach R of particle i (each j once). */
typedef void (*visit_fn)(void *ud, int32_t j);

static void cells_visit(const orc_params *p, const cells_t *cl, const double *xi, double R,
                        char *seen, int32_t *seen_list, int32_t *nseen, visit_fn fn, void *ud)
{
    int ci[3], reach[3];
    for (int d = 0; d < 3; ++d) {
        ci[d] = clampi((int)floor((xi[d] - cl->lo[d]) / cl->h[d]), 0, cl->nc[d] - 1);
        reach[d] = (int)ceil(R / cl->h[d]);
    }
    int periodic_y = !p->walls;
    /* Lees-Edwards: images across y are shifted in x by a non-cell offset;
     * for rows that reach across the y boundary, scan the full x range. */
    for (int oz = -reach[2]; oz <= reach[2]; ++oz) {
        for (int oy = -reach[1]; oy <= reach[1]; ++oy) {
            int cy = ci[1] + oy;
            int crosses = cy < 0 || cy >= cl->nc[1];
            if (crosses && !periodic_y) continue;
            cy = ((cy % cl->nc[1]) + cl->nc[1]) % cl->nc[1];
            int cz = ((ci[2] + oz) % cl->nc[2] + cl->nc[2]) % cl->nc[2];
            int full_x = p->le && crosses;
            int x_lo = full_x ? 0 : ci[0] - reach[0];
            int x_hi = full_x ? cl->nc[0] - 1 : ci[0] + reach[0];
            for (int ox = x_lo; ox <= x_hi; ++ox) {
                int cx = ((ox % cl->nc[0]) + cl->nc[0]) % cl->nc[0];
                size_t c = ((size_t)cz * cl->nc[1] + cy) * cl->nc[0] + cx;
                for (int32_t j = cl->head[c]; j >= 0; j = cl->next[j]) {
                    if (seen[j]) continue;
                    seen[j] = 1;
                    seen_list[(*nseen)++] = j;
                    fn(ud, j);
                }
            }
        }
    }
    for (int32_t k = 0; k < *nseen; ++k) seen[seen_list[k]] = 0;
    *nseen = 0;
}

typedef struct {
    const pair_ctx *c;
    int32_t i;
    double f[3];
    int32_t *cands;
    int32_t ncand;
} visit_state;

static void collect_cand(void *ud, int32_t j)
{
    visit_state *s = (visit_state *)ud;
    if (j != s->i) s->cands[s->ncand++] = j;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Forces (levels in level_mask) on the ns particles listed in sample[] (or on
 * all particles when sample == NULL, ns == n), found through a cell list.
 * Partners are summed in ascending index order, like orc_forces_brute.
 * Bond terms need a CSR adjacency: bond_off[n+1], bond_nbr[], bond_r0[]
 * (each bond listed under both ends); pass bond_off = NULL for none.
 */
void orc_forces_cells(const orc_params *p, int32_t n, const double *x, const double *v,
                      const int32_t *id, const int32_t *tag, const double *X0,
                      const int32_t *bond_off, const int32_t *bond_nbr, const double *bond_r0,
                      uint32_t level_mask, uint32_t n_time_f, uint32_t c_sub_f, double dt_f,
                      uint32_t n_time_m, uint32_t c_sub_m, double dt_m,
                      int32_t ns, const int32_t *sample, double *f_out, double *acc_out)
{
    pair_ctx c = {p, n, x, v, X0, id, tag, level_mask, n_time_f, c_sub_f, n_time_m, c_sub_m,
                  1.0 / sqrt(dt_f), 1.0 / sqrt(dt_m)};
    double cell = p->rc;
    cells_t cl;
    cells_build(p, n, x, cell, &cl);
    double Rmax_plt = p->lj_rc > p->m_rc ? p->lj_rc : p->m_rc;
    orc_acc acc;
    memset(&acc, 0, sizeof acc);
    /* angle terms: every triplet once into a full array, read per sample */
    double *fang = NULL;
    if ((level_mask & LVL_PLT) && p->n_angles > 0) {
        fang = (double *)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
        add_angle_forces(p, x, tag, fang, NULL);
    }
#pragma omp parallel
    {
        orc_acc la;
        memset(&la, 0, sizeof la);
        char *seen = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
        int32_t *seen_list = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int32_t *cands = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
        int32_t nseen = 0;
#pragma omp for schedule(dynamic, 16)
        for (int32_t s = 0; s < ns; ++s) {
            int32_t i = sample ? sample[s] : s;
            visit_state st = {&c, i, {0, 0, 0}, cands, 0};
            double R = p->rc;
            if (tag[i] >= 0 && (level_mask & LVL_PLT)) R = Rmax_plt;
            cells_visit(p, &cl, x + 3 * i, R, seen, seen_list, &nseen, collect_cand, &st);
            qsort(cands, (size_t)st.ncand, sizeof(int32_t), cmp_i32);
            double fi[3] = {0, 0, 0};
            for (int32_t k = 0; k < st.ncand; ++k) {
                double F[3], Fc[3], u, rij[3];
                if (!pair_force(&c, i, cands[k], F, Fc, &u, rij)) continue;
                fi[0] += F[0]; fi[1] += F[1]; fi[2] += F[2];
                /* each pair is visited from both ends: half of its energy and virial per visit */
                la.epot += 0.5 * u;
                acc_pair(&la, rij[0], rij[1], rij[2], F[0], F[1], F[2], Fc[0], Fc[1], Fc[2], 0.5);
            }
            if ((level_mask & LVL_FLUID) && tag[i] != TAG_WALL) fi[0] += p->g;
            if ((level_mask & LVL_PLT) && bond_off) {
                for (int32_t b = bond_off[i]; b < bond_off[i + 1]; ++b) {
                    double F[3], u, rij[3];
                    if (!term_selected(p, tag[i], tag[bond_nbr[b]])) continue;
                    bond_force(p, x, i, bond_nbr[b], bond_r0[b], F, &u, rij);
                    fi[0] += F[0]; fi[1] += F[1]; fi[2] += F[2];
                }
            }
            if (fang) { fi[0] += fang[3 * i]; fi[1] += fang[3 * i + 1]; fi[2] += fang[3 * i + 2]; }
            f_out[3 * s] = fi[0]; f_out[3 * s + 1] = fi[1]; f_out[3 * s + 2] = fi[2];
        }
        free(seen); free(seen_list); free(cands);
#pragma omp critical
        {
            acc.epot += la.epot;
            for (int k = 0; k < 9; ++k) { acc.vir[k] += la.vir[k]; acc.vir_c[k] += la.vir_c[k]; }
        }
    }
    cells_free(&cl);
    free(fang);
    /* pair sums of every particle (sample == NULL) give the system's pair
     * energy and virial; bond terms are not included */
    if (acc_out) {
        acc_out[0] = acc.epot;
        memcpy(acc_out + 1, acc.vir, 9 * sizeof(double));
        memcpy(acc_out + 10, acc.vir_c, 9 * sizeof(double));
    }
}

/* ------------------------------------------------------------------------ */
/* neighbour sets under the FP32 predicate                                   */
/* ------------------------------------------------------------------------ */

/*
 * The list predicate is evaluated in binary32, operation by operation, so a
 * device implementation of the same sequence produces the identical set:
 *   d = a - b; if d > L/2: d = (a - L) - b; elif d < -L/2: d = a - (b - L)
 *   Lees-Edwards y-crossing: xj' = xj -/+ delta, wrapped once into [0,Lx),
 *   then the x rule above;  r2 = (dx*dx + dy*dy) + dz*dz  (no FMA)
 * This file is compiled with -ffp-contract=off.
 */
static float f32_img(float a, float b, float L, float hL)
{
    float d = a - b;
    if (d > hL) d = (a - L) - b;
    else if (d < -hL) d = a - (b - L);
    return d;
}

float orc_r2_f32(const float *xi, const float *xj, const float *Lf, int32_t walls, int32_t le,
                 float delta)
{
    float hx = 0.5f * Lf[0], hy = 0.5f * Lf[1], hz = 0.5f * Lf[2];
    float xj0 = xj[0];
    float dy;
    if (walls) {
        dy = xi[1] - xj[1];
    } else if (le) {
        dy = xi[1] - xj[1];
        if (dy > hy) {
            dy = (xi[1] - Lf[1]) - xj[1];
            xj0 = xj0 + delta;
            if (xj0 >= Lf[0]) xj0 = xj0 - Lf[0];
        } else if (dy < -hy) {
            dy = xi[1] - (xj[1] - Lf[1]);
            xj0 = xj0 - delta;
            if (xj0 < 0.0f) xj0 = xj0 + Lf[0];
        }
    } else {
        dy = f32_img(xi[1], xj[1], Lf[1], hy);
    }
    float dx = f32_img(xi[0], xj0, Lf[0], hx);
    float dz = f32_img(xi[2], xj[2], Lf[2], hz);
    float r2 = dx * dx;
    r2 = r2 + dy * dy;
    r2 = r2 + dz * dz;
    return r2;
}

/* List kinds: 0 = fluid level (plasma-plasma, plasma-wall), 1 = interface
 * (plasma/wall - platelet), 2 = platelet LJ (rest-distance exclusion),
 * 3 = receptor Morse (different platelets). */
static int in_kind(int kind, int32_t ti, int32_t tj, const float *X0i, const float *X0j, float excl2)
{
    int pk = pair_kind(ti, tj);
    switch (kind) {
    case 0: return pk == PK_DPD_FF || pk == PK_DPD_FW;
    case 1: return pk == PK_DPD_FP;
    case 2: {
        if (pk != PK_PLT) return 0;
        if ((ti & ~REC_BIT) != (tj & ~REC_BIT)) return 1;
        float ex = X0i[0] - X0j[0], ey = X0i[1] - X0j[1], ez = X0i[2] - X0j[2];
        float d2 = ex * ex;
        d2 = d2 + ey * ey;
        d2 = d2 + ez * ez;
        return !(d2 < excl2);
    }
    case 3:
        return pk == PK_PLT && (ti & REC_BIT) && (tj & REC_BIT) &&
               (ti & ~REC_BIT) != (tj & ~REC_BIT);
    default: return 0;
    }
}

/*
 * All unordered pairs (i<j by index) of list kind `kind` with r2 < cut2 under
 * the FP32 predicate.  Brute force over all pairs; writes at most cap pairs
 * into out[2*cap] and returns the total count.
 */
int64_t orc_pairs_f32(int32_t n, const float *x32, const int32_t *tag, const float *X0f,
                      const float *Lf, int32_t walls, int32_t le, float delta,
                      int32_t kind, float cut2, float excl2, int64_t cap, int32_t *out)
{
    int64_t cnt = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = i + 1; j < n; ++j) {
            if (!in_kind(kind, tag[i], tag[j], X0f + 3 * i, X0f + 3 * j, excl2)) continue;
            float r2 = orc_r2_f32(x32 + 3 * i, x32 + 3 * j, Lf, walls, le, delta);
            if (r2 < cut2) {
                if (cnt < cap) { out[2 * cnt] = i; out[2 * cnt + 1] = j; }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* integrators (Table 1)                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n, nb;
    double *x, *v;             /* [3n] */
    const int32_t *id, *tag;
    const double *X0;
    const int32_t *bonds;      /* [2nb] */
    const double *r0;
} orc_state;

/*
 * Wrap / bounce a particle after a drift; Lees-Edwards images move x and v_x.
 * No-slip walls (Sec. 3.1) bounce back: the particle retraces the part of the
 * drift it spent beyond the wall (time tau = overshoot / v_y) with reversed
 * velocity.  This equals a continuous-time reflection, so the result does not
 * depend on how a drift is split into substeps.
 */
static void apply_boundaries(const orc_params *p, double *xi, double *vi)
{
    const double Lx = p->L[0], Ly = p->L[1], Lz = p->L[2];
    if (p->walls) {
        double wall = -1.0;
        if (xi[1] < 0.0) wall = 0.0;
        else if (xi[1] >= Ly) wall = Ly;
        if (wall >= 0.0) {
            double tau = vi[1] != 0.0 ? (xi[1] - wall) / vi[1] : 0.0;
            xi[0] -= 2.0 * vi[0] * tau;
            xi[2] -= 2.0 * vi[2] * tau;
            xi[1] = 2.0 * wall - xi[1];
            vi[0] = -vi[0]; vi[1] = -vi[1]; vi[2] = -vi[2];
        }
    } else if (p->le) {
        if (xi[1] >= Ly) { xi[1] -= Ly; xi[0] -= p->le_offset; vi[0] -= p->le_rate * Ly; }
        else if (xi[1] < 0.0) { xi[1] += Ly; xi[0] += p->le_offset; vi[0] += p->le_rate * Ly; }
    } else {
        xi[1] -= Ly * floor(xi[1] / Ly);
    }
    xi[0] -= Lx * floor(xi[0] / Lx);
    xi[2] -= Lz * floor(xi[2] / Lz);
}

typedef struct {
    int32_t *off, *nbr;
    double *r0;
} bond_csr_t;

/* Each bond listed under both of its ends, partners in ascending order. */
static void bond_csr_build(int32_t n, int32_t nb, const int32_t *bonds, const double *r0,
                           bond_csr_t *csr)
{
    csr->off = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    csr->nbr = (int32_t *)malloc((size_t)(2 * nb + 1) * sizeof(int32_t));
    csr->r0 = (double *)malloc((size_t)(2 * nb + 1) * sizeof(double));
    for (int32_t b = 0; b < nb; ++b) { csr->off[bonds[2 * b] + 1]++; csr->off[bonds[2 * b + 1] + 1]++; }
    for (int32_t i = 0; i < n; ++i) csr->off[i + 1] += csr->off[i];
    int32_t *fill = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t b = 0; b < nb; ++b) {
        int32_t i = bonds[2 * b], j = bonds[2 * b + 1];
        int32_t pi = csr->off[i] + fill[i]++, pj = csr->off[j] + fill[j]++;
        csr->nbr[pi] = j; csr->r0[pi] = r0[b];
        csr->nbr[pj] = i; csr->r0[pj] = r0[b];
    }
    free(fill);
    for (int32_t i = 0; i < n; ++i) {  /* insertion sort each row by partner */
        for (int32_t a = csr->off[i] + 1; a < csr->off[i + 1]; ++a) {
            int32_t kj = csr->nbr[a]; double kr = csr->r0[a]; int32_t b = a - 1;
            while (b >= csr->off[i] && csr->nbr[b] > kj) { csr->nbr[b + 1] = csr->nbr[b]; csr->r0[b + 1] = csr->r0[b]; --b; }
            csr->nbr[b + 1] = kj; csr->r0[b + 1] = kr;
        }
    }
}

static void eval_level(orc_params *p, const orc_state *s, const bond_csr_t *csr, unsigned mask,
                       uint32_t nt, uint32_t cs, double dt_f, double dt_m, double *f)
{
    orc_forces_cells(p, s->n, s->x, s->v, s->id, s->tag, s->X0, csr->off, csr->nbr, csr->r0,
                     mask, nt, cs, dt_f, nt, cs, dt_m, s->n, NULL, f, NULL);
}

static void kick(const orc_state *s, const double *f, double h)
{
    for (int32_t i = 0; i < s->n; ++i) {
        if (s->tag[i] == TAG_WALL) continue;
        for (int k = 0; k < 3; ++k) s->v[3 * i + k] += h * f[3 * i + k];
    }
}

static void drift(orc_params *p, const orc_state *s, double dt, double *t)
{
    *t += dt;
    if (p->le) {
        p->le_offset = fmod(p->le_rate * p->L[1] * (*t), p->L[0]);
        if (p->le_offset < 0.0) p->le_offset += p->L[0];
    }
    for (int32_t i = 0; i < s->n; ++i) {
        if (s->tag[i] == TAG_WALL) continue;
        for (int k = 0; k < 3; ++k) s->x[3 * i + k] += dt * s->v[3 * i + k];
        apply_boundaries(p, s->x + 3 * i, s->v + 3 * i);
    }
}

/*
 * Multi-level RESPA (Table 1), read symmetrically.  With k_m = k_p = 1 it is
 * plain velocity-Verlet (STS).  The fluid level holds plasma-plasma and
 * plasma-wall DPD plus the body force; the interface level the DPD pairs
 * between platelets and plasma/wall; the platelet level bonds, LJ, Morse.
 * Forces at time t = n dt_f + c dt_m draw zeta with time index (n, c).
 * t0: time at entry (sets the Lees-Edwards offset); n0: outer index at entry.
 * f_f, f_m, f_p: level forces [3n] -- on entry the forces at the entry state
 * (pass compute_initial = 1 to have them evaluated), on exit the final ones.
 */
void orc_run_respa(orc_params *p, int32_t n, int32_t nb, double *x, double *v,
                   const int32_t *id, const int32_t *tag, const double *X0,
                   const int32_t *bonds, const double *r0,
                   double dt_f, int32_t k_m, int32_t k_p, int32_t n_outer,
                   uint32_t n0, double t0, int32_t compute_initial,
                   double *f_f, double *f_m, double *f_p)
{
    orc_state s = {n, nb, x, v, id, tag, X0, bonds, r0};
    bond_csr_t csr;
    bond_csr_build(n, nb, bonds, r0, &csr);
    double dt_m = dt_f / k_m, dt_p = dt_m / k_p;
    double t = t0;
    if (p->le) {
        p->le_offset = fmod(p->le_rate * p->L[1] * t, p->L[0]);
        if (p->le_offset < 0.0) p->le_offset += p->L[0];
    }
    if (compute_initial) {
        eval_level(p, &s, &csr, LVL_FLUID, n0, 0, dt_f, dt_m, f_f);
        eval_level(p, &s, &csr, LVL_IFACE, n0, 0, dt_f, dt_m, f_m);
        eval_level(p, &s, &csr, LVL_PLT, n0, 0, dt_f, dt_m, f_p);
    }
    for (int32_t so = 0; so < n_outer; ++so) {
        uint32_t nn = n0 + (uint32_t)so;
        kick(&s, f_f, 0.5 * dt_f);
        for (int32_t c = 0; c < k_m; ++c) {
            kick(&s, f_m, 0.5 * dt_m);
            for (int32_t q = 0; q < k_p; ++q) {
                kick(&s, f_p, 0.5 * dt_p);
                drift(p, &s, dt_p, &t);
                eval_level(p, &s, &csr, LVL_PLT, 0, 0, dt_f, dt_m, f_p);
                kick(&s, f_p, 0.5 * dt_p);
            }
            uint32_t nt = (c + 1 == k_m) ? nn + 1 : nn;
            uint32_t cs = (c + 1 == k_m) ? 0u : (uint32_t)(c + 1);
            eval_level(p, &s, &csr, LVL_IFACE, nt, cs, dt_f, dt_m, f_m);
            kick(&s, f_m, 0.5 * dt_m);
        }
        eval_level(p, &s, &csr, LVL_FLUID, nn + 1, 0, dt_f, dt_m, f_f);
        kick(&s, f_f, 0.5 * dt_f);
    }
    free(csr.off); free(csr.nbr); free(csr.r0);
}

/*
 * AI-MTS (Sec. 3.3): Table 1 with a step ratio k_p per platelet (plt_k[P]).
 * The interface step is cut into K = lcm(k_p) fine substeps dts = dt_m / K,
 * and every mobile particle drifts by dts in each of them.  A platelet-level
 * term (a bond, an LJ or a Morse pair) belongs to the grid of the finer of
 * its two platelets, c = max(k_i, k_j), and is integrated by velocity-Verlet
 * with the step dt_m / c on that grid: a half kick at the start of the
 * interface step, a full kick (closing + opening) at each interior point
 * K/c, 2K/c, ..., and a half kick at the end.  The kicks of the terms due at
 * one point are summed as the impulse J = sum_c (dt_m / c) F^(c).  With all
 * k_p equal this is the RESPA loop above.  f_p holds J of the last point
 * (all terms due) instead of a force.
 */
static void eval_impulse(orc_params *p, const orc_state *s, const bond_csr_t *csr, const int32_t *plt_k,
                         int32_t P, int32_t K, int32_t qe, double dt_m, double *tmp, double *J)
{
    memset(J, 0, (size_t)3 * s->n * sizeof(double));
    for (int32_t c = 1; c <= K; ++c) {
        if (K % c != 0 || qe % (K / c) != 0) continue;
        int used = 0;
        for (int32_t q = 0; q < P; ++q) used |= plt_k[q] == c;
        if (!used) continue;
        p->plt_k = plt_k;
        p->lvl_k = c;
        eval_level(p, s, csr, LVL_PLT, 0, 0, 1.0, dt_m, tmp);
        p->plt_k = NULL;
        for (int64_t k = 0; k < 3 * (int64_t)s->n; ++k) J[k] += dt_m / c * tmp[k];
    }
}

void orc_run_ai_respa(orc_params *p, int32_t n, int32_t nb, double *x, double *v,
                      const int32_t *id, const int32_t *tag, const double *X0,
                      const int32_t *bonds, const double *r0, const int32_t *plt_k, int32_t P, int32_t K,
                      double dt_f, int32_t k_m, int32_t n_outer, uint32_t n0, double t0,
                      int32_t compute_initial, double *f_f, double *f_m, double *f_p)
{
    orc_state s = {n, nb, x, v, id, tag, X0, bonds, r0};
    bond_csr_t csr;
    bond_csr_build(n, nb, bonds, r0, &csr);
    double *tmp = (double *)malloc((size_t)3 * (n > 0 ? n : 1) * sizeof(double));
    const double dt_m = dt_f / k_m, dts = dt_m / K;
    double t = t0;
    if (p->le) {
        p->le_offset = fmod(p->le_rate * p->L[1] * t, p->L[0]);
        if (p->le_offset < 0.0) p->le_offset += p->L[0];
    }
    if (compute_initial) {
        eval_level(p, &s, &csr, LVL_FLUID, n0, 0, dt_f, dt_m, f_f);
        eval_level(p, &s, &csr, LVL_IFACE, n0, 0, dt_f, dt_m, f_m);
        eval_impulse(p, &s, &csr, plt_k, P, K, K, dt_m, tmp, f_p);
    }
    for (int32_t so = 0; so < n_outer; ++so) {
        uint32_t nn = n0 + (uint32_t)so;
        kick(&s, f_f, 0.5 * dt_f);
        for (int32_t c = 0; c < k_m; ++c) {
            kick(&s, f_m, 0.5 * dt_m);
            for (int32_t q = 0; q < K; ++q) {
                kick(&s, f_p, q == 0 ? 0.5 : 1.0);
                drift(p, &s, dts, &t);
                eval_impulse(p, &s, &csr, plt_k, P, K, q + 1, dt_m, tmp, f_p);
            }
            kick(&s, f_p, 0.5);
            uint32_t nt = (c + 1 == k_m) ? nn + 1 : nn;
            uint32_t cs = (c + 1 == k_m) ? 0u : (uint32_t)(c + 1);
            eval_level(p, &s, &csr, LVL_IFACE, nt, cs, dt_f, dt_m, f_m);
            kick(&s, f_m, 0.5 * dt_m);
        }
        eval_level(p, &s, &csr, LVL_FLUID, nn + 1, 0, dt_f, dt_m, f_f);
        kick(&s, f_f, 0.5 * dt_f);
    }
    free(tmp);
    free(csr.off); free(csr.nbr); free(csr.r0);
}

/*
 * Table 1 as printed: the platelet subsystem in nested sublevels inside each
 * interface substep.  Level 1 takes one step dt_1 = dt_m per interface
 * substep (the flowing platelets), level l > 1 takes kr[l - 1] steps
 * dt_l = dt_{l-1} / kr[l - 1] inside each step of level l - 1, and the
 * innermost level C (the aggregating platelets) drifts every particle.  A
 * step of level l: half kick with the level-l forces, the substeps of the
 * next level (or the drift), the level-l forces at the new state, half kick.
 * The level-l forces are the platelet-level terms whose finer platelet is on
 * level l (plt_level[P] in 1..C).
 */
typedef struct {
    orc_params *p;
    const orc_state *s;
    const bond_csr_t *csr;
    int32_t C;
    const int32_t *kr;          /* kr[0] = 1, kr[l - 1] = dt_{l-1} / dt_l */
    const int32_t *pK;          /* per platelet: dt_m / dt of its level */
    int32_t *Kl;                /* per level: dt_m / dt_l */
    double **F;                 /* per level forces [3n] */
    double dt_m;
    double *t;
} nest_ctx;

static void nest_forces(nest_ctx *c, int32_t l)
{
    c->p->plt_k = c->pK;
    c->p->lvl_k = c->Kl[l - 1];
    eval_level(c->p, c->s, c->csr, LVL_PLT, 0, 0, 1.0, c->dt_m, c->F[l - 1]);
    c->p->plt_k = NULL;
}

static void nest_step(nest_ctx *c, int32_t l, double dt_l)
{
    kick(c->s, c->F[l - 1], 0.5 * dt_l);
    if (l == c->C) {
        drift(c->p, c->s, dt_l, c->t);
    } else {
        const int32_t k = c->kr[l];
        for (int32_t q = 0; q < k; ++q) nest_step(c, l + 1, dt_l / k);
    }
    nest_forces(c, l);
    kick(c->s, c->F[l - 1], 0.5 * dt_l);
}

void orc_run_nested(orc_params *p, int32_t n, int32_t nb, double *x, double *v,
                    const int32_t *id, const int32_t *tag, const double *X0,
                    const int32_t *bonds, const double *r0, const int32_t *plt_level, int32_t P,
                    const int32_t *kr, int32_t C, double dt_f, int32_t k_m, int32_t n_outer, uint32_t n0,
                    double t0, double *f_f, double *f_m)
{
    orc_state s = {n, nb, x, v, id, tag, X0, bonds, r0};
    bond_csr_t csr;
    bond_csr_build(n, nb, bonds, r0, &csr);
    const double dt_m = dt_f / k_m;
    double t = t0;
    if (p->le) {
        p->le_offset = fmod(p->le_rate * p->L[1] * t, p->L[0]);
        if (p->le_offset < 0.0) p->le_offset += p->L[0];
    }
    int32_t *Kl = (int32_t *)malloc((size_t)C * sizeof(int32_t));
    int32_t *pK = (int32_t *)malloc((size_t)(P > 0 ? P : 1) * sizeof(int32_t));
    double **F = (double **)malloc((size_t)C * sizeof(double *));
    Kl[0] = 1;
    for (int32_t l = 1; l < C; ++l) Kl[l] = Kl[l - 1] * kr[l];
    for (int32_t q = 0; q < P; ++q) pK[q] = Kl[plt_level[q] - 1];
    for (int32_t l = 0; l < C; ++l) F[l] = (double *)calloc((size_t)3 * (n > 0 ? n : 1), sizeof(double));
    nest_ctx c = {p, &s, &csr, C, kr, pK, Kl, F, dt_m, &t};
    eval_level(p, &s, &csr, LVL_FLUID, n0, 0, dt_f, dt_m, f_f);
    eval_level(p, &s, &csr, LVL_IFACE, n0, 0, dt_f, dt_m, f_m);
    for (int32_t l = 1; l <= C; ++l) nest_forces(&c, l);
    for (int32_t so = 0; so < n_outer; ++so) {
        uint32_t nn = n0 + (uint32_t)so;
        kick(&s, f_f, 0.5 * dt_f);
        for (int32_t cm = 0; cm < k_m; ++cm) {
            kick(&s, f_m, 0.5 * dt_m);
            nest_step(&c, 1, dt_m);
            uint32_t nt = (cm + 1 == k_m) ? nn + 1 : nn;
            uint32_t cs = (cm + 1 == k_m) ? 0u : (uint32_t)(cm + 1);
            eval_level(p, &s, &csr, LVL_IFACE, nt, cs, dt_f, dt_m, f_m);
            kick(&s, f_m, 0.5 * dt_m);
        }
        eval_level(p, &s, &csr, LVL_FLUID, nn + 1, 0, dt_f, dt_m, f_f);
        kick(&s, f_f, 0.5 * dt_f);
    }
    for (int32_t l = 0; l < C; ++l) free(F[l]);
    free(F); free(Kl); free(pK);
    free(csr.off); free(csr.nbr); free(csr.r0);
}

/*
 * Single time step (STS, the reference run of Sec. 4.1): velocity-Verlet in
 * which all forces of Eq. 1-4 are evaluated together, at the drifted
 * positions and the half-kicked velocities:
 *   v += dt/2 F;  x += dt v;  F = F(x, v) at time index (n+1, 0);  v += dt/2 F.
 * f: total force [3n] at entry (compute_initial = 1: evaluated first) and exit.
 */
void orc_run_sts(orc_params *p, int32_t n, int32_t nb, double *x, double *v,
                 const int32_t *id, const int32_t *tag, const double *X0,
                 const int32_t *bonds, const double *r0,
                 double dt, int32_t n_steps, uint32_t n0, double t0, int32_t compute_initial,
                 double *f)
{
    orc_state s = {n, nb, x, v, id, tag, X0, bonds, r0};
    bond_csr_t csr;
    bond_csr_build(n, nb, bonds, r0, &csr);
    double t = t0;
    if (p->le) {
        p->le_offset = fmod(p->le_rate * p->L[1] * t, p->L[0]);
        if (p->le_offset < 0.0) p->le_offset += p->L[0];
    }
    if (compute_initial) eval_level(p, &s, &csr, LVL_FLUID | LVL_IFACE | LVL_PLT, n0, 0, dt, dt, f);
    for (int32_t k = 0; k < n_steps; ++k) {
        kick(&s, f, 0.5 * dt);
        drift(p, &s, dt, &t);
        eval_level(p, &s, &csr, LVL_FLUID | LVL_IFACE | LVL_PLT, n0 + (uint32_t)k + 1, 0, dt, dt, f);
        kick(&s, f, 0.5 * dt);
    }
    free(csr.off); free(csr.nbr); free(csr.r0);
}

/* ------------------------------------------------------------------------ */
/* observables (Sec. 4.2)                                                     */
/* ------------------------------------------------------------------------ */

/*
 * out[0..2]  total momentum of mobile particles
 * out[3]     kinetic energy  1/2 sum m v^2 (mobile)
 * out[4]     kinetic temperature of the peculiar velocity  sum m|v-u|^2 / N_dof,
 *            N_dof = 3N - 3 with periodic/Lees-Edwards y, 3N with walls;
 *            u = shear_rate (y - Ly/2) x^ under Lees-Edwards; with walls u is the
 *            mean v_x of the y-bin (nbins bins over [0, Ly)) when nbins > 0
 * out[5..13] peculiar kinetic tensor sum m (v-u)_a (v-u)_b
 * nbins > 0: prof_vx[nbins], prof_rho[nbins] -- mean v_x and number density of
 *            mobile plasma in equal y-bins over [0, Ly)
 */
void orc_kinetics(const orc_params *p, int32_t n, const double *x, const double *v,
                  const int32_t *tag, int32_t nbins, double *out, double *prof_vx, double *prof_rho)
{
    double *bin_u = NULL;
    if (nbins > 0) {
        double *cnt = (double *)calloc((size_t)nbins, sizeof(double));
        double *cntm = (double *)calloc((size_t)nbins, sizeof(double));
        double *sum = (double *)calloc((size_t)nbins, sizeof(double));
        bin_u = (double *)calloc((size_t)nbins, sizeof(double));
        for (int b = 0; b < nbins; ++b) prof_vx[b] = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            if (tag[i] == TAG_WALL) continue;
            double y = x[3 * i + 1];
            if (y < 0.0 || y >= p->L[1]) continue;
            int b = (int)floor(y / p->L[1] * nbins);
            if (b >= nbins) b = nbins - 1;
            cntm[b] += 1.0;
            sum[b] += v[3 * i];
            if (tag[i] == TAG_FLUID) { cnt[b] += 1.0; prof_vx[b] += v[3 * i]; }
        }
        double vol = p->L[0] * p->L[2] * p->L[1] / nbins;
        for (int b = 0; b < nbins; ++b) {
            prof_rho[b] = cnt[b] / vol;
            prof_vx[b] = cnt[b] > 0 ? prof_vx[b] / cnt[b] : 0.0;
            bin_u[b] = cntm[b] > 0 ? sum[b] / cntm[b] : 0.0;
        }
        free(cnt); free(cntm); free(sum);
    }
    double P[3] = {0, 0, 0}, ke = 0.0, K[9] = {0};
    int64_t nm = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (tag[i] == TAG_WALL) continue;
        ++nm;
        double u = 0.0;
        if (p->le) {
            u = p->le_rate * (x[3 * i + 1] - 0.5 * p->L[1]);
        } else if (p->walls && bin_u) {
            double y = x[3 * i + 1];
            int b = (int)floor(y / p->L[1] * nbins);
            if (b < 0) b = 0;
            if (b >= nbins) b = nbins - 1;
            u = bin_u[b];
        }
        double w[3] = {v[3 * i] - u, v[3 * i + 1], v[3 * i + 2]};
        for (int k = 0; k < 3; ++k) {
            P[k] += v[3 * i + k];
            ke += 0.5 * v[3 * i + k] * v[3 * i + k];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) K[3 * a + b] += w[a] * w[b];
    }
    out[0] = P[0]; out[1] = P[1]; out[2] = P[2];
    out[3] = ke;
    double ndof = p->walls ? 3.0 * (double)nm : 3.0 * (double)nm - 3.0;
    out[4] = ndof > 0 ? (K[0] + K[4] + K[8]) / ndof : 0.0;
    memcpy(out + 5, K, 9 * sizeof(double));
    free(bin_u);
}
