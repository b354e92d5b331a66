/*
 * oracle.c -- plain, slow, FP64 CPU reference of the pore-scale LBM hot path of
 * Fattahi et al., "Pore-scale lattice Boltzmann simulation of laminar and turbulent
 * flow through a sphere pack" (arXiv:1508.02960).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may include, link or
 * call this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg use it, through the ctypes wrapper in oracle/__init__.py.  It shares no code,
 * header, table or constant with the CUDA path: lattice tables, voxeliser, wall
 * distances, MRT matrix and every update rule are written out again here.
 *
 * Every routine follows the paper's notation (k, k-bar, x_f1, x_f2, q, f-tilde) and
 * takes the steps in the order the paper states them.  Where the paper is silent or
 * ambiguous, the reading taken is stated in the comment (readings O1..O17).
 *
 * Compiled as C99 with -O2 -ffp-contract=off (no fused multiply-add), optionally
 * with OpenMP over z.  All arithmetic is IEEE double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* ------------------------------------------------------------------------------
 * D3Q19 lattice (Sec. 2, "D3Q19 model"; Eq. equilibrium: weights normalised to
 * unity, c_s^2 = 1/3).  The paper lists neither velocities nor weights (reading O1):
 * the rest velocity first, then the six axis velocities, then the twelve
 * face diagonals, opposite pairs adjacent.  The weights are the unique D3Q19 set
 * that makes the lattice isotropic to fourth order with c_s^2 = 1/3; the tests pin
 * them by those isotropy identities.
 * ---------------------------------------------------------------------------- */
static const int E[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double W[Q];
static int OPP[Q];
static int lattice_ready = 0;

static void lattice_init(void)
{
    if (lattice_ready) return;
    for (int k = 0; k < Q; ++k) {
        int n2 = E[k][0] * E[k][0] + E[k][1] * E[k][1] + E[k][2] * E[k][2];
        W[k] = (n2 == 0) ? 1.0 / 3.0 : (n2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
        /* k-bar: the diametrically opposite direction (Sec. 2.1, TRT paragraph). */
        for (int j = 0; j < Q; ++j)
            if (E[j][0] == -E[k][0] && E[j][1] == -E[k][1] && E[j][2] == -E[k][2])
                OPP[k] = j;
    }
    lattice_ready = 1;
}

void orc_lattice(int *e_out, double *w_out, int *opp_out)
{
    lattice_init();
    for (int k = 0; k < Q; ++k) {
        for (int a = 0; a < 3; ++a) e_out[3 * k + a] = E[k][a];
        w_out[k] = W[k];
        opp_out[k] = OPP[k];
    }
}

/* ------------------------------------------------------------------------------
 * Equilibrium, Eq. (equilibrium), He & Luo incompressible form, c_s^2 = 1/3:
 *   f_k^eq = w_k { rho + rho0 [ 3 e_k.u + 9/2 (e_k.u)^2 - 3/2 u.u ] }
 * ---------------------------------------------------------------------------- */
static void equilibrium(double rho, const double *u, double rho0, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int k = 0; k < Q; ++k) {
        double eu = E[k][0] * u[0] + E[k][1] * u[1] + E[k][2] * u[2];
        feq[k] = W[k] * (rho + rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
    }
}

void orc_equilibrium(double rho, const double *u, double rho0, double *feq)
{
    lattice_init();
    equilibrium(rho, u, rho0, feq);
}

/* Moments, Eq. (Macro): rho = sum_k f_k, u = rho0^-1 sum_k e_k f_k. */
static void moments(const double *f, double rho0, double *rho, double *u)
{
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int k = 0; k < Q; ++k) {
        r += f[k];
        jx += E[k][0] * f[k];
        jy += E[k][1] * f[k];
        jz += E[k][2] * f[k];
    }
    *rho = r;
    u[0] = jx / rho0;
    u[1] = jy / rho0;
    u[2] = jz / rho0;
}

/* ------------------------------------------------------------------------------
 * MRT moment matrix (Sec. 2.1, Eq. MRT): rows obtained by Gram-Schmidt
 * orthogonalisation of polynomials in the velocity components.  The polynomials
 * are taken in d'Humieres' order (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx,
 * 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m_x, m_y, m_z); each raw polynomial is a
 * monomial-type product, and the Gram-Schmidt step (plain Euclidean inner product
 * over the 19 velocities) removes from it its projection on all earlier rows.
 * Reading O7: rows are orthogonal but not normalised, so R = M^-1 S M.
 * ---------------------------------------------------------------------------- */
static double MRT_M[Q][Q];
static int mrt_ready = 0;

static double raw_poly(int i, const int *e)
{
    double x = e[0], y = e[1], z = e[2];
    double n2 = x * x + y * y + z * z;
    switch (i) {
    case 0: return 1.0;
    case 1: return n2;
    case 2: return n2 * n2;
    case 3: return x;
    case 4: return n2 * x;
    case 5: return y;
    case 6: return n2 * y;
    case 7: return z;
    case 8: return n2 * z;
    case 9: return 3.0 * x * x - n2;
    case 10: return n2 * (3.0 * x * x - n2);
    case 11: return y * y - z * z;
    case 12: return n2 * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
    }
}

static void mrt_init(void)
{
    if (mrt_ready) return;
    lattice_init();
    for (int i = 0; i < Q; ++i) {
        double v[Q];
        for (int k = 0; k < Q; ++k) v[k] = raw_poly(i, E[k]);
        for (int j = 0; j < i; ++j) {
            double num = 0.0, den = 0.0;
            for (int k = 0; k < Q; ++k) {
                num += v[k] * MRT_M[j][k];
                den += MRT_M[j][k] * MRT_M[j][k];
            }
            for (int k = 0; k < Q; ++k) v[k] -= (num / den) * MRT_M[j][k];
        }
        for (int k = 0; k < Q; ++k) MRT_M[i][k] = v[k];
    }
    mrt_ready = 1;
}

void orc_mrt_matrix(double *m_out)
{
    mrt_init();
    for (int i = 0; i < Q; ++i)
        for (int k = 0; k < Q; ++k) m_out[i * Q + k] = MRT_M[i][k];
}

/* ------------------------------------------------------------------------------
 * Collision parameters.
 * ---------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    int collision;       /* 0 = SRT, 1 = TRT, 2 = MRT */
    int wall;            /* 0 = SBB, 1 = CLI, 2 = LIBB, 3 = QIBB, 4 = IEBB, 5 = MR */
    double tau;          /* omega = omega+ = s_nu = 1/tau, nu = (tau - 1/2)/3 */
    double delta_rho;    /* periodic pressure drop, Eqs. generalPeriodicRho..PeriodicfunkownRight */
    double rho0;         /* mean density (the paper sets rho0 = 1) */
    double magic_lambda; /* TRT magic parameter Lambda */
    double mrt_ratio;    /* (1/s_nu - 1/2)/(1/s_i - 1/2) for the energy modes s_1, s_2 */
    const double *mrt_s; /* optional: 19 explicit MRT rates (overrides the rule) */
} orc_params;

/* MRT rates (Sec. 2.1, after Eq. MRT).  s_0, s_3, s_5, s_7 = 0 (conserved rho, j);
 * s_9, s_11, s_13, s_14, s_15 = s_nu; the kinetic modes s_4, s_6, s_8, s_10, s_12,
 * s_16, s_17, s_18 = s_zeta = 8(2 - s_nu)/(8 - s_nu); the energy modes s_1, s_2 keep
 * (1/s_nu - 1/2)/(1/s_i - 1/2) = ratio (reading O8: the ratio rule overrides the
 * s_zeta value the paper first lists for s_1, s_2). */
void orc_mrt_rates(double tau, double ratio, double *s)
{
    double snu = 1.0 / tau;
    double szeta = 8.0 * (2.0 - snu) / (8.0 - snu);
    double se = 1.0 / (0.5 + (1.0 / snu - 0.5) / ratio);
    for (int i = 0; i < Q; ++i) s[i] = szeta;
    s[0] = s[3] = s[5] = s[7] = 0.0;
    s[9] = s[11] = s[13] = s[14] = s[15] = snu;
    s[1] = s[2] = se;
}

/* TRT rates (Sec. 2.1, Eq. TRT and the magic-parameter definition):
 * omega+ = 1/tau, Lambda = (1/omega+ - 1/2)(1/omega- - 1/2). */
static double trt_omega_minus(double tau, double lambda)
{
    return 1.0 / (0.5 + lambda / (tau - 0.5));
}

/* One node's collision, Eqs. (SRT), (TRT), (MRT): f-tilde = f - R (f - f^eq). */
static void collide_node(const orc_params *p, const double *f, double *ft)
{
    double rho, u[3], feq[Q];
    moments(f, p->rho0, &rho, u);
    equilibrium(rho, u, p->rho0, feq);

    if (p->collision == 0) { /* SRT / BGK: R = omega I */
        double omega = 1.0 / p->tau;
        for (int k = 0; k < Q; ++k) ft[k] = f[k] - omega * (f[k] - feq[k]);
    } else if (p->collision == 1) { /* TRT: R = omega+ R+ + omega- R- */
        double wp = 1.0 / p->tau;
        double wm = trt_omega_minus(p->tau, p->magic_lambda);
        for (int k = 0; k < Q; ++k) {
            int kb = OPP[k];
            double fp = 0.5 * (f[k] + f[kb]), fm = 0.5 * (f[k] - f[kb]);
            double ep = 0.5 * (feq[k] + feq[kb]), em = 0.5 * (feq[k] - feq[kb]);
            ft[k] = f[k] - wp * (fp - ep) - wm * (fm - em);
        }
    } else { /* MRT: R = M^-1 S M */
        double s[Q], neq[Q], m[Q], dm[Q];
        if (p->mrt_s)
            for (int i = 0; i < Q; ++i) s[i] = p->mrt_s[i];
        else
            orc_mrt_rates(p->tau, p->mrt_ratio, s);
        for (int k = 0; k < Q; ++k) neq[k] = f[k] - feq[k];
        for (int i = 0; i < Q; ++i) {
            double acc = 0.0;
            for (int k = 0; k < Q; ++k) acc += MRT_M[i][k] * neq[k];
            m[i] = acc;
        }
        /* M^-1 = M^T diag(1/|M_i|^2) because the rows are orthogonal. */
        for (int i = 0; i < Q; ++i) {
            double n2 = 0.0;
            for (int k = 0; k < Q; ++k) n2 += MRT_M[i][k] * MRT_M[i][k];
            dm[i] = s[i] * m[i] / n2;
        }
        for (int k = 0; k < Q; ++k) {
            double acc = 0.0;
            for (int i = 0; i < Q; ++i) acc += MRT_M[i][k] * dm[i];
            ft[k] = f[k] - acc;
        }
    }
}

void orc_collide(const orc_params *p, const double *f, double *ft)
{
    lattice_init();
    mrt_init();
    collide_node(p, f, ft);
}

/* ------------------------------------------------------------------------------
 * Geometry (Sec. 3: one sphere per periodic cell; wall distances computed once
 * before time stepping).  Reading O2: cell (i,j,k) has centre (i+1/2, j+1/2, k+1/2)
 * in lattice units; it is solid iff its minimum-image distance to some sphere
 * centre is <= r.  Spheres are given as (cx, cy, cz, r) quadruples.
 * ---------------------------------------------------------------------------- */
static double min_image(double d, int n)
{
    /* nearest periodic image of a displacement d along an axis of length n */
    while (d > 0.5 * n) d -= n;
    while (d < -0.5 * n) d += n;
    return d;
}

static int64_t cell_index(int x, int y, int z, int nx, int ny)
{
    return (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
}

static int wrap(int a, int n) { return ((a % n) + n) % n; }

/* Sphere centres farther than MAX_CENTRE_BOXES box lengths from the origin are refused:
 * min_image folds a displacement into the box one box length at a time. */
#define MAX_CENTRE_BOXES 64

static int centres_in_range(int nx, int ny, int nz, const double *sph, int nsph)
{
    for (int i = 0; i < nsph; ++i)
        if (!(fabs(sph[4 * i + 0]) <= (double)MAX_CENTRE_BOXES * nx) ||
            !(fabs(sph[4 * i + 1]) <= (double)MAX_CENTRE_BOXES * ny) ||
            !(fabs(sph[4 * i + 2]) <= (double)MAX_CENTRE_BOXES * nz))
            return 0;
    return 1;
}

int orc_voxelize(int nx, int ny, int nz, const double *sph, int nsph, uint8_t *solid)
{
    lattice_init();
    if (nx <= 0 || ny <= 0 || nz <= 0 || nsph < 0) return -1;
    if (!centres_in_range(nx, ny, nz, sph, nsph)) return -1;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                uint8_t s = 0;
                for (int i = 0; i < nsph; ++i) {
                    double dx = min_image(x + 0.5 - sph[4 * i + 0], nx);
                    double dy = min_image(y + 0.5 - sph[4 * i + 1], ny);
                    double dz = min_image(z + 0.5 - sph[4 * i + 2], nz);
                    double r = sph[4 * i + 3];
                    if (dx * dx + dy * dy + dz * dz <= r * r) s = 1;
                }
                solid[cell_index(x, y, z, nx, ny)] = s;
            }
    return 0;
}

/* Normalised wall distance q = |x_f1 - x_w| / |x_f1 - x_b| (Sec. 2.2.1, before
 * Eq. LIBB), for every link from a fluid node x_f1 along e_k into a solid node
 * x_b = x_f1 + e_k.  The wall point x_w is where the segment x_f1 -> x_b first
 * meets a sphere surface; among the spheres whose (nearest periodic image) contains
 * x_b, the nearest crossing counts.  Output q[k*N + cell]; NaN where the link is
 * not cut (fluid neighbour, or the node itself is solid).  Roots that round just
 * outside (0, 1] are clamped to [1e-6, 1]. */
int orc_wall_distances(int nx, int ny, int nz, const uint8_t *solid, const double *sph,
                       int nsph, double *q)
{
    lattice_init();
    const int64_t n = (int64_t)nx * ny * nz;
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    if (!centres_in_range(nx, ny, nz, sph, nsph)) return -1;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = cell_index(x, y, z, nx, ny);
                for (int k = 0; k < Q; ++k) q[(int64_t)k * n + c] = NAN;
                if (solid[c]) continue;
                for (int k = 1; k < Q; ++k) {
                    int64_t b = cell_index(wrap(x + E[k][0], nx), wrap(y + E[k][1], ny),
                                           wrap(z + E[k][2], nz), nx, ny);
                    if (!solid[b]) continue;
                    /* ray p + t e_k, t in (0,1]; p = centre of x_f1 */
                    double best = INFINITY;
                    for (int i = 0; i < nsph; ++i) {
                        double r = sph[4 * i + 3];
                        /* sphere image nearest to the solid end point x_b */
                        double bx = x + E[k][0] + 0.5, by = y + E[k][1] + 0.5, bz = z + E[k][2] + 0.5;
                        double cx = bx - min_image(bx - sph[4 * i + 0], nx);
                        double cy = by - min_image(by - sph[4 * i + 1], ny);
                        double cz = bz - min_image(bz - sph[4 * i + 2], nz);
                        double ebx = bx - cx, eby = by - cy, ebz = bz - cz;
                        if (ebx * ebx + eby * eby + ebz * ebz > r * r) continue;
                        double px = x + 0.5 - cx, py = y + 0.5 - cy, pz = z + 0.5 - cz;
                        double a = (double)(E[k][0] * E[k][0] + E[k][1] * E[k][1] + E[k][2] * E[k][2]);
                        double hb = px * E[k][0] + py * E[k][1] + pz * E[k][2];
                        double cc = px * px + py * py + pz * pz - r * r;
                        double disc = hb * hb - a * cc;
                        if (disc < 0.0) disc = 0.0;
                        double t = (-hb - sqrt(disc)) / a;
                        if (t < best) best = t;
                    }
                    if (!(best < INFINITY)) best = 0.5; /* solid from a flag field only */
                    if (best < 1e-6) best = 1e-6;
                    if (best > 1.0) best = 1.0;
                    q[(int64_t)k * n + c] = best;
                }
            }
    return 0;
}

/* ------------------------------------------------------------------------------
 * Periodic pressure drop (Sec. 2.2.2, Eqs. Periodicfunkown / PeriodicfunkownRight):
 * a population that crosses the streamwise (x) boundary from right to left gains
 * w_k delta_rho, one that crosses from left to right loses it.  With rho_L = rho_R +
 * delta_rho (Eq. generalPeriodicRho) the flow runs along +x.  Reading O3: the index
 * of w is the population's own direction.  Reading O5: every value read from a
 * periodic image in x carries the shift, including the x_f2 value of CLI.
 *
 * read_pop returns f_k at the virtual lattice position (xv, y, z), where xv may lie
 * one cell outside [0, nx): it reads the stored value of the periodic image and
 * adds the density shift of the crossing.
 * ---------------------------------------------------------------------------- */
static double read_pop(const double *f, int64_t n, int k, int xv, int yv, int zv,
                       const orc_params *p)
{
    int xs = wrap(xv, p->nx);
    double v = f[(int64_t)k * n + cell_index(xs, wrap(yv, p->ny), wrap(zv, p->nz), p->nx, p->ny)];
    if (xv < 0) v += W[k] * p->delta_rho;      /* came in through the left boundary */
    if (xv >= p->nx) v -= W[k] * p->delta_rho; /* came in through the right boundary */
    return v;
}

/* ------------------------------------------------------------------------------
 * Interpolated bounce-back rules (Sec. 2.2.1, Eqs. LIBB, QIBB, fstar, IEBB, MR, CLI), in
 * the paper's notation: k points from x_f1 into the wall (x_f1 + e_k solid), the unknown
 * is f_kbar(x_f1, t+1), x_f2 = x_f1 - e_k, x_f3 = x_f1 - 2 e_k, q the link's wall
 * distance, all f~ at time t.  wall_rule returns the unknown.  Reading O16: a rule falls
 * back when a node it reads is solid -- to SBB when x_f2 is needed and solid, QIBB to
 * LIBB and MR to CLI when only x_f3 is solid.  Reading O15: the density in f* (printed
 * as Delta rho) is the density of x_f1, so that f* is the equilibrium of Eq. equilibrium
 * at x_f1 with the first-order velocity term taken at u_bf (Mei et al.).
 * ---------------------------------------------------------------------------- */
typedef struct {
    int wall;
    double q, tau, rho0;
    int f2_fluid, f3_fluid;
    double fk_1, fkb_1;   /* f~_k(x_f1), f~_kbar(x_f1) */
    double fk_2, fkb_2;   /* f~_k(x_f2), f~_kbar(x_f2) */
    double fk_3;          /* f~_k(x_f3) */
    double rho_1, u_1[3]; /* density and velocity of x_f1 at t */
    double u_2[3];        /* velocity of x_f2 at t */
    int k;                /* link direction (into the wall) */
} wall_link;

static double rule_sbb(const wall_link *L) { return L->fk_1; }

static double rule_cli(const wall_link *L)
{
    double c = (1.0 - 2.0 * L->q) / (1.0 + 2.0 * L->q);
    return c * L->fk_2 - c * L->fkb_1 + L->fk_1;
}

static double rule_libb(const wall_link *L)
{
    double q = L->q;
    if (q < 0.5) return (1.0 - 2.0 * q) * L->fk_2 + 2.0 * q * L->fk_1;
    return (1.0 - 1.0 / (2.0 * q)) * L->fkb_1 + 1.0 / (2.0 * q) * L->fk_1;
}

static double rule_qibb(const wall_link *L)
{
    double q = L->q;
    if (q < 0.5)
        return q * (1.0 + 2.0 * q) * L->fk_1 + (1.0 - 4.0 * q * q) * L->fk_2 - q * (1.0 - 2.0 * q) * L->fk_3;
    return (2.0 * q - 1.0) / q * L->fkb_1 + 1.0 / (q * (2.0 * q + 1.0)) * L->fk_1 +
           (1.0 - 2.0 * q) / (2.0 * q + 1.0) * L->fkb_2;
}

/* Reading O17: the first MR coefficient is printed over (1+2q)^2; read over (1+q)^2, as
 * the second one.  As printed, the rule is inconsistent: it converges at first order in
 * the plane channel, worse than SBB; read so, at second order like the other rules. */
static double rule_mr(const wall_link *L)
{
    double q = L->q;
    double a = (1.0 - 2.0 * q - 2.0 * q * q) / ((1.0 + q) * (1.0 + q));
    double b = q * q / ((1.0 + q) * (1.0 + q));
    return a * L->fk_2 + b * L->fk_3 - a * L->fkb_1 - b * L->fkb_2 + L->fk_1;
}

static double rule_iebb(const wall_link *L)
{
    double q = L->q, inv_omega = L->tau; /* 1/omega = tau for omega+ (TRT) and s_nu (MRT) */
    double ubf[3], X;
    if (q < 0.5) {
        for (int a = 0; a < 3; ++a) ubf[a] = L->u_2[a];
        X = (2.0 * q - 1.0) / (inv_omega - 2.0);
    } else {
        for (int a = 0; a < 3; ++a) ubf[a] = (1.0 - 3.0 / (2.0 * q)) * L->u_1[a];
        X = (2.0 * q - 1.0) / (inv_omega + 0.5);
    }
    const int *e = E[L->k];
    double eub = e[0] * ubf[0] + e[1] * ubf[1] + e[2] * ubf[2];
    double eu1 = e[0] * L->u_1[0] + e[1] * L->u_1[1] + e[2] * L->u_1[2];
    double uu1 = L->u_1[0] * L->u_1[0] + L->u_1[1] * L->u_1[1] + L->u_1[2] * L->u_1[2];
    double fstar = W[L->k] * (L->rho_1 + L->rho0 * (3.0 * eub + 4.5 * eu1 * eu1 - 1.5 * uu1));
    return (1.0 - X) * L->fk_1 + X * fstar;
}

static double wall_rule(const wall_link *L)
{
    switch (L->wall) {
    case 1: return L->f2_fluid ? rule_cli(L) : rule_sbb(L);
    case 2: return (L->q < 0.5 && !L->f2_fluid) ? rule_sbb(L) : rule_libb(L);
    case 3:
        if (!L->f2_fluid) return L->q < 0.5 ? rule_sbb(L) : rule_libb(L);
        if (L->q < 0.5 && !L->f3_fluid) return rule_libb(L);
        return rule_qibb(L);
    case 4: return (L->q < 0.5 && !L->f2_fluid) ? rule_sbb(L) : rule_iebb(L);
    case 5:
        if (!L->f2_fluid) return rule_sbb(L);
        if (!L->f3_fluid) return rule_cli(L);
        return rule_mr(L);
    default: return rule_sbb(L);
    }
}

/* Density and velocity of the populations of the node at virtual position (xv, yv, zv)
 * (periodic image, with the pressure shift of read_pop).  For post-collision values these
 * are the node's moments at t: the collision conserves mass and momentum. */
static void node_moments(const double *f, int64_t n, int xv, int yv, int zv, const orc_params *p, double *rho,
                         double *u)
{
    double fl[Q];
    for (int m = 0; m < Q; ++m) fl[m] = read_pop(f, n, m, xv, yv, zv, p);
    moments(fl, p->rho0, rho, u);
}

/* ------------------------------------------------------------------------------
 * One time step, stream first then collide (Sec. 2, Eqs. collision, streaming and
 * the remark that waLBerla streams first, then collides).  Input f holds the
 * post-collision values f-tilde(t) of every fluid node; output ft holds
 * f-tilde(t+1).  Solid nodes are never updated and are written as 0.
 *
 * For each fluid node x and each direction k, the incoming population is pulled
 * from x - e_k.  If x - e_k is solid, the link from x along k-bar hits the wall and
 * f_k(x, t+1) is the unknown of the wall rule:
 *   SBB, Eq. (noslip):  f_k(x,t+1) = f~_kbar(x,t)
 *   CLI, Eq. (CLI) with c = (1-2q)/(1+2q), q the wall distance of link (x, kbar),
 *        x_f2 = x - e_kbar = x + e_k:
 *        f_k(x,t+1) = c f~_kbar(x_f2,t) - c f~_k(x,t) + f~_kbar(x,t)
 * Reading O4: where x_f2 is solid (one-cell gap), CLI falls back to SBB.  LIBB, QIBB,
 * IEBB and MR: wall_rule above.
 *
 * sums (optional, 4 doubles): sum over fluid nodes of rho, u_x, u_y, u_z of the
 * streamed moments (Eq. Macro) -- reading O9.  uvec (optional, 3*N): per-node u.
 *
 * force (optional, 3 doubles): the drag F_D of Sec. 3 (Eq. AnalyticForce) on all solid nodes
 * during this step, by momentum exchange (reading O13): every wall link (x, kbar) with
 * x - e_k solid carries f~_kbar(x, t) into the wall and brings f_k(x, t+1) back, so the
 * solid receives e_kbar (f~_kbar(x, t) + f_k(x, t+1)).
 * ---------------------------------------------------------------------------- */
static void step_once(const orc_params *p, const uint8_t *solid, const double *q,
                      const double *f, double *ft, double *sums, double *uvec, double *force)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const int64_t n = (int64_t)nx * ny * nz;
    double srho = 0.0, sux = 0.0, suy = 0.0, suz = 0.0;
    double sfx = 0.0, sfy = 0.0, sfz = 0.0;

#pragma omp parallel for schedule(static) reduction(+ : srho, sux, suy, suz, sfx, sfy, sfz)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = cell_index(x, y, z, nx, ny);
                if (solid[c]) {
                    for (int k = 0; k < Q; ++k) ft[(int64_t)k * n + c] = 0.0;
                    if (uvec) uvec[c] = uvec[n + c] = uvec[2 * n + c] = 0.0;
                    continue;
                }
                double fin[Q], fout[Q];
                for (int k = 0; k < Q; ++k) {
                    int xv = x - E[k][0], yv = y - E[k][1], zv = z - E[k][2];
                    int64_t s = cell_index(wrap(xv, nx), wrap(yv, ny), wrap(zv, nz), nx, ny);
                    if (!solid[s]) {
                        fin[k] = read_pop(f, n, k, xv, yv, zv, p);
                        continue;
                    }
                    /* the link of the paper's rules points into the wall: kk = kbar, and
                     * the unknown is f_k = f_{kk-bar} */
                    int kb = OPP[k];
                    double own_kb = f[(int64_t)kb * n + c]; /* f~_kbar(x_f1, t) */
                    int x2 = x + E[k][0], y2 = y + E[k][1], z2 = z + E[k][2];
                    int x3 = x + 2 * E[k][0], y3 = y + 2 * E[k][1], z3 = z + 2 * E[k][2];
                    int64_t s2 = cell_index(wrap(x2, nx), wrap(y2, ny), wrap(z2, nz), nx, ny);
                    int64_t s3 = cell_index(wrap(x3, nx), wrap(y3, ny), wrap(z3, nz), nx, ny);
                    if (p->wall == 0) {
                        fin[k] = own_kb;
                    } else {
                        wall_link L;
                        memset(&L, 0, sizeof(L));
                        L.wall = p->wall;
                        L.q = q[(int64_t)kb * n + c];
                        L.tau = p->tau;
                        L.rho0 = p->rho0;
                        L.k = kb;
                        L.f2_fluid = !solid[s2];
                        L.f3_fluid = L.f2_fluid && !solid[s3];
                        L.fk_1 = own_kb;
                        L.fkb_1 = f[(int64_t)k * n + c];
                        if (L.f2_fluid) {
                            L.fk_2 = read_pop(f, n, kb, x2, y2, z2, p);
                            L.fkb_2 = read_pop(f, n, k, x2, y2, z2, p);
                            if (p->wall == 4) {
                                double r2;
                                node_moments(f, n, x2, y2, z2, p, &r2, L.u_2);
                            }
                        }
                        if (L.f3_fluid) L.fk_3 = read_pop(f, n, kb, x3, y3, z3, p);
                        if (p->wall == 4) node_moments(f, n, x, y, z, p, &L.rho_1, L.u_1);
                        fin[k] = wall_rule(&L);
                    }
                    /* momentum given to the solid through link (x, kbar) */
                    double ex_in = own_kb + fin[k];
                    sfx += E[kb][0] * ex_in;
                    sfy += E[kb][1] * ex_in;
                    sfz += E[kb][2] * ex_in;
                }
                double rho, u[3];
                moments(fin, p->rho0, &rho, u);
                srho += rho;
                sux += u[0];
                suy += u[1];
                suz += u[2];
                if (uvec) {
                    uvec[c] = u[0];
                    uvec[n + c] = u[1];
                    uvec[2 * n + c] = u[2];
                }
                collide_node(p, fin, fout);
                for (int k = 0; k < Q; ++k) ft[(int64_t)k * n + c] = fout[k];
            }
    if (sums) {
        sums[0] = srho;
        sums[1] = sux;
        sums[2] = suy;
        sums[3] = suz;
    }
    if (force) {
        force[0] = sfx;
        force[1] = sfy;
        force[2] = sfz;
    }
}

/* Run nsteps time steps.  f (19*N, [k][z][y][x]) holds f-tilde on entry and on exit.
 * sums / uvec / force describe the last step (see step_once); each may be NULL. */
int orc_run(const orc_params *p, const uint8_t *solid, const double *q, double *f,
            int nsteps, double *sums, double *uvec, double *force)
{
    lattice_init();
    mrt_init();
    if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || nsteps < 0) return -1;
    if (!(p->tau > 0.5)) return -1;
    if (p->wall < 0 || p->wall > 5) return -1;
    if (p->wall >= 1 && !q) return -1;
    const int64_t n = (int64_t)p->nx * p->ny * p->nz;
    double *g = (double *)malloc(sizeof(double) * Q * n);
    if (!g) return -2;
    double *a = f, *b = g;
    for (int t = 0; t < nsteps; ++t) {
        int last = (t == nsteps - 1);
        step_once(p, solid, q, a, b, last ? sums : NULL, last ? uvec : NULL, last ? force : NULL);
        double *tmp = a;
        a = b;
        b = tmp;
    }
    if (a != f) memcpy(f, a, sizeof(double) * Q * n);
    free(g);
    return 0;
}

/* Initial state (reading of Sec. 3 setup): every fluid node at f^eq(rho0, u = 0) = w_k rho0,
 * taken as the post-collision state at t = 0.  Solid nodes are 0. */
int orc_init_rest(int nx, int ny, int nz, const uint8_t *solid, double rho0, double *f)
{
    lattice_init();
    const int64_t n = (int64_t)nx * ny * nz;
    for (int k = 0; k < Q; ++k)
        for (int64_t c = 0; c < n; ++c) f[(int64_t)k * n + c] = solid[c] ? 0.0 : W[k] * rho0;
    return 0;
}

/* ------------------------------------------------------------------------------
 * Observables (Sec. 1 Eqs. Darcy, Forchheimer; Sec. 4 Eq. frictionFactor), lattice
 * units with rho = rho0 (reading O11):
 *   mu = nu = (tau - 1/2)/3, dp = delta_rho/3 (p = rho c_s^2), gradP = dp / L_x,
 *   K = mu U / gradP, Re_p = U d_p / nu, and with a Darcy permeability K_D:
 *   beta = (gradP - mu U / K_D) / (rho U^2), C_F = beta sqrt(K_D),
 *   F_K = gradP sqrt(K_D) / (rho U^2), Re_K = rho U sqrt(K_D) / mu.
 * out: [U, K, Re_p, beta, C_F, F_K, Re_K]
 * ---------------------------------------------------------------------------- */
void orc_observables(double U, double tau, double delta_rho, double rho0, int lx, double d_p,
                     double K_D, double *out)
{
    double mu = rho0 * (tau - 0.5) / 3.0;
    double nu = (tau - 0.5) / 3.0;
    double gradP = (delta_rho / 3.0) / lx;
    out[0] = U;
    out[1] = mu * U / gradP;
    out[2] = U * d_p / nu;
    if (K_D > 0.0) {
        out[3] = (gradP - mu * U / K_D) / (rho0 * U * U);
        out[4] = out[3] * sqrt(K_D);
        out[5] = gradP * sqrt(K_D) / (rho0 * U * U);
        out[6] = rho0 * U * sqrt(K_D) / mu;
    } else {
        out[3] = out[4] = out[5] = out[6] = NAN;
    }
}

/* ------------------------------------------------------------------------------
 * Drag coefficients from the streamwise drag F_D (Sec. 3 Eq. AnalyticForce and the
 * resolution study of Sec. 4), lattice units, U = U_sup, mu = rho0 (tau - 1/2)/3:
 *   C_D   = F_D / (6 pi mu U r)       -- Stokes normalisation; for several spheres r is
 *                                        the sum of their radii (reading O14)
 *   C_D,A = F_D / (rho0 A U^2)        -- A = sum of the spheres' frontal areas pi r^2
 *                                        (reading O14)
 * out: [C_D, C_D,A]
 * ---------------------------------------------------------------------------- */
void orc_drag_coefficients(double F_D, double U, double tau, double rho0, double r_sum,
                           double area_sum, double *out)
{
    const double pi = 3.14159265358979323846;
    double mu = rho0 * (tau - 0.5) / 3.0;
    out[0] = F_D / (6.0 * pi * mu * U * r_sum);
    out[1] = F_D / (rho0 * area_sum * U * U);
}

/* Thread control for the timed CPU baseline (OpenMP over z when compiled with it). */
#ifdef _OPENMP
#include <omp.h>
void orc_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }
int orc_max_threads(void) { return omp_get_max_threads(); }
#else
void orc_set_threads(int n) { (void)n; }
int orc_max_threads(void) { return 1; }
#endif
