/*
 * lelbm_oracle.c -- plain, slow, FP64 CPU reference of the per-timestep cell
 * update of the Lagrangian entropic lattice Boltzmann method (LELBM),
 * W. Noh and C. Lee, arXiv:2508.06911.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed CPU
 * baseline of the benchmark load this library.  It shares no code, header or
 * table with the CUDA library; the product path never calls it.
 *
 * Every function follows the paper's equations in the paper's order and
 * notation, in lattice units (dx = dt = dV = 1, dC = 1 at refinement level 0,
 * Sec. II.A):
 *   macroscopic variables ............ Eq. (IIB6)
 *   equilibrium raw moments .......... Eq. (IIB7), App. A Eq. (A3), (A7)
 *   non-equilibrium central moments .. Eq. (IIB9)
 *   shear / bulk split ............... Eq. (IIB10)-(IIB11)
 *   heat-flux split .................. Eq. (IIB14)
 *   collision ........................ Eq. (IIB16)-(IIB17)
 *   normalisation .................... Eq. (IIB18)
 *   relaxation frequencies ........... App. C Eq. (C7)-(C8)
 *   Knudsen limiter .................. App. D Eq. (D2)-(D3)
 *   LAS stencil and refinement ....... Eq. (IIC6), (IIC9)-(IIC11)
 *   EPR Newton, Maxwellian start ..... Eq. (IID7)-(IID13)
 *   moment streaming ................. Eq. (IIE3)
 *   fluid boundaries ................. Sec. III.A
 *   solid boundaries ................. Sec. III.B, Eq. (IIIB10)-(IIIB15)
 *     (slip walls, no-slip walls at rest and moving no-slip walls)
 * Readings of passages the paper leaves open are marked "reading:" below.
 *
 * Parity unpinned (no test independent of this file fixes them; each place is
 * marked "parity unpinned" below):
 *   - how a refined point's share spreads beyond its centre of mass (the
 *     cloud-in-cell reading in orc_step; the centre of mass itself is pinned);
 *   - the quadrature weights dC inside the last-resort Maxwellian weights of
 *     solve_cell (the weights' mean, variance and mass are pinned);
 *   - the wall rules at an isolated convex corner in orc_trace_path (flat
 *     walls and box corners are pinned by the method of images).
 *
 * Build with -ffp-contract=off: every operation then rounds once, on x86-64
 * and on aarch64 alike, so the stencil membership tests are reproducible.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXD 3  /* translational dimensions D = 1, 2, 3                  */
#define ORC_MAXF 19 /* N_f in 3D: 1 + D + D(D+1)/2 + D^2 (Eq. IIB14-16) */
#define ORC_MAXG 10 /* N_g in 3D: 1 + D + D(D+1)/2 (Eq. IIB16-17)        */
#define ORC_MAXM 17 /* stored moments in 3D: 13 fluon + 4 phonon (Eq. IIB5) */

/* ------------------------------------------------------------------------ */
/* parameters and results shared with the Python loader (ctypes layout)      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int D;             /* translational dimensions, 1, 2 or 3                */
    double K;          /* internal degrees of freedom                        */
    double nu_s;       /* kinematic shear viscosity, lattice units           */
    double nu_b;       /* kinematic bulk viscosity; < 0 selects omega_b = 1  */
    double Pr;         /* Prandtl number                                     */
    int limiter;       /* 1: Knudsen limiter on (App. D)                     */
    double n_conf;     /* conformation number n, 4 (Eq. IIC6)                */
    double r_min;      /* minimum acoustic radius, 2 (Eq. IIC6)              */
    double refine_div; /* divisor 3 in N_r (Eq. IIC9)                        */
    double refine_rad; /* factor 3 in the refinement radius (Eq. IIC10)      */
    int max_refine;    /* cap on N_r                                         */
    double tol;        /* EPR residual tolerance, 1e-12 (Sec. II.D)          */
    int max_iter;      /* Newton iteration cap                               */
} orc_params;

typedef struct {
    double rho, u[ORC_MAXD], RT;
    double cf[ORC_MAXF]; /* normalised post-collision fluon constraints    */
    double cg[ORC_MAXG]; /* normalised post-collision phonon constraints   */
    double omega[3];     /* omega_f, omega_b, omega_h after the limiter    */
    double Kn;           /* local Knudsen number, Eq. (D2)                 */
} orc_collision;

typedef struct {
    double c[ORC_MAXD]; /* particle velocity c_i (lattice frame)             */
    double dC;   /* velocity volume Delta C_i (Eq. IIA8, IIC11)              */
    int level;   /* refinement level of the point                           */
} orc_point;

typedef struct {
    long long cells;         /* emitting cells processed                    */
    long long newton_hist[64];/* Newton updates per solve (f and g)          */
    long long fallback_eq;   /* solves redone with equilibrium constraints  */
    long long fallback_mx;   /* solves that fell back to Maxwellian weights */
    long long q_max;         /* largest stencil                             */
    double disp_max;         /* largest |c_i| (lattice Courant, Eq. IIC3)   */
    long long wall_hits;     /* populations reflected at solid faces        */
} orc_stats;

typedef struct {
    int D, nx, ny, nz;       /* interior size (ny = 1 in 1D, nz = 1 below 3D) */
    int periodic[3];         /* per axis                                    */
    int pad;                 /* pad layers on every non-periodic side       */
    int bc[6];               /* x-, x+, y-, y+, z-, z+: 0 outflow, 1 inflow */
    double inlet[5];         /* rho, ux, uy, uz, RT of the inflow state     */
    const unsigned char* solid; /* padded-grid wall kinds or NULL (1D, 2D): 0 fluid,
                                   1 slip wall, 2 no-slip wall at rest, 3 no-slip wall
                                   moving at wall_u                            */
    double wall_u[2];        /* velocity u_w of the kind-3 walls (Eq. IIIB2-IIIB4) */
} orc_grid;

/* N_M = 1 + D + D(D+1)/2 + D (fluons) plus 1 + D (phonons), Eq. (IIB5) */
int orc_nmom(int D) { return 2 + 3 * D + D * (D + 1) / 2; }
int orc_nf(int D) { return 1 + D + D * (D + 1) / 2 + D * D; }
int orc_ng(int D) { return 1 + D + D * (D + 1) / 2; }

/* Stored-moment positions (Eq. IIB5): M0, M_a, M_ab (a <= b, row by row),
 * M_Dg, G0, G_g.  1D {M0,Mx,Mxx,MDx,G0,Gx},
 * 2D {M0,Mx,My,Mxx,Mxy,Myy,MDx,MDy,G0,Gx,Gy},
 * 3D {M0,Mx,My,Mz,Mxx,Mxy,Mxz,Myy,Myz,Mzz,MDx,MDy,MDz,G0,Gx,Gy,Gz}.        */
static int tri(int D, int a, int b) /* position of (a <= b) among the pairs */
{
    if (a > b) { int t = a; a = b; b = t; }
    return a * D - a * (a - 1) / 2 + (b - a);
}
static int iM1(int D, int a) { (void)D; return 1 + a; }
static int iM2(int D, int a, int b) { return 1 + D + tri(D, a, b); }
static int iMD(int D, int g) { return 1 + D + D * (D + 1) / 2 + g; }
static int iG0(int D) { return 1 + 2 * D + D * (D + 1) / 2; }
static int iG1(int D, int g) { return iG0(D) + 1 + g; }

/* ------------------------------------------------------------------------ */
/* Eq. (IIB7) with App. A Eq. (A3a-b), (A3g), (A7a-b): equilibrium raw moments */
/* ------------------------------------------------------------------------ */
void orc_eq_moments(int D, double K, double rho, const double* u, double RT, double* M)
{
    double usq = 0.0;
    for (int a = 0; a < D; a++) usq += u[a] * u[a];
    for (int i = 0; i < orc_nmom(D); i++) M[i] = 0.0;
    M[0] = rho;                                             /* (A3a) */
    for (int a = 0; a < D; a++) M[iM1(D, a)] = rho * u[a]; /* (A3b) */
    for (int a = 0; a < D; a++)
        for (int b = a; b < D; b++)                          /* (IIB7a) */
            M[iM2(D, a, b)] = rho * (u[a] * u[b] + (a == b ? RT : 0.0));
    for (int g = 0; g < D; g++)                              /* (IIB7b) */
        M[iMD(D, g)] = rho * (usq + (D + 2) * RT) * u[g];
    M[iG0(D)] = rho * K * RT;                                /* (IIB7c) */
    for (int g = 0; g < D; g++) M[iG1(D, g)] = rho * K * RT * u[g]; /* (IIB7d) */
}

/* Eq. (IIB6): density, velocity and temperature from the raw moments. */
void orc_macros(int D, double K, const double* M, double* rho, double* u, double* RT)
{
    double r = M[0];
    double usq = 0.0, trace = 0.0;
    for (int a = 0; a < D; a++) {
        u[a] = M[iM1(D, a)] / r;
        usq += u[a] * u[a];
        trace += M[iM2(D, a, a)];
    }
    *rho = r;
    *RT = ((trace + M[iG0(D)]) / r - usq) / (D + K);
}

/* Eq. (IIB9): non-equilibrium central moments.
 * out: P[a][b] = M~neq_ab, Q[g] = M~neq_Dg, *G0n = G~neq_0, Gn[g] = G~neq_g. */
void orc_neq(int D, double K, const double* M, double rho, const double* u, double RT,
             double* P /* [3][3] */, double* Q, double* G0n, double* Gn)
{
    double usq = 0.0;
    for (int a = 0; a < D; a++) usq += u[a] * u[a];
    for (int a = 0; a < D; a++)                               /* (IIB9a) */
        for (int b = 0; b < D; b++)
            P[3 * a + b] = M[iM2(D, a, b)] - rho * (u[a] * u[b] + (a == b ? RT : 0.0));
    double trP = 0.0;
    for (int a = 0; a < D; a++) trP += P[3 * a + a];
    for (int g = 0; g < D; g++) {                             /* (IIB9b) */
        double s = 0.0;
        for (int a = 0; a < D; a++) s += u[a] * P[3 * a + g];
        Q[g] = M[iMD(D, g)] - 2.0 * s - u[g] * trP - rho * (usq + (D + 2) * RT) * u[g];
    }
    *G0n = M[iG0(D)] - rho * K * RT;                          /* (IIB9c) */
    for (int g = 0; g < D; g++) Gn[g] = M[iG1(D, g)] - u[g] * M[iG0(D)]; /* (IIB9d) */
}

/* App. C Eq. (C7)-(C8): implicit collision frequencies from the kinematic
 * transport coefficients.  nu_s = mu_s/rho = RT (1/omega_f - 1/2);
 * Pr = mu_s C_p / kappa gives 1/omega_h - 1/2 = (1/omega_f - 1/2) / Pr;
 * nu_b = RT (2/D - 2/(D+K)) (1/omega_b - 1/2), or omega_b = 1 (Sec. II.B). */
void orc_omegas(int D, double K, double RT, double nu_s, double nu_b, double Pr, double* om)
{
    double inv_f = nu_s / RT + 0.5;
    om[0] = 1.0 / inv_f;
    double fb = 2.0 / D - 2.0 / (D + K);
    if (nu_b < 0.0 || fb <= 0.0)
        om[1] = 1.0;
    else
        om[1] = 1.0 / (nu_b / (RT * fb) + 0.5);
    om[2] = 1.0 / ((inv_f - 0.5) / Pr + 0.5);
}

/* App. D Eq. (D2): local Knudsen number.  reading: every moment is
 * normalised by rho (G too), the first sum runs over all index pairs
 * (alpha, beta), the second over the components gamma. */
double orc_knudsen(int D, double K, double rho, double RT, const double* P, const double* Q,
                   double G0n, const double* Gn)
{
    double s2 = 0.0, s3 = 0.0;
    for (int a = 0; a < D; a++)
        for (int b = 0; b < D; b++) s2 += fabs(P[3 * a + b] / rho);
    s2 += fabs(G0n / rho);
    for (int g = 0; g < D; g++) s3 += fabs(Q[g] / rho) + fabs(Gn[g] / rho);
    double k2 = s2 / ((D + K) * RT);
    double k3 = s3 / ((D + K + 2) * pow(RT, 1.5));
    return k2 > k3 ? k2 : k3;
}

/* App. D Eq. (D3) with the thresholds stated after it (Kn*_L = -2,
 * Kn*_H = -1, omega_H = 1).  reading: the case labels of (D3b) are taken
 * from the text: no change below Kn = 0.01, equilibrium above Kn = 0.1,
 * linear in log10 Kn in between. */
double orc_limit_omega(double Kn, double omega)
{
    const double kl = -2.0, kh = -1.0, wh = 1.0;
    if (!(Kn > 0.0)) return omega;
    double ks = log10(Kn);
    if (ks <= kl) return omega;
    if (ks >= kh) return wh;
    return (wh - omega) / (kh - kl) * (ks - kl) + omega;
}

/* Collision module (Fig. collision_module): Eq. (IIB6), (IIB9)-(IIB18). */
void orc_collide(const orc_params* p, const double* M, orc_collision* out)
{
    int D = p->D;
    double K = p->K;
    double rho, u[ORC_MAXD] = {0, 0, 0}, RT;
    orc_macros(D, K, M, &rho, u, &RT);
    double P[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, Q[ORC_MAXD] = {0, 0, 0}, G0n, Gn[ORC_MAXD] = {0, 0, 0};
    orc_neq(D, K, M, rho, u, RT, P, Q, &G0n, Gn);

    double om[3];
    orc_omegas(D, K, RT, p->nu_s, p->nu_b, p->Pr, om);
    double Kn = orc_knudsen(D, K, rho, RT, P, Q, G0n, Gn);
    if (p->limiter)
        for (int i = 0; i < 3; i++) om[i] = orc_limit_omega(Kn, om[i]);
    double wf = om[0], wb = om[1], wh = om[2];

    /* Eq. (IIB10)-(IIB11): bulk and shear parts of M~neq_ab. */
    double bulk = -G0n / D;
    double shear[9];
    for (int a = 0; a < D; a++)
        for (int b = 0; b < D; b++) shear[3 * a + b] = P[3 * a + b] - (a == b ? bulk : 0.0);

    /* Eq. (IIB14): per-dimension heat-flux constraints M~neq_{aa|g}. */
    double h[ORC_MAXD][ORC_MAXD];
    for (int a = 0; a < D; a++)
        for (int g = 0; g < D; g++) h[a][g] = (1.0 + 2.0 * (a == g)) / (D + 2) * Q[g];

    /* Eq. (IIB16)-(IIB17), normalised by Eq. (IIB18).  Constraint order
     * follows the basis T_j of orc_basis_f / orc_basis_g below. */
    double *cf = out->cf, *cg = out->cg;
    for (int j = 0; j < ORC_MAXF; j++) cf[j] = 0.0;
    for (int j = 0; j < ORC_MAXG; j++) cg[j] = 0.0;
    cf[0] = (rho) / rho;                   /* (IIB16a) M~*_0 = rho        */
    /* (IIB16b): M~*_a = 0 -> cf[1..D] stay zero                          */
    int j = 1 + D;
    for (int a = 0; a < D; a++)
        for (int b = a; b < D; b++) {      /* (IIB16c)                     */
            double m = rho * RT * (a == b) + (1.0 - wf) * shear[3 * a + b] +
                       (1.0 - wb) * (a == b ? bulk : 0.0);
            cf[j++] = m / rho;
        }
    for (int g = 0; g < D; g++)            /* (IIB16d)                     */
        for (int a = 0; a < D; a++) cf[j++] = (1.0 - wh) * h[a][g] / rho;

    if (K > 0.0) {
        double nrm = rho * K * RT;
        cg[0] = (rho * K * RT + (1.0 - wb) * G0n) / nrm;          /* (IIB16e) */
        for (int g = 0; g < D; g++) cg[1 + g] = (1.0 - wh) * Gn[g] / nrm; /* (IIB16f) */
        int k = 1 + D;
        for (int a = 0; a < D; a++)
            for (int b = a; b < D; b++)                            /* (IIB17) */
                cg[k++] = (a == b) ? rho * K * RT * RT / nrm : 0.0;
    }
    out->rho = rho;
    for (int a = 0; a < ORC_MAXD; a++) out->u[a] = a < D ? u[a] : 0.0;
    out->RT = RT;
    out->omega[0] = wf;
    out->omega[1] = wb;
    out->omega[2] = wh;
    out->Kn = Kn;
}

/* ------------------------------------------------------------------------ */
/* Lagrangian acoustic stencils, Eq. (IIC6), (IIC9)-(IIC11)                 */
/* ------------------------------------------------------------------------ */

/* [x]: round half away from zero (C99 round). */
static double rnd(double x) { return round(x); }

/* Eq. (IIC6): R_ac = max([n sqrt(RT)], r_min). */
int orc_acoustic_radius(const orc_params* p, double RT)
{
    double r = rnd(p->n_conf * sqrt(RT));
    if (r < p->r_min) r = p->r_min;
    return (int)r;
}

/* Eq. (IIC9): N_r = [1 / (3 sqrt(RT))], capped at max_refine. */
int orc_refine_levels(const orc_params* p, double RT)
{
    double n = rnd(1.0 / (p->refine_div * sqrt(RT)));
    if (n > p->max_refine) n = p->max_refine;
    return (int)n;
}

static double dist2(int D, const double* c, const double* u)
{
    double s = 0.0;
    for (int a = 0; a < D; a++) {
        double d = c[a] - u[a];
        s = s + d * d;
    }
    return s;
}

/* LAS module (Fig. las_module).  reading of Eq. (IIC6): level-0 points are
 * the integer velocities whose distance to the unrounded bulk velocity is at
 * most R_ac + 1/2 (inclusive); this reproduces the 284 points of Fig. 3.
 * reading of Eq. (IIC10)-(IIC11): for Lvl = 1..N_r every point of level
 * Lvl-1 within 3 * 0.5^Lvl of u is replaced by 2^D children at +-h/4 per
 * axis (h = its spacing) with dC scaled by 0.5^D; this reproduces the 41
 * points of Fig. 4.  Returns q, or -q_needed when max_pts is too small. */
int orc_las(int D, const double* u_in, double RT, const orc_params* p, orc_point* pts, int max_pts)
{
    double u[ORC_MAXD];
    for (int a = 0; a < ORC_MAXD; a++) u[a] = a < D ? u_in[a] : 0.0;
    int R = orc_acoustic_radius(p, RT);
    double rr = R + 0.5;
    double rr2 = rr * rr;
    int Nr = orc_refine_levels(p, RT);

    /* level 0: scan the bounding box, keep the disk (ball in 3D) */
    int lo[ORC_MAXD], hi[ORC_MAXD];
    for (int a = 0; a < ORC_MAXD; a++) {
        if (a < D) {
            lo[a] = (int)floor(u[a] - rr) - 1;
            hi[a] = (int)ceil(u[a] + rr) + 1;
        } else {
            lo[a] = hi[a] = 0;
        }
    }
    int cap = 64;
    orc_point* cur = (orc_point*)malloc(sizeof(orc_point) * cap);
    int n = 0;
    for (int cz = lo[2]; cz <= hi[2]; cz++)
        for (int cy = lo[1]; cy <= hi[1]; cy++)
            for (int cx = lo[0]; cx <= hi[0]; cx++) {
                double c[ORC_MAXD] = {(double)cx, (double)cy, (double)cz};
                if (dist2(D, c, u) <= rr2) {
                    if (n == cap) {
                        cap *= 2;
                        cur = (orc_point*)realloc(cur, sizeof(orc_point) * cap);
                    }
                    for (int a = 0; a < ORC_MAXD; a++) cur[n].c[a] = a < D ? c[a] : 0.0;
                    cur[n].dC = 1.0;
                    cur[n].level = 0;
                    n++;
                }
            }

    /* internal refinement, one level at a time */
    double h = 1.0;
    for (int L = 1; L <= Nr; L++) {
        double rad = p->refine_rad * pow(0.5, L);
        double rad2 = rad * rad;
        int cap2 = n * (1 << D) + 8;
        orc_point* nxt = (orc_point*)malloc(sizeof(orc_point) * cap2);
        int m = 0;
        for (int i = 0; i < n; i++) {
            if (cur[i].level == L - 1 && dist2(D, cur[i].c, u) <= rad2) {
                double q4 = h / 4.0;
                int nch = 1 << D;
                for (int k = 0; k < nch; k++) {
                    orc_point ch = cur[i];
                    ch.c[0] = cur[i].c[0] + ((k & 1) ? q4 : -q4);
                    if (D >= 2) ch.c[1] = cur[i].c[1] + ((k & 2) ? q4 : -q4);
                    if (D == 3) ch.c[2] = cur[i].c[2] + ((k & 4) ? q4 : -q4);
                    ch.dC = cur[i].dC * pow(0.5, D);
                    ch.level = L;
                    nxt[m++] = ch;
                }
            } else {
                nxt[m++] = cur[i];
            }
        }
        free(cur);
        cur = nxt;
        n = m;
        h = h / 2.0;
    }
    if (n > max_pts) {
        free(cur);
        return -n;
    }
    memcpy(pts, cur, sizeof(orc_point) * n);
    free(cur);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Entropic population reconstruction, Eq. (IID7)-(IID13)                   */
/* ------------------------------------------------------------------------ */

/* Fluon basis T_j(c~): 1, c~_a, c~_a c~_b (a <= b), c~_a^2 c~_g (Eq. IIB14-16),
 * ordered g-major: (xx|x, yy|x, xx|y, yy|y) in 2D, (xx|x, yy|x, zz|x, xx|y, ...)
 * in 3D. Order of each in ord. */
void orc_basis_f(int D, const double* ct, double* T, int* ord)
{
    int j = 0;
    T[j] = 1.0; if (ord) ord[j] = 0; j++;
    for (int a = 0; a < D; a++) { T[j] = ct[a]; if (ord) ord[j] = 1; j++; }
    for (int a = 0; a < D; a++)
        for (int b = a; b < D; b++) { T[j] = ct[a] * ct[b]; if (ord) ord[j] = 2; j++; }
    for (int g = 0; g < D; g++)
        for (int a = 0; a < D; a++) { T[j] = ct[a] * ct[a] * ct[g]; if (ord) ord[j] = 3; j++; }
}

/* Phonon basis: 1, c~_g, c~_a c~_b (a <= b) (Eq. IIB16e-f, IIB17). */
void orc_basis_g(int D, const double* ct, double* T, int* ord)
{
    int j = 0;
    T[j] = 1.0; if (ord) ord[j] = 0; j++;
    for (int a = 0; a < D; a++) { T[j] = ct[a]; if (ord) ord[j] = 1; j++; }
    for (int a = 0; a < D; a++)
        for (int b = a; b < D; b++) { T[j] = ct[a] * ct[b]; if (ord) ord[j] = 2; j++; }
}

/* Plain Cholesky factorisation A = L L^T and solve A x = b (Golub & Van Loan).
 * A is n x n row-major and is overwritten by L; b is overwritten by x.
 * Returns 0, or -1 on a non-positive pivot. */
int orc_cholesky_solve(int n, double* A, double* b)
{
    for (int j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (int k = 0; k < j; k++) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (int k = 0; k < j; k++) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / d;
        }
    }
    for (int i = 0; i < n; i++) { /* L y = b */
        double t = b[i];
        for (int k = 0; k < i; k++) t -= A[i * n + k] * b[k];
        b[i] = t / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) { /* L^T x = y */
        double t = b[i];
        for (int k = i + 1; k < n; k++) t -= A[k * n + i] * b[k];
        b[i] = t / A[i * n + i];
    }
    return 0;
}

/* Eq. (IID13): Maxwellian start, lambda_0 = -1 + D/2 ln(2 pi RT),
 * lambda_ab = delta_ab / (2 RT), all others 0 (for f and g alike). */
void orc_maxwell_lambda(int D, int kind, double RT, double* lam)
{
    int n = kind == 0 ? orc_nf(D) : orc_ng(D);
    for (int j = 0; j < n; j++) lam[j] = 0.0;
    lam[0] = -1.0 + 0.5 * D * log(2.0 * M_PI * RT);
    int j = 1 + D;
    for (int a = 0; a < D; a++)
        for (int b = a; b < D; b++) { lam[j] = (a == b) ? 1.0 / (2.0 * RT) : 0.0; j++; }
}

/* EPR module (Fig. epr_module).  Newton-Raphson on the Lagrange multipliers
 * of f'_i = dC_i exp[-(1 + sum_j lambda_j T_j(c~_i))] (Eq. IID7), with
 * A_ij = sum_k T_i f_k T_j (IID11a), dM_i = sum_k T_i f_k - M~'_i (IID11c),
 * A dLambda = dM (IID10) solved by Cholesky (Sec. II.D), lambda += dLambda
 * (IID9).  reading: converged when max_j |dM_j| / sqrt(RT)^order_j <= tol
 * (the residual in thermal units), followed by one more (polishing) update.
 * kind 0: fluons (basis orc_basis_f), 1: phonons (orc_basis_g).
 * lam holds the start on entry (NULL-equivalent: caller fills Eq. IID13) and
 * the solution on exit; pop receives f'_i.  Returns the number of updates,
 * or -1 (Cholesky breakdown or non-finite value), -2 (iteration cap). */
int orc_epr(int D, int kind, int q, const orc_point* pts, const double* u, double RT,
            const double* con, const orc_params* p, double* lam, double* pop)
{
    int n = kind == 0 ? orc_nf(D) : orc_ng(D);
    int ord[ORC_MAXF];
    double T[ORC_MAXF];
    double scale[ORC_MAXF];
    double ct0[ORC_MAXD] = {0.0, 0.0, 0.0};
    if (kind == 0) orc_basis_f(D, ct0, T, ord); else orc_basis_g(D, ct0, T, ord);
    for (int j = 0; j < n; j++) scale[j] = pow(sqrt(RT), ord[j]);

    int updates = 0, polished = 0;
    for (int it = 0;; it++) {
        double r[ORC_MAXF];
        for (int j = 0; j < n; j++) r[j] = 0.0;
        for (int k = 0; k < q; k++) {
            double ct[ORC_MAXD];
            for (int a = 0; a < ORC_MAXD; a++) ct[a] = a < D ? pts[k].c[a] - u[a] : 0.0;
            if (kind == 0) orc_basis_f(D, ct, T, NULL); else orc_basis_g(D, ct, T, NULL);
            double e = 1.0;
            for (int j = 0; j < n; j++) e += lam[j] * T[j];
            pop[k] = pts[k].dC * exp(-e);                       /* (IID7)  */
            for (int j = 0; j < n; j++) r[j] += T[j] * pop[k];
        }
        double rmax = 0.0;
        for (int j = 0; j < n; j++) {
            r[j] -= con[j];                                    /* (IID11c) */
            if (!isfinite(r[j])) return -1;
            double a = fabs(r[j]) / scale[j];
            if (a > rmax) rmax = a;
        }
        if (polished) return updates;
        int conv = rmax <= p->tol;
        if (!conv && it >= p->max_iter) return -2;

        double A[ORC_MAXF * ORC_MAXF];                          /* (IID11a) */
        for (int i = 0; i < n * n; i++) A[i] = 0.0;
        for (int k = 0; k < q; k++) {
            double ct[ORC_MAXD];
            for (int a = 0; a < ORC_MAXD; a++) ct[a] = a < D ? pts[k].c[a] - u[a] : 0.0;
            if (kind == 0) orc_basis_f(D, ct, T, NULL); else orc_basis_g(D, ct, T, NULL);
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) A[i * n + j] += T[i] * pop[k] * T[j];
        }
        if (orc_cholesky_solve(n, A, r) != 0) return -1;        /* (IID10) */
        for (int j = 0; j < n; j++) lam[j] += r[j];            /* (IID9)  */
        updates++;
        if (conv) polished = 1;
    }
}

/* ------------------------------------------------------------------------ */
/* single-cell operation and moment streaming                               */
/* ------------------------------------------------------------------------ */

static void equilibrium_constraints(int D, double RT, double* cf, double* cg)
{
    for (int j = 0; j < ORC_MAXF; j++) cf[j] = 0.0;
    for (int j = 0; j < ORC_MAXG; j++) cg[j] = 0.0;
    cf[0] = 1.0;
    cg[0] = 1.0;
    int j = 1 + D;
    for (int a = 0; a < D; a++)
        for (int b = a; b < D; b++) {
            cf[j] = (a == b) ? RT : 0.0;
            cg[j] = (a == b) ? RT : 0.0;
            j++;
        }
}

/* reading (failure handling, not in the paper): a solve that breaks down
 * is redone for f and g with the equilibrium constraints (omega = 1, the
 * Knudsen limiter's end state); if that also fails, the populations are the
 * Maxwellian weights of Eq. (IID12) scaled to carry the exact mass.
 * parity unpinned: the dC factor of those weights (it moves their moments by
 * less than the quadrature error the pins allow). */
static int solve_cell(const orc_params* p, int q, const orc_point* pts, const orc_collision* co,
                      double* popf, double* popg, orc_stats* st)
{
    int D = p->D;
    int has_g = p->K > 0.0;
    double lf[ORC_MAXF], lg[ORC_MAXG];
    orc_maxwell_lambda(D, 0, co->RT, lf);
    int sf = orc_epr(D, 0, q, pts, co->u, co->RT, co->cf, p, lf, popf);
    int sg = 0;
    if (has_g) {
        orc_maxwell_lambda(D, 1, co->RT, lg);
        sg = orc_epr(D, 1, q, pts, co->u, co->RT, co->cg, p, lg, popg);
    }
    if (sf >= 0 && sg >= 0) {
        if (st) {
            st->newton_hist[sf < 63 ? sf : 63]++;
            if (has_g) st->newton_hist[sg < 63 ? sg : 63]++;
        }
        return 0;
    }
    double cf[ORC_MAXF], cg[ORC_MAXG];
    equilibrium_constraints(D, co->RT, cf, cg);
    orc_maxwell_lambda(D, 0, co->RT, lf);
    sf = orc_epr(D, 0, q, pts, co->u, co->RT, cf, p, lf, popf);
    sg = 0;
    if (has_g) {
        orc_maxwell_lambda(D, 1, co->RT, lg);
        sg = orc_epr(D, 1, q, pts, co->u, co->RT, cg, p, lg, popg);
    }
    if (sf >= 0 && sg >= 0) {
        if (st) st->fallback_eq++;
        return 1;
    }
    double s = 0.0;
    for (int k = 0; k < q; k++) {
        double ct[ORC_MAXD];
        for (int a = 0; a < ORC_MAXD; a++) ct[a] = a < D ? pts[k].c[a] - co->u[a] : 0.0;
        double w = pts[k].dC * exp(-dist2(D, ct, (double[ORC_MAXD]){0.0, 0.0, 0.0}) / (2.0 * co->RT));
        popf[k] = w;
        s += w;
    }
    for (int k = 0; k < q; k++) {
        popf[k] /= s;
        if (has_g) popg[k] = popf[k];
    }
    if (st) st->fallback_mx++;
    return 2;
}

/* Populations of one cell: collision, LAS and EPR (Fig. LELBM_algorithm
 * steps 1-3).  pts, popf, popg must hold max_pts entries.  Returns q (or
 * -q_needed), *status the fallback level (0, 1 or 2). */
int orc_cell_populations(const orc_params* p, const double* M, orc_collision* co, orc_point* pts,
                         double* popf, double* popg, int max_pts, int* status)
{
    orc_collide(p, M, co);
    int q = orc_las(p->D, co->u, co->RT, p, pts, max_pts);
    if (q < 0) return q;
    *status = solve_cell(p, q, pts, co, popf, popg, NULL);
    return q;
}

/* Raw moment basis of the stored moments (Eq. IIB5, IIE3a):
 * fluons 1, c_a, c_a c_b (a <= b), |c|^2 c_g; phonons 1, c_g. */
static void raw_contrib(int D, const double* c, double mf, double mg, double* dM)
{
    double csq = 0.0;
    for (int a = 0; a < D; a++) csq += c[a] * c[a];
    dM[0] = mf;
    for (int a = 0; a < D; a++) dM[iM1(D, a)] = c[a] * mf;
    for (int a = 0; a < D; a++)
        for (int b = a; b < D; b++) dM[iM2(D, a, b)] = c[a] * c[b] * mf;
    for (int g = 0; g < D; g++) dM[iMD(D, g)] = csq * c[g] * mf;
    dM[iG0(D)] = mg;
    for (int g = 0; g < D; g++) dM[iG1(D, g)] = c[g] * mg;
}

static int grid_NX(const orc_grid* g) { return g->nx + (g->periodic[0] ? 0 : 2 * g->pad); }
static int grid_NY(const orc_grid* g)
{
    if (g->D == 1) return 1;
    return g->ny + (g->periodic[1] ? 0 : 2 * g->pad);
}
static int grid_NZ(const orc_grid* g)
{
    if (g->D < 3) return 1;
    return g->nz + (g->periodic[2] ? 0 : 2 * g->pad);
}

/* Sec. III.A fluid boundary: pad cells take, on an inflow side, the
 * equilibrium moments of the prescribed state (non-equilibrium dropped),
 * elsewhere the full raw moments of the nearest interior cell.
 * reading: "first-order extrapolation" is the zero-gradient copy; an inflow
 * side wins at corners (x sides before y sides). */
void orc_fill_pads(const orc_grid* g, const orc_params* p, double* M)
{
    int D = g->D, NX = grid_NX(g), NY = grid_NY(g), NZ = grid_NZ(g), nm = orc_nmom(D);
    long ncell = (long)NX * NY * NZ;
    int px = g->periodic[0] ? 0 : g->pad;
    int py = (D == 1 || g->periodic[1]) ? 0 : g->pad;
    int pz = (D < 3 || g->periodic[2]) ? 0 : g->pad;
    int ny = D == 1 ? 1 : g->ny;
    int nz = D < 3 ? 1 : g->nz;
    double Meq[ORC_MAXM];
    double uin[ORC_MAXD] = {g->inlet[1], g->inlet[2], g->inlet[3]};
    orc_eq_moments(D, p->K, g->inlet[0], uin, g->inlet[4], Meq);
    for (int iz = 0; iz < NZ; iz++)
        for (int iy = 0; iy < NY; iy++)
            for (int ix = 0; ix < NX; ix++) {
                int inx = ix >= px && ix < px + g->nx;
                int iny = iy >= py && iy < py + ny;
                int inz = iz >= pz && iz < pz + nz;
                if (inx && iny && inz) continue;
                int inflow = 0;
                if (ix < px && g->bc[0] == 1) inflow = 1;
                if (ix >= px + g->nx && g->bc[1] == 1) inflow = 1;
                if (D >= 2 && iy < py && g->bc[2] == 1) inflow = 1;
                if (D >= 2 && iy >= py + ny && g->bc[3] == 1) inflow = 1;
                if (D == 3 && iz < pz && g->bc[4] == 1) inflow = 1;
                if (D == 3 && iz >= pz + nz && g->bc[5] == 1) inflow = 1;
                long dst = ((long)iz * NY + iy) * NX + ix;
                if (inflow) {
                    for (int m = 0; m < nm; m++) M[m * ncell + dst] = Meq[m];
                } else {
                    int sx = ix < px ? px : (ix >= px + g->nx ? px + g->nx - 1 : ix);
                    int sy = iy < py ? py : (iy >= py + ny ? py + ny - 1 : iy);
                    int sz = iz < pz ? pz : (iz >= pz + nz ? pz + nz - 1 : iz);
                    long src = ((long)sz * NY + sy) * NX + sx;
                    for (int m = 0; m < nm; m++) M[m * ncell + dst] = M[m * ncell + src];
                }
            }
}

/* Landing cell along one axis; returns -1 when the population leaves the
 * interior of a padded axis (it is discarded, Sec. III) . */
static int land_axis(int i, int n, int pad, int periodic)
{
    if (periodic) {
        int r = i % n;
        return r < 0 ? r + n : r;
    }
    if (i < pad || i >= pad + n) return -1;
    return i;
}

/* Solid flag of padded cell (i, j) inside the array.  Interior cells carry the
 * caller's flags.  reading (Sec. III.A with Sec. III.B): a pad cell of an outflow side
 * whose nearest interior cell is solid is solid too -- the wall continues through the
 * pads instead of a pad copying the empty state of a solid cell; inflow pads are
 * never solid. */
static int solid_flag(const orc_grid* g, int NX, int i, int j)
{
    int px = g->periodic[0] ? 0 : g->pad;
    int py = (g->D == 1 || g->periodic[1]) ? 0 : g->pad;
    int ny = g->D == 1 ? 1 : g->ny;
    int inx = i >= px && i < px + g->nx, iny = j >= py && j < py + ny;
    if (inx && iny) return g->solid[(long)j * NX + i];
    if ((i < px && g->bc[0] == 1) || (i >= px + g->nx && g->bc[1] == 1)) return 0;
    if (g->D >= 2 && ((j < py && g->bc[2] == 1) || (j >= py + ny && g->bc[3] == 1))) return 0;
    int si = i < px ? px : (i >= px + g->nx ? px + g->nx - 1 : i);
    int sj = j < py ? py : (j >= py + ny ? py + ny - 1 : j);
    return g->solid[(long)sj * NX + si];
}

/* The bit a wall kind sets in a path's contact record: 1 slip wall, 2 no-slip wall at
 * rest, 4 moving no-slip wall. */
static int kind_bit(int kind) { return kind == 0 ? 0 : (kind == 2 ? 2 : (kind == 3 ? 4 : 1)); }
/* The no-slip boundary n (Eq. IIIB8) a contact belongs to: 1 at rest, 2 moving, 0 none. */
static int noslip_of(int kind) { return kind == 2 ? 1 : (kind == 3 ? 2 : 0); }

/* Sec. III.B: the wall kind of padded cell (i, j): 0 fluid, 1 slip wall, 2 no-slip
 * wall (stationary).  Cells outside the array are fluid (their populations are
 * discarded later). */
static int solid_at(const orc_grid* g, int NX, int NY, int i, int j)
{
    if (!g->solid) return 0;
    if (g->periodic[0]) i = ((i % NX) + NX) % NX;
    if (g->D == 2 && g->periodic[1]) j = ((j % NY) + NY) % NY;
    if (i < 0 || i >= NX || j < 0 || j >= NY) return 0;
    return solid_flag(g, NX, i, j);
}

/* Sec. III.B, first step of the extended bounce-back: the path x -> x + c is
 * followed cell by cell, and at a face of a solid cell the population is
 * specularly reflected (the normal component of its velocity flips) until the
 * whole displacement is used.  reading: for a stationary adiabatic slip wall the
 * image populations of Eq. (IIIB10)-(IIIB15) are built from the cell's own
 * post-collision moments (u_n = u, Eq. IIIB11-12), so they are the reflected
 * real populations and the mass ratio of Eq. (IIIB15) is one.  Face crossings
 * are ordered exactly in integer units of 1/64 cell.  reading: a path through a
 * cell corner whose diagonal cell is solid reflects only the component normal
 * to a flat wall (one of the two side cells solid, the other fluid) and both
 * components otherwise; with the diagonal cell fluid it passes the corner.
 * parity unpinned: the corner rule at an isolated convex corner, which has no
 * image construction (conservation and mirror symmetry still hold there).
 * Returns the walls the path touched (bit 1: a slip wall, bit 2: a no-slip wall at rest,
 * bit 4: a moving no-slip wall; 0: none) and, in bits 4-5, the last no-slip boundary it
 * touched (1 at rest, 2 moving); *fi, *fj receive the final cell, off[] the final offset
 * from its centre, cs[] the reflected velocity c*. */
int orc_trace_path(const orc_grid* g, int NX, int NY, int ix, int iy, const double* c, int* fi, int* fj,
                      double* off, double* cs)
{
    const long S = 64;
    int D = g->D;
    long qx = lround(S * c[0]), qy = D == 2 ? lround(S * c[1]) : 0;
    int sx = qx > 0 ? 1 : (qx < 0 ? -1 : 0), sy = qy > 0 ? 1 : (qy < 0 ? -1 : 0);
    long ax = labs(qx), ay = labs(qy);
    int i = ix, j = iy, touched = 0, last_ns = 0;
    long kx = 0, ky = 0;
    for (;;) {
        long Xn = S / 2 + S * kx, Yn = S / 2 + S * ky;
        int hx = ax > 0 && Xn < ax, hy = ay > 0 && Yn < ay;
        if (!hx && !hy) break;
        int stx = hx, sty = hy;
        if (hx && hy) {
            long l = Xn * ay, r = Yn * ax;
            stx = l <= r;
            sty = r <= l;
        }
        if (stx && sty) {
            /* through a cell corner: a flat wall along one axis reflects only
             * that component, a corner of solid cells reflects both */
            if (!solid_at(g, NX, NY, i + sx, j + sy)) {
                i += sx;
                j += sy;
            } else {
                int sd = solid_at(g, NX, NY, i + sx, j + sy);
                int sa = solid_at(g, NX, NY, i + sx, j), sb = solid_at(g, NX, NY, i, j + sy);
                if (sa && !sb) {
                    touched |= kind_bit(sa);
                    if (noslip_of(sa)) last_ns = noslip_of(sa);
                    sx = -sx;
                    j += sy;
                } else if (sb && !sa) {
                    touched |= kind_bit(sb);
                    if (noslip_of(sb)) last_ns = noslip_of(sb);
                    sy = -sy;
                    i += sx;
                } else {
                    touched |= kind_bit(sd) | kind_bit(sa) | kind_bit(sb);
                    /* a corner: the diagonal cell, else a side cell, names the boundary */
                    int k = noslip_of(sd) ? sd : (noslip_of(sa) ? sa : sb);
                    if (noslip_of(k)) last_ns = noslip_of(k);
                    sx = -sx;
                    sy = -sy;
                }
            }
        } else {
            int ti = i + (stx ? sx : 0), tj = j + (sty ? sy : 0);
            int st = solid_at(g, NX, NY, ti, tj);
            if (st) {
                if (stx) sx = -sx;
                if (sty) sy = -sy;
                touched |= kind_bit(st);
                if (noslip_of(st)) last_ns = noslip_of(st);
            } else {
                i = ti;
                j = tj;
            }
        }
        if (stx) kx++;
        if (sty) ky++;
    }
    *fi = i;
    *fj = j;
    off[0] = sx * (double)(ax - S * kx) / S;
    off[1] = sy * (double)(ay - S * ky) / S;
    cs[0] = sx * fabs(c[0]);
    cs[1] = D == 2 ? sy * fabs(c[1]) : 0.0;
    return touched | (last_ns << 4);
}

enum { STREAM_REAL = 0, STREAM_IMAGE_SUM = 1, STREAM_IMAGE_PUT = 2 };

/* Lands one population of padded cell (ix, iy, iz) with velocity c, mass fraction mf
 * and phonon energy fraction mg (Eq. IIE3).  Without walls it goes to x + c; with
 * walls its path is traced (Sec. III.B).  The landing point is shared between the
 * cells it overlaps by cloud-in-cell weights.
 *   STREAM_REAL: a path that touched a no-slip wall is absorbed by the last no-slip
 *     boundary n it touched (acc[2(n-1)] += mf, acc[2(n-1)+1] += mg; Eq. IIIB8), as is a
 *     share that would fall on a no-slip cell (by that cell's boundary); a share that
 *     would fall on a slip cell is mirrored back (the slip-wall reading); the rest is
 *     deposited.
 *   STREAM_IMAGE_SUM / _PUT (c is the reversed velocity -c_i of an image population of
 *     boundary sel, Eq. IIIB13): only a path whose last no-slip contact is boundary sel
 *     enters; shares that would fall on a wall cell are dropped.  _SUM adds the mass of
 *     what enters to acc[0..1] (Eq. IIIB14), _PUT deposits it scaled by sf (f) and sg
 *     (g) (Eq. IIIB15). */
static void stream_one(const orc_grid* g, int NX, int NY, int NZ, int ix, int iy, int iz, const double* c,
                       double mf, double mg, int mode, int sel, double sf, double sg, double* Mout, double* acc,
                       orc_stats* st)
{
    int D = g->D, nm = orc_nmom(D);
    long ncell = (long)NX * NY * NZ;
    int px = g->periodic[0] ? 0 : g->pad;
    int py = (D == 1 || g->periodic[1]) ? 0 : g->pad;
    int pz = (D < 3 || g->periodic[2]) ? 0 : g->pad;
    int ny = D == 1 ? 1 : g->ny;
    int nz = D < 3 ? 1 : g->nz;
    const unsigned char* solid = D <= 2 ? g->solid : NULL;
    /* landing point: x + c, or the end of the reflected path (Sec. III.B) */
    double cl[ORC_MAXD] = {c[0], D >= 2 ? c[1] : 0.0, D == 3 ? c[2] : 0.0}, pos[ORC_MAXD];
    int fi = ix, fj = iy;
    if (solid) {
        double off[2];
        int touched = orc_trace_path(g, NX, NY, ix, iy, c, &fi, &fj, off, cl);
        int ns = touched >> 4; /* the last no-slip boundary the path touched */
        if (mode == STREAM_REAL) {
            if (st && (touched & 15)) st->wall_hits++;
            if (ns) {
                acc[2 * (ns - 1)] += mf;
                acc[2 * (ns - 1) + 1] += mg;
                return;
            }
        } else if (ns != sel) {
            return;
        }
        pos[0] = fi + off[0];
        pos[1] = fj + off[1];
        pos[2] = 0.0;
    } else {
        pos[0] = ix + c[0];
        pos[1] = iy + (D >= 2 ? c[1] : 0.0);
        pos[2] = iz + (D == 3 ? c[2] : 0.0);
    }
    /* cloud-in-cell split of the landing position */
    int i0[ORC_MAXD] = {0, 0, 0};
    double w1[ORC_MAXD] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; a++) {
        double fl = floor(pos[a]);
        i0[a] = (int)fl;
        w1[a] = pos[a] - fl;
    }
    int ncx = w1[0] > 0.0 ? 2 : 1;
    int ncy = (D >= 2 && w1[1] > 0.0) ? 2 : 1;
    int ncz = (D == 3 && w1[2] > 0.0) ? 2 : 1;
    for (int sz = 0; sz < ncz; sz++)
        for (int sy = 0; sy < ncy; sy++)
            for (int sx = 0; sx < ncx; sx++) {
                double w = (sx ? w1[0] : 1.0 - w1[0]);
                if (D >= 2) w *= (sy ? w1[1] : 1.0 - w1[1]);
                if (D == 3) w *= (sz ? w1[2] : 1.0 - w1[2]);
                int cx_ = i0[0] + sx, cy_ = D >= 2 ? i0[1] + sy : 0, cz_ = D == 3 ? i0[2] + sz : 0;
                double cw[ORC_MAXD] = {cl[0], cl[1], cl[2]};
                int kind = solid ? solid_at(g, NX, NY, cx_, cy_) : 0;
                if (kind && mode != STREAM_REAL) continue;
                if (noslip_of(kind)) {
                    acc[2 * (noslip_of(kind) - 1)] += w * mf;
                    acc[2 * (noslip_of(kind) - 1) + 1] += w * mg;
                    continue;
                }
                /* reading: a share that would fall on a slip-wall cell is the mirror
                 * image of one arriving from the image lattice, so it is mirrored
                 * back across the wall with the normal velocity component reversed
                 * (exact for flat walls, Sec. III.B).  A diagonal share behind a
                 * flat wall (one side cell fluid) goes to that side cell; behind a
                 * corner of solid cells it goes to the final cell, both reversed. */
                if (kind) {
                    int ox = cx_ != fi, oy = cy_ != fj;
                    if (ox && oy) {
                        int sa = solid_at(g, NX, NY, cx_, fj), sb = solid_at(g, NX, NY, fi, cy_);
                        if (!sa && sb) {
                            ox = 0; /* keep x: mirror across the y wall */
                        } else if (sa && !sb) {
                            oy = 0; /* keep y: mirror across the x wall */
                        }
                    }
                    if (ox) {
                        cw[0] = -cw[0];
                        cx_ = fi;
                    }
                    if (oy) {
                        cw[1] = -cw[1];
                        cy_ = fj;
                    }
                }
                /* px = 0 on a periodic axis, py and pz likewise */
                int tx = land_axis(cx_, g->nx, px, g->periodic[0]);
                int ty = 0, tz = 0;
                if (D >= 2) ty = land_axis(cy_, ny, py, g->periodic[1]);
                if (D == 3) tz = land_axis(cz_, nz, pz, g->periodic[2]);
                if (mode == STREAM_IMAGE_SUM) {
                    acc[0] += w * mf;
                    acc[1] += w * mg;
                    continue;
                }
                if (tx < 0 || ty < 0 || tz < 0) continue;
                double dM[ORC_MAXM];
                if (mode == STREAM_IMAGE_PUT)
                    raw_contrib(D, cw, sf * mf, sg * mg, dM);
                else
                    raw_contrib(D, cw, mf, mg, dM);
                long tgt = ((long)tz * NY + ty) * NX + tx;
                for (int m = 0; m < nm; m++) Mout[m * ncell + tgt] += w * dM[m];
            }
}

/* One time step over a padded grid: fill the pads, then for every non-solid
 * cell run collision, LAS and EPR and stream the moment fractions
 * T_N(c_i) rho f'_i and T_N(c_i) rho K RT g'_i to x + c_i (Eq. IIE3).
 * reading: a refined point lands off the lattice; its fractions are shared
 * between the cells it overlaps by cloud-in-cell weights (cell averaging,
 * Eq. IIA10-11).  parity unpinned: that spread beyond the share's centre of
 * mass.  Min and Mout are SoA [nmom][NY*NX]; Min is not modified.
 * Returns 0, or -1 on allocation failure. */
int orc_step(const orc_grid* g, const orc_params* p, const double* Min, double* Mout, orc_stats* st)
{
    int D = g->D, NX = grid_NX(g), NY = grid_NY(g), NZ = grid_NZ(g), nm = orc_nmom(D);
    long ncell = (long)NX * NY * NZ;
    int px = g->periodic[0] ? 0 : g->pad;
    int py = (D == 1 || g->periodic[1]) ? 0 : g->pad;
    int pz = (D < 3 || g->periodic[2]) ? 0 : g->pad;
    int ny = D == 1 ? 1 : g->ny;
    int nz = D < 3 ? 1 : g->nz;
    const unsigned char* solid = D <= 2 ? g->solid : NULL; /* solid cells: 1D and 2D only */
    double* W = (double*)malloc(sizeof(double) * nm * ncell);
    if (!W) return -1;
    memcpy(W, Min, sizeof(double) * nm * ncell);
    orc_fill_pads(g, p, W);
    memset(Mout, 0, sizeof(double) * nm * ncell);

    int cap = 4096;
    orc_point* pts = (orc_point*)malloc(sizeof(orc_point) * cap);
    double* popf = (double*)malloc(sizeof(double) * cap);
    double* popg = (double*)malloc(sizeof(double) * cap);
    int icap = 0; /* image velocity sets of moving walls */
    orc_point* imp = NULL;
    double *imf = NULL, *img = NULL;
    for (int iz = 0; iz < NZ; iz++)
    for (int iy = 0; iy < NY; iy++)
        for (int ix = 0; ix < NX; ix++) {
            long cell = ((long)iz * NY + iy) * NX + ix;
            if (solid && solid_flag(g, NX, ix, iy)) continue;
            double M[ORC_MAXM];
            for (int m = 0; m < nm; m++) M[m] = W[m * ncell + cell];
            orc_collision co;
            orc_collide(p, M, &co);
            int q = orc_las(D, co.u, co.RT, p, pts, cap);
            if (q < 0) {
                cap = -q;
                pts = (orc_point*)realloc(pts, sizeof(orc_point) * cap);
                popf = (double*)realloc(popf, sizeof(double) * cap);
                popg = (double*)realloc(popg, sizeof(double) * cap);
                q = orc_las(D, co.u, co.RT, p, pts, cap);
            }
            solve_cell(p, q, pts, &co, popf, popg, st);
            if (st) {
                st->cells++;
                if (q > st->q_max) st->q_max = q;
            }
            double mscale = co.rho;                  /* rho dV f'   (IIE3a) */
            double gscale = co.rho * p->K * co.RT;   /* rho K RT dV g'      */
            double absorbed[4] = {0.0, 0.0, 0.0, 0.0}; /* Eq. (IIIB8): Delta m (f, g) of the
                                                         no-slip boundaries at rest, moving */
            for (int k = 0; k < q; k++) {
                const double* c = pts[k].c;
                if (st) {
                    double cm = sqrt(dist2(D, c, (double[ORC_MAXD]){0.0, 0.0, 0.0}));
                    if (cm > st->disp_max) st->disp_max = cm;
                }
                double mf = mscale * popf[k], mg = p->K > 0.0 ? gscale * popg[k] : 0.0;
                stream_one(g, NX, NY, NZ, ix, iy, iz, c, mf, mg, STREAM_REAL, 0, 1.0, 1.0, Mout, absorbed, st);
            }
            for (int n = 1; n <= 2; n++) {
                double* dm = absorbed + 2 * (n - 1);
                if (!(dm[0] > 0.0 || dm[1] > 0.0)) continue;
                /* Eq. (IIIB10)-(IIIB15): the image populations of boundary n are the EPR
                 * populations of the cell's post-collision central moments at the bulk
                 * velocity u_n = u - 2 u_w (Eq. IIIB11; both components: no slip),
                 * launched with -c_i; those whose last no-slip contact is boundary n enter
                 * the domain, scaled so that their mass equals what boundary n absorbed.
                 * At rest (u_w = 0) they are the cell's own populations. */
                int qi = q;
                orc_point* ipts = pts;
                double *ipf = popf, *ipg = popg;
                if (n == 2) {
                    orc_collision cn = co;
                    for (int a = 0; a < D; a++) cn.u[a] = co.u[a] - 2.0 * g->wall_u[a];
                    if (icap < cap) {
                        icap = cap;
                        imp = (orc_point*)realloc(imp, sizeof(orc_point) * icap);
                        imf = (double*)realloc(imf, sizeof(double) * icap);
                        img = (double*)realloc(img, sizeof(double) * icap);
                    }
                    qi = orc_las(D, cn.u, co.RT, p, imp, icap);
                    if (qi < 0) {
                        icap = -qi;
                        imp = (orc_point*)realloc(imp, sizeof(orc_point) * icap);
                        imf = (double*)realloc(imf, sizeof(double) * icap);
                        img = (double*)realloc(img, sizeof(double) * icap);
                        qi = orc_las(D, cn.u, co.RT, p, imp, icap);
                    }
                    solve_cell(p, qi, imp, &cn, imf, img, NULL);
                    ipts = imp;
                    ipf = imf;
                    ipg = img;
                }
                double kept[2] = {0.0, 0.0};
                for (int pass = 0; pass < 2; pass++) {
                    double sf = kept[0] > 0.0 ? dm[0] / kept[0] : 0.0;
                    double sg = kept[1] > 0.0 ? dm[1] / kept[1] : 0.0;
                    for (int k = 0; k < qi; k++) {
                        double cm[ORC_MAXD] = {-ipts[k].c[0], -ipts[k].c[1], -ipts[k].c[2]};
                        double mf = mscale * ipf[k], mg = p->K > 0.0 ? gscale * ipg[k] : 0.0;
                        stream_one(g, NX, NY, NZ, ix, iy, iz, cm, mf, mg,
                                   pass == 0 ? STREAM_IMAGE_SUM : STREAM_IMAGE_PUT, n, sf, sg, Mout, kept, st);
                    }
                }
                /* reading: no image reaches the domain (a cell boxed in by walls): the
                 * absorbed mass and internal energy stay in the cell, at rest */
                int sxi = land_axis(ix, g->nx, px, g->periodic[0]);
                int syi = D >= 2 ? land_axis(iy, ny, py, g->periodic[1]) : 0;
                if (sxi >= 0 && syi >= 0) {
                    long self = ((long)iz * NY + iy) * NX + ix;
                    if (kept[0] <= 0.0) Mout[self] += dm[0];
                    if (kept[1] <= 0.0) Mout[(long)iG0(D) * ncell + self] += dm[1];
                }
            }
        }
    free(pts);
    free(popf);
    free(popg);
    free(imp);
    free(imf);
    free(img);
    free(W);
    return 0;
}
