/*
 * axilbm_oracle.c -- plain FP64 CPU oracle of the axisymmetric Allen-Cahn
 * phase-field MRT lattice Boltzmann model (Liang et al., arXiv 1810.09299).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the CUDA product path never does.  It
 * shares no code with the CUDA library.
 *
 * Deliberately written in velocity space, one equation at a time, from the
 * paper's discrete-velocity formulas (Eq. 9-11, 14-17, 24-35, 38-40) with the
 * explicit 9x9 matrices M and M^-1.  The moment-space closed forms
 * (Eq. 21-23, 36-37) that the CUDA path uses are NOT used here; the tests
 * check the two against each other.  No blocking, fusion or reordering beyond
 * the paper's algorithm:
 *   Eq. 16 phi -> Eq. 39/40 stencils (ghosts per Sec. 2.3) -> Eq. 17, 35, 4 ->
 *   Eq. 32 u and Eq. 33 p (solved together per node) -> Eq. 30 F -> Eq. 19 f-collision
 *   (Eq. 10, 11, 14, 15, 38) -> Eq. 24 g-collision (Eq. 25-29) ->
 *   Eq. 20 streaming with axis symmetry and halfway bounce-back.
 *
 * Readings of points on which the paper is silent (each listed in the design
 * notes): Eq. 32 and Eq. 33 solved together per node (the lagged p^{n-1} is an
 * option), n = grad/(|grad|+eps),
 * d(r rho) taken analytically from grad(phi), halfway mirror ghosts, axis
 * specular reflection, corner links bounced back, G = ((rho-rho_l) g_z, 0),
 * initial state f = f^eq(phi0, 0), g = 0, chi^{-1} = chi^0, p^{-1} = 0.
 *
 * Option: the non-orthogonal (raw-moment) MRT that the paper's summary
 * (Sec. 4) names as a direct extension -- the same Eq. 10 / Eq. 24 collisions
 * with M replaced by the raw-moment basis, and s_p of Eq. 33 re-derived for it
 * (see node_macros).
 */
#include "axilbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2/3 with c = 1 (Eq. 12) */

/* ------------------------------------------------------------------ */
/* Lattice (Eq. 12) and the transformation matrix M (Sec. 2.2)          */
/* ------------------------------------------------------------------ */
static int g_cz[Q], g_cr[Q];
static double g_w[Q];
static double g_M[Q * Q], g_Minv[Q * Q];
static double g_T[Q * Q], g_Tinv[Q * Q];
static int g_opp[Q], g_rmirror[Q];
static int g_ready = 0;

/* c_i from Eq. 12: the paper's first component is z (x), the second r (y). */
static void build_lattice(void)
{
    const double pi = acos(-1.0);
    g_cz[0] = 0;
    g_cr[0] = 0;
    for (int i = 1; i <= 4; ++i) {
        double a = (i - 1) * pi / 2.0;
        g_cz[i] = (int)lround(cos(a));
        g_cr[i] = (int)lround(sin(a));
    }
    for (int i = 5; i <= 8; ++i) {
        double a = (i - 5) * pi / 2.0 + pi / 4.0;
        g_cz[i] = (int)lround(sqrt(2.0) * cos(a));
        g_cr[i] = (int)lround(sqrt(2.0) * sin(a));
    }
    g_w[0] = 4.0 / 9.0;
    for (int i = 1; i <= 4; ++i) g_w[i] = 1.0 / 9.0;
    for (int i = 5; i <= 8; ++i) g_w[i] = 1.0 / 36.0;
    /* opposite and r-mirror directions, found by search over the vectors */
    for (int i = 0; i < Q; ++i) {
        for (int j = 0; j < Q; ++j) {
            if (g_cz[j] == -g_cz[i] && g_cr[j] == -g_cr[i]) g_opp[i] = j;
            if (g_cz[j] == g_cz[i] && g_cr[j] == -g_cr[i]) g_rmirror[i] = j;
        }
    }
}

/* The matrix M printed in Sec. 2.2 (Lallemand-Luo ordering). */
static const double M_PAPER[Q * Q] = {
     1,  1,  1,  1,  1,  1,  1,  1,  1,
    -4, -1, -1, -1, -1,  2,  2,  2,  2,
     4, -2, -2, -2, -2,  1,  1,  1,  1,
     0,  1,  0, -1,  0,  1, -1, -1,  1,
     0, -2,  0,  2,  0,  1, -1, -1,  1,
     0,  0,  1,  0, -1,  1,  1, -1, -1,
     0,  0, -2,  0,  2,  1,  1, -1, -1,
     0,  1, -1,  1, -1,  0,  0,  0,  0,
     0,  0,  0,  0,  0,  1, -1,  1, -1,
};

/* Gauss-Jordan inversion with partial pivoting (a library-style primitive). */
static void invert9(const double* A, double* Ainv)
{
    double a[Q][2 * Q];
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < 2 * Q; ++j)
            a[i][j] = (j < Q) ? A[i * Q + j] : (j - Q == i ? 1.0 : 0.0);
    for (int c = 0; c < Q; ++c) {
        int piv = c;
        for (int i = c + 1; i < Q; ++i)
            if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
        if (piv != c)
            for (int j = 0; j < 2 * Q; ++j) {
                double t = a[c][j];
                a[c][j] = a[piv][j];
                a[piv][j] = t;
            }
        double d = a[c][c];
        for (int j = 0; j < 2 * Q; ++j) a[c][j] /= d;
        for (int i = 0; i < Q; ++i) {
            if (i == c) continue;
            double m = a[i][c];
            if (m == 0.0) continue;
            for (int j = 0; j < 2 * Q; ++j) a[i][j] -= m * a[c][j];
        }
    }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) Ainv[i * Q + j] = a[i][Q + j];
}

/* The non-orthogonal (raw-moment) basis that the paper's summary (Sec. 4)
 * names as the direct extension of its orthogonal MRT: row k holds the
 * polynomial p_k(c) at every lattice vector, with
 *   p = 1, c_z, c_r, c_z^2 + c_r^2, c_z^2 - c_r^2, c_z c_r, c_z^2 c_r, c_z c_r^2,
 *       c_z^2 c_r^2. */
static void build_raw_basis(void)
{
    for (int i = 0; i < Q; ++i) {
        const double z = g_cz[i], r = g_cr[i];
        const double row[Q] = {1.0, z, r, z * z + r * r, z * z - r * r, z * r, z * z * r, z * r * r, z * z * r * r};
        for (int k = 0; k < Q; ++k) g_T[k * Q + i] = row[k];
    }
}

static void ensure_tables(void)
{
    if (g_ready) return;
    build_lattice();
    memcpy(g_M, M_PAPER, sizeof(g_M));
    invert9(g_M, g_Minv);
    build_raw_basis();
    invert9(g_T, g_Tinv);
    g_ready = 1;
}

static void matvec9(const double* A, const double* x, double* y)
{
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int j = 0; j < Q; ++j) s += A[i * Q + j] * x[j];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Equilibria, sources and the collision operator                        */
/* ------------------------------------------------------------------ */

/* Eq. 11: f_i^eq = w_i [ r phi + c_ia (r phi u_a + M phi delta_ar) / cs2 ] */
void orc_feq(double r, double phi, double uz, double ur, double mobility, double* feq)
{
    ensure_tables();
    double chi_z = r * phi * uz;
    double chi_r = r * phi * ur + mobility * phi;
    for (int i = 0; i < Q; ++i)
        feq[i] = g_w[i] * (r * phi + (g_cz[i] * chi_z + g_cr[i] * chi_r) / CS2);
}

/* Eq. 15: R_i = w_i c_ia [ d_t chi_a + cs2 r n_a lambda ] / cs2,
 * chi = (r phi u_z, r phi u_r + M phi). */
void orc_R(double r, double dchi_z, double dchi_r, double nz_, double nr_, double lam, double* R)
{
    ensure_tables();
    double az = dchi_z + CS2 * r * nz_ * lam;
    double ar = dchi_r + CS2 * r * nr_ * lam;
    for (int i = 0; i < Q; ++i) R[i] = g_w[i] * (g_cz[i] * az + g_cr[i] * ar) / CS2;
}

/* Eq. 26: s_i(u) */
static double s_of_u(int i, double uz, double ur)
{
    double cu = g_cz[i] * uz + g_cr[i] * ur;
    double uu = uz * uz + ur * ur;
    return g_w[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 25 */
void orc_geq(double r, double p, double rho, double uz, double ur, double* geq)
{
    ensure_tables();
    for (int i = 0; i < Q; ++i) {
        double wi = (i == 0) ? (g_w[i] - 1.0) : g_w[i];
        geq[i] = r * p / CS2 * wi + r * rho * s_of_u(i, uz, ur);
    }
}

/* Eq. 29: T_i = w_i [ c_ia F_a / cs2 + u_a d_b(r rho) c_ia c_ib / cs2 - rho u_r ] */
void orc_T(double rho, double uz, double ur, double Fz, double Fr,
           double dz_rrho, double dr_rrho, double* T)
{
    ensure_tables();
    double u[2] = {uz, ur};
    double d[2] = {dz_rrho, dr_rrho};
    for (int i = 0; i < Q; ++i) {
        double c[2] = {(double)g_cz[i], (double)g_cr[i]};
        double quad = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) quad += u[a] * d[b] * c[a] * c[b];
        T[i] = g_w[i] * ((c[0] * Fz + c[1] * Fr) / CS2 + quad / CS2 - rho * ur);
    }
}

/* Eq. 19 with Eq. 10 and Eq. 14 (and the same form, Eq. 24 + Eq. 27, for g)
 * in the moment basis B:
 * x+ = x - B^-1 S B (x - xeq) + B^-1 (I - S/2) B src.
 * The matrix products are applied right to left to the vectors. */
static void collide_in_basis(const double* B, const double* Binv, const double* x, const double* xeq,
                             const double* src, const double* S, double* xpost)
{
    double d[Q], md[Q], ms[Q], msrc[Q], back1[Q], back2[Q];
    for (int i = 0; i < Q; ++i) d[i] = x[i] - xeq[i];
    matvec9(B, d, md);
    for (int i = 0; i < Q; ++i) md[i] *= S[i];
    matvec9(Binv, md, back1);
    matvec9(B, src, msrc);
    for (int i = 0; i < Q; ++i) ms[i] = (1.0 - 0.5 * S[i]) * msrc[i];
    matvec9(Binv, ms, back2);
    for (int i = 0; i < Q; ++i) xpost[i] = x[i] - back1[i] + back2[i];
}

/* the paper's orthogonal MRT: B = M of Sec. 2.2 */
void orc_mrt_collide(const double* x, const double* xeq, const double* src, const double* S,
                     double* xpost)
{
    ensure_tables();
    collide_in_basis(g_M, g_Minv, x, xeq, src, S, xpost);
}

/* the raw-moment (non-orthogonal) MRT: B = the raw basis above, S the rates of
 * its nine moments */
void orc_raw_collide(const double* x, const double* xeq, const double* src, const double* S,
                     double* xpost)
{
    ensure_tables();
    collide_in_basis(g_T, g_Tinv, x, xeq, src, S, xpost);
}

/* ------------------------------------------------------------------ */
/* Stencils, Eq. 39-40, with the ghost rules of Sec. 2.3                 */
/* ------------------------------------------------------------------ */

/* Ghost lookup: mirror about the axis (r = 0, between j = -1 and j = 0),
 * mirror about the halfway wall planes, periodic wrap in z when enabled. */
static double field_at(int nr, int nz, int zper, const double* f, int k, int j)
{
    while (j < 0 || j >= nr) {
        if (j < 0) j = -1 - j;
        if (j >= nr) j = 2 * nr - 1 - j;
    }
    if (zper) {
        k %= nz;
        if (k < 0) k += nz;
    } else {
        while (k < 0 || k >= nz) {
            if (k < 0) k = -1 - k;
            if (k >= nz) k = 2 * nz - 1 - k;
        }
    }
    return f[(size_t)k * nr + j];
}

static void stencil_at(int nr, int nz, int zper, const double* f, int k, int j,
                       double* dz, double* dr, double* lap)
{
    double c0 = f[(size_t)k * nr + j];
    double gz = 0.0, gr = 0.0, lp = 0.0;
    for (int i = 1; i < Q; ++i) {
        double x1 = field_at(nr, nz, zper, f, k + g_cz[i], j + g_cr[i]);
        double x2 = field_at(nr, nz, zper, f, k + 2 * g_cz[i], j + 2 * g_cr[i]);
        gz += g_w[i] * g_cz[i] * (8.0 * x1 - x2);
        gr += g_w[i] * g_cr[i] * (8.0 * x1 - x2);
        lp += g_w[i] * (16.0 * x1 - x2 - 15.0 * c0);
    }
    *dz = gz / (6.0 * CS2);
    *dr = gr / (6.0 * CS2);
    *lap = lp / (6.0 * CS2);
}

void orc_stencil(int nr, int nz, int z_periodic, const double* field,
                 double* dz, double* dr, double* lap)
{
    ensure_tables();
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nr; ++j) {
            size_t n = (size_t)k * nr + j;
            stencil_at(nr, nz, z_periodic, field, k, j, &dz[n], &dr[n], &lap[n]);
        }
}

/* ------------------------------------------------------------------ */
/* State                                                                 */
/* ------------------------------------------------------------------ */
struct orc_state {
    orc_params prm;
    size_t n;            /* nodes */
    double *f, *g;       /* [9][nz][nr] post-streaming populations at time n */
    double *fn, *gn;     /* streaming targets */
    double *chi_z, *chi_r, *p_prev; /* chi^{n-1}, p^{n-1} */
    double *phi;         /* work: phi^n */
    int64_t steps;
    double tau_f;        /* from Eq. 18 */
};

void orc_lattice(int* cz, int* cr, double* w)
{
    ensure_tables();
    for (int i = 0; i < Q; ++i) {
        cz[i] = g_cz[i];
        cr[i] = g_cr[i];
        w[i] = g_w[i];
    }
}
void orc_matrix_M(double* M) { ensure_tables(); memcpy(M, g_M, sizeof(g_M)); }
void orc_matrix_Minv(double* Minv) { ensure_tables(); memcpy(Minv, g_Minv, sizeof(g_Minv)); }
void orc_matrix_T(double* T) { ensure_tables(); memcpy(T, g_T, sizeof(g_T)); }
void orc_matrix_Tinv(double* Tinv) { ensure_tables(); memcpy(Tinv, g_Tinv, sizeof(g_Tinv)); }

void orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

orc_state* orc_create(const orc_params* prm)
{
    ensure_tables();
    if (!prm || prm->nr < 2 || prm->nz < 2) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->prm = *prm;
    s->n = (size_t)prm->nr * prm->nz;
    s->f = (double*)calloc(Q * s->n, sizeof(double));
    s->g = (double*)calloc(Q * s->n, sizeof(double));
    s->fn = (double*)calloc(Q * s->n, sizeof(double));
    s->gn = (double*)calloc(Q * s->n, sizeof(double));
    s->chi_z = (double*)calloc(s->n, sizeof(double));
    s->chi_r = (double*)calloc(s->n, sizeof(double));
    s->p_prev = (double*)calloc(s->n, sizeof(double));
    s->phi = (double*)calloc(s->n, sizeof(double));
    if (!s->f || !s->g || !s->fn || !s->gn || !s->chi_z || !s->chi_r || !s->p_prev || !s->phi) {
        orc_destroy(s);
        return NULL;
    }
    /* Eq. 18: M = cs2 (tau_f - 1/2) */
    s->tau_f = prm->mobility / CS2 + 0.5;
    return s;
}

void orc_destroy(orc_state* s)
{
    if (!s) return;
    free(s->f);
    free(s->g);
    free(s->fn);
    free(s->gn);
    free(s->chi_z);
    free(s->chi_r);
    free(s->p_prev);
    free(s->phi);
    free(s);
}

static double radius(int j) { return j + 0.5; } /* first lattice line at r = 0.5 */

int orc_init(orc_state* s, const double* phi0)
{
    const orc_params* P = &s->prm;
    const int nr = P->nr, nz = P->nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nr; ++j) {
            size_t n = (size_t)k * nr + j;
            double r = radius(j), feq[Q];
            orc_feq(r, phi0[n], 0.0, 0.0, P->mobility, feq);
            for (int i = 0; i < Q; ++i) {
                s->f[i * s->n + n] = feq[i];
                s->g[i * s->n + n] = 0.0; /* g^eq(p = 0, u = 0) = 0 */
            }
            s->chi_z[n] = 0.0;
            s->chi_r[n] = P->mobility * phi0[n];
            s->p_prev[n] = 0.0;
        }
    s->steps = 0;
    return 0;
}

/* Per-node macroscopic quantities of one time level. */
typedef struct {
    double r, phi, rho, nu, dphiz, dphir, lap;
    double mu, mut, Fsz, Fsr, Gz, Gr;
    double uz, ur, p, pstar;
    double Fz, Fr;
    double nz_, nr_, lam;
    double sf[Q], sg[Q];
} node_macro;

/* Eq. 16 for every node. */
static void compute_phi(orc_state* s)
{
    const int nr = s->prm.nr, nz = s->prm.nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nr; ++j) {
            size_t n = (size_t)k * nr + j;
            double sum = 0.0;
            for (int i = 0; i < Q; ++i) sum += s->f[i * s->n + n];
            s->phi[n] = sum / radius(j);
        }
}

/* Everything a node needs before collision: Eq. 4, 17, 35, 2, 31-33, 30. */
static void node_macros(const orc_state* s, int k, int j, node_macro* m)
{
    const orc_params* P = &s->prm;
    const int nr = P->nr, nz = P->nz;
    const size_t n = (size_t)k * nr + j;
    const double r = radius(j);
    m->r = r;
    m->phi = s->phi[n];
    stencil_at(nr, nz, P->z_periodic, s->phi, k, j, &m->dphiz, &m->dphir, &m->lap);
    /* Eq. 17, Eq. 35 */
    m->rho = m->phi * P->rho_l + (1.0 - m->phi) * P->rho_g;
    m->nu = m->phi * P->nu_l + (1.0 - m->phi) * P->nu_g;
    /* rates: Eq. 13 with Eq. 18; Eq. 28 with Eq. 34 */
    double tau_g = m->nu / CS2 + 0.5;
    for (int i = 0; i < Q; ++i) {
        m->sf[i] = (P->sf[i] < 0.0) ? 1.0 / s->tau_f : P->sf[i];
        m->sg[i] = (P->sg[i] < 0.0) ? 1.0 / tau_g : P->sg[i];
    }
    /* Eq. 4 and the axisymmetric potential mu~ = mu - k d_r phi / r (Sec. 2.1) */
    double beta = 12.0 * P->sigma / P->W;
    double kap = 1.5 * P->sigma * P->W;
    m->mu = 4.0 * beta * m->phi * (m->phi - 1.0) * (m->phi - 0.5) - kap * m->lap;
    m->mut = m->mu - kap * m->dphir / r;
    m->Fsz = m->mut * m->dphiz;
    m->Fsr = m->mut * m->dphir;
    m->Gz = (m->rho - P->rho_l) * P->grav_z;
    m->Gr = 0.0;
    /* Eq. 2 and the interface normal */
    double gnorm = sqrt(m->dphiz * m->dphiz + m->dphir * m->dphir);
    m->nz_ = m->dphiz / (gnorm + P->n_eps);
    m->nr_ = m->dphir / (gnorm + P->n_eps);
    m->lam = -4.0 * (m->phi - 1.0) * m->phi / P->W;
    /* first moments of g and the sum over i != 0 */
    double Jz = 0.0, Jr = 0.0, S0 = 0.0;
    for (int i = 0; i < Q; ++i) {
        double gi = s->g[i * s->n + n];
        Jz += g_cz[i] * gi;
        Jr += g_cr[i] * gi;
        if (i != 0) S0 += gi;
    }
    double drho = P->rho_l - P->rho_g;
    double dzrho = drho * m->dphiz, drrho = drho * m->dphir;
    /* s_p of Eq. 33 (Appendix C).  In the raw basis the i = 0 row of
     * T^-1 S^-1 T takes raw moments 0, 3 and 8 (x_0 = k_0 - k_3 + k_8), and the
     * appendix's argument, with the moments of its Eq. C.7 matched term by term,
     * gives s_p = 3 / (2 s_3) - 1 / (2 s_8) - 1/2 (equal to the orthogonal s_p
     * whenever the two collisions coincide, e.g. for a single rate). */
    double sp = (P->collision == 1)
                    ? 1.5 / m->sg[3] - 0.5 / m->sg[8] - 0.5
                    : (m->sg[1] + m->sg[2] - m->sg[1] * m->sg[2]) / (2.0 * m->sg[1] * m->sg[2]);
    double w0 = g_w[0];
    /* Eq. 32, z component (independent of p) */
    m->uz = (Jz + 0.5 * r * (m->Fsz + m->Gz)) / (r * m->rho);
    double Dr = r * m->rho + m->nu * m->rho / r;
    if (P->p_coupling == 1) {
        /* lagged pressure p^{n-1} in Eq. 32 and Eq. 30 */
        m->pstar = s->p_prev[n];
        m->ur = (Jr + 0.5 * (r * (m->Fsr + m->Gr) + m->pstar)) / Dr;
        /* Eq. 33 */
        double uu = m->uz * m->uz + m->ur * m->ur;
        double s0u = w0 * (-uu / (2.0 * CS2));
        m->p = CS2 / (1.0 - w0) *
               (S0 / r + 0.5 * (m->uz * dzrho + m->ur * drrho) + m->rho * s0u -
                sp * w0 * m->rho * m->ur / r);
    } else {
        /* exact node-local solve of Eq. 32 (r) with Eq. 33: u_r = a + b p,
         * p = A0 + A1 u_r - A2 u_r^2 -> quadratic in p; take the root that
         * tends to the linear solution as A2 -> 0. */
        double a = (Jr + 0.5 * r * (m->Fsr + m->Gr)) / Dr;
        double b = 0.5 / Dr;
        double c = CS2 / (1.0 - w0);
        double A0 = c * (S0 / r + 0.5 * m->uz * dzrho - w0 * m->rho * m->uz * m->uz / (2.0 * CS2));
        double A1 = c * (0.5 * drrho - sp * w0 * m->rho / r);
        double A2 = c * w0 * m->rho / (2.0 * CS2);
        double qa = A2 * b * b;
        double qb = 1.0 - A1 * b + 2.0 * A2 * a * b;
        double qc = -(A0 + A1 * a - A2 * a * a);
        double disc = qb * qb - 4.0 * qa * qc;
        double p = (disc >= 0.0) ? (-2.0 * qc / (qb + sqrt(disc))) : (-qc / qb);
        m->p = p;
        m->pstar = p;
        m->ur = a + b * p;
    }
    /* Eq. 30 */
    m->Fz = r * (m->Fsz + m->Gz);
    m->Fr = r * (m->Fsr + m->Gr) + (m->pstar - 2.0 * m->rho * m->nu * m->ur / r);
}

int orc_step(orc_state* s, int64_t nsteps)
{
    const orc_params* P = &s->prm;
    const int nr = P->nr, nz = P->nz, zper = P->z_periodic;
    const size_t N = s->n;
    for (int64_t t = 0; t < nsteps; ++t) {
        compute_phi(s);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k) {
            for (int j = 0; j < nr; ++j) {
                const size_t n = (size_t)k * nr + j;
                node_macro m;
                node_macros(s, k, j, &m);
                const double r = m.r;
                /* ---- phase-field LBE: Eq. 19 with Eq. 11, 14, 15, 38 ---- */
                double f[Q], feq[Q], R[Q], fpost[Q];
                for (int i = 0; i < Q; ++i) f[i] = s->f[i * N + n];
                orc_feq(r, m.phi, m.uz, m.ur, P->mobility, feq);
                double chiz = r * m.phi * m.uz;
                double chir = r * m.phi * m.ur + P->mobility * m.phi;
                orc_R(r, chiz - s->chi_z[n], chir - s->chi_r[n], m.nz_, m.nr_, m.lam, R);
                if (P->collision == 1) orc_raw_collide(f, feq, R, m.sf, fpost);
                else orc_mrt_collide(f, feq, R, m.sf, fpost);
                /* ---- hydrodynamic LBE: Eq. 24 with Eq. 25-30 ---- */
                double g[Q], geq[Q], T[Q], gpost[Q];
                for (int i = 0; i < Q; ++i) g[i] = s->g[i * N + n];
                orc_geq(r, m.p, m.rho, m.uz, m.ur, geq);
                double drho = P->rho_l - P->rho_g;
                double dz_rrho = r * drho * m.dphiz;            /* d_z (r rho) */
                double dr_rrho = m.rho + r * drho * m.dphir;    /* d_r (r rho) */
                orc_T(m.rho, m.uz, m.ur, m.Fz, m.Fr, dz_rrho, dr_rrho, T);
                if (P->collision == 1) orc_raw_collide(g, geq, T, m.sg, gpost);
                else orc_mrt_collide(g, geq, T, m.sg, gpost);
                /* time-level bookkeeping for Eq. 38 and the lagged p */
                s->chi_z[n] = chiz;
                s->chi_r[n] = chir;
                s->p_prev[n] = m.p;
                /* ---- Eq. 20: streaming with boundary rules ---- */
                for (int i = 0; i < Q; ++i) {
                    int kt = k + g_cz[i], jt = j + g_cr[i];
                    int zout = 0;
                    if (zper) {
                        kt %= nz;
                        if (kt < 0) kt += nz;
                    } else if (kt < 0 || kt >= nz) {
                        zout = 1;
                    }
                    if (zout || jt >= nr) {
                        /* halfway bounce-back at a wall (also at any corner) */
                        s->fn[g_opp[i] * N + n] = fpost[i];
                        s->gn[g_opp[i] * N + n] = gpost[i];
                    } else if (jt < 0) {
                        /* specular reflection at the symmetry axis */
                        size_t t2 = (size_t)kt * nr + 0;
                        s->fn[g_rmirror[i] * N + t2] = fpost[i];
                        s->gn[g_rmirror[i] * N + t2] = gpost[i];
                    } else {
                        size_t t2 = (size_t)kt * nr + jt;
                        s->fn[i * N + t2] = fpost[i];
                        s->gn[i * N + t2] = gpost[i];
                    }
                }
            }
        }
        double* tmp = s->f;
        s->f = s->fn;
        s->fn = tmp;
        tmp = s->g;
        s->g = s->gn;
        s->gn = tmp;
        s->steps += 1;
    }
    return 0;
}

int orc_fields(orc_state* s, double* phi, double* rho, double* uz, double* ur, double* p)
{
    const int nr = s->prm.nr, nz = s->prm.nz;
    compute_phi(s);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nr; ++j) {
            size_t n = (size_t)k * nr + j;
            node_macro m;
            node_macros(s, k, j, &m);
            if (phi) phi[n] = m.phi;
            if (rho) rho[n] = m.rho;
            if (uz) uz[n] = m.uz;
            if (ur) ur[n] = m.ur;
            if (p) p[n] = m.p;
        }
    return 0;
}

int orc_get_populations(const orc_state* s, double* f, double* g)
{
    if (f) memcpy(f, s->f, Q * s->n * sizeof(double));
    if (g) memcpy(g, s->g, Q * s->n * sizeof(double));
    return 0;
}

int orc_set_populations(orc_state* s, const double* f, const double* g)
{
    if (f) memcpy(s->f, f, Q * s->n * sizeof(double));
    if (g) memcpy(s->g, g, Q * s->n * sizeof(double));
    return 0;
}

int orc_get_aux(const orc_state* s, double* chi_z, double* chi_r, double* p_prev)
{
    if (chi_z) memcpy(chi_z, s->chi_z, s->n * sizeof(double));
    if (chi_r) memcpy(chi_r, s->chi_r, s->n * sizeof(double));
    if (p_prev) memcpy(p_prev, s->p_prev, s->n * sizeof(double));
    return 0;
}

int orc_set_aux(orc_state* s, const double* chi_z, const double* chi_r, const double* p_prev)
{
    if (chi_z) memcpy(s->chi_z, chi_z, s->n * sizeof(double));
    if (chi_r) memcpy(s->chi_r, chi_r, s->n * sizeof(double));
    if (p_prev) memcpy(s->p_prev, p_prev, s->n * sizeof(double));
    return 0;
}

int64_t orc_step_count(const orc_state* s) { return s->steps; }

/* Diagnostics: plain FP64 sums in node order.  A node whose phi, u_z, u_r or
 * p is not finite is counted in `nonfinite` and left out of every sum and
 * extremum (the paper defines these quantities for finite states only; the
 * count says how many nodes were left out). */
int orc_diagnostics(orc_state* s, orc_diag* out)
{
    const int nr = s->prm.nr, nz = s->prm.nz;
    const size_t N = s->n;
    double* ph = (double*)malloc(N * sizeof(double));
    double* rh = (double*)malloc(N * sizeof(double));
    double* uz = (double*)malloc(N * sizeof(double));
    double* ur = (double*)malloc(N * sizeof(double));
    double* p = (double*)malloc(N * sizeof(double));
    if (!ph || !rh || !uz || !ur || !p) {
        free(ph); free(rh); free(uz); free(ur); free(p);
        return -1;
    }
    orc_fields(s, ph, rh, uz, ur, p);
    double mass = 0, ke = 0, zm = 0, umax = 0, pin = 0, win = 0, pout = 0, wout = 0;
    double pmin = 1e300, pmax = -1e300, bad = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nr; ++j) {
            size_t n = (size_t)k * nr + j;
            double r = radius(j), z = k + 0.5;
            if (!isfinite(ph[n]) || !isfinite(uz[n]) || !isfinite(ur[n]) || !isfinite(p[n])) {
                bad += 1;
                continue;
            }
            mass += r * ph[n];
            double uu = uz[n] * uz[n] + ur[n] * ur[n];
            ke += 0.5 * r * rh[n] * uu;
            zm += r * z * ph[n];
            double um = sqrt(uu);
            if (um > umax) umax = um;
            if (ph[n] > 0.99) { pin += r * p[n]; win += r; }
            if (ph[n] < 0.01) { pout += r * p[n]; wout += r; }
            if (ph[n] < pmin) pmin = ph[n];
            if (ph[n] > pmax) pmax = ph[n];
        }
    out->step = (double)s->steps;
    out->mass = mass;
    out->kinetic = ke;
    out->z_centroid = zm / mass;
    out->dp = (win > 0 ? pin / win : 0.0) - (wout > 0 ? pout / wout : 0.0);
    out->umax = umax;
    out->phi_min = pmin;
    out->phi_max = pmax;
    /* half-length of the phi > 1/2 set along the axis row j = 0 (linear crossings) */
    double len = 0.0;
    for (int k = 0; k < nz; ++k) {
        double a = ph[(size_t)k * nr] - 0.5;
        int kn = k + 1;
        if (kn >= nz) {
            if (!s->prm.z_periodic) {
                if (a > 0) len += 0.5; /* half cell to the wall plane */
                break;
            }
            kn = 0;
        }
        double b = ph[(size_t)kn * nr] - 0.5;
        if (a > 0 && b > 0) len += 1.0;
        else if (a > 0 && b <= 0) len += a / (a - b);
        else if (a <= 0 && b > 0) len += b / (b - a);
    }
    if (!s->prm.z_periodic && ph[0] - 0.5 > 0) len += 0.5;
    out->axis_half_length = 0.5 * len;
    /* radial crossing on the row nearest the centroid */
    int kc = (int)floor(out->z_centroid);
    if (kc < 0) kc = 0;
    if (kc >= nz) kc = nz - 1;
    double rc = 0.0;
    for (int j = 0; j + 1 < nr; ++j) {
        double a = ph[(size_t)kc * nr + j] - 0.5, b = ph[(size_t)kc * nr + j + 1] - 0.5;
        if (a > 0 && b <= 0) {
            rc = radius(j) + a / (a - b);
            break;
        }
    }
    out->radial_half_length = rc;
    out->nonfinite = bad;
    free(ph); free(rh); free(uz); free(ur); free(p);
    return 0;
}

/* Drops on the axis (the bodies a breaking thread forms, Sec. 3.3): maximal
 * runs of axis nodes (j = 0) with phi > 1/2.  Written in two passes: first the
 * runs, then for each gas gap between two runs the row of least sum_j r phi
 * (first such row) where the rows are split between the two drops; a drop's
 * volume is 2 pi sum r phi over its rows.  In a walled case the rows before the
 * first run and after the last one belong to those runs; in a periodic case
 * the gap that wraps around is split like the others. */
int orc_axis_drops(orc_state* s, int max_drops, double* out, int* n_drops, double* axis_min)
{
    const int nr = s->prm.nr, nz = s->prm.nz, zper = s->prm.z_periodic;
    const double two_pi = 2.0 * acos(-1.0);
    double* ph = (double*)malloc(s->n * sizeof(double));
    double* w = (double*)malloc((size_t)nz * sizeof(double));
    int* rs = (int*)malloc((size_t)(nz + 1) * sizeof(int)); /* first row of each run */
    int* re = (int*)malloc((size_t)(nz + 1) * sizeof(int)); /* last row of each run */
    if (!ph || !w || !rs || !re) {
        free(ph); free(w); free(rs); free(re);
        return -1;
    }
    orc_fields(s, ph, NULL, NULL, NULL, NULL);
    for (int k = 0; k < nz; ++k) {
        w[k] = 0.0;
        for (int j = 0; j < nr; ++j) w[k] += radius(j) * ph[(size_t)k * nr + j];
    }
    int kmin = 0;
    for (int k = 1; k < nz; ++k)
        if (ph[(size_t)k * nr] < ph[(size_t)kmin * nr]) kmin = k;
    if (axis_min) {
        axis_min[0] = ph[(size_t)kmin * nr];
        axis_min[1] = kmin + 0.5;
    }
#define LIQ(k) (ph[(size_t)(k) * nr] > 0.5)
    /* pass 1: runs, in rows 0 .. nz-1 */
    int nruns = 0;
    for (int k = 0; k < nz; ++k) {
        if (LIQ(k) && (k == 0 || !LIQ(k - 1))) rs[nruns] = k;
        if (LIQ(k) && (k == nz - 1 || !LIQ(k + 1))) re[nruns++] = k;
    }
    /* periodic: a run through z = 0 and one through z = nz are one drop */
    int all_liquid = (nruns == 1 && rs[0] == 0 && re[0] == nz - 1);
    if (zper && nruns >= 2 && rs[0] == 0 && re[nruns - 1] == nz - 1) {
        rs[0] = rs[nruns - 1];   /* the merged drop starts in the last run */
        nruns -= 1;
        /* rotate so that the merged drop comes last (scan order starts after a gap) */
        int s0 = rs[0], e0 = re[0];
        for (int m = 0; m + 1 < nruns; ++m) { rs[m] = rs[m + 1]; re[m] = re[m + 1]; }
        rs[nruns - 1] = s0;
        re[nruns - 1] = e0;
    } else if (zper && nruns >= 1 && !all_liquid) {
        /* order the runs from the first gap after z = 0: a run starting at row 0
         * (the gap before it wraps) is kept last */
        if (rs[0] == 0) {
            int s0 = rs[0], e0 = re[0];
            for (int m = 0; m + 1 < nruns; ++m) { rs[m] = rs[m + 1]; re[m] = re[m + 1]; }
            rs[nruns - 1] = s0;
            re[nruns - 1] = e0;
        }
    }
    *n_drops = nruns;
    if (nruns == 0) {
        free(ph); free(w); free(rs); free(re);
        return 0;
    }
    if (all_liquid && zper) {
        double v = 0.0;
        for (int k = 0; k < nz; ++k) v += w[k];
        if (max_drops > 0) {
            out[0] = 0.0;
            out[1] = nz;
            out[2] = two_pi * v;
            out[3] = cbrt(3.0 * out[2] / (4.0 * acos(-1.0)));
        }
        free(ph); free(w); free(rs); free(re);
        return 0;
    }
    /* pass 2: the cut row of the gap after each run (cyclic in periodic cases);
     * walled: the last run takes every row up to nz */
    for (int m = 0; m < nruns && m < max_drops; ++m) {
        double* d = out + 4 * m;
        /* ends: crossings between the run's outer rows and the gas rows next to them */
        int kb = rs[m] - 1, ka = re[m] + 1;
        if (!zper && rs[m] == 0) d[0] = 0.0;
        else {
            int k0 = (kb + nz) % nz;
            double a = ph[(size_t)k0 * nr], b = ph[(size_t)rs[m] * nr];
            double z = (kb + 0.5) + (0.5 - a) / (b - a);
            d[0] = z < 0.0 ? z + nz : z;
        }
        if (!zper && re[m] == nz - 1) d[1] = nz;
        else {
            int k1 = ka % nz;
            double a = ph[(size_t)re[m] * nr], b = ph[(size_t)k1 * nr];
            double z = (re[m] + 0.5) + (0.5 - a) / (b - a);
            d[1] = z >= nz ? z - nz : z;
        }
    }
    /* cut rows: cut[m] = first row of drop m's share (rows cut[m] .. cut[m+1]-1, cyclic) */
    int* cut = (int*)malloc((size_t)(nruns + 1) * sizeof(int));
    if (!cut) {
        free(ph); free(w); free(rs); free(re);
        return -1;
    }
    for (int m = 0; m < nruns; ++m) {
        /* the gap before run m: from the row after the previous run's end */
        int prev = (m == 0) ? (zper ? nruns - 1 : -1) : m - 1;
        if (prev < 0) {
            cut[m] = 0;
            continue;
        }
        int g0 = (re[prev] + 1) % nz, len = (rs[m] - g0 + nz) % nz;
        int best = g0;
        for (int q = 1; q < len; ++q) {
            int k = (g0 + q) % nz;
            if (w[k] < w[best]) best = k;
        }
        cut[m] = best;
    }
    for (int m = 0; m < nruns && m < max_drops; ++m) {
        int a = cut[m];
        int b = (m + 1 < nruns) ? cut[m + 1] : (zper ? cut[0] : nz);
        int len = zper ? ((b - a + nz) % nz) : (b - a);
        if (zper && len == 0) len = nz;
        double v = 0.0;
        for (int q = 0; q < len; ++q) v += w[(a + q) % nz];
        out[4 * m + 2] = two_pi * v;
        out[4 * m + 3] = cbrt(3.0 * out[4 * m + 2] / (4.0 * acos(-1.0)));
    }
#undef LIQ
    free(cut);
    free(ph); free(w); free(rs); free(re);
    return 0;
}
