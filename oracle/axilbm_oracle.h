/*
 * axilbm_oracle.h -- plain FP64 CPU oracle of the axisymmetric Allen-Cahn
 * phase-field MRT lattice Boltzmann step (Liang et al., arXiv 1810.09299).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * restatement of the paper's equations that the CUDA path is checked against.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or helper with the CUDA
 * library, and it never calls it.
 *
 * Lattice: D2Q9 on the (z, r) plane, node (k, j) with k = 0..nz-1 along z and
 * j = 0..nr-1 along r; the first lattice line sits at r = 0.5 (Sec. 2.3), so
 * r_j = j + 0.5.  Arrays are row-major [z][r] (r fastest); population arrays
 * are [9][nz][nr].
 */
#ifndef AXILBM_ORACLE_H
#define AXILBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Physical and numerical parameters of one case.
 * sf / sg: diagonal MRT rates (Eq. 13, Eq. 28).  A negative entry means
 * "derived": sf[i] < 0 -> 1/tau_f with M = cs2 (tau_f - 1/2) (Eq. 18);
 * sg[i] < 0 -> 1/tau_g(x) with nu(x) = cs2 (tau_g - 1/2) (Eq. 34) and
 * nu(x) from Eq. 35 at each node.
 * grav_z: z-component of the gravitational acceleration; the body force is
 * G = ((rho - rho_l) grav_z, 0) (buoyancy relative to the liquid).
 * p_coupling: 0 = node-local exact solve of Eq. 32 + Eq. 33 for (u, p)
 *                 (p appears in u_r and u in p; the pair is a quadratic in p);
 *             1 = lagged pressure p^{n-1} in Eq. 32 and Eq. 30.
 * n_eps: n = grad(phi) / (|grad(phi)| + n_eps).
 * collision: 0 = the paper's orthogonal MRT (M of Sec. 2.2);
 *            1 = raw-moment MRT: M replaced by the non-orthogonal basis
 *                1, c_z, c_r, c_z^2 + c_r^2, c_z^2 - c_r^2, c_z c_r, c_z^2 c_r,
 *                c_z c_r^2, c_z^2 c_r^2 (the extension named in Sec. 4); sf / sg
 *                are then the rates of these moments. */
typedef struct {
    int32_t nr, nz, z_periodic;
    int32_t p_coupling;
    int32_t collision;
    double rho_l, rho_g, nu_l, nu_g, sigma, W, mobility, grav_z;
    double sf[9], sg[9];
    double n_eps;
} orc_params;

typedef struct orc_state orc_state;

/* Diagnostics record (all FP64).  Nodes whose phi, u_z, u_r or p is not
 * finite are left out of every sum and extremum and counted in nonfinite. */
typedef struct {
    double step;            /* number of completed time steps */
    double mass;            /* sum_nodes r*phi (= sum of all f) */
    double kinetic;         /* sum_nodes 0.5 r rho |u|^2 */
    double z_centroid;      /* sum r z phi / sum r phi, z_k = k + 0.5 */
    double dp;              /* <p>_{phi>0.99} - <p>_{phi<0.01}, r-weighted means */
    double umax;            /* max |u| */
    double phi_min, phi_max;
    double axis_half_length;   /* half the length of phi>1/2 along the axis row j=0 */
    double radial_half_length; /* phi=1/2 crossing along r on the row nearest z_centroid */
    double nonfinite;       /* number of nodes with a non-finite phi, u or p */
} orc_diag;

orc_state* orc_create(const orc_params* prm);
void orc_destroy(orc_state* s);
/* phi0: [nz][nr]. Sets f = f^eq(phi0, u=0), g = 0, chi^{-1} = (0, M phi0), p^{-1} = 0. */
int orc_init(orc_state* s, const double* phi0);
int orc_step(orc_state* s, int64_t nsteps);
/* Any pointer may be NULL. Each output is [nz][nr]. */
int orc_fields(orc_state* s, double* phi, double* rho, double* uz, double* ur, double* p);
int orc_get_populations(const orc_state* s, double* f, double* g);
int orc_set_populations(orc_state* s, const double* f, const double* g);
int orc_get_aux(const orc_state* s, double* chi_z, double* chi_r, double* p_prev);
int orc_set_aux(orc_state* s, const double* chi_z, const double* chi_r, const double* p_prev);
int orc_diagnostics(orc_state* s, orc_diag* out);
/* Drops on the axis row (phi > 1/2 runs; Sec. 3.3): *n_drops found, out[4 m ..]
 * = (z_start, z_end, volume, equivalent radius) for m < max_drops; axis_min
 * (may be NULL) = (least phi of the axis row, its z). */
int orc_axis_drops(orc_state* s, int max_drops, double* out, int* n_drops, double* axis_min);
int64_t orc_step_count(const orc_state* s);
void orc_set_threads(int nthreads);

/* ---- building blocks, exposed for the pin tests ---- */
void orc_lattice(int* cz, int* cr, double* w);          /* 9 each */
void orc_matrix_M(double* M);                           /* 81, row-major */
void orc_matrix_Minv(double* Minv);                     /* 81, Gauss-Jordan inverse of M */
void orc_matrix_T(double* T);                           /* 81, raw-moment basis */
void orc_matrix_Tinv(double* Tinv);                     /* 81, Gauss-Jordan inverse of T */
/* Eq. 11 */
void orc_feq(double r, double phi, double uz, double ur, double mobility, double* feq);
/* Eq. 15 */
void orc_R(double r, double dchi_z, double dchi_r, double nz_, double nr_, double lam, double* R);
/* Eq. 25-26 */
void orc_geq(double r, double p, double rho, double uz, double ur, double* geq);
/* Eq. 29; drz_rho = d(r rho)/dz, drr_rho = d(r rho)/dr */
void orc_T(double rho, double uz, double ur, double Fz, double Fr,
           double dz_rrho, double dr_rrho, double* T);
/* Eq. 10 + Eq. 14 / Eq. 24 + Eq. 27: x+ = x - M^-1 S M (x - xeq) + M^-1 (I - S/2) M src */
void orc_mrt_collide(const double* x, const double* xeq, const double* src, const double* S,
                     double* xpost);
/* the same with the raw-moment basis T in place of M */
void orc_raw_collide(const double* x, const double* xeq, const double* src, const double* S,
                     double* xpost);
/* Eq. 39 and Eq. 40 on an arbitrary [nz][nr] field with the ghost rules of Sec. 2.3 */
void orc_stencil(int nr, int nz, int z_periodic, const double* field,
                 double* dz, double* dr, double* lap);

#ifdef __cplusplus
}
#endif
#endif
