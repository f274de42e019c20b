/*
 * gks_oracle.h -- interface of the plain FP64 CPU oracle (test infrastructure
 * only; see gks_oracle.c). Not included by, and not linked into, the CUDA
 * library.
 */
#ifndef GKS_ORACLE_H
#define GKS_ORACLE_H

#define OG_GHOST 3
#define OG_MAX_OBJECTS 16
#define OG_MAX_BLADES 8

/* Boundary kinds. Their numeric values are part of the public interface of
 * the method (the C-ABI library uses the same numbers). */
enum { OG_BC_PERIODIC = 0, OG_BC_NOSLIP = 1, OG_BC_SLIP = 2, OG_BC_INFLOW = 3, OG_BC_OUTFLOW = 4 };

typedef struct og_grid og_grid;

og_grid *og_create(const int n[3], const double *xf0, const double *xf1, const double *xf2,
                   double mach, double u_ref, double mu, const int bc[6], double cfl,
                   double dt_fixed);
void og_destroy(og_grid *g);
const char *og_last_error(og_grid *g);
long og_num_cells(const og_grid *g);
void og_set_inflow(og_grid *g, double rho, double u, double v, double w);
void og_set_body_force(og_grid *g, double fx, double fy, double fz);
void og_set_state(og_grid *g, const double *Q);
void og_get_state(const og_grid *g, double *Q);
double og_time(const og_grid *g);
double og_last_dt(const og_grid *g);
void og_set_time(og_grid *g, double t);
double og_cfl_dt(const og_grid *g);
int og_step(og_grid *g, int nsteps);
void og_rhs(og_grid *g, const double *Q, double *L, double *Lt);
void og_ghost_filled(og_grid *g, const double *Q, double *out);
void og_diagnostics(const og_grid *g, double out[5]);
int og_add_rotor(og_grid *g, int nb, int np, const double hub[3], double omega, double azimuth0,
                 double radius, double eps, double rho_inf, double u_inf_ref, const double *r,
                 const double *chord, const double *twist, const double *width, int correction,
                 int tip_correction);
int og_set_force_scales(og_grid *g, int id, const double *s);
int og_add_body(og_grid *g, int n, const double *xyz, const double *dS, const double *vel,
                double eps, int niter, double tol);
long og_body_fields(og_grid *g, int id, long bb[6], double *Vbar, double *phi);
int og_forces(og_grid *g, int id, double *out, double *points);
void og_set_threads(int n);
int og_get_threads(void);

/* building blocks exposed for the pins */
double og_weno5(const double q[5]);
void og_weno5_parts(const double q[5], double p[3], double beta[3], double w[3]);
double og_normal_derivative(double q0, const double c[4]);
void og_tangential(const double q[5], double val[2], double der[2]);
double og_linear5_face(const double q[5]);
void og_stencil_table(double dn_w[5], double tv_w[10], double td_w[10], double weno_d[3]);
void og_moments(double U, double lambda, int kmax, double *M);
void og_half_moments(double U, double lambda, int sign, double out[2]);
void og_coeff_solve(double U, double V, double W, double lambda, const double d[4], double a[4]);
void og_flux_local(double lambda, double mu, const double Q[4], const double Dn[4],
                   const double Dt1[4], const double Dt2[4], double F0[4], double F1[4]);
void og_equilibrium_local(double lambda, const double Ql[4], const double Qr[4], double Q0[4]);
double og_gauss_kernel(double r, double eps);
void og_s2o4_stage1(long n, double dt, const double *W, const double *L, const double *Lt,
                    double *Ws);
void og_s2o4_stage2(long n, double dt, const double *W, const double *L, const double *Lt,
                    const double *Lts, double *Wn);

#endif
