/*
 * FP64 CPU oracle for the chemical-potential multiphase LBM step
 * (Qin, Chen, Qin, Xu, Wen, "Spurious currents suppression by accurate
 * difference schemes in multiphase lattice Boltzmann method").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include,
 * link or call this code: only the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg use it.  It shares no header, table or
 * helper with the CUDA library.
 *
 * Everything is plain double precision, plain nested loops, in the order the
 * paper states the algorithm (Sec. 2.1-2.3).  Built with -ffp-contract=off so
 * that results do not depend on whether the host has FMA.
 *
 * Parity pins: every function here is pinned by a CPU test against a
 * property fixed by the paper or by mathematics (see tests/test_oracle_*.py).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* lattices */
#define OR_D2Q9 0
#define OR_D3Q19 1

/* finite-difference schemes (Sec. 2.3) */
#define OR_EFDS2 0  /* Eq. 18 */
#define OR_EFDS4 1  /* Eq. 19 */
#define OR_EFDS6 2  /* Eq. 20 */
#define OR_CFDS4 3  /* Eq. 22 */
#define OR_CFDS6 4  /* Eq. 23 */
#define OR_CFDS8 5  /* Eq. 24 */
#define OR_OCFDS4 6 /* Sec. 3.1 optimal fourth-order compact */
#define OR_E4 7     /* Eq. 25, fourth-order isotropic */
#define OR_E8 8     /* Eq. 25, eighth-order isotropic (2D only) */
#define OR_NSCHEMES 9

/* status codes */
#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2
#define OR_EUNSTABLE -4

/* collision operators */
#define OR_BGK 0 /* every MRT rate 1/tau: single relaxation (Sec. 2.1, after Eq. 5) */
#define OR_MRT 1 /* Eq. 1 with M of Eq. 3 and S of Eq. 5 (D2Q9 only) */

typedef struct {
  int lattice;          /* OR_D2Q9 or OR_D3Q19 */
  int nx, ny, nz;       /* nz = 1 for D2Q9; x fastest */
  double a, b, R, Tr;   /* Carnahan-Starling constants and reduced temperature */
  double k, kappa, tau; /* proportional coefficient (Eq. 16), kappa-hat, BGK tau */
  int scheme;           /* OR_EFDS2 .. OR_E8 */
  int collision;        /* OR_BGK or OR_MRT */
  double mrt_s[9];      /* OR_MRT: s_1 .. s_9 of Eq. 5 */
  int eos;              /* OR_EOS_CS, OR_EOS_PR, OR_EOS_VDW or OR_EOS_RKS */
  double acentric;      /* OR_EOS_PR: acentric factor of alpha(T) (Eq. 15) */
} or_params;

typedef struct {
  double max_v, max_u, rho_center, rho_corner, mass, max_drho;
  long long step;
  int status;
} or_obs;

typedef struct or_sim or_sim;

/* ---- lattice, equilibrium, forcing (Sec. 2.1) ---- */
int or_lattice_q(int lattice);
void or_lattice_e(int lattice, int* e /* Q*3 */, double* w /* Q */);
void or_feq(int lattice, double rho, const double u[3], double* feq);
void or_edm(int lattice, double rho, const double u[3], const double F[3], double* Fi);

/* ---- Carnahan-Starling EOS and chemical potential (Eq. 10-13, 16) ---- */
double or_cs_pressure(double rho, double a, double b, double R, double T);
double or_cs_mu(double rho, double a, double b, double R, double T);
int or_cs_critical(double a, double b, double R, double* rho_c, double* T_c);
int or_maxwell(double a, double b, double R, double T, double* rho_g, double* rho_l);

/* ---- Peng-Robinson EOS and chemical potential (Eq. 14-15) ---- */
double or_pr_alpha(double T, double Tc, double acentric);
double or_pr_pressure(double rho, double a, double b, double R, double T, double alpha);
double or_pr_mu(double rho, double a, double b, double R, double T, double alpha);
int or_pr_critical(double a, double b, double R, double* rho_c, double* T_c);

/* ---- an EOS of either kind at one temperature ---- */
#define OR_EOS_CS 0
#define OR_EOS_PR 1
#define OR_EOS_VDW 2 /* van der Waals, mu by Eq. 13 */
#define OR_EOS_RKS 3 /* Redlich-Kwong-Soave, mu by Eq. 13 */
double or_vdw_pressure(double rho, double a, double b, double R, double T);
double or_vdw_mu(double rho, double a, double b, double R, double T);
double or_rks_alpha(double T, double Tc, double acentric);
double or_rks_pressure(double rho, double a, double b, double R, double T, double alpha);
double or_rks_mu(double rho, double a, double b, double R, double T, double alpha);
int or_cubic_critical(int kind, double a, double b, double R, double* rho_c, double* T_c);
typedef struct {
  int kind;
  double a, b, R, T, Tc, rho_c, alpha, rho_max;
} or_eos;
int or_eos_make(int kind, double a, double b, double R, double Tr, double acentric, or_eos* e);
int or_eos_critical(int kind, double a, double b, double R, double* rho_c, double* T_c);
double or_eos_pressure(const or_eos* e, double rho);
double or_eos_mu(const or_eos* e, double rho);
double or_eos_dpdrho(const or_eos* e, double rho);
int or_eos_maxwell(const or_eos* e, double* rho_g, double* rho_l);

/* Equilibrium flat interface (Eq. 29) along one axis: rho and its analytic
 * derivative at nodes j = 0..n-1, gas for j < y0 and liquid beyond, rho(y0) =
 * (rho_g + rho_l) / 2, for the EOS, T_r, k and kappa-hat of p. */
int or_flat_profile(const or_params* p, int n, double y0, double* rho, double* drho);

/* ---- finite differences on periodic lattices (Sec. 2.3) ---- */
void or_scheme_coeffs(int scheme, double* alpha, double* a, double* b, double* c);
int or_deriv_line(int scheme, const double* f, int n, double* d);
int or_deriv2_line(int scheme, const double* f, int n, double* d2);
int or_gradient(int scheme, int dim, int nx, int ny, int nz, const double* phi, double* g /* dim*N */);
int or_laplacian(int scheme, int dim, int nx, int ny, int nz, const double* phi, double* lap);

/* ---- the simulation ---- */
or_sim* or_create(const or_params* p);

/* MRT (Eq. 1, 3-5), D2Q9: the transformation matrix M of Eq. 3 (row-major,
 * rows rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy; columns in the
 * velocity order of Eq. 2) and its inverse by Gauss-Jordan elimination. */
void or_mrt_matrix(double M[81]);
int or_mrt_inverse(double Minv[81]);
/* post-collision populations f* = f - M^-1 S (M f - M f_eq) + F_i (Eq. 1, 4) */
void or_mrt_collide(const double* f, const double* feq, const double* Fi, const double s[9], double* post);
void or_destroy(or_sim* s);

/* Walls (Appendix A; explicit schemes EFDS2/4/6): mask[N] nonzero marks a wall
 * node.  Wall nodes do not collide; populations reaching them bounce back
 * (halfway) to the opposite direction at the fluid node; their densities are
 * the Eq. A.1 averages over the previous layer, layer by layer, and their
 * chemical potential is mu_w.  Observables cover fluid nodes only. */
int or_set_solid(or_sim* s, const unsigned char* mask, double mu_w);
int or_solid_layers(const or_sim* s, int* layer /* N */);
int or_init_droplet(or_sim* s, const double center[3], double radius, double width, double rho_l, double rho_g);
int or_init_slab(or_sim* s, int axis, double thickness, double width, double rho_l, double rho_g);
int or_init_profile(or_sim* s, const double center[3], const double* r, const double* rho, int n);
int or_set_f(or_sim* s, const double* f);
int or_get_f(const or_sim* s, double* f);
int or_get_density(const or_sim* s, double* rho);
int or_get_fields(or_sim* s, double* rho, double* u, double* F, double* mu);
int or_step(or_sim* s, long long n);
int or_observables(or_sim* s, or_obs* out);
double or_temperature(const or_sim* s);

/* ---- warm-start MLP (FP64 reference of the network the solver trains) ---- */
int or_mlp_forward(const int* sizes, int nlayers, const double* params, const double* x, int batch,
                   double* y, double* acts);
int or_mlp_loss_grad(const int* sizes, int nlayers, const double* params, const double* x,
                     const double* target, int batch, double* loss, double* grad);
int or_adam_step(int n, double* params, double* m, double* v, const double* grad, double lr,
                 double beta1, double beta2, double eps, int t);

#ifdef __cplusplus
}
#endif
#endif
