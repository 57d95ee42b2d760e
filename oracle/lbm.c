/*
 * Oracle (test infrastructure only): the chemical-potential multiphase LBM
 * time step on D2Q9 and D3Q19, plain FP64 loops.
 *
 * One step, in the paper's order (Sec. 2.1-2.2):
 *   1. moments rho = sum f_i, rho u = sum e_i f_i                       (Eq. 7)
 *   2. mu = k^2 psi'(rho) - kappa lap(rho)                              (Eq. 16)
 *   3. grad mu, grad rho with the selected difference scheme            (Eq. 17-25)
 *   4. nonideal force F = -rho grad mu + c_s^2 grad rho                 (Eq. 12)
 *   5. collision: the MRT operator of Eq. 1 with every rate s_i = 1/tau,
 *      which the paper states reduces to single relaxation (BGK) with the
 *      equilibrium of Eq. 6:  f*_i = f_i - (f_i - f_i^eq(rho, u)) / tau + F_i
 *   6. forcing by the exact difference method,
 *      F_i = f_i^eq(rho, u + F/rho) - f_i^eq(rho, u)                      (Eq. 8)
 *   7. streaming f_i(x + e_i, t + 1) = f*_i(x, t), periodic             (Eq. 1, left side)
 * Lattice units: dx = dt = c = 1, c_s^2 = 1/3.
 *
 * Observables at time t are taken from rho(t), u(t) and F(t); the physical
 * velocity is v = u + F / (2 rho) (Sec. 2.1, after Eq. 8).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* D2Q9 velocities in the order of Eq. 2: rest; i = 1..4 at angles (i-1) pi/2;
 * i = 5..8 diagonal at angles (2i - 9) pi / 4.  Weights 4/9, 1/9, 1/36. */
static const int E2[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W2[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* D3Q19 (the paper runs 3D cases but does not name the lattice; this is the
 * standard nineteen-velocity set): rest; +-x, +-y, +-z; the twelve edge
 * diagonals.  Weights 1/3, 1/18, 1/36. */
static const int E3[19][3] = {{0, 0, 0},
                              {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
                              {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
                              {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W3[19] = {1.0 / 3,
                              1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                              1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

int or_lattice_q(int lattice) { return lattice == OR_D2Q9 ? 9 : lattice == OR_D3Q19 ? 19 : 0; }

static const int (*lat_e(int lattice))[3] { return lattice == OR_D2Q9 ? E2 : E3; }
static const double* lat_w(int lattice) { return lattice == OR_D2Q9 ? W2 : W3; }

void or_lattice_e(int lattice, int* e, double* w) {
  int q = or_lattice_q(lattice);
  for (int i = 0; i < q; ++i) {
    for (int d = 0; d < 3; ++d) e[i * 3 + d] = lat_e(lattice)[i][d];
    w[i] = lat_w(lattice)[i];
  }
}

/* Eq. 6 with c_s^2 = 1/3 */
void or_feq(int lattice, double rho, const double u[3], double* feq) {
  int q = or_lattice_q(lattice);
  const int(*e)[3] = lat_e(lattice);
  const double* w = lat_w(lattice);
  const double cs2 = 1.0 / 3.0;
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < q; ++i) {
    double eu = e[i][0] * u[0] + e[i][1] * u[1] + e[i][2] * u[2];
    feq[i] = w[i] * rho * (1.0 + eu / cs2 + eu * eu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
  }
}

/* Eq. 8 with delta u = F / rho (dt = 1) */
void or_edm(int lattice, double rho, const double u[3], const double F[3], double* Fi) {
  double a[19], b[19];
  double up[3] = {u[0] + F[0] / rho, u[1] + F[1] / rho, u[2] + F[2] / rho};
  or_feq(lattice, rho, up, a);
  or_feq(lattice, rho, u, b);
  int q = or_lattice_q(lattice);
  for (int i = 0; i < q; ++i) Fi[i] = a[i] - b[i];
}

struct or_sim {
  or_params p;
  int q, dim;
  long n;
  double T;
  or_eos eos;                           /* the equation of state at T */
  double *f, *fn;                       /* f[i*n + node] */
  unsigned char* solid;                 /* wall nodes (Appendix A), NULL: none */
  int* layer;                           /* 0 fluid, 1..3 wall layers, 4 deeper wall */
  double mu_w;                          /* chemical potential assigned to wall nodes */
  double *rho, *u, *F, *mu, *lap, *gmu, *grho;
  double* rho_snap;
  long long t, t_snap;
  int status;
  long long bad_step;
};

static long node_index(const or_sim* s, int x, int y, int z) {
  return (long)x + (long)s->p.nx * ((long)y + (long)s->p.ny * z);
}

or_sim* or_create(const or_params* p) {
  if (!p) return NULL;
  if (p->lattice != OR_D2Q9 && p->lattice != OR_D3Q19) return NULL;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
  if (p->lattice == OR_D2Q9 && p->nz != 1) return NULL;
  if (p->scheme < 0 || p->scheme >= OR_NSCHEMES) return NULL;
  if (p->scheme == OR_E8 && p->lattice != OR_D2Q9) return NULL;
  if (!(p->tau > 0.5) || !(p->k > 0) || !(p->kappa >= 0) || !(p->Tr > 0)) return NULL;
  if (p->collision != OR_BGK && p->collision != OR_MRT) return NULL;
  if (p->collision == OR_MRT && p->lattice != OR_D2Q9) return NULL;
  if (p->eos < OR_EOS_CS || p->eos > OR_EOS_RKS) return NULL;
  or_eos eos;
  if (or_eos_make(p->eos, p->a, p->b, p->R, p->Tr, p->acentric, &eos) != OR_OK) return NULL;
  or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
  s->p = *p;
  s->q = or_lattice_q(p->lattice);
  s->dim = p->lattice == OR_D2Q9 ? 2 : 3;
  s->n = (long)p->nx * p->ny * p->nz;
  s->eos = eos;
  s->T = eos.T;
  long n = s->n;
  s->f = (double*)calloc((size_t)s->q * n, sizeof(double));
  s->fn = (double*)calloc((size_t)s->q * n, sizeof(double));
  s->rho = (double*)calloc(n, sizeof(double));
  s->u = (double*)calloc(3 * n, sizeof(double));
  s->F = (double*)calloc(3 * n, sizeof(double));
  s->mu = (double*)calloc(n, sizeof(double));
  s->lap = (double*)calloc(n, sizeof(double));
  s->gmu = (double*)calloc(3 * n, sizeof(double));
  s->grho = (double*)calloc(3 * n, sizeof(double));
  s->rho_snap = (double*)calloc(n, sizeof(double));
  if (!s->f || !s->fn || !s->rho || !s->u || !s->F || !s->mu || !s->lap || !s->gmu || !s->grho ||
      !s->rho_snap) {
    or_destroy(s);
    return NULL;
  }
  return s;
}

void or_destroy(or_sim* s) {
  if (!s) return;
  free(s->f); free(s->fn); free(s->rho); free(s->u); free(s->F);
  free(s->mu); free(s->lap); free(s->gmu); free(s->grho); free(s->rho_snap);
  free(s->solid); free(s->layer);
  free(s);
}

double or_temperature(const or_sim* s) { return s->T; }

/* f_i = f_i^eq(rho, 0) = w_i rho; resets time, status and the rate snapshot */
static void init_from_rho(or_sim* s, const double* rho) {
  const double* w = lat_w(s->p.lattice);
  for (long x = 0; x < s->n; ++x)
    for (int i = 0; i < s->q; ++i) s->f[i * s->n + x] = w[i] * rho[x];
  s->t = 0;
  s->t_snap = 0;
  s->status = OR_OK;
  s->bad_step = -1;
  memcpy(s->rho_snap, rho, sizeof(double) * s->n);
}

static int default_densities(or_sim* s, double* rho_l, double* rho_g) {
  if (*rho_l > 0 && *rho_g > 0) return OR_OK;
  double g, l;
  int rc = or_eos_maxwell(&s->eos, &g, &l);
  if (rc != OR_OK) return rc;
  *rho_l = l;
  *rho_g = g;
  return OR_OK;
}

/* Eq. 26: rho = (rho_l + rho_g)/2 - (rho_l - rho_g)/2 tanh(2 (r - r0) / W), r the
 * Euclidean distance to the centre (no periodic image). */
int or_init_droplet(or_sim* s, const double center[3], double radius, double width, double rho_l,
                    double rho_g) {
  if (!(width > 0) || !(radius >= 0)) return OR_EINVAL;
  int rc = default_densities(s, &rho_l, &rho_g);
  if (rc != OR_OK) return rc;
  double c[3] = {s->p.nx / 2, s->p.ny / 2, s->p.nz / 2};
  if (center) { c[0] = center[0]; c[1] = center[1]; c[2] = center[2]; }
  if (s->dim == 2) c[2] = 0;
  for (int z = 0; z < s->p.nz; ++z)
    for (int y = 0; y < s->p.ny; ++y)
      for (int x = 0; x < s->p.nx; ++x) {
        double dx = x - c[0], dy = y - c[1], dz = z - c[2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        s->rho[node_index(s, x, y, z)] =
            0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * tanh(2.0 * (r - radius) / width);
      }
  init_from_rho(s, s->rho);
  return OR_OK;
}

/* flat liquid slab of the given thickness centred on the mid-plane of `axis`
 * (the coexistence test of Sec. 3.4) */
int or_init_slab(or_sim* s, int axis, double thickness, double width, double rho_l, double rho_g) {
  if (axis < 0 || axis >= s->dim || !(width > 0) || !(thickness >= 0)) return OR_EINVAL;
  int rc = default_densities(s, &rho_l, &rho_g);
  if (rc != OR_OK) return rc;
  int dims[3] = {s->p.nx, s->p.ny, s->p.nz};
  double c0 = dims[axis] / 2;
  for (int z = 0; z < s->p.nz; ++z)
    for (int y = 0; y < s->p.ny; ++y)
      for (int x = 0; x < s->p.nx; ++x) {
        int p[3] = {x, y, z};
        double d = fabs(p[axis] - c0);
        s->rho[node_index(s, x, y, z)] =
            0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * tanh(2.0 * (d - 0.5 * thickness) / width);
      }
  init_from_rho(s, s->rho);
  return OR_OK;
}

/* radial profile (r_j increasing, rho_j) linearly interpolated in r, held at
 * the end values outside [r_0, r_{n-1}] */
int or_init_profile(or_sim* s, const double center[3], const double* r, const double* rho, int n) {
  if (n < 2) return OR_EINVAL;
  for (int j = 1; j < n; ++j)
    if (!(r[j] > r[j - 1])) return OR_EINVAL;
  for (int j = 0; j < n; ++j)
    if (!(rho[j] > 0)) return OR_EINVAL;
  double c[3] = {s->p.nx / 2, s->p.ny / 2, s->p.nz / 2};
  if (center) { c[0] = center[0]; c[1] = center[1]; c[2] = center[2]; }
  if (s->dim == 2) c[2] = 0;
  for (int z = 0; z < s->p.nz; ++z)
    for (int y = 0; y < s->p.ny; ++y)
      for (int x = 0; x < s->p.nx; ++x) {
        double dx = x - c[0], dy = y - c[1], dz = z - c[2];
        double rr = sqrt(dx * dx + dy * dy + dz * dz), v;
        if (rr <= r[0]) v = rho[0];
        else if (rr >= r[n - 1]) v = rho[n - 1];
        else {
          int j = 0;
          while (r[j + 1] < rr) ++j;
          double t = (rr - r[j]) / (r[j + 1] - r[j]);
          v = rho[j] + t * (rho[j + 1] - rho[j]);
        }
        s->rho[node_index(s, x, y, z)] = v;
      }
  init_from_rho(s, s->rho);
  return OR_OK;
}

int or_set_f(or_sim* s, const double* f) {
  memcpy(s->f, f, sizeof(double) * s->q * s->n);
  for (long x = 0; x < s->n; ++x) {
    double r = 0;
    for (int i = 0; i < s->q; ++i) r += s->f[i * s->n + x];
    s->rho_snap[x] = r;
  }
  s->t = 0;
  s->t_snap = 0;
  s->status = OR_OK;
  s->bad_step = -1;
  return OR_OK;
}

int or_get_f(const or_sim* s, double* f) {
  memcpy(f, s->f, sizeof(double) * s->q * s->n);
  return OR_OK;
}

/* index of the velocity opposite to e_i */
static int opposite(const or_sim* s, int i) {
  const int(*e)[3] = lat_e(s->p.lattice);
  for (int j = 0; j < s->q; ++j)
    if (e[j][0] == -e[i][0] && e[j][1] == -e[i][1] && e[j][2] == -e[i][2]) return j;
  return i;
}

/*
 * Wall nodes (Appendix A).  Layer 1: wall nodes with a fluid neighbour along
 * some lattice velocity; layer L: not in an earlier layer, with a neighbour in
 * layer L - 1 (up to 3 layers: the reach of the sixth-order stencil).  Each
 * step the densities of layers 1, 2, 3 are, in that order, the w_i-weighted
 * average of the neighbours in the layer before (Eq. A.1: the switching
 * function selects those neighbours), and every wall node carries the chemical
 * potential mu_w.  Deeper wall nodes take the fluid's mean density (no
 * stencil of a fluid node reaches them).
 */
int or_set_solid(or_sim* s, const unsigned char* mask, double mu_w) {
  if (!s || !mask) return OR_EINVAL;
  if (s->p.scheme != OR_EFDS2 && s->p.scheme != OR_EFDS4 && s->p.scheme != OR_EFDS6) return OR_EINVAL;
  long n = s->n;
  if (!s->solid) {
    s->solid = (unsigned char*)calloc(n, 1);
    s->layer = (int*)calloc(n, sizeof(int));
  }
  const int(*e)[3] = lat_e(s->p.lattice);
  int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  long nfluid = 0;
  for (long x = 0; x < n; ++x) {
    s->solid[x] = mask[x] ? 1 : 0;
    s->layer[x] = mask[x] ? 4 : 0;
    nfluid += !mask[x];
  }
  if (nfluid == 0) return OR_EINVAL;
  for (int L = 1; L <= 3; ++L) {
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          long c = node_index(s, x, y, z);
          if (s->layer[c] != 4) continue;
          for (int i = 1; i < s->q; ++i) {
            long t = node_index(s, (x + e[i][0] + nx) % nx, (y + e[i][1] + ny) % ny, (z + e[i][2] + nz) % nz);
            if (s->layer[t] == L - 1) { s->layer[c] = -L; break; }
          }
        }
    /* marks of this pass become layer L only after it, so that a node does
     * not join layer L through a neighbour marked in the same pass */
    for (long x = 0; x < n; ++x)
      if (s->layer[x] < 0) s->layer[x] = -s->layer[x];
  }
  s->mu_w = mu_w;
  return OR_OK;
}

int or_solid_layers(const or_sim* s, int* layer) {
  if (!s || !layer) return OR_EINVAL;
  for (long x = 0; x < s->n; ++x) layer[x] = s->layer ? s->layer[x] : 0;
  return OR_OK;
}

static void wall_densities(or_sim* s) {
  const int(*e)[3] = lat_e(s->p.lattice);
  const double* w = lat_w(s->p.lattice);
  int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  long n = s->n;
  double mean = 0;
  long nf = 0;
  for (long x = 0; x < n; ++x)
    if (!s->solid[x]) { mean += s->rho[x]; ++nf; }
  mean /= (double)nf;
  for (int L = 1; L <= 3; ++L)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          long c = node_index(s, x, y, z);
          if (s->layer[c] != L) continue;
          double num = 0, den = 0;
          for (int i = 1; i < s->q; ++i) {
            long t = node_index(s, (x + e[i][0] + nx) % nx, (y + e[i][1] + ny) % ny, (z + e[i][2] + nz) % nz);
            if (s->layer[t] == L - 1) { num += w[i] * s->rho[t]; den += w[i]; }
          }
          s->rho[c] = num / den;
        }
  for (long x = 0; x < n; ++x)
    if (s->solid[x] && s->layer[x] == 4) s->rho[x] = mean;
}

/* steps 1-4 for the current state: rho, u, mu, grad mu, grad rho, F */
static int macro_fields(or_sim* s) {
  const int(*e)[3] = lat_e(s->p.lattice);
  long n = s->n;
  int ok = 1;
  for (long x = 0; x < n; ++x) {
    if (s->solid && s->solid[x]) {
      for (int d = 0; d < 3; ++d) s->u[d * n + x] = 0.0;
      continue;
    }
    double r = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < s->q; ++i) {
      double fi = s->f[i * n + x];
      r += fi;
      for (int d = 0; d < 3; ++d) j[d] += e[i][d] * fi;
    }
    s->rho[x] = r;
    for (int d = 0; d < 3; ++d) s->u[d * n + x] = j[d] / r;
    if (!(r > 0) || !isfinite(r)) ok = 0;
  }
  if (!ok) return OR_EUNSTABLE;
  if (s->solid) wall_densities(s);
  const or_params* p = &s->p;
  int rc = or_laplacian(p->scheme, s->dim, p->nx, p->ny, p->nz, s->rho, s->lap);
  if (rc != OR_OK) return rc;
  for (long x = 0; x < n; ++x)
    s->mu[x] = (s->solid && s->solid[x]) ? s->mu_w
                                         : p->k * p->k * or_eos_mu(&s->eos, s->rho[x]) - p->kappa * s->lap[x];
  rc = or_gradient(p->scheme, s->dim, p->nx, p->ny, p->nz, s->mu, s->gmu);
  if (rc != OR_OK) return rc;
  rc = or_gradient(p->scheme, s->dim, p->nx, p->ny, p->nz, s->rho, s->grho);
  if (rc != OR_OK) return rc;
  for (int d = 0; d < 3; ++d)
    for (long x = 0; x < n; ++x)
      s->F[d * n + x] = (d < s->dim && !(s->solid && s->solid[x])) ? -s->rho[x] * s->gmu[d * n + x] + s->grho[d * n + x] / 3.0 : 0.0;
  return OR_OK;
}

int or_get_density(const or_sim* s, double* rho) {
  for (long x = 0; x < s->n; ++x) {
    double r = 0;
    for (int i = 0; i < s->q; ++i) r += s->f[i * s->n + x];
    rho[x] = r;
  }
  return OR_OK;
}

int or_get_fields(or_sim* s, double* rho, double* u, double* F, double* mu) {
  int rc = macro_fields(s);
  if (rc != OR_OK) return rc;
  if (rho) memcpy(rho, s->rho, sizeof(double) * s->n);
  if (u) memcpy(u, s->u, sizeof(double) * 3 * s->n);
  if (F) memcpy(F, s->F, sizeof(double) * 3 * s->n);
  if (mu) memcpy(mu, s->mu, sizeof(double) * s->n);
  return OR_OK;
}

int or_step(or_sim* s, long long nsteps) {
  const int(*e)[3] = lat_e(s->p.lattice);
  long n = s->n;
  int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
  for (long long it = 0; it < nsteps; ++it) {
    if (s->status != OR_OK) return s->status;
    int rc = macro_fields(s);
    if (rc == OR_EUNSTABLE) {
      s->status = OR_EUNSTABLE;
      s->bad_step = s->t;
      return rc;
    }
    if (rc != OR_OK) return rc;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          long c = node_index(s, x, y, z);
          double u[3] = {s->u[c], s->u[n + c], s->u[2 * n + c]};
          double F[3] = {s->F[c], s->F[n + c], s->F[2 * n + c]};
          double feq[19], Fi[19];
          or_feq(s->p.lattice, s->rho[c], u, feq);
          or_edm(s->p.lattice, s->rho[c], u, F, Fi);
          if (s->solid && s->solid[c]) continue; /* wall nodes do not collide */
          double fc[19], post[19];
          for (int i = 0; i < s->q; ++i) fc[i] = s->f[i * n + c];
          if (s->p.collision == OR_MRT) {
            or_mrt_collide(fc, feq, Fi, s->p.mrt_s, post);
          } else {
            for (int i = 0; i < s->q; ++i) post[i] = fc[i] - (fc[i] - feq[i]) / s->p.tau + Fi[i];
          }
          for (int i = 0; i < s->q; ++i) {
            int xd = (x + e[i][0] + nx) % nx, yd = (y + e[i][1] + ny) % ny, zd = (z + e[i][2] + nz) % nz;
            long t = node_index(s, xd, yd, zd);
            if (s->solid && s->solid[t])
              s->fn[opposite(s, i) * n + c] = post[i]; /* halfway bounce-back off a wall */
            else
              s->fn[i * n + t] = post[i];
          }
        }
    double* tmp = s->f; s->f = s->fn; s->fn = tmp;
    s->t += 1;
  }
  return OR_OK;
}

int or_observables(or_sim* s, or_obs* o) {
  memset(o, 0, sizeof(*o));
  o->step = s->t;
  if (s->status == OR_OK) {
    int rc = macro_fields(s);
    if (rc == OR_EUNSTABLE) { s->status = OR_EUNSTABLE; s->bad_step = s->t; }
    else if (rc != OR_OK) return rc;
  }
  if (s->status != OR_OK) {
    o->status = s->status;
    o->step = s->bad_step;
    return s->status;
  }
  long n = s->n;
  double max_v = 0, max_u = 0, mass = 0, max_dr = 0;
  for (long x = 0; x < n; ++x) {
    if (s->solid && s->solid[x]) continue; /* fluid nodes only */
    double r = s->rho[x], uu = 0, vv = 0;
    for (int d = 0; d < 3; ++d) {
      double ud = s->u[d * n + x];
      double vd = ud + s->F[d * n + x] / (2.0 * r);
      uu += ud * ud;
      vv += vd * vd;
    }
    if (sqrt(uu) > max_u) max_u = sqrt(uu);
    if (sqrt(vv) > max_v) max_v = sqrt(vv);
    mass += r;
    double dr = fabs(r - s->rho_snap[x]);
    if (dr > max_dr) max_dr = dr;
  }
  o->max_v = max_v;
  o->max_u = max_u;
  o->mass = mass;
  o->max_drho = (s->t > s->t_snap) ? max_dr / (double)(s->t - s->t_snap) : 0.0;
  o->rho_center = s->rho[node_index(s, s->p.nx / 2, s->p.ny / 2, s->p.nz / 2)];
  o->rho_corner = s->rho[0];
  o->status = OR_OK;
  memcpy(s->rho_snap, s->rho, sizeof(double) * n);
  s->t_snap = s->t;
  return OR_OK;
}

/* ---------------------------------------------------------------- MRT (D2Q9) */

/* The matrix of Eq. 3 as printed; columns follow the velocity order of Eq. 2. */
static const double MRT_M[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},         {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},     {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},      {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},      {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

void or_mrt_matrix(double M[81]) {
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) M[r * 9 + c] = MRT_M[r][c];
}

/* Gauss-Jordan elimination with partial pivoting on [M | I]. */
int or_mrt_inverse(double Minv[81]) {
  double a[9][18];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 18; ++c) a[r][c] = c < 9 ? MRT_M[r][c] : (c - 9 == r ? 1.0 : 0.0);
  for (int col = 0; col < 9; ++col) {
    int piv = col;
    for (int r = col + 1; r < 9; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (fabs(a[piv][col]) < 1e-12) return OR_EINVAL;
    if (piv != col)
      for (int c = 0; c < 18; ++c) {
        double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t;
      }
    double d = a[col][col];
    for (int c = 0; c < 18; ++c) a[col][c] /= d;
    for (int r = 0; r < 9; ++r) {
      if (r == col) continue;
      double m = a[r][col];
      for (int c = 0; c < 18; ++c) a[r][c] -= m * a[col][c];
    }
  }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) Minv[r * 9 + c] = a[r][c + 9];
  return OR_OK;
}

void or_mrt_collide(const double* f, const double* feq, const double* Fi, const double s[9], double* post) {
  double Minv[81];
  or_mrt_inverse(Minv);
  double dm[9];
  for (int k = 0; k < 9; ++k) {
    double m = 0.0, meq = 0.0;
    for (int i = 0; i < 9; ++i) {
      m += MRT_M[k][i] * f[i];
      meq += MRT_M[k][i] * feq[i];
    }
    dm[k] = s[k] * (m - meq);
  }
  for (int i = 0; i < 9; ++i) {
    double corr = 0.0;
    for (int k = 0; k < 9; ++k) corr += Minv[i * 9 + k] * dm[k];
    post[i] = f[i] - corr + Fi[i];
  }
}
