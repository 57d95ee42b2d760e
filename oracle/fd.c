/*
 * Oracle (test infrastructure only): finite-difference operators on periodic
 * lattices, Sec. 2.3 of the paper.  Grid spacing h = 1 (lattice units).
 *
 *   EFDS2/4/6   explicit central first derivative, Eq. 18, 19, 20.
 *   CFDS4/6/8   compact (alpha-family tridiagonal, beta = 0) first derivative,
 *               Eq. 21 with the coefficients of Eq. 22, 23, 24.
 *   OCFDS4      the optimal fourth-order compact scheme of Sec. 3.1 with the
 *               printed alpha = 0.446776 and c = -0.0541132; a and b are taken
 *               from the two fourth-order Taylor conditions of Eq. 21,
 *                   a + b + c = 1 + 2 alpha,   a + 4 b + 9 c = 6 alpha,
 *               because the printed a = 1.541, b = 0.40667 are rounded and do
 *               not satisfy the first condition to better than 5e-6.
 *   E4, E8      isotropic gradient and Laplacian, Eq. 25a and 25b.
 *
 * On a periodic lattice the compact relation Eq. 21 is a cyclic tridiagonal
 * system (alpha, 1, alpha) per grid line; it is solved here by the Thomas
 * algorithm plus a Sherman-Morrison correction for the two corner entries.
 *
 * The paper does not state which Laplacian accompanies each first-derivative
 * scheme in mu = k^2 psi' - kappa lap(rho) (Eq. 16).  Reading used here:
 * E4/E8 use Eq. 25b with the same weights; the explicit and compact schemes
 * use the explicit central second-derivative stencil of matching formal order
 * (2nd for EFDS2, 4th for EFDS4, CFDS4 and OCFDS4, 6th for EFDS6 and CFDS6,
 * 8th for CFDS8), summed over the axes.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

void or_scheme_coeffs(int scheme, double* alpha, double* a, double* b, double* c) {
  *alpha = 0; *a = 0; *b = 0; *c = 0;
  switch (scheme) {
    case OR_EFDS2: *a = 1.0; break;                                   /* Eq. 18 */
    case OR_EFDS4: *a = 4.0 / 3.0; *b = -1.0 / 3.0; break;            /* Eq. 19 */
    case OR_EFDS6: *a = 3.0 / 2.0; *b = -3.0 / 5.0; *c = 1.0 / 10.0; break; /* Eq. 20 */
    case OR_CFDS4: *alpha = 1.0 / 4.0; *a = 3.0 / 2.0; break;         /* Eq. 22 */
    case OR_CFDS6: *alpha = 1.0 / 3.0; *a = 14.0 / 9.0; *b = 1.0 / 9.0; break; /* Eq. 23 */
    case OR_CFDS8:                                                    /* Eq. 24 */
      *alpha = 3.0 / 8.0; *a = 25.0 / 16.0; *b = 1.0 / 5.0; *c = -1.0 / 80.0; break;
    case OR_OCFDS4: {
      double al = 0.446776, cc = -0.0541132;
      double bb = (4.0 * al - 1.0 - 8.0 * cc) / 3.0;
      *alpha = al; *c = cc; *b = bb; *a = 1.0 + 2.0 * al - bb - cc;
      break;
    }
    default: break;
  }
}

static int is_compact(int s) { return s == OR_CFDS4 || s == OR_CFDS6 || s == OR_CFDS8 || s == OR_OCFDS4; }

static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

/* Explicit part of Eq. 21 (the whole derivative when alpha = 0). */
static void rhs_line(double a, double b, double c, const double* f, int n, double* r) {
  for (int i = 0; i < n; ++i) {
    r[i] = a * (f[wrap(i + 1, n)] - f[wrap(i - 1, n)]) / 2.0
         + b * (f[wrap(i + 2, n)] - f[wrap(i - 2, n)]) / 4.0
         + c * (f[wrap(i + 3, n)] - f[wrap(i - 3, n)]) / 6.0;
  }
}

/* Thomas algorithm for the plain tridiagonal system
 *   lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1] = r[i],  lo[0] = up[n-1] = 0. */
static void thomas(const double* lo, const double* di, const double* up, const double* r, int n,
                   double* x, double* cp, double* dp) {
  cp[0] = up[0] / di[0];
  dp[0] = r[0] / di[0];
  for (int i = 1; i < n; ++i) {
    double m = di[i] - lo[i] * cp[i - 1];
    cp[i] = up[i] / m;
    dp[i] = (r[i] - lo[i] * dp[i - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
}

/* Cyclic system with diagonal 1 and off-diagonals alpha (including the two
 * corner entries A[0][n-1] = A[n-1][0] = alpha).  Write A = T + u v^T with
 * u = (g, 0, ..., 0, alpha)^T and v = (1, 0, ..., 0, alpha/g)^T, g = -1, so that T is
 * the tridiagonal matrix with T[0][0] = 1 - g and T[n-1][n-1] = 1 - alpha^2/g.
 * Then x = y - (v.y)/(1 + v.z) z with T y = r and T z = u (Sherman-Morrison). */
static void cyclic_solve(double alpha, const double* r, int n, double* x) {
  double* lo = (double*)malloc(sizeof(double) * n * 7);
  double *di = lo + n, *up = di + n, *y = up + n, *z = y + n, *cp = z + n, *dp = cp + n;
  double g = -1.0;
  for (int i = 0; i < n; ++i) { lo[i] = alpha; di[i] = 1.0; up[i] = alpha; }
  lo[0] = 0.0; up[n - 1] = 0.0;
  di[0] = 1.0 - g;
  di[n - 1] = 1.0 - alpha * alpha / g;
  thomas(lo, di, up, r, n, y, cp, dp);
  double* u = (double*)calloc(n, sizeof(double));
  u[0] = g; u[n - 1] = alpha;
  thomas(lo, di, up, u, n, z, cp, dp);
  double vy = y[0] + (alpha / g) * y[n - 1];
  double vz = z[0] + (alpha / g) * z[n - 1];
  double fac = vy / (1.0 + vz);
  for (int i = 0; i < n; ++i) x[i] = y[i] - fac * z[i];
  free(u);
  free(lo);
}

/* First derivative of one periodic line (explicit or compact scheme).  The
 * isotropic E4/E8 stencils are not line operators; they act on whole fields. */
int or_deriv_line(int scheme, const double* f, int n, double* d) {
  if (scheme < OR_EFDS2 || scheme > OR_OCFDS4 || n < 1) return OR_EINVAL;
  if (is_compact(scheme) && n < 3) return OR_EINVAL;
  double al, a, b, c;
  or_scheme_coeffs(scheme, &al, &a, &b, &c);
  if (!is_compact(scheme)) { rhs_line(a, b, c, f, n, d); return OR_OK; }
  double* r = (double*)malloc(sizeof(double) * n);
  rhs_line(a, b, c, f, n, r);
  cyclic_solve(al, r, n, d);
  free(r);
  return OR_OK;
}

/* Central second-derivative stencils of formal order 2, 4, 6, 8 (half-width
 * 1..4), from Taylor matching: d2 = sum_m s[|m|] f[i+m]. */
static int lap_order(int scheme) {
  switch (scheme) {
    case OR_EFDS2: return 2;
    case OR_EFDS4: case OR_CFDS4: case OR_OCFDS4: return 4;
    case OR_EFDS6: case OR_CFDS6: return 6;
    case OR_CFDS8: return 8;
    default: return 0;
  }
}

static void d2_stencil(int order, double* s /* s[0..4] */) {
  for (int m = 0; m < 5; ++m) s[m] = 0;
  switch (order) {
    case 2: s[0] = -2.0; s[1] = 1.0; break;
    case 4: s[0] = -5.0 / 2.0; s[1] = 4.0 / 3.0; s[2] = -1.0 / 12.0; break;
    case 6: s[0] = -49.0 / 18.0; s[1] = 3.0 / 2.0; s[2] = -3.0 / 20.0; s[3] = 1.0 / 90.0; break;
    case 8:
      s[0] = -205.0 / 72.0; s[1] = 8.0 / 5.0; s[2] = -1.0 / 5.0; s[3] = 8.0 / 315.0; s[4] = -1.0 / 560.0;
      break;
    default: break;
  }
}

int or_deriv2_line(int scheme, const double* f, int n, double* d2) {
  int order = lap_order(scheme);
  if (order == 0 || n < 1) return OR_EINVAL;
  double s[5];
  d2_stencil(order, s);
  for (int i = 0; i < n; ++i) {
    double acc = s[0] * f[i];
    for (int m = 1; m <= 4; ++m) acc += s[m] * (f[wrap(i + m, n)] + f[wrap(i - m, n)]);
    d2[i] = acc;
  }
  return OR_OK;
}

/* Isotropic neighbour sets with weights w(|e|^2) (Eq. 25).
 * E4, 2D: the eight D2Q9 neighbours, w(1) = 1/3, w(2) = 1/12 (Sec. 2.3.3).
 * E4, 3D: the eighteen D3Q19 neighbours, w(1) = 1/6, w(2) = 1/12 (the D3Q19
 *         weights divided by c_s^2; sum_i w e_x^2 = 1).
 * E8, 2D: shells |e|^2 = 1, 2, 4, 5, 8 with w = 4/21, 4/45, 1/60, 2/315, 1/5040
 *         (the paper names E8 but does not print weights; these satisfy the
 *         isotropy conditions up to eighth rank, checked in the tests). */
static int iso_stencil(int scheme, int dim, int (*e)[3], double* w) {
  int n = 0;
  if (scheme == OR_E4 && dim == 2) {
    for (int y = -1; y <= 1; ++y)
      for (int x = -1; x <= 1; ++x) {
        int s2 = x * x + y * y;
        if (s2 == 0) continue;
        e[n][0] = x; e[n][1] = y; e[n][2] = 0;
        w[n++] = (s2 == 1) ? 1.0 / 3.0 : 1.0 / 12.0;
      }
  } else if (scheme == OR_E4 && dim == 3) {
    for (int z = -1; z <= 1; ++z)
      for (int y = -1; y <= 1; ++y)
        for (int x = -1; x <= 1; ++x) {
          int s2 = x * x + y * y + z * z;
          if (s2 == 0 || s2 == 3) continue;
          e[n][0] = x; e[n][1] = y; e[n][2] = z;
          w[n++] = (s2 == 1) ? 1.0 / 6.0 : 1.0 / 12.0;
        }
  } else if (scheme == OR_E8 && dim == 2) {
    for (int y = -2; y <= 2; ++y)
      for (int x = -2; x <= 2; ++x) {
        int s2 = x * x + y * y;
        double ww;
        switch (s2) {
          case 1: ww = 4.0 / 21.0; break;
          case 2: ww = 4.0 / 45.0; break;
          case 4: ww = 1.0 / 60.0; break;
          case 5: ww = 2.0 / 315.0; break;
          case 8: ww = 1.0 / 5040.0; break;
          default: ww = 0.0; break;
        }
        if (ww == 0.0) continue;
        e[n][0] = x; e[n][1] = y; e[n][2] = 0;
        w[n++] = ww;
      }
  }
  return n;
}

static long idx3(int x, int y, int z, int nx, int ny, int nz) {
  return (long)wrap(x, nx) + (long)nx * ((long)wrap(y, ny) + (long)ny * wrap(z, nz));
}

/* gather one grid line along `axis` through (x, y, z) */
static void get_line(const double* phi, int axis, int x, int y, int z, int nx, int ny, int nz, double* line) {
  int n = axis == 0 ? nx : axis == 1 ? ny : nz;
  for (int i = 0; i < n; ++i) {
    int p[3] = {x, y, z};
    p[axis] = i;
    line[i] = phi[idx3(p[0], p[1], p[2], nx, ny, nz)];
  }
}

static void put_line(double* out, int axis, int x, int y, int z, int nx, int ny, int nz, const double* line) {
  int n = axis == 0 ? nx : axis == 1 ? ny : nz;
  for (int i = 0; i < n; ++i) {
    int p[3] = {x, y, z};
    p[axis] = i;
    out[idx3(p[0], p[1], p[2], nx, ny, nz)] = line[i];
  }
}

static int check_dims(int dim, int nx, int ny, int nz) {
  if (dim == 2) return nx > 0 && ny > 0 && nz == 1;
  if (dim == 3) return nx > 0 && ny > 0 && nz > 0;
  return 0;
}

/* g[axis * N + node] = D_S phi along axis, for every lattice node */
int or_gradient(int scheme, int dim, int nx, int ny, int nz, const double* phi, double* g) {
  if (!check_dims(dim, nx, ny, nz)) return OR_EINVAL;
  long N = (long)nx * ny * nz;
  if (scheme == OR_E4 || scheme == OR_E8) {
    int e[32][3];
    double w[32];
    int ne = iso_stencil(scheme, dim, e, w);
    if (ne == 0) return OR_EINVAL;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          double acc[3] = {0, 0, 0};
          for (int i = 0; i < ne; ++i) {
            double v = phi[idx3(x + e[i][0], y + e[i][1], z + e[i][2], nx, ny, nz)];
            for (int d = 0; d < dim; ++d) acc[d] += w[i] * e[i][d] * v;
          }
          for (int d = 0; d < dim; ++d) g[d * N + idx3(x, y, z, nx, ny, nz)] = acc[d];
        }
    return OR_OK;
  }
  if (scheme < OR_EFDS2 || scheme > OR_OCFDS4) return OR_EINVAL;
  int dims[3] = {nx, ny, nz};
  int nmax = nx > ny ? nx : ny;
  if (nz > nmax) nmax = nz;
  double* line = (double*)malloc(sizeof(double) * nmax * 2);
  double* dl = line + nmax;
  int rc = OR_OK;
  for (int axis = 0; axis < dim && rc == OR_OK; ++axis) {
    /* iterate over all lines parallel to axis */
    for (int z = 0; z < (axis == 2 ? 1 : nz) && rc == OR_OK; ++z)
      for (int y = 0; y < (axis == 1 ? 1 : ny) && rc == OR_OK; ++y)
        for (int x = 0; x < (axis == 0 ? 1 : nx) && rc == OR_OK; ++x) {
          get_line(phi, axis, x, y, z, nx, ny, nz, line);
          rc = or_deriv_line(scheme, line, dims[axis], dl);
          if (rc == OR_OK) put_line(g + axis * N, axis, x, y, z, nx, ny, nz, dl);
        }
  }
  free(line);
  return rc;
}

int or_laplacian(int scheme, int dim, int nx, int ny, int nz, const double* phi, double* lap) {
  if (!check_dims(dim, nx, ny, nz)) return OR_EINVAL;
  long N = (long)nx * ny * nz;
  if (scheme == OR_E4 || scheme == OR_E8) {
    int e[32][3];
    double w[32];
    int ne = iso_stencil(scheme, dim, e, w);
    if (ne == 0) return OR_EINVAL;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          double c0 = phi[idx3(x, y, z, nx, ny, nz)], acc = 0;
          for (int i = 0; i < ne; ++i)
            acc += w[i] * (phi[idx3(x + e[i][0], y + e[i][1], z + e[i][2], nx, ny, nz)] - c0);
          lap[idx3(x, y, z, nx, ny, nz)] = 2.0 * acc;  /* Eq. 25b */
        }
    return OR_OK;
  }
  if (scheme < OR_EFDS2 || scheme > OR_OCFDS4) return OR_EINVAL;
  int dims[3] = {nx, ny, nz};
  int nmax = nx > ny ? nx : ny;
  if (nz > nmax) nmax = nz;
  double* line = (double*)malloc(sizeof(double) * nmax * 2);
  double* dl = line + nmax;
  double* tmp = (double*)malloc(sizeof(double) * N);
  for (long i = 0; i < N; ++i) lap[i] = 0.0;
  int rc = OR_OK;
  for (int axis = 0; axis < dim && rc == OR_OK; ++axis) {
    for (int z = 0; z < (axis == 2 ? 1 : nz) && rc == OR_OK; ++z)
      for (int y = 0; y < (axis == 1 ? 1 : ny) && rc == OR_OK; ++y)
        for (int x = 0; x < (axis == 0 ? 1 : nx) && rc == OR_OK; ++x) {
          get_line(phi, axis, x, y, z, nx, ny, nz, line);
          rc = or_deriv2_line(scheme, line, dims[axis], dl);
          if (rc == OR_OK) put_line(tmp, axis, x, y, z, nx, ny, nz, dl);
        }
    for (long i = 0; i < N && rc == OR_OK; ++i) lap[i] += tmp[i];
  }
  free(tmp);
  free(line);
  return rc;
}
