/*
 * Oracle (test infrastructure only): Carnahan-Starling equation of state, its
 * chemical potential, critical point and Maxwell equal-area coexistence.
 *
 * The paper prints the Peng-Robinson pair (Eq. 14-15) and only names the
 * Carnahan-Starling EOS (Sec. 3.4, Fig. 13).  The CS pressure used here is the
 * textbook form
 *     p0 = rho R T (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2,  eta = b rho / 4,
 * and the bulk chemical potential psi'(rho) follows from it by the route of
 * Eq. 10 and Eq. 13: psi = rho (int p0/rho^2 drho + C), so
 *     psi'(rho) = int p0/rho^2 drho + p0/rho.
 * Carrying out the integral (with d rho / rho = d eta / eta) gives
 *     psi'(rho) = R T [ ln rho + (8 eta - 9 eta^2 + 3 eta^3) / (1 - eta)^3 ] - 2 a rho + const,
 * and the additive constant drops out of every gradient and of the Maxwell
 * conditions, so it is set to zero.
 */
#include <math.h>
#include "oracle.h"

double or_cs_pressure(double rho, double a, double b, double R, double T) {
  double eta = b * rho / 4.0;
  double one_m = 1.0 - eta;
  double z = (1.0 + eta + eta * eta - eta * eta * eta) / (one_m * one_m * one_m);
  return rho * R * T * z - a * rho * rho;
}

double or_cs_mu(double rho, double a, double b, double R, double T) {
  double eta = b * rho / 4.0;
  double one_m = 1.0 - eta;
  double hs = (8.0 * eta - 9.0 * eta * eta + 3.0 * eta * eta * eta) / (one_m * one_m * one_m);
  return R * T * (log(rho) + hs) - 2.0 * a * rho;
}

/*
 * Critical point: dp0/drho = d2p0/drho2 = 0.  With g(eta) = eta Z(eta), the
 * pressure is p0 = (4/b) R T g(eta) - a rho^2, so the two conditions become
 *     R T g'(eta) = 8 a eta / b    and    R T g''(eta) = 8 a / b,
 * hence g'(eta) = eta g''(eta) fixes eta_c and then T_c = 8 a / (b R g''(eta_c)).
 * g' and g'' are taken analytically below; eta_c is bracketed and bisected.
 */
static void cs_g_derivs(double eta, double* g1, double* g2) {
  /* g = (eta + eta^2 + eta^3 - eta^4) / (1 - eta)^3 */
  double n = eta + eta * eta + eta * eta * eta - eta * eta * eta * eta;
  double n1 = 1.0 + 2.0 * eta + 3.0 * eta * eta - 4.0 * eta * eta * eta;
  double n2 = 2.0 + 6.0 * eta - 12.0 * eta * eta;
  double q = 1.0 - eta;
  double d = q * q * q;            /* (1-eta)^3 */
  double d1 = -3.0 * q * q;        /* derivative of (1-eta)^3 */
  double d2 = 6.0 * q;
  /* quotient rule, first and second derivative */
  *g1 = (n1 * d - n * d1) / (d * d);
  *g2 = (n2 * d * d - n * d * d2 - 2.0 * n1 * d * d1 + 2.0 * n * d1 * d1) / (d * d * d);
}

int or_cs_critical(double a, double b, double R, double* rho_c, double* T_c) {
  if (!(a > 0 && b > 0 && R > 0)) return OR_EINVAL;
  /* h(eta) = g'(eta) - eta g''(eta): positive at eta -> 0 (g' -> 1), negative near
   * eta = 0.5; the root is unique in between. */
  double lo = 1e-6, hi = 0.5;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi), g1, g2;
    cs_g_derivs(mid, &g1, &g2);
    double h = g1 - mid * g2;
    if (h > 0) lo = mid; else hi = mid;
  }
  double eta = 0.5 * (lo + hi), g1, g2;
  cs_g_derivs(eta, &g1, &g2);
  *rho_c = 4.0 * eta / b;
  *T_c = 8.0 * a / (b * R * g2);
  return OR_OK;
}

/*
 * Maxwell equal-area construction: the two coexisting bulk phases have equal
 * chemical potential and equal pressure,
 *     mu(rho_g) = mu(rho_l),   p0(rho_g) = p0(rho_l).
 * Solved by bisection on the common pressure P: for a trial P the gas density
 * is the root of p0 = P on the gas branch (0, spinodal_g) and the liquid
 * density the root on the liquid branch (spinodal_l, 4/b); both branches are
 * monotonic.  By Gibbs-Duhem (d mu = dp / rho) the difference
 * mu_g(P) - mu_l(P) rises with P, so the equal-mu pressure is bracketed and
 * bisected (in ln P, because the gas pressure spans many decades at low T).
 */
static double cs_dpdrho(double rho, double a, double b, double R, double T) {
  double eta = b * rho / 4.0, g1, g2;
  cs_g_derivs(eta, &g1, &g2);
  return R * T * g1 - 2.0 * a * rho;
}

static double gas_root(double P, double sp_g, double a, double b, double R, double T) {
  double lo = -700.0, hi = log(sp_g); /* ln rho */
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (or_cs_pressure(exp(mid), a, b, R, T) < P) lo = mid; else hi = mid;
  }
  return exp(0.5 * (lo + hi));
}

static double liquid_root(double P, double sp_l, double a, double b, double R, double T) {
  double lo = sp_l, hi = 4.0 / b;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (or_cs_pressure(mid, a, b, R, T) < P) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

int or_maxwell(double a, double b, double R, double T, double* rho_g, double* rho_l) {
  double rc, Tc;
  if (or_cs_critical(a, b, R, &rc, &Tc) != OR_OK) return OR_EINVAL;
  if (!(T > 0 && T < Tc)) return OR_EINVAL;
  /* spinodals: dp0/drho = 0 on either side of rho_c */
  double lo = -700.0, hi = log(rc);
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (cs_dpdrho(exp(mid), a, b, R, T) > 0) lo = mid; else hi = mid;
  }
  double sp_g = exp(lo);
  lo = rc; hi = 4.0 / b;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (cs_dpdrho(mid, a, b, R, T) < 0) lo = mid; else hi = mid;
  }
  double sp_l = hi;
  /* pressure bracket: gas branch covers (0, p(sp_g)), liquid branch (p(sp_l), inf) */
  double p_hi = or_cs_pressure(sp_g, a, b, R, T);
  double p_lo = or_cs_pressure(sp_l, a, b, R, T);
  double lp_hi = log(p_hi);
  double lp_lo = (p_lo > 0) ? log(p_lo) : -700.0;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lp_lo + lp_hi), P = exp(mid);
    double rg = gas_root(P, sp_g, a, b, R, T), rl = liquid_root(P, sp_l, a, b, R, T);
    if (or_cs_mu(rg, a, b, R, T) - or_cs_mu(rl, a, b, R, T) < 0) lp_lo = mid; else lp_hi = mid;
  }
  double P = exp(0.5 * (lp_lo + lp_hi));
  *rho_g = gas_root(P, sp_g, a, b, R, T);
  *rho_l = liquid_root(P, sp_l, a, b, R, T);
  double r1 = fabs(or_cs_mu(*rho_g, a, b, R, T) - or_cs_mu(*rho_l, a, b, R, T));
  if (!(r1 < 1e-9)) return OR_EINVAL;
  return OR_OK;
}

/* ---------------------------------------------------------------- Peng-Robinson */
/*
 * Eq. 14:  p0 = rho R T / (1 - b rho) - a alpha(T) rho^2 / (1 + 2 b rho - b^2 rho^2)
 * Eq. 15:  mu = R T ln(rho / (1 - b rho)) - a alpha / (2 sqrt2 b) ln((sqrt2 - 1 + b rho) / (sqrt2 + 1 - b rho))
 *               + R T / (1 - b rho) - a alpha rho / (1 + 2 b rho - b^2 rho^2)      (bulk part, kappa term apart)
 * alpha(T) = [1 + (0.37464 + 1.54226 w - 0.26992 w^2)(1 - sqrt(T / T_c))]^2, w the acentric factor.
 * The critical point is that of alpha = 1 (alpha(T_c) = 1).
 */
double or_pr_alpha(double T, double Tc, double w) {
  double kap = 0.37464 + 1.54226 * w - 0.26992 * w * w;
  double s = 1.0 + kap * (1.0 - sqrt(T / Tc));
  return s * s;
}

double or_pr_pressure(double rho, double a, double b, double R, double T, double alpha) {
  double br = b * rho;
  return rho * R * T / (1.0 - br) - a * alpha * rho * rho / (1.0 + 2.0 * br - br * br);
}

double or_pr_mu(double rho, double a, double b, double R, double T, double alpha) {
  double br = b * rho, s2 = sqrt(2.0);
  return R * T * log(rho / (1.0 - br)) - a * alpha / (2.0 * s2 * b) * log((s2 - 1.0 + br) / (s2 + 1.0 - br)) +
         R * T / (1.0 - br) - a * alpha * rho / (1.0 + 2.0 * br - br * br);
}

static double pr_dpdrho(double rho, double a, double b, double R, double T, double alpha) {
  double br = b * rho, D = 1.0 + 2.0 * br - br * br;
  return R * T / ((1.0 - br) * (1.0 - br)) - 2.0 * a * alpha * rho * (1.0 + br) / (D * D);
}

/* With x = b rho and h(x) = x^2 / (1 + 2x - x^2) the alpha = 1 pressure is
 * p0 = (R T / b) x / (1 - x) - (a / b^2) h(x); p0' = p0'' = 0 give
 * (1 - x) / 2 = h'(x) / h''(x), then R T_c = (a / b) (1 - x)^2 h'(x). */
static void pr_h_derivs(double x, double* h1, double* h2) {
  double D = 1.0 + 2.0 * x - x * x, D1 = 2.0 - 2.0 * x;
  /* h' = 2x(1 + x) / D^2 (quotient rule, simplified) */
  double n = 2.0 * x * (1.0 + x), n1 = 2.0 + 4.0 * x;
  *h1 = n / (D * D);
  *h2 = (n1 * D - 2.0 * n * D1) / (D * D * D);
}

int or_pr_critical(double a, double b, double R, double* rho_c, double* T_c) {
  if (!(a > 0 && b > 0 && R > 0)) return OR_EINVAL;
  double lo = 1e-6, hi = 0.9;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi), h1, h2;
    pr_h_derivs(mid, &h1, &h2);
    /* g(x) = (1 - x) h'' - 2 h': positive for small x, negative near x -> 1 */
    if ((1.0 - mid) * h2 - 2.0 * h1 > 0) lo = mid; else hi = mid;
  }
  double x = 0.5 * (lo + hi), h1, h2;
  pr_h_derivs(x, &h1, &h2);
  *rho_c = x / b;
  *T_c = (a / b) * (1.0 - x) * (1.0 - x) * h1 / R;
  return OR_OK;
}

/* ---------------------------------------------------------------- EOS by kind */
static double vdw_dpdrho(double rho, double a, double b, double R, double T) {
  double om = 1.0 - b * rho;
  return R * T / (om * om) - 2.0 * a * rho;
}
static double rks_dpdrho(double rho, double a, double b, double R, double T, double alpha) {
  double br = b * rho, om = 1.0 - br, q = 1.0 + br;
  return R * T / (om * om) - a * alpha * rho * (2.0 + br) / (q * q);
}

double or_eos_pressure(const or_eos* e, double rho) {
  switch (e->kind) {
    case OR_EOS_PR: return or_pr_pressure(rho, e->a, e->b, e->R, e->T, e->alpha);
    case OR_EOS_VDW: return or_vdw_pressure(rho, e->a, e->b, e->R, e->T);
    case OR_EOS_RKS: return or_rks_pressure(rho, e->a, e->b, e->R, e->T, e->alpha);
    default: return or_cs_pressure(rho, e->a, e->b, e->R, e->T);
  }
}

double or_eos_mu(const or_eos* e, double rho) {
  switch (e->kind) {
    case OR_EOS_PR: return or_pr_mu(rho, e->a, e->b, e->R, e->T, e->alpha);
    case OR_EOS_VDW: return or_vdw_mu(rho, e->a, e->b, e->R, e->T);
    case OR_EOS_RKS: return or_rks_mu(rho, e->a, e->b, e->R, e->T, e->alpha);
    default: return or_cs_mu(rho, e->a, e->b, e->R, e->T);
  }
}

double or_eos_dpdrho(const or_eos* e, double rho) {
  switch (e->kind) {
    case OR_EOS_PR: return pr_dpdrho(rho, e->a, e->b, e->R, e->T, e->alpha);
    case OR_EOS_VDW: return vdw_dpdrho(rho, e->a, e->b, e->R, e->T);
    case OR_EOS_RKS: return rks_dpdrho(rho, e->a, e->b, e->R, e->T, e->alpha);
    default: return cs_dpdrho(rho, e->a, e->b, e->R, e->T);
  }
}

int or_eos_critical(int kind, double a, double b, double R, double* rho_c, double* T_c) {
  switch (kind) {
    case OR_EOS_PR: return or_pr_critical(a, b, R, rho_c, T_c);
    case OR_EOS_VDW: case OR_EOS_RKS: return or_cubic_critical(kind, a, b, R, rho_c, T_c);
    default: return or_cs_critical(a, b, R, rho_c, T_c);
  }
}

int or_eos_make(int kind, double a, double b, double R, double Tr, double acentric, or_eos* e) {
  double rc, Tc;
  if (kind < OR_EOS_CS || kind > OR_EOS_RKS) return OR_EINVAL;
  if (or_eos_critical(kind, a, b, R, &rc, &Tc) != OR_OK) return OR_EINVAL;
  e->kind = kind; e->a = a; e->b = b; e->R = R; e->T = Tr * Tc; e->Tc = Tc; e->rho_c = rc;
  e->alpha = kind == OR_EOS_PR ? or_pr_alpha(e->T, Tc, acentric)
             : kind == OR_EOS_RKS ? or_rks_alpha(e->T, Tc, acentric) : 1.0;
  e->rho_max = kind == OR_EOS_CS ? 4.0 / b : 1.0 / b;
  return OR_OK;
}

/* The same equal-pressure, equal-mu bisection as or_maxwell, for either EOS.
 * At the PR critical point alpha = 1; below it alpha > 1 and the spinodals
 * lie on either side of rho_c as for CS. */
int or_eos_maxwell(const or_eos* e, double* rho_g, double* rho_l) {
  if (!(e->T > 0 && e->T < e->Tc)) return OR_EINVAL;
  double lo = -700.0, hi = log(e->rho_c);
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (or_eos_dpdrho(e, exp(mid)) > 0) lo = mid; else hi = mid;
  }
  double sp_g = exp(lo);
  lo = e->rho_c; hi = e->rho_max;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (or_eos_dpdrho(e, mid) < 0) lo = mid; else hi = mid;
  }
  double sp_l = hi;
  double p_hi = or_eos_pressure(e, sp_g), p_lo = or_eos_pressure(e, sp_l);
  double lp_hi = log(p_hi), lp_lo = (p_lo > 0) ? log(p_lo) : -700.0;
  double rg = 0, rl = 0;
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lp_lo + lp_hi), P = exp(mid);
    double glo = -700.0, ghi = log(sp_g);
    for (int k = 0; k < 300; ++k) {
      double m = 0.5 * (glo + ghi);
      if (or_eos_pressure(e, exp(m)) < P) glo = m; else ghi = m;
    }
    double llo = sp_l, lhi = e->rho_max;
    for (int k = 0; k < 300; ++k) {
      double m = 0.5 * (llo + lhi);
      if (or_eos_pressure(e, m) < P) llo = m; else lhi = m;
    }
    rg = exp(0.5 * (glo + ghi));
    rl = 0.5 * (llo + lhi);
    if (or_eos_mu(e, rg) - or_eos_mu(e, rl) < 0) lp_lo = mid; else lp_hi = mid;
  }
  *rho_g = rg;
  *rho_l = rl;
  if (!(fabs(or_eos_mu(e, rg) - or_eos_mu(e, rl)) < 1e-9)) return OR_EINVAL;
  return OR_OK;
}

/* ---------------------------------------------------------------- van der Waals, Redlich-Kwong-Soave */
/*
 * Not printed by the paper; their chemical potentials follow from Eq. 13 the
 * way Eq. 15 does for PR (psi = rho (int p0 / rho^2 drho + C), mu = psi'):
 *   VDW  p0 = rho R T / (1 - b rho) - a rho^2
 *        mu = R T [ln(rho / (1 - b rho)) + 1 / (1 - b rho)] - 2 a rho
 *   RKS  p0 = rho R T / (1 - b rho) - a alpha rho^2 / (1 + b rho)
 *        mu = R T [ln(rho / (1 - b rho)) + 1 / (1 - b rho)] - (a alpha / b) ln(1 + b rho) - a alpha rho / (1 + b rho)
 *        alpha(T) = [1 + (0.480 + 1.574 w - 0.176 w^2)(1 - sqrt(T / T_c))]^2
 * Critical points (p0' = p0'' = 0; RKS with alpha = 1) by bisection on x = b rho.
 */
double or_vdw_pressure(double rho, double a, double b, double R, double T) {
  return rho * R * T / (1.0 - b * rho) - a * rho * rho;
}
double or_vdw_mu(double rho, double a, double b, double R, double T) {
  double om = 1.0 - b * rho;
  return R * T * (log(rho / om) + 1.0 / om) - 2.0 * a * rho;
}
double or_rks_alpha(double T, double Tc, double w) {
  double s = 1.0 + (0.480 + 1.574 * w - 0.176 * w * w) * (1.0 - sqrt(T / Tc));
  return s * s;
}
double or_rks_pressure(double rho, double a, double b, double R, double T, double alpha) {
  double br = b * rho;
  return rho * R * T / (1.0 - br) - a * alpha * rho * rho / (1.0 + br);
}
double or_rks_mu(double rho, double a, double b, double R, double T, double alpha) {
  double br = b * rho, om = 1.0 - br;
  return R * T * (log(rho / om) + 1.0 / om) - a * alpha / b * log(1.0 + br) - a * alpha * rho / (1.0 + br);
}

/* critical x = b rho from the attractive term h(x) (p0 = (R T / b) x / (1 - x) - (a / b^2) h):
 * 2 h'(x) = (1 - x) h''(x); R T_c = (a / b) (1 - x)^2 h'(x).  h = x^2 (VDW) or x^2 / (1 + x) (RKS). */
static void attr_derivs(int kind, double x, double* h1, double* h2) {
  if (kind == OR_EOS_VDW) { *h1 = 2.0 * x; *h2 = 2.0; return; }
  /* x^2 / (1 + x): h' = (2x + x^2) / (1 + x)^2, h'' = 2 / (1 + x)^3 */
  double q = 1.0 + x;
  *h1 = (2.0 * x + x * x) / (q * q);
  *h2 = 2.0 / (q * q * q);
}

int or_cubic_critical(int kind, double a, double b, double R, double* rho_c, double* T_c) {
  if (!(a > 0 && b > 0 && R > 0)) return OR_EINVAL;
  double lo = 1e-6, hi = 0.9;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi), h1, h2;
    attr_derivs(kind, mid, &h1, &h2);
    if ((1.0 - mid) * h2 - 2.0 * h1 > 0) lo = mid; else hi = mid;
  }
  double x = 0.5 * (lo + hi), h1, h2;
  attr_derivs(kind, x, &h1, &h2);
  *rho_c = x / b;
  *T_c = (a / b) * (1.0 - x) * (1.0 - x) * h1 / R;
  return OR_OK;
}

/* ---------------------------------------------------------------- flat interface (Eq. 29) */
/*
 * A flat liquid-vapour interface in equilibrium (Eq. 29, with rho(-inf) =
 * rho_g, rho(+inf) = rho_l) has a uniform chemical potential in mesh units
 * (Eq. 16):  k^2 psi'(rho) - kappa rho'' = mu_0 = k^2 psi'(rho_g).
 * Multiplying by rho' and integrating from the gas side,
 *     (kappa / 2) rho'^2 = k^2 W(rho),
 *     W(rho) = psi(rho) - psi(rho_g) - psi'(rho_g) (rho - rho_g),
 * and with psi = rho psi' - p0 (Eq. 10),
 *     W(rho) = rho (psi'(rho) - psi'(rho_g)) - (p0(rho) - p0(rho_g)).
 * So rho' = k sqrt(2 W / kappa) and y(rho) = int_{rho_m}^{rho} dr / rho'(r),
 * rho_m = (rho_g + rho_l) / 2 at y = y0.  The integral is taken in the logit
 * variable s, rho = rho_g + (rho_l - rho_g) / (1 + e^-s), where dy/ds stays
 * finite, with 3-point Gauss-Legendre on a table of steps 0.01 over |s| <= 14;
 * the node values by bisection on the table and Newton within a step.
 * Beyond the table (rho within 1e-6 of a bulk value, where W is a difference
 * of nearly equal terms) the profile follows the linearised equation
 * kappa d'' = k^2 psi''(rho_b) d, psi'' = p0' / rho: exponential tails.
 */
#define FLAT_S 14.0
#define FLAT_H 0.01
#define FLAT_M 2800 /* 2 FLAT_S / FLAT_H */

typedef struct {
  const or_eos* e;
  double g, l, mug, pg, k, kappa;
} flat_ctx;

static double flat_rho(const flat_ctx* c, double s) { return c->g + (c->l - c->g) / (1.0 + exp(-s)); }

static double flat_drho(const flat_ctx* c, double rho) {
  double W = rho * (or_eos_mu(c->e, rho) - c->mug) - (or_eos_pressure(c->e, rho) - c->pg);
  if (W < 0) W = 0;
  return c->k * sqrt(2.0 * W / c->kappa);
}

static double flat_dyds(const flat_ctx* c, double s) {
  double sig = 1.0 / (1.0 + exp(-s));
  double drds = (c->l - c->g) * sig * (1.0 - sig);
  return drds / flat_drho(c, flat_rho(c, s));
}

/* int_a^b dy/ds ds, 3-point Gauss-Legendre */
static double flat_gl3(const flat_ctx* c, double a, double b) {
  const double x = sqrt(0.6), m = 0.5 * (a + b), h = 0.5 * (b - a);
  return h * (5.0 / 9.0 * flat_dyds(c, m - h * x) + 8.0 / 9.0 * flat_dyds(c, m) + 5.0 / 9.0 * flat_dyds(c, m + h * x));
}

int or_flat_profile(const or_params* p, int n, double y0, double* rho, double* drho) {
  if (!p || n < 1 || !rho || !(p->k > 0) || !(p->kappa > 0)) return OR_EINVAL;
  or_eos e;
  if (or_eos_make(p->eos, p->a, p->b, p->R, p->Tr, p->acentric, &e) != OR_OK) return OR_EINVAL;
  double g, l;
  if (or_eos_maxwell(&e, &g, &l) != OR_OK) return OR_EINVAL;
  flat_ctx c = {&e, g, l, or_eos_mu(&e, g), or_eos_pressure(&e, g), p->k, p->kappa};
  static double Y[FLAT_M + 1]; /* y(s_i) - y0, s_i = -FLAT_S + i FLAT_H; y(0) = 0 at i = FLAT_M / 2 */
  const int mid = FLAT_M / 2;
  Y[mid] = 0.0;
  for (int i = mid + 1; i <= FLAT_M; ++i)
    Y[i] = Y[i - 1] + flat_gl3(&c, -FLAT_S + (i - 1) * FLAT_H, -FLAT_S + i * FLAT_H);
  for (int i = mid - 1; i >= 0; --i) Y[i] = Y[i + 1] - flat_gl3(&c, -FLAT_S + i * FLAT_H, -FLAT_S + (i + 1) * FLAT_H);
  /* tail rates from the linearised equation */
  const double lam_g = p->k * sqrt(or_eos_dpdrho(&e, g) / g / p->kappa);
  const double lam_l = p->k * sqrt(or_eos_dpdrho(&e, l) / l / p->kappa);
  for (int j = 0; j < n; ++j) {
    const double t = (double)j - y0;
    double r, d;
    if (t <= Y[0]) {
      const double d0 = flat_rho(&c, -FLAT_S) - g;
      r = g + d0 * exp(lam_g * (t - Y[0]));
      d = lam_g * (r - g);
    } else if (t >= Y[FLAT_M]) {
      const double d0 = l - flat_rho(&c, FLAT_S);
      r = l - d0 * exp(-lam_l * (t - Y[FLAT_M]));
      d = lam_l * (l - r);
    } else {
      int lo = 0, hi = FLAT_M;
      while (hi - lo > 1) {
        const int m = (lo + hi) / 2;
        if (Y[m] <= t) lo = m; else hi = m;
      }
      const double sa = -FLAT_S + lo * FLAT_H;
      double s = sa + FLAT_H * (t - Y[lo]) / (Y[hi] - Y[lo]);
      for (int it = 0; it < 6; ++it) s -= (Y[lo] + flat_gl3(&c, sa, s) - t) / flat_dyds(&c, s);
      r = flat_rho(&c, s);
      d = flat_drho(&c, r);
    }
    rho[j] = r;
    if (drho) drho[j] = d;
  }
  return OR_OK;
}
