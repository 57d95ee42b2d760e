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
