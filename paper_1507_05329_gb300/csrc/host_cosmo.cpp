// Host FP64 cosmology and COLA time coefficients of the library (independent of the test oracle).
//
//   H(a) = sqrt(Om a^-3 + 1 - Om) (flat LCDM, H0 = 1)
//   D1(a) = H(a) int_0^a da'/(a'H)^3 / (same at a = 1)                 §2.1 growing mode
//   D2(a) = -3/7 D1^2 Omega(a)^(-1/143), Omega(a) = Om/(Om + OL a^3)    §2.1 and its footnote
//   drift = int_{a_i}^{a_{i+1}} (a/a_{i+1/2})^n da / (a^3 H)             §2.2 eq. (cola-drift)
//   kick  = (a_hi^n - a_lo^n) / (n a_i^n H(a_i))                        §2.2 eq. (cola-kick)
//   2LPT acceleration F_2LPT = (3/2)(Om/a)[D1 Psi1 + (D2 - D1^2) Psi2] (the growth equations)
//   P(k) = A k^ns T_BBKS(k)^2, Gamma = Om h, A from sigma8 (8 Mpc/h top hat) at a = 1.
//
// Quadrature: adaptive Gauss-Kronrod 7/15 on bisected intervals to 1e-13 relative.
#include "cola_internal.h"

#include <cmath>
#include <functional>

namespace cola {
namespace {

// Gauss-Kronrod 7/15 nodes and weights (Kronrod 1965; the standard published table).
const double kXgk[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                        0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                        0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                        0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
const double kWgk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                        0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                        0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                        0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
const double kWg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                       0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

void gk15(const std::function<double(double)>& f, double a, double b, double* res, double* err) {
  const double c = 0.5 * (a + b), h = 0.5 * (b - a);
  const double fc = f(c);
  double rk = fc * kWgk[7], rg = fc * kWg[3];
  for (int j = 0; j < 7; ++j) {
    const double dx = h * kXgk[j];
    const double f1 = f(c - dx), f2 = f(c + dx);
    rk += kWgk[j] * (f1 + f2);
    if (j % 2 == 1) rg += kWg[j / 2] * (f1 + f2);
  }
  *res = rk * h;
  *err = std::fabs((rk - rg) * h);
}

double adapt(const std::function<double(double)>& f, double a, double b, double whole, double tol,
             int depth) {
  double r, e;
  gk15(f, a, b, &r, &e);
  if (depth > 60 || e <= tol * std::fabs(whole) || e < 1e-300) return r;
  const double m = 0.5 * (a + b);
  return adapt(f, a, m, whole, tol, depth + 1) + adapt(f, m, b, whole, tol, depth + 1);
}

double integrate(const std::function<double(double)>& f, double a, double b) {
  double r, e;
  gk15(f, a, b, &r, &e);
  // a first estimate fixes the absolute target; refinement is then relative to the whole integral
  double whole = r;
  for (int pass = 0; pass < 3; ++pass) {
    const double next = adapt(f, a, b, whole, 1e-14, 0);
    if (std::fabs(next - whole) <= 1e-13 * std::fabs(next)) return next;
    whole = next;
  }
  return whole;
}

}  // namespace

double hubble(double a, double om) { return std::sqrt(om / (a * a * a) + (1.0 - om)); }

static double growth_integral(double a, double om) {
  if (a <= 0.0) return 0.0;
  return integrate([om](double x) { const double ah = x * hubble(x, om); return 1.0 / (ah * ah * ah); },
                   0.0, a);
}

Cosmo::Cosmo(double om_, double h_, double ns_, double s8_) : om(om_), h(h_), ns(ns_), sigma8(s8_) {
  i1 = growth_integral(1.0, om);
  // sigma^2(8 Mpc/h) for A = 1, integrated in ln k over [1e-7, 1e3] h/Mpc in decades
  auto integrand = [this](double lnk) {
    const double k = std::exp(lnk);
    const double x = 8.0 * k;
    double w;
    if (x < 1e-3) w = 1.0 - x * x / 10.0;
    else w = 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
    const double t = transfer(k);
    return k * k * k * std::pow(k, ns) * t * t * w * w / (2.0 * M_PI * M_PI);
  };
  double s2 = 0.0;
  for (int d = -7; d < 3; ++d) s2 += integrate(integrand, d * M_LN10, (d + 1) * M_LN10);
  amp = sigma8 * sigma8 / s2;
}

double Cosmo::transfer(double k) const {
  const double q = k / (om * h);
  if (q <= 0.0) return 1.0;
  const double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
  return std::log1p(2.34 * q) / (2.34 * q) * std::pow(poly, -0.25);
}

double Cosmo::power(double k) const { return amp * std::pow(k, ns) * std::pow(transfer(k), 2); }

double Cosmo::omega_a(double a) const { return om / (om + (1.0 - om) * a * a * a); }

double Cosmo::d1(double a) const { return hubble(a, om) * growth_integral(a, om) / i1; }

double Cosmo::d1_da(double a) const {
  const double hh = hubble(a, om);
  const double dh = -1.5 * om / (a * a * a * a) / hh;
  return (dh * growth_integral(a, om) + hh / std::pow(a * hh, 3)) / i1;
}

double Cosmo::d2(double a) const {
  const double g = d1(a);
  return -3.0 / 7.0 * g * g * std::pow(omega_a(a), -1.0 / 143.0);
}

double Cosmo::d2_da(double a) const {
  const double ol = 1.0 - om, oa = omega_a(a);
  const double dom = -3.0 * om * ol * a * a / ((om + ol * a * a * a) * (om + ol * a * a * a));
  const double g = d1(a), gp = d1_da(a);
  return -3.0 / 7.0 * (2.0 * g * gp * std::pow(oa, -1.0 / 143.0) +
                       g * g * (-1.0 / 143.0) * std::pow(oa, -1.0 / 143.0 - 1.0) * dom);
}

double Cosmo::drift(double a0, double a1, double ahalf, double nlpt, int ansatz) const {
  const double om_ = om;
  if (ansatz == 0)
    return integrate([=](double a) { return std::pow(a / ahalf, nlpt) / (a * a * a * hubble(a, om_)); },
                     a0, a1);
  return integrate([=](double a) { return 1.0 / (a * a * a * hubble(a, om_)); }, a0, a1);
}

double Cosmo::kick(double alo, double ahi, double ai, double nlpt) const {
  return (std::pow(ahi, nlpt) - std::pow(alo, nlpt)) / (nlpt * std::pow(ai, nlpt) * hubble(ai, om));
}

StepScalars step_scalars(const cola_params& p, const Cosmo& c, int i) {
  StepScalars s{};
  const double ns = p.nstep;
  s.a = i / ns;
  s.a_lo = (i - 0.5) / ns;
  if (i == 1 && p.ic_mode == 1) s.a_lo = s.a;
  const bool last = (i == p.nstep);
  s.a_hi = last ? s.a : (i + 0.5) / ns;
  const double g1 = c.d1(s.a), g2 = c.d2(s.a);
  s.force_scale = 1.5 * p.omega_m / s.a;
  s.c1 = s.force_scale * g1;
  s.c2 = s.force_scale * (g2 - g1 * g1);
  s.kick = c.kick(s.a_lo, s.a_hi, s.a, p.nlpt);
  s.d1 = g1;
  s.d2 = g2;
  if (last) {
    s.drift = s.dd1 = s.dd2 = 0.0;
  } else {
    const double an = (i + 1) / ns;
    s.drift = c.drift(s.a, an, (i + 0.5) / ns, p.nlpt, p.drift_ansatz);
    s.dd1 = c.d1(an) - g1;
    s.dd2 = c.d2(an) - g2;
  }
  return s;
}

}  // namespace cola
