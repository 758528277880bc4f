// Host FP64 cosmology for the PM engine: linear power spectrum (Sec. 2.1, Eq. 7) with
// the Eisenstein & Hu (1998) no-wiggle transfer function, the linear growth ODE in the
// suppression factor G1 = D1/a (App. A, Eqs. 52-58), the FastPM drift/kick factors
// (Sec. 2.3, Eq. 15) and their derivatives with respect to theta.
//
// Derivatives are taken by the complex step, d f / d x = Im f(x + i eps) / eps, which
// is exact to rounding for the analytic expressions here; every routine is templated on
// the scalar type (double or std::complex<double>).
#include <cmath>
#include <complex>
#include <vector>

#include "cosmo.h"

namespace pmgb {
namespace cosmo {

using cd = std::complex<double>;

static const double kCoverH0 = 2997.92458;  // c / (100 km/s/Mpc), Mpc/h
static const double kTcmb = 2.7255;         // K
static const double kPivot = 0.05;          // 1/Mpc
static const double kAic = 1e-4;            // start of the growth integration
static const double kLnaStep = 1.0 / 1024;  // largest RK4 step in ln a

template <class R> static R hubble(double a, R om) { return std::sqrt(om / (a * a * a) + (1.0 - om)); }

// y = (G1, G1'), ' = d / d ln a.  G1'' = -(4 + H'/H) G1' - (3 + H'/H - 3/2 Om(a)) G1,
// with H'/H = -3/2 Om(a) in flat LCDM (App. A, Eq. 56).
template <class R> static void rhs(double lna, const R y[2], R om, R out[2]) {
  const double a = std::exp(lna);
  const R h2 = om / (a * a * a) + (1.0 - om);
  const R oma = om / (a * a * a) / h2;
  const R dlnh = -1.5 * oma;
  out[0] = y[1];
  out[1] = -(4.0 + dlnh) * y[1] - (3.0 + dlnh - 1.5 * oma) * y[0];
}

// G1 and G1' at ascending scale factors (RK4 from a = 1e-4, G1 = 1, G1' = 0: Eq. 57).
template <class R>
static void growth(const std::vector<double>& a, R om, std::vector<R>& g, std::vector<R>& dg) {
  g.assign(a.size(), R(0));
  dg.assign(a.size(), R(0));
  R y[2] = {R(1.0), R(0.0)};
  double lna = std::log(kAic);
  for (size_t idx = 0; idx < a.size(); ++idx) {
    const double target = std::log(a[idx]);
    const double span = target - lna;
    if (span > 0) {
      const int nsub = (int)std::ceil(span / kLnaStep);
      const double h = span / nsub;
      for (int s = 0; s < nsub; ++s) {
        R k1[2], k2[2], k3[2], k4[2], t[2];
        rhs(lna, y, om, k1);
        for (int c = 0; c < 2; ++c) t[c] = y[c] + 0.5 * h * k1[c];
        rhs(lna + 0.5 * h, t, om, k2);
        for (int c = 0; c < 2; ++c) t[c] = y[c] + 0.5 * h * k2[c];
        rhs(lna + 0.5 * h, t, om, k3);
        for (int c = 0; c < 2; ++c) t[c] = y[c] + h * k3[c];
        rhs(lna + h, t, om, k4);
        for (int c = 0; c < 2; ++c) y[c] += (h / 6.0) * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
        lna += h;
      }
      lna = target;
    }
    g[idx] = y[0];
    dg[idx] = y[1];
  }
}

// D1, G_D = a^2 H D1', G_K = 3/2 Om D1 (App. A, Eq. 58 with the D1 ODE) at ascending a.
template <class R>
static void factors(const std::vector<double>& a, R om, std::vector<R>& d1, std::vector<R>& gd,
                    std::vector<R>& gk) {
  std::vector<R> g, dg;
  growth(a, om, g, dg);
  d1.resize(a.size());
  gd.resize(a.size());
  gk.resize(a.size());
  for (size_t i = 0; i < a.size(); ++i) {
    d1[i] = a[i] * g[i];
    gd[i] = a[i] * a[i] * hubble(a[i], om) * (a[i] * (g[i] + dg[i]));
    gk[i] = 1.5 * om * d1[i];
  }
}

// y = (G1, G1', G2, G2'): both suppression-factor ODEs of App. A (Eq. 56) with
// G2'' = -(6 + H'/H) G2' - (8 + 2 H'/H - 3/2 Om(a)) G2 + 3/2 Om(a) G1^2.
template <class R> static void rhs2(double lna, const R y[4], R om, R out[4]) {
  rhs(lna, y, om, out);
  const double a = std::exp(lna);
  const R h2 = om / (a * a * a) + (1.0 - om);
  const R oma = om / (a * a * a) / h2;
  const R dlnh = -1.5 * oma;
  out[2] = y[3];
  out[3] = -(6.0 + dlnh) * y[3] - (8.0 + 2.0 * dlnh - 1.5 * oma) * y[2] + 1.5 * oma * y[0] * y[0];
}

// Second-order growth at one scale factor a: D2 = a^2 G2 and G_D2 = a^2 H D2' with
// D2' = a^2 (2 G2 + G2') (App. A, Eq. 59 for m = 2), by RK4 in ln a from a_ic with
// G1 = 1, G1' = 0, G2 = 3/7, G2' = 0 (Eq. 57).
template <class R> static void factors2(double a, R om, R& d2, R& gd2) {
  R y[4] = {R(1.0), R(0.0), R(3.0 / 7.0), R(0.0)};
  double lna = std::log(kAic);
  const double span = std::log(a) - lna;
  if (span > 0) {
    const int nsub = (int)std::ceil(span / kLnaStep);
    const double h = span / nsub;
    for (int s = 0; s < nsub; ++s) {
      R k1[4], k2[4], k3[4], k4[4], t[4];
      rhs2(lna, y, om, k1);
      for (int c = 0; c < 4; ++c) t[c] = y[c] + 0.5 * h * k1[c];
      rhs2(lna + 0.5 * h, t, om, k2);
      for (int c = 0; c < 4; ++c) t[c] = y[c] + 0.5 * h * k2[c];
      rhs2(lna + 0.5 * h, t, om, k3);
      for (int c = 0; c < 4; ++c) t[c] = y[c] + h * k3[c];
      rhs2(lna + h, t, om, k4);
      for (int c = 0; c < 4; ++c) y[c] += (h / 6.0) * (k1[c] + 2.0 * k2[c] + 2.0 * k3[c] + k4[c]);
      lna += h;
    }
  }
  d2 = a * a * y[2];
  gd2 = a * a * hubble(a, om) * (a * a * (2.0 * y[2] + y[3]));
}

// Eisenstein & Hu 1998 no-wiggle T(k), k in h/Mpc: their Eqs. 26 (sound horizon),
// 28 (q), 29 (T0), 30 (Gamma_eff), 31 (alpha_Gamma).
template <class R> static R transfer(double k, R om, R ob, R h) {
  const double th = kTcmb / 2.7;
  const R omh2 = om * h * h, obh2 = ob * h * h, fb = ob / om;
  const R s = 44.5 * std::log(9.83 / omh2) / std::sqrt(1.0 + 10.0 * std::pow(obh2, 0.75));
  const R alpha = 1.0 - 0.328 * std::log(431.0 * omh2) * fb + 0.38 * std::log(22.3 * omh2) * fb * fb;
  const R ks = 0.43 * k * h * s;
  const R ks2 = ks * ks;
  const R gam = om * h * (alpha + (1.0 - alpha) / (1.0 + ks2 * ks2));
  const R q = k * th * th / gam;
  const R l0 = std::log(2.0 * M_E + 1.8 * q);
  const R c0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
  return l0 / (l0 + c0 * q * q);
}

// P_lin(k) (Sec. 2.1, Eq. 7) in (Mpc/h)^3, k in h/Mpc, k_pivot = 0.05/Mpc.
template <class R> static R plin(double k, const R th[5]) {
  const R t = transfer(k, th[2], th[3], th[4]);
  const double ck = kCoverH0 * k;
  return 2.0 * M_PI * M_PI / (k * k * k) * 0.16 * th[0] * std::pow(k * th[4] / kPivot, th[1] - 1.0) * t * t *
         (ck * ck * ck * ck) / (th[2] * th[2]);
}

static const double kEps = 1e-30;

double transfer_eh(double k, double om, double ob, double h) { return transfer(k, om, ob, h); }

double plin_value(double k, const double theta[5]) { return plin(k, theta); }

void plin_tables(const double theta[5], double kf, int maxn2, std::vector<double>& p,
                 std::vector<double>& dlnp /* [5][maxn2+1] */) {
  p.assign(maxn2 + 1, 0.0);
  dlnp.assign(5 * (size_t)(maxn2 + 1), 0.0);
  for (int n2 = 1; n2 <= maxn2; ++n2) {
    const double k = kf * std::sqrt((double)n2);
    p[n2] = plin(k, theta);
    for (int j = 0; j < 5; ++j) {
      cd th[5];
      for (int i = 0; i < 5; ++i) th[i] = cd(theta[i], 0.0);
      th[j] += cd(0.0, kEps);
      dlnp[(size_t)j * (maxn2 + 1) + n2] = std::imag(std::log(plin(k, th))) / kEps;
    }
  }
}

void time_coefficients(double a0, double a1, int n, double om, TimeCoef& out) {
  // a_i linear in a, a_{i-1/2} the arithmetic mean (reading); all nodes in ascending order
  std::vector<double> a(2 * n + 1);
  for (int i = 0; i <= 2 * n; ++i) a[i] = a0 + (a1 - a0) * (0.5 * i) / n;
  std::vector<double> d1, gd, gk;
  std::vector<cd> cd1, cgd, cgk;
  factors(a, om, d1, gd, gk);
  factors(a, cd(om, kEps), cd1, cgd, cgk);
  out.k1.resize(n);
  out.dd.resize(n);
  out.k2.resize(n);
  out.dk1.resize(n);
  out.ddd.resize(n);
  out.dk2.resize(n);
  for (int i = 1; i <= n; ++i) {
    const int im = 2 * (i - 1), ih = 2 * i - 1, ii = 2 * i;
    // K1_i = [G_D(a_{i-1/2}) - G_D(a_{i-1})] / G_K(a_{i-1}), D_i, K2_i  (Eq. 15)
    out.k1[i - 1] = (gd[ih] - gd[im]) / gk[im];
    out.dd[i - 1] = (d1[ii] - d1[im]) / gd[ih];
    out.k2[i - 1] = (gd[ii] - gd[ih]) / gk[ii];
    out.dk1[i - 1] = std::imag((cgd[ih] - cgd[im]) / cgk[im]) / kEps;
    out.ddd[i - 1] = std::imag((cd1[ii] - cd1[im]) / cgd[ih]) / kEps;
    out.dk2[i - 1] = std::imag((cgd[ii] - cgd[ih]) / cgk[ii]) / kEps;
  }
  out.d1_a0 = d1[0];
  out.gd_a0 = gd[0];
  out.dd1_a0 = std::imag(cd1[0]) / kEps;
  out.dgd_a0 = std::imag(cgd[0]) / kEps;
  cd cd2, cgd2;
  factors2(a0, om, out.d2_a0, out.gd2_a0);
  factors2(a0, cd(om, kEps), cd2, cgd2);
  out.dd2_a0 = std::imag(cd2) / kEps;
  out.dgd2_a0 = std::imag(cgd2) / kEps;
}

void partial_drift(double a0, double a1, int n, double om, double a, PartialDrift& out) {
  auto node = [&](int i) { return a0 + (a1 - a0) * (0.5 * (2 * i)) / n; };   // a_i as in time_coefficients
  int j = (int)std::ceil((a - a0) / (a1 - a0) * n) - 1;
  j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
  while (j > 0 && !(node(j) < a)) --j;
  while (j < n - 1 && node(j + 1) < a) ++j;
  const double aj = node(j), ah = a0 + (a1 - a0) * (0.5 * (2 * j + 1)) / n;
  std::vector<double> d1, gd, gk, d1h, gdh, gkh;
  std::vector<cd> cd1, cgd, cgk, cd1h, cgdh, cgkh;
  factors(std::vector<double>{aj, a}, om, d1, gd, gk);
  factors(std::vector<double>{ah}, om, d1h, gdh, gkh);
  factors(std::vector<double>{aj, a}, cd(om, kEps), cd1, cgd, cgk);
  factors(std::vector<double>{ah}, cd(om, kEps), cd1h, cgdh, cgkh);
  out.j = j;
  out.fac = (d1[1] - d1[0]) / gdh[0];
  out.dfac = std::imag((cd1[1] - cd1[0]) / cgdh[0]) / kEps;
}

}  // namespace cosmo
}  // namespace pmgb
