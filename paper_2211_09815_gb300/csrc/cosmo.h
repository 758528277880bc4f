// Host FP64 cosmology tables for the PM engine (see cosmo.cpp).
#pragma once
#include <vector>

namespace pmgb {
namespace cosmo {

struct TimeCoef {
  // per step i = 1..n (index i-1): FastPM factors of Sec. 2.3, Eq. 15 and d/dOmega_m
  std::vector<double> k1, dd, k2, dk1, ddd, dk2;
  double d1_a0, gd_a0, dd1_a0, dgd_a0;  // D1, G_D at a0 and d/dOmega_m
  double d2_a0, gd2_a0, dd2_a0, dgd2_a0; // D2, G_D2 = a^2 H D2' at a0 and d/dOmega_m (2LPT)
};

// K1_i, D_i, K2_i for a linear-in-a grid a0..a1 with n steps.
void time_coefficients(double a0, double a1, int n, double omega_m, TimeCoef& out);

// P_lin(kf sqrt(n2)) for n2 = 0..maxn2 (p[0] = 0) and d ln P / d theta_j ([5][maxn2+1]).
void plin_tables(const double theta[5], double kf, int maxn2, std::vector<double>& p,
                 std::vector<double>& dlnp);

// Drift factor of a position observed at scale factor a inside step j + 1, a_j < a <=
// a_{j+1} of the linear-in-a grid: the FastPM drift of Sec. 2.3 (Eq. 15) stopped at a,
// Dp_j(a) = [D1(a) - D1(a_j)] / G_D(a_{j+1/2}), and its d/dOmega_m.
struct PartialDrift {
  int j;
  double fac, dfac;
};
void partial_drift(double a0, double a1, int n, double omega_m, double a, PartialDrift& out);

double transfer_eh(double k, double om, double ob, double h);
double plin_value(double k, const double theta[5]);

}  // namespace cosmo
}  // namespace pmgb
