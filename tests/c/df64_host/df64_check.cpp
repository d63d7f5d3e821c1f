// CPU check of the double-float arithmetic of df64.cuh against double
// precision libm: exp over [-60, 0] (relative error over max(1, |x|)), log1p
// over [0, 1] (absolute), and the two per-sample entropy functions of the
// certified ordering, |u| + log1p(e^{-2|u|}) (absolute over max(1, value))
// and u e^{-u^2/2} (absolute), on light- and heavy-tailed samples.  Prints one line per function:
// "<name> <max error> <argument>".
#include <cstdio>
#include <cstdint>
#include <cmath>
#include <random>

#include "df64.cuh"

using namespace vl::df;

static double to_d(F2 x) { return (double)x.hi + (double)x.lo; }

int main() {
  float2 tab[32];
  for (int j = 0; j < 32; ++j) tab[j] = kExp2Frac[j];
  std::mt19937_64 g(2409);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  std::normal_distribution<double> N(0.0, 1.0);
  const int n = 400000;
  double e_exp = 0, a_exp = 0, e_log = 0, a_log = 0, e_lc = 0, a_lc = 0, e_g = 0, a_g = 0;
  for (int k = 0; k < n; ++k) {
    // exp: arguments spread over [-60, 0] (below, the low part of a pair
    // leaves the normal FP32 range) and dense in [-1, 0]
    const F2 x = from_double(k & 1 ? -60.0 * U(g) : -U(g));
    const double xr = to_d(x), ref = std::exp(xr);
    // relative error per unit of |x| (the reduction x - k ln2/32 carries an
    // absolute error proportional to |x|)
    const double e = std::fabs(to_d(dexp(x, tab)) - ref) / ref / std::fmax(1.0, std::fabs(xr));
    if (e > e_exp) { e_exp = e; a_exp = xr; }
    // log1p on [0, 1]
    const F2 y = from_double(k & 3 ? U(g) : 1e-6 * U(g));
    const double yr = to_d(y);
    const double el = std::fabs(to_d(dlog1p(y, tab)) - std::log1p(yr));
    if (el > e_log) { e_log = el; a_log = yr; }
    // per-sample entropy functions on light and heavy tails
    const double z = N(g);
    const double u0 = k & 1 ? z * (k % 3 == 0 ? 4.0 : 1.0)
                            : z / std::sqrt(std::fmax(1e-3, -2.0 * std::log(std::fmax(1e-300, U(g))) / 3.0));
    const F2 u = from_double(u0);
    const double ur = to_d(u);
    const F2 au = u.hi < 0.0f ? neg(u) : u;
    const double lc = to_d(add(au, dlog1p(dexp(scale(au, -2.0f), tab), tab)));
    const double lref = std::fabs(ur) + std::log1p(std::exp(-2.0 * std::fabs(ur)));
    const double elc = std::fabs(lc - lref) / std::fmax(1.0, std::fabs(lref));
    if (elc > e_lc) { e_lc = elc; a_lc = ur; }
    const double gv = to_d(mul(u, dexp(scale(sqr(u), -0.5f), tab)));
    const double eg = std::fabs(gv - ur * std::exp(-0.5 * ur * ur));
    if (eg > e_g) { e_g = eg; a_g = ur; }
  }
  std::printf("exp %.6e %.17g\n", e_exp, a_exp);
  std::printf("log1p %.6e %.17g\n", e_log, a_log);
  std::printf("logcosh %.6e %.17g\n", e_lc, a_lc);
  std::printf("gauss %.6e %.17g\n", e_g, a_g);
  return 0;
}
