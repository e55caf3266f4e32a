// Equal-acceptance update of a parallel-tempering ladder (Sec. II: the
// temperature set is chosen so that the exchange acceptance rate does not
// depend on the temperature).  Host code: the ladder has at most a few
// dozen couplings.
//
// Model: near a pair (beta_k, beta_k+1) the energy distributions are
// Gaussians of a common width sigma_k, for which the exchange acceptance of
// Eq. 3 is A_k = erfc(Delta_k sigma_k / 2), Delta_k = beta_k+1 - beta_k.
// Inverting the measured rates gives sigma_k = 2 erfcinv(A_k) / Delta_k;
// widths proportional to 1 / sigma_k give every pair the same acceptance,
// so the target widths are Delta*_k = W (Delta_k / x_k) / sum_j (Delta_j /
// x_j), x_k = erfcinv(A_k), W = beta_R-1 - beta_0.  The new ladder keeps both
// ends and moves each width a fraction `damping` of the way to its target.
#include <cmath>
#include <vector>

#include "../../include/xy.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

// erfc(x) = a for a in (0, 2), by Newton's method on erfc from a bracketing
// start (erfc is decreasing and convex for x > 0).
double erfc_inverse(double a) {
  if (a >= 1.0) return -erfc_inverse(2.0 - a);
  double x = std::sqrt(-std::log(a / 2.0));  // within a few percent for small a
  if (a > 0.5) x = (1.0 - a) * std::sqrt(kPi) / 2.0;  // erfc(x) ~ 1 - 2x / sqrt(pi)
  for (int it = 0; it < 100; ++it) {
    const double f = std::erfc(x) - a;
    const double df = -2.0 / std::sqrt(kPi) * std::exp(-x * x);
    const double dx = f / df;
    x -= dx;
    if (std::fabs(dx) <= 1e-16 * (1.0 + std::fabs(x))) break;
  }
  return x;
}

}  // namespace

extern "C" {

int xy_ladder_update(int R, const double* betas, const double* acceptance, double damping, double* new_betas) {
  if (R < 2 || !betas || !acceptance || !new_betas || !(damping >= 0.0 && damping <= 1.0)) return XY_ERR_ARG;
  for (int k = 0; k < R; ++k) {
    if (!std::isfinite(betas[k]) || (k > 0 && !(betas[k] > betas[k - 1]))) return XY_ERR_ARG;
  }
  for (int k = 0; k + 1 < R; ++k)
    if (!(acceptance[k] >= 0.0 && acceptance[k] <= 1.0)) return XY_ERR_ARG;
  const double W = betas[R - 1] - betas[0];
  std::vector<double> q(R - 1);
  double qs = 0.0;
  for (int k = 0; k + 1 < R; ++k) {
    // rates of 0 or 1 carry no width information beyond their bound
    const double a = std::fmin(std::fmax(acceptance[k], 1e-6), 1.0 - 1e-9);
    q[k] = (betas[k + 1] - betas[k]) / erfc_inverse(a);
    qs += q[k];
  }
  double b = betas[0];
  new_betas[0] = betas[0];
  for (int k = 0; k + 1 < R; ++k) {
    const double d = betas[k + 1] - betas[k];
    b += (1.0 - damping) * d + damping * W * q[k] / qs;
    new_betas[k + 1] = b;
  }
  new_betas[R - 1] = betas[R - 1];
  for (int k = 1; k < R; ++k)
    if (!(new_betas[k] > new_betas[k - 1])) return XY_ERR_STATE;  // cannot happen for 0 <= damping <= 1
  return XY_OK;
}

}  // extern "C"
