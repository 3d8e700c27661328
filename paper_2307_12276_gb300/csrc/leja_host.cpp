// Host-side scalar work of the Leja method (Section 2): the Leja sequence on
// [-2, 2] and Newton divided differences of the interpolated scalar function.
// O(M^2) scalars per series configuration; the matrix work runs on the GPU.
#include "leja_host.h"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

namespace ad {

// Leja points: xi_0 = 2 (so z = c + 2 gamma = 0 is a node), then each new
// point maximises prod_j |xi - xi_j| over [-2, 2].  Inside a gap (a, b)
// between neighbouring points the maximiser is the zero of
//   q(xi) = (xi - a) + (xi - b) + (xi - a)(xi - b) * sum_{other j} 1/(xi - xi_j),
// which rises from a - b < 0 to b - a > 0; bracketed Newton finds it to
// working precision.  Ties (relative 1e-12 in the log-product) go to the
// larger point.
static std::vector<double> compute_leja(int n) {
  std::vector<double> pts;
  pts.reserve(n);
  pts.push_back(2.0);
  if (n > 1) pts.push_back(-2.0);
  std::vector<double> sorted;
  while ((int)pts.size() < n) {
    sorted = pts;
    std::sort(sorted.begin(), sorted.end());
    const int k = (int)pts.size();
    const int ngaps = (int)sorted.size() - 1;
    std::vector<double> gx(ngaps), gv(ngaps);
    for (int gi = 0; gi < ngaps; ++gi) {
      const double a = sorted[gi], b = sorted[gi + 1];
      double lo = a, hi = b, x = 0.5 * (a + b);
      for (int it = 0; it < 200; ++it) {
        double R = 0.0, Rp = 0.0;
        for (int j = 0; j < k; ++j) {
          const double pj = pts[j];
          if (pj == a || pj == b) continue;
          const double inv = 1.0 / (x - pj);
          R += inv;
          Rp -= inv * inv;
        }
        const double q = (x - a) + (x - b) + (x - a) * (x - b) * R;
        const double qp = 2.0 + (2.0 * x - a - b) * R + (x - a) * (x - b) * Rp;
        const double step = q / qp;
        if (std::fabs(step) <= 2e-16 * std::max(1.0, std::fabs(x))) break;
        if (q < 0) lo = x; else hi = x;
        double xn = x - step;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        x = xn;
      }
      double v = 0.0;
      for (int j = 0; j < k; ++j) v += std::log(std::fabs(x - pts[j]));
      gx[gi] = x;
      gv[gi] = v;
    }
    const double best = *std::max_element(gv.begin(), gv.end());
    const double thr = best - 1e-12 * std::max(1.0, std::fabs(best));
    double best_x = -INFINITY;
    for (int gi = 0; gi < ngaps; ++gi)
      if (gv[gi] >= thr && gx[gi] > best_x) best_x = gx[gi];
    pts.push_back(best_x);
  }
  return pts;
}

const std::vector<double>& leja_points() {
  static std::vector<double> pts;
  static std::once_flag once;
  std::call_once(once, [] { pts = compute_leja(kLejaPoints); });
  return pts;
}

void divided_differences(const double* x, const double* f, int n, double* d) {
  for (int i = 0; i < n; ++i) d[i] = f[i];
  for (int j = 1; j < n; ++j)
    for (int i = n - 1; i >= j; --i) d[i] = (d[i] - d[i - 1]) / (x[i] - x[i - j]);
}

double phi1(double z) {
  if (std::fabs(z) < 1e-8) return 1.0 + z * (0.5 + z / 6.0);
  return std::expm1(z) / z;
}

}  // namespace ad
