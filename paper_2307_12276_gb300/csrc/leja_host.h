#pragma once
#include <vector>

namespace ad {

constexpr int kLejaPoints = 502;   // enough for kMaxIters + 1 terms

// The Leja sequence on [-2, 2] (computed once per process, thread-safe).
const std::vector<double>& leja_points();
// Newton divided differences d_m = f[x_0, ..., x_m], m < n.
void divided_differences(const double* x, const double* f, int n, double* d);
// phi_1(z) = (e^z - 1)/z, phi_1(0) = 1.
double phi1(double z);

}  // namespace ad
