// FP64 folded 9-weight stencil (A y at one cell), shared by the apply kernel
// and the fused step prologue of the persistent tile kernel.
#pragma once

namespace ad {

// FP64: folded 9-weight stencil, branch-free.  Periodic: neighbour indices
// wrap.  Dirichlet: the ghosts are folded into the interior slots, so every
// out-of-domain slot has weight exactly 0; its index is clamped into the
// domain (any finite value times 0 adds nothing), which keeps all nine loads
// unconditional and independent.
__device__ __forceinline__ double stencil9(const double* __restrict__ W, long long n,
                                           const double* __restrict__ u, int i, int j, int nx,
                                           int ny, int bc, long long idx) {
  int im, ip, jm, jp;
  if (bc == 0) {
    im = i ? i - 1 : nx - 1;
    ip = (i + 1 < nx) ? i + 1 : 0;
    jm = j ? j - 1 : ny - 1;
    jp = (j + 1 < ny) ? j + 1 : 0;
  } else {
    im = i ? i - 1 : 0;
    ip = (i + 1 < nx) ? i + 1 : i;
    jm = j ? j - 1 : 0;
    jp = (j + 1 < ny) ? j + 1 : j;
  }
  const double* rm = u + (long long)jm * nx;
  const double* r0 = u + (long long)j * nx;
  const double* rp = u + (long long)jp * nx;
  double acc = W[4 * n + idx] * r0[i];
  acc = fma(W[0 * n + idx], rm[im], acc);
  acc = fma(W[1 * n + idx], rm[i], acc);
  acc = fma(W[2 * n + idx], rm[ip], acc);
  acc = fma(W[3 * n + idx], r0[im], acc);
  acc = fma(W[5 * n + idx], r0[ip], acc);
  acc = fma(W[6 * n + idx], rp[im], acc);
  acc = fma(W[7 * n + idx], rp[i], acc);
  acc = fma(W[8 * n + idx], rp[ip], acc);
  return acc;
}

}  // namespace ad
