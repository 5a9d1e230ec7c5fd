// Largest eigenvalue modulus of a small upper Hessenberg matrix (the Arnoldi Ritz values
// used for the relaxation weight 1/rho(D^-1 A)).  Plain C++ usable on host and device.
//
// Francis double-shift QR iteration (Francis 1961; Golub & Van Loan, Matrix
// Computations, Sec. 7.5) on the active window only, deflating 1x1 and 2x2 blocks.  The
// work of each Householder reflector is split among `nlanes` cooperating threads (one
// warp on the device, a single thread on the host): every thread computes the scalars
// (shifts, reflectors, deflation tests) identically from the shared matrix, column
// updates of the left multiplication and row updates of the right multiplication are
// divided among the threads, and `sync()` separates the phases.
#pragma once
#include <math.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace clair {

struct NoSync {
  __host__ __device__ void operator()() const {}
};

template <class Sync>
__host__ __device__ double hessenberg_spectral_radius_lanes(double* H, int ld, int m, int lane,
                                                            int nlanes, Sync sync) {
#define HH(r, c) H[(r) + (long long)(c) * ld]
  double rho = 0.0;
  int hi = m - 1;
  int iter = 0;
  const double eps = 2.220446049250313e-16;
  while (hi >= 0) {
    // lowest l with a negligible subdiagonal H[l][l-1]
    int l = hi;
    while (l > 0) {
      const double s = fabs(HH(l - 1, l - 1)) + fabs(HH(l, l));
      if (fabs(HH(l, l - 1)) <= eps * (s > 0.0 ? s : 1.0)) break;
      --l;
    }
    sync();
    if (l > 0 && lane == 0) HH(l, l - 1) = 0.0;
    sync();
    if (l == hi) {  // 1x1 block
      rho = fmax(rho, fabs(HH(hi, hi)));
      --hi;
      iter = 0;
      continue;
    }
    if (l == hi - 1) {  // 2x2 block
      const double a = HH(hi - 1, hi - 1), b = HH(hi - 1, hi), c = HH(hi, hi - 1), d = HH(hi, hi);
      const double tr = 0.5 * (a + d), det = a * d - b * c;
      const double disc = tr * tr - det;
      if (disc >= 0.0) {
        const double sq = sqrt(disc);
        rho = fmax(rho, fmax(fabs(tr + sq), fabs(tr - sq)));
      } else {
        rho = fmax(rho, sqrt(fmax(det, 0.0)));  // |complex pair|^2 = det
      }
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++iter > 200) {  // no convergence: the Frobenius norm of the block bounds rho
      double f = 0.0;
      for (int r = l; r <= hi; ++r)
        for (int c = l; c <= hi; ++c) f += HH(r, c) * HH(r, c);
      rho = fmax(rho, sqrt(f));
      break;
    }
    // shifts: eigenvalues of the trailing 2x2 (an exceptional shift every 10 iterations)
    double s, t;
    if (iter % 10 == 0) {
      const double w = fabs(HH(hi, hi - 1)) + fabs(HH(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    } else {
      s = HH(hi - 1, hi - 1) + HH(hi, hi);
      t = HH(hi - 1, hi - 1) * HH(hi, hi) - HH(hi - 1, hi) * HH(hi, hi - 1);
    }
    // first column of (H - s1 I)(H - s2 I) = H^2 - s H + t I
    double x = HH(l, l) * HH(l, l) + HH(l, l + 1) * HH(l + 1, l) - s * HH(l, l) + t;
    double y = HH(l + 1, l) * (HH(l, l) + HH(l + 1, l + 1) - s);
    double z = HH(l + 1, l) * HH(l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      // reflector P = I - 2 v v^T / (v^T v) with P (x, y, z)^T = (beta, 0, 0)^T
      const double alpha = sqrt(x * x + y * y + z * z);
      const double beta = x > 0.0 ? -alpha : alpha;
      const double v0 = x - beta, v1 = y, v2 = z;
      const double vv = v0 * v0 + v1 * v1 + v2 * v2;
      sync();
      if (alpha > 0.0 && vv > 0.0) {
        const double f = 2.0 / vv;
        const int c0 = k > l ? k - 1 : l;
        for (int c = c0 + lane; c <= hi; c += nlanes) {  // rows k..k+2 (left multiply)
          const double d = f * (v0 * HH(k, c) + v1 * HH(k + 1, c) + v2 * HH(k + 2, c));
          HH(k, c) -= d * v0;
          HH(k + 1, c) -= d * v1;
          HH(k + 2, c) -= d * v2;
        }
        sync();
        const int r1 = k + 3 < hi ? k + 3 : hi;
        for (int r = l + lane; r <= r1; r += nlanes) {  // columns k..k+2 (right multiply)
          const double d = f * (v0 * HH(r, k) + v1 * HH(r, k + 1) + v2 * HH(r, k + 2));
          HH(r, k) -= d * v0;
          HH(r, k + 1) -= d * v1;
          HH(r, k + 2) -= d * v2;
        }
        sync();
      }
      x = HH(k + 1, k);
      y = HH(k + 2, k);
      if (k < hi - 2) z = HH(k + 3, k);
    }
    // final 2-element reflector on rows/columns hi-1, hi
    {
      const int k = hi - 1;
      const double alpha = sqrt(x * x + y * y);
      const double beta = x > 0.0 ? -alpha : alpha;
      const double v0 = x - beta, v1 = y;
      const double vv = v0 * v0 + v1 * v1;
      sync();
      if (alpha > 0.0 && vv > 0.0) {
        const double f = 2.0 / vv;
        for (int c = (k - 1 >= l ? k - 1 : l) + lane; c <= hi; c += nlanes) {
          const double d = f * (v0 * HH(k, c) + v1 * HH(k + 1, c));
          HH(k, c) -= d * v0;
          HH(k + 1, c) -= d * v1;
        }
        sync();
        for (int r = l + lane; r <= hi; r += nlanes) {
          const double d = f * (v0 * HH(r, k) + v1 * HH(r, k + 1));
          HH(r, k) -= d * v0;
          HH(r, k + 1) -= d * v1;
        }
      }
      sync();
    }
  }
  return rho;
#undef HH
}

// Single-thread form (host tests and any one-thread caller); works on H in place.
__host__ __device__ inline double hessenberg_spectral_radius(double* H, int ld, int m) {
  return hessenberg_spectral_radius_lanes(H, ld, m, 0, 1, NoSync{});
}

}  // namespace clair
