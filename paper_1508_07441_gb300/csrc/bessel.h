// exp(-z) i_l(z), the scaled modified spherical Bessel functions of the
// Gaussian-term pair potential in the free-packet basis (Sec. 2.2 Eq. vpot),
// for the host (setup.cpp) and the device (pair.cu) alike.
//
// Small z: leading power-series terms.  Moderate z: Miller's downward
// recurrence i_{n-1} = i_{n+1} + (2n+1)/z i_n (stable: i_n is the minimal
// solution) normalised by exp(-z) i_0 = (1 - exp(-2z)) / (2z).  Large z: the
// terminating expansion of i_l in powers of 1/(2z).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define WPCD_HD __host__ __device__
#else
#define WPCD_HD
#endif

namespace wpcd {

constexpr int kBesselLmax = 4;  // channels l = 0 .. 4

WPCD_HD inline double bessel_i_scaled(int l, double z) {
  if (z == 0.0) return l == 0 ? 1.0 : 0.0;
  if (z < 1e-3) {
    double df = 1.0;
    for (int m = 3; m <= 2 * l + 1; m += 2) df *= m;
    const double lead = pow(z, (double)l) / df;
    return lead * (1.0 + z * z / (2.0 * (2 * l + 3))) * exp(-z);
  }
  if (z > 40.0) {
    const double inv = 1.0 / (2.0 * z);
    double term = 1.0, s_alt = 0.0, s_pos = 0.0;
    for (int k = 0; k <= l; ++k) {
      if (k > 0) term *= (double)(l + k) * (l - k + 1) / k * inv;  // (l+k)!/(k!(l-k)!) (2z)^-k
      s_alt += (k % 2 ? -term : term);
      s_pos += term;
    }
    const double tail = ((l + 1) % 2 ? -1.0 : 1.0) * exp(-2.0 * z) * s_pos;
    return (s_alt + tail) / (2.0 * z);
  }
  const int top = l + 30 + (int)(2.0 * z);
  double up = 0.0, cur = 1e-300, want = 0.0;
  for (int n = top; n >= 1; --n) {
    const double down = up + (2.0 * n + 1.0) / z * cur;  // i_{n-1}
    up = cur;
    cur = down;
    if (n - 1 == l) want = cur;
    if (fabs(cur) > 1e250) {  // rescale to stay in range
      cur *= 1e-250;
      up *= 1e-250;
      want *= 1e-250;
    }
  }
  // cur = i_0 (unnormalised)
  const double i0s = -expm1(-2.0 * z) / (2.0 * z);
  return want / cur * i0s;
}

// l = 0 .. lmax at once (out[lmax + 1], lmax <= kBesselLmax): the same three
// regimes; in the middle one a single downward recurrence (started above
// lmax) yields every order
WPCD_HD inline void bessel_i_scaled_all(int lmax, double z, double *out) {
  if (z == 0.0 || z < 1e-3 || z > 40.0) {
    for (int l = 0; l <= lmax; ++l) out[l] = bessel_i_scaled(l, z);
    return;
  }
  for (int l = 0; l <= lmax; ++l) out[l] = 0.0;
  const int top = lmax + 30 + (int)(2.0 * z);
  const double inv_z = 1.0 / z;
  double up = 0.0, cur = 1e-300;
  for (int n = top; n >= 1; --n) {
    const double down = up + (2.0 * n + 1.0) * inv_z * cur;  // i_{n-1}
    up = cur;
    cur = down;
    if (n - 1 <= lmax) out[n - 1] = cur;
    if (fabs(cur) > 1e250) {  // rescale to stay in range
      cur *= 1e-250;
      up *= 1e-250;
      for (int l = 0; l <= lmax; ++l) out[l] *= 1e-250;
    }
  }
  // cur = i_0 (unnormalised)
  const double scale = -expm1(-2.0 * z) / (2.0 * z) / cur;
  for (int l = 0; l <= lmax; ++l) out[l] *= scale;
}

}  // namespace wpcd
