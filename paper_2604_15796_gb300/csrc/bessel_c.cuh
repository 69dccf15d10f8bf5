// Bessel and Hankel functions of complex argument, FP64, for the 2-D
// Green's function of an attenuating background, G = (i/4) H0^(1)(k r) with
// Im k > 0, and its cell integral (J1, H1^(1)).  Written from the classical
// expansions (Abramowitz & Stegun 9.1.10-9.1.13: ascending series of J_n and
// Y_n; 9.2.7: Hankel's asymptotic expansion) for arguments in the first
// quadrant: the series for |z| <= kSeriesMax, the asymptotic expansion
// above it (its smallest term there is below 1e-12 of the sum).  Relative
// accuracy about 1e-10 for arg z <= 0.1 (Im k up to a tenth of Re k; tissue
// attenuation gives arg k ~ 1e-3); the series' cancellation grows like
// e^{Im z} near the switch for larger arguments.  Host and device code (the
// tests compile this header on the host).
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define FWI_HD __host__ __device__ __forceinline__
#else
#define FWI_HD inline
#endif

namespace fwi {
namespace bes {

struct cd {
  double re, im;
};

FWI_HD cd mkc(double a, double b) { return cd{a, b}; }
FWI_HD cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
FWI_HD cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
FWI_HD cd operator*(cd a, cd b) {
  return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
FWI_HD cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
FWI_HD cd cdiv(cd a, cd b) {
  const double d = b.re * b.re + b.im * b.im;
  return cd{(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
FWI_HD double cabs2(cd a) { return a.re * a.re + a.im * a.im; }
FWI_HD cd cexp_(cd a) {
  const double e = exp(a.re);
  return cd{e * cos(a.im), e * sin(a.im)};
}
FWI_HD cd clog_(cd a) { return cd{0.5 * log(cabs2(a)), atan2(a.im, a.re)}; }
FWI_HD cd csqrt_(cd a) {
  const double r = sqrt(sqrt(cabs2(a)));
  const double t = 0.5 * atan2(a.im, a.re);
  return cd{r * cos(t), r * sin(t)};
}

constexpr double kSeriesMax = 14.0;
constexpr double kEulerGamma = 0.57721566490153286060651209008240243;
constexpr double kPi = 3.141592653589793238462643383279502884;

// J0, J1, Y0, Y1 by their ascending series (q = z^2 / 4):
//   J0 = sum (-q)^m / m!^2,            J1 = (z/2) sum (-q)^m / (m! (m+1)!),
//   Y0 = (2/pi)(ln(z/2) + gamma) J0 + (2/pi) sum_{m>=1} (-1)^{m+1} H_m q^m / m!^2,
//   Y1 = -2/(pi z) + (2/pi) ln(z/2) J1
//        - (1/pi)(z/2) sum (-q)^m (psi(m+1) + psi(m+2)) / (m! (m+1)!),
// with H_m the harmonic numbers and psi(m+1) = H_m - gamma.
FWI_HD void series01(cd z, cd& j0, cd& j1, cd& y0, cd& y1) {
  const cd h = 0.5 * z;
  const cd q = h * h;
  const cd mq = cd{-q.re, -q.im};
  cd t0 = cd{1.0, 0.0};     // (-q)^m / m!^2
  cd t1 = cd{1.0, 0.0};     // (-q)^m / (m! (m+1)!)
  cd sj0 = t0, sj1 = t1;
  cd sy0 = cd{0.0, 0.0};    // sum_{m>=1} (-1)^{m+1} H_m q^m / m!^2 = -sum H_m t0_m
  cd sy1 = cd{2.0 * (-kEulerGamma) + 1.0, 0.0};  // (psi(1) + psi(2)) t1_0
  double hm = 0.0;          // H_m
  for (int m = 1; m < 120; ++m) {
    t0 = (1.0 / ((double)m * m)) * (t0 * mq);
    t1 = (1.0 / ((double)m * (m + 1))) * (t1 * mq);
    hm += 1.0 / m;
    sj0 = sj0 + t0;
    sj1 = sj1 + t1;
    sy0 = sy0 - hm * t0;
    const double psi = 2.0 * (hm - kEulerGamma) + 1.0 / (m + 1);  // psi(m+1) + psi(m+2)
    sy1 = sy1 + psi * t1;
    if (cabs2(t0) < 1e-36 * cabs2(sj0) && cabs2(t1) < 1e-36 * cabs2(sj1) && m > 4) break;
  }
  j0 = sj0;
  j1 = h * sj1;
  const cd lg = clog_(h);
  y0 = (2.0 / kPi) * ((lg + cd{kEulerGamma, 0.0}) * j0 + sy0);
  y1 = (-2.0 / kPi) * cdiv(cd{1.0, 0.0}, z) + (2.0 / kPi) * (lg * j1) - (1.0 / kPi) * (h * sy1);
}

// Hankel's expansion H_nu^(1,2)(z) ~ sqrt(2/(pi z)) exp(+-i chi)
// sum_k (+-i)^k a_k(nu) / z^k, chi = z - (nu/2 + 1/4) pi,
// a_k(nu) = prod_{j=1..k} (4 nu^2 - (2j - 1)^2) / (k! 8^k); summed while the
// terms decrease.
FWI_HD cd hankel_asym(int nu, int kind, cd z) {
  const double mu = 4.0 * nu * nu;
  const cd iz = cdiv(cd{1.0, 0.0}, z);
  const double sgn = (kind == 1) ? 1.0 : -1.0;
  cd term = cd{1.0, 0.0}, sum = term;
  double prev = 1.0;
  for (int k = 1; k < 60; ++k) {
    const double f = (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k);
    term = f * (term * iz);
    term = cd{-sgn * term.im, sgn * term.re};  // times (+-i)
    const double a = cabs2(term);
    if (a > prev) break;
    sum = sum + term;
    prev = a;
    if (a < 1e-36 * cabs2(sum)) break;
  }
  const double phase0 = -(0.5 * nu + 0.25) * kPi;
  const cd chi = cd{z.re + phase0, z.im};
  const cd e = cexp_(cd{-sgn * chi.im, sgn * chi.re});  // exp(+-i chi)
  const cd pre = csqrt_(cdiv(cd{2.0 / kPi, 0.0}, z));
  return pre * (e * sum);
}

// H0^(1)(z), H1^(1)(z), J1(z) for z in the first quadrant (Im z >= 0).
FWI_HD cd hankel1_0(cd z) {
  if (cabs2(z) <= kSeriesMax * kSeriesMax) {
    cd j0, j1, y0, y1;
    series01(z, j0, j1, y0, y1);
    return cd{j0.re - y0.im, j0.im + y0.re};  // J0 + i Y0
  }
  return hankel_asym(0, 1, z);
}
FWI_HD cd hankel1_1(cd z) {
  if (cabs2(z) <= kSeriesMax * kSeriesMax) {
    cd j0, j1, y0, y1;
    series01(z, j0, j1, y0, y1);
    return cd{j1.re - y1.im, j1.im + y1.re};  // J1 + i Y1
  }
  return hankel_asym(1, 1, z);
}
FWI_HD cd besselj_1(cd z) {
  if (cabs2(z) <= kSeriesMax * kSeriesMax) {
    cd j0, j1, y0, y1;
    series01(z, j0, j1, y0, y1);
    return j1;
  }
  return 0.5 * (hankel_asym(1, 1, z) + hankel_asym(1, 2, z));
}

}  // namespace bes
}  // namespace fwi
