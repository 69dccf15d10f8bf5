// Per-context precomputation (Sec. II, Sec. IV-A): the cell-integrated
// Green's function on the doubled offset lattice and its spectrum, the
// incident fields of the array elements, contrast conversions.
//
// Discretisation: pixel collocation with the Green's function integrated
// exactly over a disc (2D) or ball (3D) of the pixel's area / volume:
//   2D  Ghat(r>0) = (i pi a/(2k)) J1(ka) H0(kr),  Ghat(0) = (i pi a/(2k)) H1(ka) - 1/k^2,
//       a = h / sqrt(pi), H_n = J_n + i Y_n
//   3D  Ghat(r>0) = 4 pi (sin ka - ka cos ka)/k^3 * e^{ikr}/(4 pi r),
//       Ghat(0) = ((1 - ika) e^{ika} - 1)/k^2,  a = h (3/(4 pi))^(1/3)
// Bessel functions come from the CUDA math library (j0, j1, y0, y1).
#include <cmath>
#include <vector>

#include "bessel_c.cuh"
#include "ctx.cuh"
#include "mesh.cuh"
#include "prof.cuh"

namespace fwi {

namespace {

__device__ inline double lattice_offset(int i, int n) {
  // index i of a doubled axis of length 2n -> signed offset, NaN-free:
  // i < n -> i, i > n -> i - 2n; i == n is flagged by the caller.
  return (double)(i < n ? i : i - 2 * n);
}

__global__ void green_lattice_kernel(double2* lat, int nx, int ny, int nz, int dim,
                                     double h, double k) {
  const int lx = 2 * nx, ly = (dim == 3) ? 2 * ny : 1, lz = 2 * nz;
  const long long total = (long long)lx * ly * lz;
  const double PI = 3.141592653589793238462643383279502884;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(id % lx);
    const long long rem = id / lx;
    const int iy = (int)(rem % ly);
    const int iz = (int)(rem / ly);
    double2 out = make_double2(0.0, 0.0);
    const bool half = (ix == nx) || (iz == nz) || (dim == 3 && iy == ny);
    if (!half) {
      const double ox = lattice_offset(ix, nx) * h;
      const double oy = (dim == 3) ? lattice_offset(iy, ny) * h : 0.0;
      const double oz = lattice_offset(iz, nz) * h;
      const double r = sqrt(ox * ox + oy * oy + oz * oz);
      if (dim == 2) {
        const double a = h / sqrt(PI);
        const double ka = k * a;
        const double c = PI * a / (2.0 * k);  // Ghat = i c (...)
        if (r > 0.0) {
          const double j1a = j1(ka);
          const double kr = k * r;
          // i c J1(ka) (J0 + i Y0) = c J1(ka) (-Y0 + i J0)
          out.x = -c * j1a * y0(kr);
          out.y = c * j1a * j0(kr);
        } else {
          // i c (J1 + i Y1) - 1/k^2
          out.x = -c * y1(ka) - 1.0 / (k * k);
          out.y = c * j1(ka);
        }
      } else {
        const double a = h * cbrt(3.0 / (4.0 * PI));
        const double ka = k * a;
        if (r > 0.0) {
          const double vol = 4.0 * PI * (sin(ka) - ka * cos(ka)) / (k * k * k);
          double s, cs;
          sincos(k * r, &s, &cs);
          const double g = vol / (4.0 * PI * r);
          out.x = g * cs;
          out.y = g * s;
        } else {
          double s, cs;
          sincos(ka, &s, &cs);
          // (1 - i ka)(cs + i s) - 1 = (cs + ka s - 1) + i (s - ka cs)
          out.x = (cs + ka * s - 1.0) / (k * k);
          out.y = (s - ka * cs) / (k * k);
        }
      }
    }
    lat[id] = out;
  }
}

// Ghat of an attenuating background (complex k = kr + i ki): the closed
// forms above with complex arithmetic; 2D through the complex-argument
// Bessel / Hankel functions (bessel_c.cuh).
__global__ void green_lattice_lossy_kernel(double2* lat, int nx, int ny, int nz, int dim,
                                           double h, double kr, double ki) {
  using namespace bes;
  const int lx = 2 * nx, ly = (dim == 3) ? 2 * ny : 1, lz = 2 * nz;
  const long long total = (long long)lx * ly * lz;
  const cd k{kr, ki};
  const cd k2 = k * k;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(id % lx);
    const long long rem = id / lx;
    const int iy = (int)(rem % ly);
    const int iz = (int)(rem / ly);
    cd out{0.0, 0.0};
    const bool half = (ix == nx) || (iz == nz) || (dim == 3 && iy == ny);
    if (!half) {
      const double ox = lattice_offset(ix, nx) * h;
      const double oy = (dim == 3) ? lattice_offset(iy, ny) * h : 0.0;
      const double oz = lattice_offset(iz, nz) * h;
      const double r = sqrt(ox * ox + oy * oy + oz * oz);
      if (dim == 2) {
        const double a = h / sqrt(bes::kPi);
        const cd ka = a * k;
        const cd ic = cdiv(cd{0.0, bes::kPi * a / 2.0}, k);  // i pi a / (2k)
        if (r > 0.0) {
          out = ic * (besselj_1(ka) * hankel1_0(r * k));
        } else {
          out = ic * hankel1_1(ka) - cdiv(cd{1.0, 0.0}, k2);
        }
      } else {
        const double a = h * cbrt(3.0 / (4.0 * bes::kPi));
        const cd ka = a * k;
        const cd eika = cexp_(cd{-ka.im, ka.re});  // e^{i ka}
        const cd sn = cdiv(eika - cexp_(cd{ka.im, -ka.re}), cd{0.0, 2.0});  // sin ka
        const cd cs = 0.5 * (eika + cexp_(cd{ka.im, -ka.re}));              // cos ka
        if (r > 0.0) {
          const cd vol = cdiv((4.0 * bes::kPi) * (sn - ka * cs), k2 * k);
          const cd eikr = cexp_(cd{-r * k.im, r * k.re});
          out = (1.0 / (4.0 * bes::kPi * r)) * (vol * eikr);
        } else {
          // ((1 - i ka) e^{i ka} - 1) / k^2
          out = cdiv((cd{1.0 + ka.im, -ka.re} * eika) - cd{1.0, 0.0}, k2);
        }
      }
    }
    lat[id] = make_double2(out.re, out.im);
  }
}

template <typename T>
__global__ void scale_spectrum_c_kernel(cplx<T>* dst, const double2* src, long long n,
                                        double sr, double si) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = mk<T>((T)(v.x * sr - v.y * si), (T)(v.x * si + v.y * sr));
  }
}

// Incident fields of point elements in an attenuating background:
// 2D (i/4) H0^(1)(k r), 3D e^{ikr}/(4 pi r), complex k per frequency.
template <typename T>
__global__ void incident_lossy_kernel(cplx<T>* p0, const double* elem, const double2* kc,
                                      int n_elem, int n_freq, int nx, int ny, int nz, int dim,
                                      double h) {
  using namespace bes;
  const long long N = (long long)nx * ny * nz;
  const long long total = N * n_elem * n_freq;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const long long n = id % N;
    const long long le = id / N;
    const int e = (int)(le % n_elem);
    const int l = (int)(le / n_elem);
    const int ix = (int)(n % nx);
    const long long q = n / nx;
    const int iy = (int)(q % ny);
    const int iz = (int)(q / ny);
    const double x = (ix + 0.5 - 0.5 * nx) * h;
    const double z = iz * h;
    double dx, dy = 0.0, dz;
    if (dim == 2) {
      dx = x - elem[2 * e];
      dz = z - elem[2 * e + 1];
    } else {
      dx = x - elem[3 * e];
      dy = (iy + 0.5 - 0.5 * ny) * h - elem[3 * e + 1];
      dz = z - elem[3 * e + 2];
    }
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const cd k{kc[l].x, kc[l].y};
    cd g;
    if (dim == 2) {
      const cd hk = hankel1_0(r * k);
      g = cd{-0.25 * hk.im, 0.25 * hk.re};  // (i/4) H0
    } else {
      g = (1.0 / (4.0 * bes::kPi * r)) * cexp_(cd{-r * k.im, r * k.re});
    }
    p0[id] = mk<T>((T)g.re, (T)g.im);
  }
}

template <typename T>
__global__ void scale_spectrum_kernel(cplx<T>* dst, const double2* src, long long n,
                                      double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = mk<T>((T)(v.x * scale), (T)(v.y * scale));
  }
}

// p0_{l,e}(x_n) = G_l(x_n, x_e): 2D (i/4) H0(k r), 3D e^{ikr}/(4 pi r).
template <typename T>
__global__ void incident_kernel(cplx<T>* p0, const double* elem, const double* kw,
                                int n_elem, int n_freq, int nx, int ny, int nz,
                                int dim, double h) {
  const long long N = (long long)nx * ny * nz;
  const long long total = N * n_elem * n_freq;
  const double PI = 3.141592653589793238462643383279502884;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const long long n = id % N;
    const long long le = id / N;
    const int e = (int)(le % n_elem);
    const int l = (int)(le / n_elem);
    const int ix = (int)(n % nx);
    const long long q = n / nx;
    const int iy = (int)(q % ny);
    const int iz = (int)(q / ny);
    const double x = (ix + 0.5 - 0.5 * nx) * h;
    const double z = iz * h;
    double dx, dy = 0.0, dz;
    if (dim == 2) {
      dx = x - elem[2 * e];
      dz = z - elem[2 * e + 1];
    } else {
      const double y = (iy + 0.5 - 0.5 * ny) * h;
      dx = x - elem[3 * e];
      dy = y - elem[3 * e + 1];
      dz = z - elem[3 * e + 2];
    }
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    const double k = kw[l];
    double re, im;
    if (dim == 2) {
      re = -0.25 * y0(k * r);
      im = 0.25 * j0(k * r);
    } else {
      double s, c;
      sincos(k * r, &s, &c);
      re = c / (4.0 * PI * r);
      im = s / (4.0 * PI * r);
    }
    p0[id] = mk<T>((T)re, (T)im);
  }
}

// Gauss-Legendre rule on [-1, 1] (12 points) for the element quadrature.
struct GaussRule { double x[12], w[12]; };

// Nodes by Newton's method on P_12 (three-term recurrence), weights
// 2 / ((1 - x^2) P_12'(x)^2).
GaussRule gauss_legendre12() {
  const int n = 12;
  const double PI = 3.141592653589793238462643383279502884;
  GaussRule g;
  for (int i = 0; i < n; ++i) {
    double x = std::cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 64; ++it) {
      double p0 = 1.0, p1 = x;
      for (int j = 2; j <= n; ++j) {
        const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    g.x[i] = x;
    g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return g;
}

// Mean over a line element (length L along y, offset dy of the pixel along
// the element, distance rho from its axis) of exp(ikr) / (4 pi r).  With
// v = rho sinh t along the element, r = rho cosh t and dv / r = dt:
//   (1 / (4 pi L)) int_{t1}^{t2} exp(i k rho cosh t) dt,
// an entire integrand.  The integrand is even in t; panels end where the
// phase has advanced by 2 pi or t by 1, 12-point Gauss-Legendre on each
// (at most 4096 panels).
__device__ double2 line_mean_green(double k, double ki, double rho, double dy, double L,
                                   const GaussRule& g) {
  const double PI = 3.141592653589793238462643383279502884;
  const double a = asinh((-0.5 * L - dy) / rho), b = asinh((0.5 * L - dy) / rho);
  const double kr = k * rho, dphase = 2.0 * PI / kr;
  double re = 0.0, im = 0.0;
  auto piece = [&](double t0, double t1) {  // 0 <= t0 <= t1
    double t = t0;
    for (int p = 0; p < 4096 && t < t1; ++p) {
      double tn = acosh(cosh(t) + dphase);
      tn = fmin(fmin(tn, t + 1.0), t1);
      const double hw = 0.5 * (tn - t), mid = 0.5 * (tn + t);
      for (int q = 0; q < 12; ++q) {
        const double ch = cosh(mid + hw * g.x[q]);
        double s, c;
        sincos(kr * ch, &s, &c);
        // attenuating background (k + i ki): the factor exp(-ki rho cosh t)
        const double wq = ki > 0.0 ? g.w[q] * hw * exp(-ki * rho * ch) : g.w[q] * hw;
        re += wq * c;
        im += wq * s;
      }
      t = tn;
    }
  };
  if (a >= 0.0) {
    piece(a, b);
  } else if (b <= 0.0) {
    piece(-b, -a);
  } else {
    piece(0.0, -a);
    piece(0.0, b);
  }
  const double f = 1.0 / (4.0 * PI * L);
  return make_double2(re * f, im * f);
}

// Incident fields of 3-D line elements (finite elevation along y).
template <typename T>
__global__ void incident_line_kernel(cplx<T>* p0, const double* elem, const double* kw,
                                     const double* kwi, int n_elem, int n_freq, int nx, int ny,
                                     int nz, double h, double L, GaussRule g) {
  const long long N = (long long)nx * ny * nz;
  const long long total = N * n_elem * n_freq;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const long long n = id % N;
    const long long le = id / N;
    const int e = (int)(le % n_elem);
    const int l = (int)(le / n_elem);
    const int ix = (int)(n % nx);
    const long long q = n / nx;
    const int iy = (int)(q % ny);
    const int iz = (int)(q / ny);
    const double dx = (ix + 0.5 - 0.5 * nx) * h - elem[3 * e];
    const double dy = (iy + 0.5 - 0.5 * ny) * h - elem[3 * e + 1];
    const double dz = iz * h - elem[3 * e + 2];
    // pixels on the element's axis would make the mean singular; the array
    // sits outside the grid, so rho >= h there
    const double rho = fmax(sqrt(dx * dx + dz * dz), 1e-3 * h);
    const double2 v = line_mean_green(kw[l], kwi ? kwi[l] : 0.0, rho, dy, L, g);
    p0[id] = mk<T>((T)v.x, (T)v.y);
  }
}

template <typename T>
__global__ void convert_kernel(cplx<T>* dst, const double2* src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = mk<T>((T)src[i].x, (T)src[i].y);
}

// m = c0^2/c^2 - 1 + i alpha c0^2 / (pi c)   (Eq. 1-3, e^{-i omega t})
__global__ void contrast_kernel(double2* m, const double* sos, const double* alpha,
                                long long n, double c0, double alpha0) {
  const double PI = 3.141592653589793238462643383279502884;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double c = sos[i];
    double2 v;
    if (alpha0 > 0.0) {
      // kappa / kappa0 - 1, rho0 kappa = 1/c^2 + i a/(pi c); a pixel without
      // an attenuation value carries the background's
      const double a = alpha ? alpha[i] : alpha0;
      const double pr = 1.0 / (c * c), pi = a / (PI * c);
      const double qr = 1.0 / (c0 * c0), qi = alpha0 / (PI * c0);
      const double d = qr * qr + qi * qi;
      v.x = (pr * qr + pi * qi) / d - 1.0;
      v.y = (pi * qr - pr * qi) / d;
    } else {
      v.x = c0 * c0 / (c * c) - 1.0;
      v.y = alpha ? alpha[i] * c0 * c0 / (PI * c) : 0.0;
    }
    m[i] = v;
  }
}

// c = 1/sqrt(Re q), alpha = pi c Im q with q = rho0 kappa0 (1 + m) (the
// inverse of contrast_kernel).
__global__ void sos_alpha_kernel(const double2* m, double* sos, double* alpha, long long n,
                                 double c0, double alpha0) {
  const double PI = 3.141592653589793238462643383279502884;
  const double k0r = 1.0 / (c0 * c0), k0i = alpha0 / (PI * c0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double ar = 1.0 + m[i].x, ai = m[i].y;
    const double qr = k0r * ar - k0i * ai, qi = k0r * ai + k0i * ar;
    const double c = 1.0 / sqrt(qr);
    if (sos) sos[i] = c;
    if (alpha) alpha[i] = PI * c * qi;
  }
}

template <typename T>
cudaError_t upload_twiddles(int L, void** dst, cudaStream_t s) {
  std::vector<cplx<T>> h(L);
  for (int j = 0; j < L; ++j) {
    const double a = -2.0 * kPi * (double)j / (double)L;
    h[j] = mk<T>((T)std::cos(a), (T)std::sin(a));
  }
  cudaError_t e = cudaMallocAsync(dst, sizeof(cplx<T>) * L, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(*dst, h.data(), sizeof(cplx<T>) * L, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);  // h is released on return
}

inline int grid1d(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <typename T>
fwi_status compute_spectra(fwi_ctx* c) {
  const long long P = (long long)c->lx * c->ly * c->lz;
  double2 *lat = nullptr, *A = nullptr, *B = nullptr;
  void *tx = nullptr, *ty = nullptr, *tz = nullptr;
  fwi_status st = FWI_OK;
  cudaError_t e = cudaSuccess;
  const int cap = c->n_sm * 16;
  do {
    if ((e = cudaMallocAsync(&lat, sizeof(double2) * P, c->stream)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(&A, sizeof(double2) * P, c->stream)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(&B, sizeof(double2) * P, c->stream)) != cudaSuccess) break;
    if ((e = upload_twiddles<double>(c->lx, &tx, c->stream)) != cudaSuccess) break;
    if ((e = upload_twiddles<double>(c->lz, &tz, c->stream)) != cudaSuccess) break;
    if (c->dim == 3 && (e = upload_twiddles<double>(c->ly, &ty, c->stream)) != cudaSuccess) break;
    for (int l = 0; l < c->n_freq && e == cudaSuccess; ++l) {
      const double k = c->kwave[l];
      if (c->alpha0 > 0)
        green_lattice_lossy_kernel<<<grid1d(P, 256, cap), 256, 0, c->stream>>>(
            lat, c->nx, c->ny, c->nz, c->dim, c->h, c->kc[l].x, c->kc[l].y);
      else
        green_lattice_kernel<<<grid1d(P, 256, cap), 256, 0, c->stream>>>(
            lat, c->nx, c->ny, c->nz, c->dim, c->h, k);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      // x lines (full, unpadded input)
      RowFwdArgs<double> r{};
      r.mode = RF_PLAIN; r.full = 1; r.use_m = 0; r.in = lat; r.plane = A;
      r.tw = (const double2*)tx; r.nb = 1; r.nx = c->lx; r.rows = c->ly * c->lz;
      r.ntiles = (r.rows + Lsop<double>::row_lines_per_cta(c->lx) - 1) /
                 Lsop<double>::row_lines_per_cta(c->lx);
      r.N = P;
      if ((e = Lsop<double>::row_fwd(c->lx, r, c->stream)) != cudaSuccess) break;
      double2* res = A;
      if (c->dim == 3) {
        ColArgs<double> y{};
        y.mode = C_FWD; y.full = 1; y.in = A; y.out = B;
        y.in_rhs_stride = y.out_rhs_stride = P;
        y.in_plane_stride = y.out_plane_stride = (long long)c->ly * c->lx;
        y.line_stride = c->lx; y.ncols = c->lx; y.nplanes = c->lz;
        y.tw = (const double2*)ty; y.nb = 1; y.n_elem = 1;
        if ((e = Lsop<double>::col(c->ly, y, c->stream)) != cudaSuccess) break;
        res = B;
      }
      ColArgs<double> z{};
      z.mode = C_FWD; z.full = 1; z.in = res; z.out = (res == A) ? B : A;
      z.in_rhs_stride = z.out_rhs_stride = P;
      z.in_plane_stride = z.out_plane_stride = 0;
      z.line_stride = (long long)c->ly * c->lx; z.ncols = c->ly * c->lx; z.nplanes = 1;
      z.tw = (const double2*)tz; z.nb = 1; z.n_elem = 1;
      if ((e = Lsop<double>::col(c->lz, z, c->stream)) != cudaSuccess) break;
      if (c->alpha0 > 0) {
        // complex k^2 / P
        const double kr = c->kc[l].x, ki = c->kc[l].y;
        scale_spectrum_c_kernel<T><<<grid1d(P, 256, cap), 256, 0, c->stream>>>(
            (cplx<T>*)c->ghat + (long long)l * P, z.out, P, (kr * kr - ki * ki) / (double)P,
            2.0 * kr * ki / (double)P);
      } else {
        const double scale = k * k / (double)P;
        scale_spectrum_kernel<T><<<grid1d(P, 256, cap), 256, 0, c->stream>>>(
            (cplx<T>*)c->ghat + (long long)l * P, z.out, P, scale);
      }
      if ((e = cudaGetLastError()) != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  } while (0);
  if (e != cudaSuccess) st = cuda_fail(c, e, "Green's function spectrum");
  for (void* p : {(void*)lat, (void*)A, (void*)B, tx, ty, tz})
    if (p) cudaFreeAsync(p, c->stream);
  cudaStreamSynchronize(c->stream);
  return st;
}

template <typename T>
fwi_status setup_t(fwi_ctx* c) {
  if (!Lsop<double>::supported(c->lx) || !Lsop<double>::supported(c->lz) ||
      (c->dim == 3 && !Lsop<double>::supported(c->ly)))
    return fail(c, FWI_ERR_UNSUPPORTED, "no FFT plan for the doubled grid");
  FWI_CUDA(c, upload_twiddles<T>(c->lx, &c->tw_x, c->stream));
  FWI_CUDA(c, upload_twiddles<T>(c->lz, &c->tw_z, c->stream));
  if (c->dim == 3) FWI_CUDA(c, upload_twiddles<T>(c->ly, &c->tw_y, c->stream));
  fwi_status st = compute_spectra<T>(c);
  if (st != FWI_OK) return st;
  // incident fields
  double *elem = nullptr, *kw = nullptr;
  double2* kc = nullptr;  // complex k (lossy background)
  std::vector<double> kre(c->n_freq), kim(c->n_freq);
  for (int l = 0; l < c->n_freq; ++l) {
    kre[l] = c->alpha0 > 0 ? c->kc[l].x : c->kwave[l];
    kim[l] = c->kc[l].y;
  }
  FWI_CUDA(c, cudaMallocAsync(&elem, sizeof(double) * c->elem.size(), c->stream));
  FWI_CUDA(c, cudaMallocAsync(&kw, sizeof(double) * 2 * c->n_freq, c->stream));
  FWI_CUDA(c, cudaMallocAsync(&kc, sizeof(double2) * c->n_freq, c->stream));
  cudaError_t e = cudaMemcpyAsync(elem, c->elem.data(), sizeof(double) * c->elem.size(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(kw, kre.data(), sizeof(double) * c->n_freq, cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(kw + c->n_freq, kim.data(), sizeof(double) * c->n_freq,
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(kc, c->kc.data(), sizeof(double2) * c->n_freq, cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess) {
    const long long total = c->N * c->n_rhs;
    if (c->dim == 3 && c->elem_length > 0.0)
      incident_line_kernel<T><<<grid1d(total, 256, c->n_sm * 32), 256, 0, c->stream>>>(
          (cplx<T>*)c->p0, elem, kw, c->alpha0 > 0 ? kw + c->n_freq : nullptr, c->n_elem,
          c->n_freq, c->nx, c->ny, c->nz, c->h, c->elem_length, gauss_legendre12());
    else if (c->alpha0 > 0)
      incident_lossy_kernel<T><<<grid1d(total, 256, c->n_sm * 32), 256, 0, c->stream>>>(
          (cplx<T>*)c->p0, elem, kc, c->n_elem, c->n_freq, c->nx, c->ny, c->nz, c->dim, c->h);
    else
      incident_kernel<T><<<grid1d(total, 256, c->n_sm * 32), 256, 0, c->stream>>>(
          (cplx<T>*)c->p0, elem, kw, c->n_elem, c->n_freq, c->nx, c->ny, c->nz, c->dim, c->h);
    e = cudaGetLastError();
  }
  cudaFreeAsync(elem, c->stream);
  cudaFreeAsync(kw, c->stream);
  cudaFreeAsync(kc, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "incident fields");
  return FWI_OK;
}

template <typename T>
fwi_status set_contrast_t(fwi_ctx* c, const void* m) {
  Prof p(c, KC_MISC);
  if (c->rf > 1)
    prolong_kernel<T><<<grid1d(c->N, 256, c->n_sm * 16), 256, 0, c->stream>>>(
        (cplx<T>*)c->mF, (const double2*)m, c->nx, c->ny, c->rf, c->ry, c->N);
  else
    convert_kernel<T><<<grid1d(c->N, 256, c->n_sm * 16), 256, 0, c->stream>>>(
        (cplx<T>*)c->mF, (const double2*)m, c->N);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

}  // namespace

fwi_status setup_operator(fwi_ctx* c) {
  return c->fp64 ? setup_t<double>(c) : setup_t<float>(c);
}

fwi_status set_contrast(fwi_ctx* c, const void* m) {
  return c->fp64 ? set_contrast_t<double>(c, m) : set_contrast_t<float>(c, m);
}

fwi_status sos_attenuation_from_contrast(fwi_ctx* c, const void* m, double* sos, double* alpha) {
  Prof p(c, KC_MISC);
  sos_alpha_kernel<<<grid1d(c->Ninv, 256, c->n_sm * 16), 256, 0, c->stream>>>(
      (const double2*)m, sos, alpha, c->Ninv, c->c0, c->alpha0);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

fwi_status contrast_from_sos(fwi_ctx* c, const double* sos, const double* alpha, void* m) {
  Prof p(c, KC_MISC);
  contrast_kernel<<<grid1d(c->Ninv, 256, c->n_sm * 16), 256, 0, c->stream>>>(
      (double2*)m, sos, alpha, c->Ninv, c->c0, c->alpha0);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

}  // namespace fwi
