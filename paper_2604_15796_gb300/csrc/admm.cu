// One ADMM-TV iteration (Sec. III, Eq. 9-14, Algorithm 1 lines 4-7) after
// the forward simulation and the gradient:
//
//   b  = -grad + rho nabla^T (g + u - nabla m) + gamma (m_ref - m)
//   (J^H J + rho nabla^T nabla + gamma I) dm = b      n_cg CG iterations from 0
//   m += dm
//   g  = shrink_{lambda/rho}(nabla m - u)             isotropic, per pixel
//   u += dual_step (g - nabla m)
//   c  = c0 / sqrt(1 + Re m)                          (optional)
//
// nabla is the forward difference in index units with a zero last slice
// (Neumann); nabla^T its exact adjoint.  All ADMM vectors are complex FP64;
// CG scalars are reduced in FP64 in fixed order.
#include <cmath>

#include "ctx.cuh"
#include "prof.cuh"

namespace fwi {

namespace {

constexpr int kRedBlocks = 512;

struct Grid3 {
  int nx, ny, nz;
  long long N;
};

__device__ inline void coords(const Grid3& g, long long n, int& ix, int& iy, int& iz) {
  ix = (int)(n % g.nx);
  const long long q = n / g.nx;
  iy = (int)(q % g.ny);
  iz = (int)(q / g.ny);
}

// component q: 0 -> x (stride 1), 1 -> y (stride nx, 3D only), last -> z
__device__ inline void axis(const Grid3& g, int dim, int q, int ix, int iy, int iz,
                            long long& stride, int& i, int& n) {
  if (q == 0) { stride = 1; i = ix; n = g.nx; return; }
  if (dim == 3 && q == 1) { stride = g.nx; i = iy; n = g.ny; return; }
  stride = (long long)g.nx * g.ny; i = iz; n = g.nz;
}

__device__ inline double2 z2(double x, double y) { return make_double2(x, y); }
__device__ inline double2 operator+(double2 a, double2 b) { return z2(a.x + b.x, a.y + b.y); }
__device__ inline double2 operator-(double2 a, double2 b) { return z2(a.x - b.x, a.y - b.y); }
__device__ inline double2 operator*(double s, double2 a) { return z2(s * a.x, s * a.y); }

__device__ inline void block_reduce_store(double v, double* part) {
  __shared__ double sh[256];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// w_q = g_q + u_q - (nabla m)_q
__global__ void w_kernel(double2* w, const double2* g, const double2* u, const double2* m,
                         Grid3 G, int dim) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.N;
       n += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(G, n, ix, iy, iz);
    for (int q = 0; q < dim; ++q) {
      long long s; int i, nq;
      axis(G, dim, q, ix, iy, iz, s, i, nq);
      const double2 gm = (i < nq - 1) ? m[n + s] - m[n] : z2(0.0, 0.0);
      w[q * G.N + n] = g[q * G.N + n] + u[q * G.N + n] - gm;
    }
  }
}

// (nabla^T a)_n = sum_q [a_q(n - e_q) if i_q >= 1] - [a_q(n) if i_q <= n_q - 2]
__device__ inline double2 gradT_at(const double2* a, const Grid3& G, int dim, long long n) {
  int ix, iy, iz;
  coords(G, n, ix, iy, iz);
  double2 out = z2(0.0, 0.0);
  for (int q = 0; q < dim; ++q) {
    long long s; int i, nq;
    axis(G, dim, q, ix, iy, iz, s, i, nq);
    if (i >= 1) out = out + a[q * G.N + n - s];
    if (i <= nq - 2) out = out - a[q * G.N + n];
  }
  return out;
}

// b = -grad + rho nabla^T w + gamma (m_ref - m); x = 0; r = d = b; partial |b|^2
__global__ void rhs_kernel(double2* b, double2* x, double2* r, double2* d, const double2* grad,
                           const double2* w, const double2* m, const double2* mref, double rho,
                           double gamma, Grid3 G, int dim, double* part) {
  double acc = 0.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.N;
       n += (long long)gridDim.x * blockDim.x) {
    const double2 mr = mref ? mref[n] : z2(0.0, 0.0);
    const double2 v = (rho * gradT_at(w, G, dim, n)) - grad[n] + gamma * (mr - m[n]);
    b[n] = v;
    x[n] = z2(0.0, 0.0);
    r[n] = v;
    d[n] = v;
    acc += v.x * v.x + v.y * v.y;
  }
  block_reduce_store(acc, part);
}

// q = z + rho nabla^T nabla d + gamma d ; partial Re<d, q>
__global__ void q_kernel(double2* q, const double2* z, const double2* d, double rho, double gamma,
                         Grid3 G, int dim, double* part) {
  double acc = 0.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.N;
       n += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(G, n, ix, iy, iz);
    const double2 dn = d[n];
    double2 lap = z2(0.0, 0.0);
    for (int k = 0; k < dim; ++k) {
      long long s; int i, nq;
      axis(G, dim, k, ix, iy, iz, s, i, nq);
      if (i >= 1) lap = lap + (dn - d[n - s]);
      if (i <= nq - 2) lap = lap + (dn - d[n + s]);
    }
    const double2 v = z[n] + rho * lap + gamma * dn;
    q[n] = v;
    acc += dn.x * v.x + dn.y * v.y;
  }
  block_reduce_store(acc, part);
}

// Fixed-order block sum of np partials (one block of 256 threads).
__device__ inline double block_total(const double* part, int np) {
  __shared__ double sh[256];
  double t = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) t += part[i];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  return sh[0];
}

// scalars: s[0] = rr, s[1] = alpha, s[2] = beta, s[3] = flag (1: stop)
__global__ void cg_init_scalar(double* s, const double* part, int np) {
  const double t = block_total(part, np);
  if (threadIdx.x == 0) {
    s[0] = t;
    s[3] = (t == 0.0) ? 1.0 : 0.0;
  }
}
__global__ void cg_alpha_scalar(double* s, const double* part, int np) {
  const double t = block_total(part, np);
  if (threadIdx.x == 0) s[1] = (s[3] == 0.0 && t != 0.0) ? s[0] / t : 0.0;
}
__global__ void cg_beta_scalar(double* s, const double* part, int np) {
  const double t = block_total(part, np);
  if (threadIdx.x != 0) return;
  if (s[3] != 0.0 || s[0] == 0.0) {
    s[2] = 0.0;
    s[3] = 1.0;
    return;
  }
  s[2] = t / s[0];
  s[0] = t;
  if (t == 0.0) s[3] = 1.0;
}

// x += alpha d; r -= alpha q; partial |r|^2
__global__ void xr_kernel(double2* x, double2* r, const double2* d, const double2* q,
                          const double* s, long long N, double* part) {
  const double a = s[1];
  double acc = 0.0;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    x[n] = x[n] + a * d[n];
    const double2 rn = r[n] - a * q[n];
    r[n] = rn;
    acc += rn.x * rn.x + rn.y * rn.y;
  }
  block_reduce_store(acc, part);
}

// d = r + beta d
__global__ void d_kernel(double2* d, const double2* r, const double* s, long long N) {
  const double b = s[2];
  if (s[3] != 0.0) return;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x)
    d[n] = r[n] + b * d[n];
}

__global__ void add_kernel(double2* m, const double2* dm, long long N) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x)
    m[n] = m[n] + dm[n];
}

// g = shrink_tau(nabla m - u); u += step (g - nabla m); sos = c0/sqrt(1+Re m)
__global__ void shrink_dual_kernel(double2* g, double2* u, const double2* m, double* sos,
                                   double tau, double step, double c0, double alpha0, Grid3 G,
                                   int dim) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.N;
       n += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(G, n, ix, iy, iz);
    double2 gm[3], a[3];
    double nrm2 = 0.0;
    for (int q = 0; q < dim; ++q) {
      long long s; int i, nq;
      axis(G, dim, q, ix, iy, iz, s, i, nq);
      gm[q] = (i < nq - 1) ? m[n + s] - m[n] : z2(0.0, 0.0);
      a[q] = gm[q] - u[q * G.N + n];
      nrm2 += a[q].x * a[q].x + a[q].y * a[q].y;
    }
    const double nrm = sqrt(nrm2);
    double sc = 0.0;
    if (nrm > 0.0) {
      sc = 1.0 - tau / nrm;
      if (sc < 0.0) sc = 0.0;
    }
    for (int q = 0; q < dim; ++q) {
      const double2 gq = sc * a[q];
      g[q * G.N + n] = gq;
      u[q * G.N + n] = u[q * G.N + n] + step * (gq - gm[q]);
    }
    if (sos) {
      if (alpha0 > 0.0) {
        // 1/c^2 = Re(rho0 kappa0 (1 + m)), rho0 kappa0 = 1/c0^2 + i alpha0/(pi c0)
        const double qr = 1.0 / (c0 * c0), qi = alpha0 / (3.141592653589793238462643383279502884 * c0);
        sos[n] = 1.0 / sqrt(qr * (1.0 + m[n].x) - qi * m[n].y);
      } else {
        sos[n] = c0 / sqrt(1.0 + m[n].x);
      }
    }
  }
}

// g_q = (nabla m)_q ; u_q = 0
__global__ void admm_init_kernel(double2* g, double2* u, const double2* m, Grid3 G, int dim) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < G.N;
       n += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    coords(G, n, ix, iy, iz);
    for (int q = 0; q < dim; ++q) {
      long long s; int i, nq;
      axis(G, dim, q, ix, iy, iz, s, i, nq);
      g[q * G.N + n] = (i < nq - 1) ? m[n + s] - m[n] : z2(0.0, 0.0);
      u[q * G.N + n] = z2(0.0, 0.0);
    }
  }
}

inline int blocks_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

fwi_status admm_init(fwi_ctx* c, const void* m0, void* g, void* u) {
  Grid3 G{c->inx, c->iny, c->inz, c->Ninv};  // inversion mesh
  Prof pf(c, KC_ADMM);
  admm_init_kernel<<<blocks_for(c->Ninv, 256, kRedBlocks), 256, 0, c->stream>>>(
      (double2*)g, (double2*)u, (const double2*)m0, G, c->dim);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

fwi_status admm_step(fwi_ctx* c, void* mv, void* gv, void* uv, const void* gradv,
                     const fwi_admm_params* p, double* sos) {
  if (!c->fields_valid)
    return fail(c, FWI_ERR_INVALID_ARG, "no forward fields: call fwi_forward or fwi_gradient first");
  double2* m = (double2*)mv;
  double2* g = (double2*)gv;
  double2* u = (double2*)uv;
  const double2* grad = (const double2*)gradv;
  Grid3 G{c->inx, c->iny, c->inz, c->Ninv};  // inversion mesh
  const int dim = c->dim;
  const int nb = kRedBlocks;
  double* part = c->red + c->n_freq + 256;
  double* sc = part + kRedBlocks;
  double2* b = c->vN[0];
  double2* x = c->vN[1];
  double2* r = c->vN[2];
  double2* d = c->vN[3];
  double2* q = c->vN[4];
  double2* z = c->vN[5];
  double2* w = c->vD[0];
  cudaStream_t s = c->stream;
  const double rho = p->rho, gamma = p->gamma;
  {
    Prof pf(c, KC_ADMM);
    w_kernel<<<blocks_for(c->Ninv, 256, nb), 256, 0, s>>>(w, g, u, m, G, dim);
  }
  FWI_CUDA(c, cudaGetLastError());
  {
    Prof pf(c, KC_ADMM);
    rhs_kernel<<<nb, 256, 0, s>>>(b, x, r, d, grad, w, m, (const double2*)p->m_ref, rho, gamma,
                                  G, dim, part);
  }
  FWI_CUDA(c, cudaGetLastError());
  {
    Prof pf(c, KC_ADMM);
    cg_init_scalar<<<1, 256, 0, s>>>(sc, part, nb);
  }
  FWI_CUDA(c, cudaGetLastError());
  for (int it = 0; it < p->n_cg; ++it) {
    fwi_status st = jac_forward(c, d, c->dres);
    if (st != FWI_OK) return st;
    const double2* y = c->dres;
    if (c->n_tx > 0) {
      // plane-wave transmits: J^H J = J_point^H (W^H W) J_point
      st = synth(c, c->WhW, 0, c->n_elem, c->n_elem, c->dres, c->dsyn, nullptr);
      if (st != FWI_OK) return st;
      y = c->dsyn;
    }
    st = jac_adjoint(c, y, z);
    if (st != FWI_OK) return st;
    // frequency sharding: J^H J d summed over every rank's frequencies
    st = reduce_sum(c, z, 2 * (size_t)c->Ninv);
    if (st != FWI_OK) return st;
    {
      Prof pf(c, KC_ADMM);
      q_kernel<<<nb, 256, 0, s>>>(q, z, d, rho, gamma, G, dim, part);
    }
    FWI_CUDA(c, cudaGetLastError());
    {
      Prof pf(c, KC_ADMM);
      cg_alpha_scalar<<<1, 256, 0, s>>>(sc, part, nb);
    }
    {
      Prof pf(c, KC_ADMM);
      xr_kernel<<<nb, 256, 0, s>>>(x, r, d, q, sc, c->Ninv, part);
    }
    {
      Prof pf(c, KC_ADMM);
      cg_beta_scalar<<<1, 256, 0, s>>>(sc, part, nb);
    }
    {
      Prof pf(c, KC_ADMM);
      d_kernel<<<nb, 256, 0, s>>>(d, r, sc, c->Ninv);
    }
    FWI_CUDA(c, cudaGetLastError());
  }
  {
    Prof pf(c, KC_ADMM);
    add_kernel<<<blocks_for(c->Ninv, 256, nb), 256, 0, s>>>(m, x, c->Ninv);
  }
  const double tau = p->lambda / p->rho;
  const double step = p->dual_step > 0.0 ? p->dual_step : p->rho;
  {
    Prof pf(c, KC_ADMM);
    shrink_dual_kernel<<<blocks_for(c->Ninv, 256, nb), 256, 0, s>>>(g, u, m, sos, tau, step, c->c0,
                                                                  c->alpha0,
                                                               G, dim);
  }
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

}  // namespace fwi
