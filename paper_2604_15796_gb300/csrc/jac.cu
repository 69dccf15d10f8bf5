// Pixel contractions of the data equation, the adjoint state and the
// implicit Jacobian (Eq. 4, 15-17; Sec. IV-B, IV-C).  With receivers at the
// transmit positions the receiver rows are R_{l,j} = k_l^2 dV p0_{l,j} and
// the receiver fields ptilde_{l,j} = k_l^2 dV p_{l,j}, so every product is
// one of two complex contractions over the field arrays [l][e][N]:
//
//  contract : Y_l[e][j] = s_l sum_n X_l[e][n] a[n] Q_l[j][n]
//             (data: X = p, a = m, Q = p0; J a: X = Q = p)
//  mix      : W_l[e][n] = s_l sum_j B_l[e][j] Q'_l[j][n]   (Q' = Q or conj Q)
//             materialised (adjoint sources conj(s_e) = sum_j R_j conj(r_ej))
//             or fused with z[n] += sum_e conj(X_l[e][n]) W_l[e][n]  (J^H b)
//
// With FP32 fields the contraction and the fused J^H run on the tensor
// cores (jac_tc.cu); the kernels here are the FP64 path, the materialised
// mix, and the fallback for odd pixel counts: register-tiled CUDA-core
// kernels (64 x 64 complex output tiles, 4 x 4 per thread, operands staged
// through shared memory).  Partial sums across pixel chunks / transmit
// blocks are combined in FP64 in fixed order.
#include <cmath>
#include <type_traits>
#include <vector>

#include "ctx.cuh"
#include "mesh.cuh"
#include "prof.cuh"

namespace fwi {

namespace {

constexpr int TB = 64;   // output tile edge (complex)
constexpr int KC = 16;   // contraction chunk

inline int blocks_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// Tile (eb, jb) of grid index ty: all nbe^2 tiles, or (sym) only eb <= jb
// enumerated column by column.
__device__ inline void tile_of(int ty, int nbe, int sym, int& eb, int& jb) {
  if (!sym) {
    eb = ty % nbe;
    jb = ty / nbe;
    return;
  }
  jb = 0;
  while ((jb + 1) * (jb + 2) / 2 <= ty) ++jb;
  eb = ty - jb * (jb + 1) / 2;
}

template <typename T>
__global__ void __launch_bounds__(256)
contract_kernel(const cplx<T>* __restrict__ X, const cplx<T>* __restrict__ a,
                const cplx<T>* __restrict__ Q, cplx<T>* __restrict__ part, int NE,
                long long N, int n_freq, long long chunk, int sym) {
  using V = cplx<T>;
  __shared__ V Xs[KC][TB + 1];
  __shared__ V Qs[KC][TB + 1];
  const int s = blockIdx.x;
  const int nbe = (NE + TB - 1) / TB;
  int eb, jb;
  tile_of(blockIdx.y, nbe, sym, eb, jb);
  const int l = blockIdx.z;
  const int tid = threadIdx.x;
  const int te = tid & 15, tj = tid >> 4;
  const long long n_begin = (long long)s * chunk;
  long long n_end = n_begin + chunk;
  if (n_end > N) n_end = N;
  const V* Xl = X + (long long)l * NE * N;
  const V* Ql = Q + (long long)l * NE * N;
  V acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<T>(T(0), T(0));
  for (long long n0 = n_begin; n0 < n_end; n0 += KC) {
#pragma unroll
    for (int q = 0; q < (TB * KC) / 256; ++q) {
      const int idx = tid + q * 256;
      const int r = idx / KC, cc = idx % KC;
      const long long n = n0 + cc;
      const int e = eb * TB + r, j = jb * TB + r;
      V xv = mk<T>(T(0), T(0)), qv = mk<T>(T(0), T(0));
      if (n < n_end) {
        if (e < NE) {
          xv = Xl[(long long)e * N + n];
          if (a) xv = cmul(xv, a[n]);
        }
        if (j < NE) qv = Ql[(long long)j * N + n];
      }
      Xs[cc][r] = xv;
      Qs[cc][r] = qv;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      V xv[4], qv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = Xs[kk][te + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) qv[j] = Qs[kk][tj + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x += xv[i].x * qv[j].x - xv[i].y * qv[j].y;
          acc[i][j].y += xv[i].x * qv[j].y + xv[i].y * qv[j].x;
        }
    }
    __syncthreads();
  }
  V* out = part + ((long long)s * n_freq + l) * NE * NE;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = eb * TB + te + 16 * i, jj = jb * TB + tj + 16 * j;
      if (e < NE && jj < NE) out[(long long)e * NE + jj] = acc[i][j];
    }
}

// Y[l][e][j] = scale_l * sum_s part[s][l][e][j]  (FP64, fixed order); with
// sym, entries below the computed tiles (eb > jb) are read transposed.
template <typename T>
__global__ void contract_reduce_kernel(double2* Y, const cplx<T>* part, int split,
                                       long long per_split, int NE2, const double* scale,
                                       int NE, int sym) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per_split;
       i += (long long)gridDim.x * blockDim.x) {
    long long src = i;
    if (sym) {
      const long long l = i / NE2;
      const int e = (int)((i % NE2) / NE), j = (int)(i % NE);
      if (e / TB > j / TB) src = l * NE2 + (long long)j * NE + e;
    }
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < split; ++s) {
      const cplx<T> v = part[(long long)s * per_split + src];
      sx += (double)v.x;
      sy += (double)v.y;
    }
    const double f = scale[i / NE2];
    Y[i] = make_double2(sx * f, sy * f);
  }
}

template <typename T, bool FUSED>
__global__ void __launch_bounds__(256)
mix_kernel(const cplx<T>* __restrict__ B, const cplx<T>* __restrict__ Q, int conjQ,
           const cplx<T>* __restrict__ X, cplx<T>* __restrict__ out,
           const double* __restrict__ scale, int NE, long long N) {
  using V = cplx<T>;
  __shared__ V Bs[KC][TB + 1];
  __shared__ V Qs[KC][TB + 1];
  __shared__ V red[16][TB + 1];
  const int nbn = blockIdx.x, eb = blockIdx.y, l = blockIdx.z;
  const int nbe = gridDim.y;
  const int tid = threadIdx.x;
  const int tn = tid & 15, te = tid >> 4;
  const long long n0 = (long long)nbn * TB;
  const V* Bl = B + (long long)l * NE * NE;
  const V* Ql = Q + (long long)l * NE * N;
  V acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mk<T>(T(0), T(0));
  for (int j0 = 0; j0 < NE; j0 += KC) {
#pragma unroll
    for (int q = 0; q < (TB * KC) / 256; ++q) {
      const int idx = tid + q * 256;
      // B tile: row e (TB of them), KC consecutive j
      {
        const int r = idx / KC, cc = idx % KC;
        const int e = eb * TB + r, j = j0 + cc;
        Bs[cc][r] = (e < NE && j < NE) ? Bl[(long long)e * NE + j] : mk<T>(T(0), T(0));
      }
      // Q tile: row j (KC of them), TB consecutive n
      {
        const int kk = idx / TB, nn = idx % TB;
        const int j = j0 + kk;
        const long long n = n0 + nn;
        V v = mk<T>(T(0), T(0));
        if (j < NE && n < N) {
          v = Ql[(long long)j * N + n];
          if (conjQ) v.y = -v.y;
        }
        Qs[kk][nn] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      V bv[4], qv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) bv[i] = Bs[kk][te + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) qv[j] = Qs[kk][tn + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x += bv[i].x * qv[j].x - bv[i].y * qv[j].y;
          acc[i][j].y += bv[i].x * qv[j].y + bv[i].y * qv[j].x;
        }
    }
    __syncthreads();
  }
  const T f = (T)scale[l];
  if (!FUSED) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = eb * TB + te + 16 * i;
        const long long n = n0 + tn + 16 * j;
        if (e < NE && n < N)
          out[((long long)l * NE + e) * N + n] = mk<T>(acc[i][j].x * f, acc[i][j].y * f);
      }
    return;
  }
  // fused J^H: sum_e conj(X[e][n]) W[e][n]
  const V* Xl = X + (long long)l * NE * N;
  V zs[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    zs[j] = mk<T>(T(0), T(0));
    const long long n = n0 + tn + 16 * j;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = eb * TB + te + 16 * i;
      if (e < NE && n < N) {
        const V x = Xl[(long long)e * N + n];
        zs[j] = cadd(zs[j], cmulc(acc[i][j], x));  // W * conj(X)
      }
    }
    red[te][tn + 16 * j] = zs[j];
  }
  __syncthreads();
  if (tid < TB) {
    V s = mk<T>(T(0), T(0));
#pragma unroll
    for (int r = 0; r < 16; ++r) s = cadd(s, red[r][tid]);
    const long long n = n0 + tid;
    if (n < N) out[((long long)l * nbe + eb) * N + n] = mk<T>(s.x * f, s.y * f);
  }
}

// z[n] = sum_{p < np} part[p][n]  (FP64, fixed order)
template <typename T>
__global__ void sum_parts_kernel(double2* z, const cplx<T>* part, int np, long long N,
                                 int conj_out) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int p = 0; p < np; ++p) {
      const cplx<T> v = part[(long long)p * N + n];
      sx += (double)v.x;
      sy += (double)v.y;
    }
    z[n] = make_double2(sx, conj_out ? -sy : sy);
  }
}

// Per-pixel sum over (l, e) of p * y in chunks: part[s][n] (FP64).
template <typename T>
__global__ void grad_partial_kernel(double2* part, const cplx<T>* P, const cplx<T>* Y,
                                    int nle, int per, long long N) {
  const int s = blockIdx.y;
  const int le0 = s * per;
  int le1 = le0 + per;
  if (le1 > nle) le1 = nle;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0;
    int le = le0;
    while (le < le1) {
      T ax = 0, ay = 0;
      const int stop = (le + 16 < le1) ? le + 16 : le1;
#pragma unroll 4
      for (; le < stop; ++le) {
        const cplx<T> p = P[(long long)le * N + n];
        const cplx<T> y = Y[(long long)le * N + n];
        ax += p.x * y.x - p.y * y.y;
        ay += p.x * y.y + p.y * y.x;
      }
      sx += (double)ax;
      sy += (double)ay;
    }
    part[(long long)s * N + n] = make_double2(sx, sy);
  }
}

// grad[n] = conj(sum_s part[s][n])
__global__ void grad_reduce_kernel(double2* g, const double2* part, int ns, long long N) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < ns; ++s) {
      sx += part[(long long)s * N + n].x;
      sy += part[(long long)s * N + n].y;
    }
    g[n] = make_double2(sx, -sy);
  }
}

// r = d - d_obs (FP64); conj(r) in field precision for the adjoint sources;
// block partials of |r|^2.
template <typename T>
__global__ void residual_kernel(double2* r, cplx<T>* rconjF, const double2* d,
                                const cplx<T>* d_obs, long long n, double* part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const cplx<T> o = d_obs[i];
    const double2 v = make_double2(d[i].x - (double)o.x, d[i].y - (double)o.y);
    r[i] = v;
    rconjF[i] = mk<T>((T)v.x, (T)(-v.y));
    acc += v.x * v.x + v.y * v.y;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <typename T>
__global__ void to_field_kernel(cplx<T>* dst, const double2* src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = mk<T>((T)src[i].x, (T)src[i].y);
}

// ---------------------------------------------------------------------------
template <typename T> struct Jac {
  static std::vector<double> scales(fwi_ctx* c) {
    std::vector<double> s(c->n_freq);
    const double dv = std::pow(c->h, c->dim);
    for (int l = 0; l < c->n_freq; ++l) s[l] = c->kwave[l] * c->kwave[l] * dv;
    return s;
  }

  static int split_for(fwi_ctx* c) {
    const int nbe = (c->n_elem + TB - 1) / TB;
    const int tiles = nbe * nbe * c->n_freq;
    int split = (c->n_sm * 6 + tiles - 1) / tiles;
    const long long max_split = (c->N + KC - 1) / KC;
    if (split > max_split) split = (int)max_split;
    if (split < 1) split = 1;
    if (split > c->jsplit_n) split = c->jsplit_n;
    return split;
  }

  // Y = scale_l * contract(X, a, Q) (c128, [l][e][j]); sym when Q == X
  // (then Y_l is complex-symmetric and only tiles eb <= jb are computed).
  // FP32 fields: tensor cores (jac_tc.cu), whose TMEM accumulation runs
  // over sub-chunks of at most 512 pixels so that it stays within a few
  // 1e-6 of FMA accumulation.
  static fwi_status contract(fwi_ctx* c, const cplx<T>* X, const cplx<T>* a,
                             const cplx<T>* Q, double2* Y) {
    const long long per = (long long)c->n_freq * c->n_elem * c->n_elem;
    if constexpr (std::is_same<T, float>::value) {
      if (tc_usable(c)) {
        const int split = tc_contract_partials(c, X, a, Q, (float2*)c->jsplit);
        if (split < 0) return FWI_ERR_CUDA;
        Prof p(c, KC_MISC);
        contract_reduce_kernel<T><<<blocks_for(per, 256, c->n_sm * 8), 256, 0, c->stream>>>(
            Y, (const cplx<T>*)c->jsplit, split, per, c->n_elem * c->n_elem, c->red, c->n_elem,
            0);
        FWI_CUDA(c, cudaGetLastError());
        return FWI_OK;
      }
    }
    const int nbe = (c->n_elem + TB - 1) / TB;
    const int split = split_for(c);
    const int sym = (X == Q) ? 1 : 0;
    long long chunk = (c->N + split - 1) / split;
    chunk = ((chunk + KC - 1) / KC) * KC;
    dim3 grid(split, sym ? nbe * (nbe + 1) / 2 : nbe * nbe, c->n_freq);
    const double fe = (double)c->n_freq * c->n_elem * c->N;
    {
      Prof p(c, KC_CONTRACT, (2.0 * fe + (a ? c->N : 0)) * sizeof(cplx<T>),
             8.0 * fe * c->n_elem);
      contract_kernel<T><<<grid, 256, 0, c->stream>>>(X, a, Q, (cplx<T>*)c->jsplit, c->n_elem,
                                                      c->N, c->n_freq, chunk, sym);
    }
    FWI_CUDA(c, cudaGetLastError());
    {
      Prof p(c, KC_MISC);
      contract_reduce_kernel<T><<<blocks_for(per, 256, c->n_sm * 8), 256, 0, c->stream>>>(
          Y, (const cplx<T>*)c->jsplit, split, per, c->n_elem * c->n_elem, c->red, c->n_elem,
          sym);
    }
    FWI_CUDA(c, cudaGetLastError());
    return FWI_OK;
  }

  static fwi_status upload_scales(fwi_ctx*) { return FWI_OK; }  // set in fwi_create
};

}  // namespace

// Plane-wave synthesis in data space: out[l][r][j] = sum_k op(A)[l][r][k]
// in[l][k][j], op(A) = A (stored [l][R][K]) or, herm, A^H (A stored
// [l][K][R]).  The matrices are small (N_T, n_elem of a few hundred), so one
// thread per output entry with a fixed-order FP64 sum; conj_out (field
// precision, optional) receives conj(out) for the adjoint sources.
template <typename T>
__global__ void synth_kernel(double2* __restrict__ out, cplx<T>* __restrict__ conj_out,
                             const double2* __restrict__ A, const double2* __restrict__ in,
                             int R, int K, int J, int herm, long long total) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % J);
    const long long t = idx / J;
    const int r = (int)(t % R);
    const long long l = t / R;
    const double2* Al = A + l * (long long)R * K;
    const double2* il = in + l * (long long)K * J;
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < K; ++k) {
      const double2 a = herm ? Al[(long long)k * R + r] : Al[(long long)r * K + k];
      const double ay = herm ? -a.y : a.y;
      const double2 b = il[(long long)k * J + j];
      sx += a.x * b.x - ay * b.y;
      sy += a.x * b.y + ay * b.x;
    }
    out[idx] = make_double2(sx, sy);
    if (conj_out) conj_out[idx] = mk<T>((T)sx, (T)(-sy));
  }
}

fwi_status synth(fwi_ctx* c, const double2* A, int herm, int R, int K, const double2* in,
                 double2* out, void* conj_out) {
  const long long total = (long long)c->n_freq * R * c->n_elem;
  const int nb = blocks_for(total, 256, c->n_sm * 8);
  Prof p(c, KC_MISC);
  if (c->fp64)
    synth_kernel<double><<<nb, 256, 0, c->stream>>>(out, (cplx<double>*)conj_out, A, in, R, K,
                                                     c->n_elem, herm, total);
  else
    synth_kernel<float><<<nb, 256, 0, c->stream>>>(out, (cplx<float>*)conj_out, A, in, R, K,
                                                    c->n_elem, herm, total);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

// Attenuating background: out[l][..] = s_l in[l][..] (conj: conj(s_l)), s_l
// = k_l^2 dV complex, on [n_freq][per] data-space arrays (FP64 or field
// precision); the contraction kernels themselves scale by 1 then.
template <typename V>
__global__ void data_scale_kernel(V* out, const V* in, const double2* s, long long per,
                                  long long total, int conj) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 f = s[i / per];
    const double fr = f.x, fi = conj ? -f.y : f.y;
    const V v = in[i];
    const double vr = (double)v.x, vi = (double)v.y;
    V o;
    o.x = (decltype(o.x))(vr * fr - vi * fi);
    o.y = (decltype(o.y))(vr * fi + vi * fr);
    out[i] = o;
  }
}

template <typename V>
static fwi_status data_scale(fwi_ctx* c, V* out, const V* in, int conj) {
  if (c->alpha0 <= 0.0) return FWI_OK;
  const long long per = (long long)c->n_elem * c->n_elem;
  const long long total = per * c->n_freq;
  Prof p(c, KC_MISC);
  data_scale_kernel<V><<<blocks_for(total, 256, c->n_sm * 8), 256, 0, c->stream>>>(
      out, in, c->sdat, per, total, conj);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

// Inversion mesh: forward-mesh results written to c->vfwd are summed over
// each cell into out (no-op on the forward mesh, where they went to out).
static fwi_status to_inversion_mesh(fwi_ctx* c, double2* out) {
  if (c->rf == 1) return FWI_OK;
  Prof p(c, KC_MISC);
  restrict_kernel<<<blocks_for(c->Ninv, 256, c->n_sm * 8), 256, 0, c->stream>>>(
      out, c->vfwd, c->nx, c->ny, c->rf, c->ry, c->Ninv);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

// Layout of c->red: [0, n_freq) per-frequency scales k_l^2 dV; then misfit
// block partials.
static inline double* misfit_parts(fwi_ctx* c) { return c->red + c->n_freq; }
constexpr int kMisfitBlocks = 256;

template <typename T> static fwi_status project_data_t(fwi_ctx* c, void* data_out) {
  fwi_status st = Jac<T>::upload_scales(c);
  if (st != FWI_OK) return st;
  st = Jac<T>::contract(c, (const cplx<T>*)c->fields, (const cplx<T>*)c->mF,
                        (const cplx<T>*)c->p0, c->dres);
  if (st != FWI_OK) return st;
  st = data_scale(c, c->dres, c->dres, 0);  // lossy background: k_l^2 dV
  if (st != FWI_OK) return st;
  // plane-wave transmits: data of transmit i = sum_e w_{l,i,e} (point data of e)
  if (c->n_tx > 0) {
    st = synth(c, c->W, 0, c->n_tx, c->n_elem, c->dres, c->dpw, nullptr);
    if (st != FWI_OK) return st;
  }
  if (data_out) {
    const long long nd = (long long)c->n_freq * c->n_t * c->n_elem;
    Prof p(c, KC_MISC);
    to_field_kernel<T><<<blocks_for(nd, 256, c->n_sm * 8), 256, 0, c->stream>>>(
        (cplx<T>*)data_out, c->n_tx > 0 ? c->dpw : c->dres, nd);
    FWI_CUDA(c, cudaGetLastError());
  }
  return FWI_OK;
}

fwi_status project_data(fwi_ctx* c, const void* m, void* data_out) {
  (void)m;  // the contrast was set by the forward solve
  return c->fp64 ? project_data_t<double>(c, data_out) : project_data_t<float>(c, data_out);
}

template <typename T> static fwi_status residual_t(fwi_ctx* c, const void* d_obs, double* misfit) {
  const long long nd = (long long)c->n_freq * c->n_t * c->n_elem;
  // c->dres (plane waves: c->dpw) holds F(m); overwrite with r = F(m) - d_obs,
  // conj(r) into dF
  double2* d = c->n_tx > 0 ? c->dpw : c->dres;
  {
    Prof p(c, KC_MISC);
    residual_kernel<T><<<kMisfitBlocks, 256, 0, c->stream>>>(
        d, (cplx<T>*)c->dF, d, (const cplx<T>*)d_obs, nd, misfit_parts(c));
  }
  FWI_CUDA(c, cudaGetLastError());
  // plane waves: the point-source residual of the chain rule, y = W^H r, into
  // dres and conj(y) into dF (the adjoint sources read dF)
  if (c->n_tx > 0) {
    fwi_status st = synth(c, c->W, 1, c->n_elem, c->n_tx, c->dpw, c->dres, c->dF);
    if (st != FWI_OK) return st;
  }
  // lossy background: the receiver rows carry the complex k_l^2 dV, so the
  // adjoint sources sum_j R_j conj(r) take it on conj(r)
  {
    fwi_status st = data_scale(c, (cplx<T>*)c->dF, (const cplx<T>*)c->dF, 0);
    if (st != FWI_OK) return st;
  }
  {
    // frequency sharding: the partial sums of every rank's frequencies
    // (reduced whether or not this caller reads the misfit, so that every
    // rank makes the same reductions)
    fwi_status st = reduce_sum(c, misfit_parts(c), kMisfitBlocks);
    if (st != FWI_OK) return st;
  }
  if (misfit) {
    FWI_CUDA(c, cudaMemcpyAsync(c->h_red, misfit_parts(c), sizeof(double) * kMisfitBlocks,
                                cudaMemcpyDeviceToHost, c->stream));
    FWI_CUDA(c, cudaStreamSynchronize(c->stream));
    double s = 0.0;
    for (int i = 0; i < kMisfitBlocks; ++i) s += c->h_red[i];
    *misfit = 0.5 * s;
  }
  return FWI_OK;
}

fwi_status residual_misfit(fwi_ctx* c, const void* d_obs, double* misfit) {
  return c->fp64 ? residual_t<double>(c, d_obs, misfit) : residual_t<float>(c, d_obs, misfit);
}

// conj(s_{l,e})(n) = k_l^2 dV sum_j p0_{l,j}(n) conj(r_{l,e,j}) into `out`.
template <typename T> static fwi_status adjoint_sources_t(fwi_ctx* c, void* out) {
  fwi_status st = Jac<T>::upload_scales(c);
  if (st != FWI_OK) return st;
  if constexpr (std::is_same<T, float>::value) {
    if (tc_usable(c)) {
      if (tc_adjoint_sources(c, (const float2*)c->dF, (const float2*)c->p0, (float2*)out) < 0)
        return FWI_ERR_CUDA;
      return FWI_OK;
    }
  }
  dim3 grid((unsigned)((c->N + TB - 1) / TB), (c->n_elem + TB - 1) / TB, c->n_freq);
  const double fe = (double)c->n_freq * c->n_elem * c->N;
  Prof p(c, KC_MIX_SOURCES, 2.0 * fe * sizeof(cplx<T>), 8.0 * fe * c->n_elem);
  mix_kernel<T, false><<<grid, 256, 0, c->stream>>>(
      (const cplx<T>*)c->dF, (const cplx<T>*)c->p0, 0, nullptr, (cplx<T>*)out, c->red,
      c->n_elem, c->N);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

fwi_status adjoint_sources_conj(fwi_ctx* c, void* out) {
  return c->fp64 ? adjoint_sources_t<double>(c, out) : adjoint_sources_t<float>(c, out);
}

// grad = sum_{l,e} conj(p) lambda with lambda = conj(y), y in c->lam.
template <typename T> static fwi_status gradient_t(fwi_ctx* c, void* grad) {
  const int ns = 8;
  const int per = (c->n_rhs + ns - 1) / ns;
  double2* part = (double2*)c->jsplit;  // needs ns * N doubles2 (checked at create)
  dim3 grid(blocks_for(c->N, 256, 1 << 20), ns);
  {
    Prof p(c, KC_GRADIENT, 2.0 * c->n_rhs * c->N * sizeof(cplx<T>), 8.0 * c->n_rhs * c->N);
    grad_partial_kernel<T><<<grid, 256, 0, c->stream>>>(
        part, (const cplx<T>*)c->fields, (const cplx<T>*)c->lam, c->n_rhs, per, c->N);
  }
  FWI_CUDA(c, cudaGetLastError());
  {
    Prof p(c, KC_MISC);
    grad_reduce_kernel<<<blocks_for(c->N, 256, c->n_sm * 8), 256, 0, c->stream>>>(
        c->rf > 1 ? c->vfwd : (double2*)grad, part, ns, c->N);
  }
  FWI_CUDA(c, cudaGetLastError());
  return to_inversion_mesh(c, (double2*)grad);
}

fwi_status assemble_gradient(fwi_ctx* c, void* grad) {
  return c->fp64 ? gradient_t<double>(c, grad) : gradient_t<float>(c, grad);
}

// (J a)_{l,e,j} = k_l^2 dV sum_n p_e(n) p_j(n) a_n, p_j from the receiver
// fields (the current fields, or their frozen snapshot: Sec. IV-B)
template <typename T> static fwi_status jac_forward_t(fwi_ctx* c, const void* a, double2* y) {
  fwi_status st = Jac<T>::upload_scales(c);
  if (st != FWI_OK) return st;
  {
    Prof p(c, KC_MISC);
    if (c->rf > 1)
      prolong_kernel<T><<<blocks_for(c->N, 256, c->n_sm * 8), 256, 0, c->stream>>>(
          (cplx<T>*)c->aF, (const double2*)a, c->nx, c->ny, c->rf, c->ry, c->N);
    else
      to_field_kernel<T><<<blocks_for(c->N, 256, c->n_sm * 8), 256, 0, c->stream>>>(
          (cplx<T>*)c->aF, (const double2*)a, c->N);
  }
  FWI_CUDA(c, cudaGetLastError());
  st = Jac<T>::contract(c, (const cplx<T>*)c->fields, (const cplx<T>*)c->aF,
                        (const cplx<T>*)receiver_fields(c), y);
  if (st != FWI_OK) return st;
  return data_scale(c, y, (const double2*)y, 0);  // lossy background: k_l^2 dV
}

fwi_status jac_forward(fwi_ctx* c, const void* a, double2* y) {
  return c->fp64 ? jac_forward_t<double>(c, a, y) : jac_forward_t<float>(c, a, y);
}

// (J^H b)_n = sum_l k_l^2 dV sum_e conj(p_e(n)) sum_j conj(p_j(n)) b_ej, p_j
// from the receiver fields
template <typename T> static fwi_status jac_adjoint_t(fwi_ctx* c, const double2* y,
                                                      double2* z_out) {
  fwi_status st = Jac<T>::upload_scales(c);
  if (st != FWI_OK) return st;
  // forward-mesh result, summed over the inversion cells at the end
  double2* z = c->rf > 1 ? c->vfwd : z_out;
  if (c->alpha0 > 0.0) {
    // lossy background: J^H carries conj(k_l^2 dV)
    st = data_scale(c, c->dlossy, y, 1);
    if (st != FWI_OK) return st;
    y = c->dlossy;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (tc_usable(c)) {
      const int np = tc_jh_partials(c, y, (const float2*)receiver_fields(c),
                                    (const float2*)c->fields, (float2*)c->zpart);
      if (np < 0) return FWI_ERR_CUDA;
      Prof p(c, KC_MISC);
      sum_parts_kernel<T><<<blocks_for(c->N, 256, c->n_sm * 8), 256, 0, c->stream>>>(
          z, (const cplx<T>*)c->zpart, np, c->N, 0);
      FWI_CUDA(c, cudaGetLastError());
      return to_inversion_mesh(c, z_out);
    }
  }
  const long long nd = (long long)c->n_freq * c->n_elem * c->n_elem;
  {
    Prof p(c, KC_MISC);
    to_field_kernel<T><<<blocks_for(nd, 256, c->n_sm * 8), 256, 0, c->stream>>>(
        (cplx<T>*)c->dF, y, nd);
  }
  FWI_CUDA(c, cudaGetLastError());
  const int nbe = (c->n_elem + TB - 1) / TB;
  dim3 grid((unsigned)((c->N + TB - 1) / TB), nbe, c->n_freq);
  {
    const double fe = (double)c->n_freq * c->n_elem * c->N;
    Prof p(c, KC_MIX_JH, 2.0 * fe * sizeof(cplx<T>), 8.0 * fe * c->n_elem + 8.0 * fe);
    mix_kernel<T, true><<<grid, 256, 0, c->stream>>>(
        (const cplx<T>*)c->dF, (const cplx<T>*)receiver_fields(c), 1,
        (const cplx<T>*)c->fields, (cplx<T>*)c->zpart, c->red, c->n_elem, c->N);
  }
  FWI_CUDA(c, cudaGetLastError());
  Prof p(c, KC_MISC);
  sum_parts_kernel<T><<<blocks_for(c->N, 256, c->n_sm * 8), 256, 0, c->stream>>>(
      z, (const cplx<T>*)c->zpart, c->n_freq * nbe, c->N, 0);
  FWI_CUDA(c, cudaGetLastError());
  return to_inversion_mesh(c, z_out);
}

fwi_status jac_adjoint(fwi_ctx* c, const double2* y, double2* z) {
  return c->fp64 ? jac_adjoint_t<double>(c, y, z) : jac_adjoint_t<float>(c, y, z);
}

}  // namespace fwi

// ---------------------------------------------------------------------------
// Allocation-free variant of the pixel contraction, for callers that cannot
// call cudaMalloc (see fwi_contract_pixels_noalloc in libfwi.h).  Its split
// partial sums live in a file-scope device array instead of a context
// workspace.  Every call shares this array; concurrent calls race.
#include <mutex>

namespace fwi {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr long long kNoallocScratchElems = (long long)(kNoallocScratchBytes / sizeof(float2));
__device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchElems];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
// Per device: the array's device address and the id of the CUDA context it
// was looked up in.  A __device__ symbol's address belongs to the context
// that loaded the module: after cudaDeviceReset (or any teardown of the
// primary context) the next context loads the module again, possibly at
// another address, so the cached address is only reused while the current
// context is the one it was looked up in.
struct NoallocSlot { unsigned long long ctx_id; float2* ptr; };
NoallocSlot g_noalloc_slot[kNoallocMaxDevices] = {};

struct FreqScales { double s[FWI_NOALLOC_MAX_FREQ]; };

// Y[l][e][j] = scale_l * sum_s part[s][l][e][j]  (FP64, fixed order)
__global__ void contract_reduce_static_kernel(double2* Y, const float2* part, int split,
                                              long long per_split, int NE2, FreqScales sc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per_split;
       i += (long long)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < split; ++s) {
      const float2 v = part[(long long)s * per_split + i];
      sx += (double)v.x;
      sy += (double)v.y;
    }
    const double f = sc.s[i / NE2];
    Y[i] = make_double2(sx * f, sy * f);
  }
}

// Driver entry points for the current context and its process-unique id
// (cuCtxGetId ids are never reused, unlike context handles), taken through
// the runtime so that the library does not link libcuda.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Unique id of the current CUDA context, or 0 if the driver cannot tell.
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)f;
  });
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on device `dev` (the current
// device), looked up with cudaGetSymbolAddress (no allocation) once per
// device and context.  If the driver cannot name the context, the address
// is looked up on every call instead of being cached.
cudaError_t noalloc_scratch(int dev, float2** out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  const unsigned long long id = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  NoallocSlot& slot = g_noalloc_slot[dev];
  if (id == 0 || slot.ctx_id != id || !slot.ptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    slot.ptr = (float2*)p;
    slot.ctx_id = id;
  }
  *out = slot.ptr;
  return cudaSuccess;
}

}  // namespace
}  // namespace fwi

extern "C" fwi_status fwi_contract_pixels_noalloc(const void* X, const void* a, const void* Q,
                                                  int n_freq, int n_elem, long long N,
                                                  const double* scale, void* Y,
                                                  void* cuda_stream) {
  using namespace fwi;
  if (!X || !Q || !Y || !scale || n_freq <= 0 || n_elem <= 0 || N <= 0)
    return fail(nullptr, FWI_ERR_INVALID_ARG, "fwi_contract_pixels_noalloc: bad argument");
  if (n_freq > FWI_NOALLOC_MAX_FREQ)
    return fail(nullptr, FWI_ERR_INVALID_ARG,
                "fwi_contract_pixels_noalloc: n_freq exceeds FWI_NOALLOC_MAX_FREQ");
  const long long per = (long long)n_freq * n_elem * n_elem;
  if (per > kNoallocScratchElems)
    return fail(nullptr, FWI_ERR_INVALID_ARG,
                "fwi_contract_pixels_noalloc: n_freq * n_elem^2 exceeds the 4 MiB static "
                "scratch (at most 524288 complex partial sums)");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sdev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fwi_contract_pixels_noalloc device");
  // the array (and the SM count) are the current device's: a stream of
  // another device would run the kernels against the wrong copy
  e = cudaStreamGetDevice(s, &sdev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fwi_contract_pixels_noalloc stream");
  if (sdev != dev)
    return fail(nullptr, FWI_ERR_INVALID_ARG,
                "fwi_contract_pixels_noalloc: cuda_stream belongs to another device than "
                "the current one");
  float2* part = nullptr;
  e = noalloc_scratch(dev, &part);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fwi_contract_pixels_noalloc scratch");
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fwi_contract_pixels_noalloc");
  const int nbe = (n_elem + TB - 1) / TB;
  const int tiles = nbe * nbe * n_freq;
  long long split = (sms * 6 + tiles - 1) / tiles;
  const long long max_split_mem = kNoallocScratchElems / per;
  const long long max_split_n = (N + KC - 1) / KC;
  if (split > max_split_mem) split = max_split_mem;
  if (split > max_split_n) split = max_split_n;
  if (split < 1) split = 1;
  long long chunk = (N + split - 1) / split;
  chunk = ((chunk + KC - 1) / KC) * KC;
  FreqScales sc{};
  for (int l = 0; l < n_freq; ++l) sc.s[l] = scale[l];
  dim3 grid((unsigned)split, nbe * nbe, n_freq);
  contract_kernel<float><<<grid, 256, 0, s>>>((const float2*)X, (const float2*)a,
                                              (const float2*)Q, part, n_elem, N, n_freq, chunk,
                                              0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fwi_contract_pixels_noalloc launch");
  contract_reduce_static_kernel<<<blocks_for(per, 256, sms * 8), 256, 0, s>>>(
      (double2*)Y, part, (int)split, per, n_elem * n_elem, sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fwi_contract_pixels_noalloc launch");
  return FWI_OK;
}
