// Kernels of the Lippmann-Schwinger operator K w = IFFT(Ghat_hat .* FFT(pad(w)))
// (Eq. 5, Sec. IV-A), split into three streaming passes over HBM:
//
//   row_fwd : per grid row, w = m .* u (u produced by a BiCGSTAB prologue),
//             zero-pad to L, forward FFT along x -> plane [rows][L]
//   col     : per column tile, FFT along the remaining axis, multiply by the
//             scaled kernel spectrum, inverse FFT, crop (2D: in place on the
//             plane; 3D: separate y and z passes)
//   row_inv : per row, inverse FFT along x, crop to the grid, and a fused
//             BiCGSTAB epilogue (v = p - K m p, t = s - K m s, ...) with the
//             per-RHS partial inner products accumulated for the FP64
//             reductions.
//
// All right-hand sides of a batch are processed in one persistent launch
// (grid-stride loop over (active RHS, tile) work items).
#pragma once

#include "common.cuh"

namespace fwi {

// --------------------------------------------------------------------------
// Block-wide reduction of NV per-thread values; thread 0 receives the
// totals in fixed order (deterministic).  All threads must call it.
template <int NV, typename A>
__device__ __forceinline__ void block_sum(A (&acc)[NV], double (&out)[NV]) {
  __shared__ double red[32][NV];
  double d[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) d[k] = (double)acc[k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < NV; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp][k] = d[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w][k];
      out[k] = s;
    }
  }
}

template <typename T> struct Coef { cplx<T> alpha, omega, beta; };

template <typename T>
__device__ __forceinline__ Coef<T> load_coef(const Scal* sc) {
  Coef<T> c;
  c.alpha = mk<T>((T)sc->alpha.x, (T)sc->alpha.y);
  c.omega = mk<T>((T)sc->omega.x, (T)sc->omega.y);
  c.beta = mk<T>((T)sc->beta.x, (T)sc->beta.y);
  return c;
}

// --------------------------------------------------------------------------
// Row forward pass.  Thread t of a line owns columns n2 = t + i*TL; the
// sample x = R2*n1 + n2 of the row feeds v[i*R1 + n1].
template <class P, typename T, int MODE>
__device__ __forceinline__ void rf_load(const RowFwdArgs<T>& a, int t, int rhs,
                                        int row, cplx<T>* v, T& acc) {
  using V = cplx<T>;
  const long long vb = (long long)rhs * a.N + (long long)row * a.nx;
  const long long mb = (long long)row * a.nx;
  const int nin1 = a.full ? P::R1 : P::H1;
  Coef<T> c;
  if (MODE == RF_ITER || MODE == RF_S) c = load_coef<T>(a.scal + rhs);
#pragma unroll
  for (int i = 0; i < P::C1; ++i) {
    const int n2 = t + i * P::TL;
    if (P::C1 * P::TL == P::R2 || n2 < P::R2) {
#pragma unroll
      for (int n1 = 0; n1 < P::R1; ++n1) {
        V w = mk<T>(T(0), T(0));
        if (n1 < nin1) {
          const int x = P::R2 * n1 + n2;
          const long long idx = vb + x;
          V u;
          if (MODE == RF_PLAIN) {
            u = a.in[idx];
            if (a.conj_in) u = cconj(u);
          } else if (MODE == RF_INIT) {
            u = a.in[idx];
            if (a.conj_in) u = cconj(u);
            a.X[idx] = mk<T>(T(0), T(0));
            a.R[idx] = u;
            a.RH[idx] = u;
            a.P[idx] = u;
            acc += u.x * u.x + u.y * u.y;
          } else if (MODE == RF_START) {
            u = a.P[idx];
          } else if (MODE == RF_ITER) {
            // x += alpha p + omega s ; r = s - omega t ; p = r + beta (p - omega v)
            V xx = a.X[idx], p = a.P[idx], s = a.R[idx], tt = a.Tt[idx], vv = a.V[idx];
            xx = cadd(xx, cadd(cmul(c.alpha, p), cmul(c.omega, s)));
            V r = csub(s, cmul(c.omega, tt));
            p = cadd(r, cmul(c.beta, csub(p, cmul(c.omega, vv))));
            a.X[idx] = xx;
            a.R[idx] = r;
            a.P[idx] = p;
            u = p;
          } else {  // RF_S: s = r - alpha v, stored over r
            V s = csub(a.R[idx], cmul(c.alpha, a.V[idx]));
            a.R[idx] = s;
            u = s;
          }
          if (a.use_m) u = cmul(a.m[mb + x], u);
          w = u;
        }
        v[i * P::R1 + n1] = w;
      }
    }
  }
}

template <class P, typename T, int LPC>
__global__ void __launch_bounds__(LPC * P::TL)
row_fwd_kernel(const RowFwdArgs<T> a) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  constexpr int LSTR = P::span(1) + 1;
  const int line = threadIdx.x / P::TL;
  const int t = threadIdx.x - line * P::TL;
  V* sml = sm + line * LSTR;
  const int nact = a.active ? *a.n_active : a.nb;
  const long long items = (long long)nact * a.ntiles;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int slot = (int)(item / a.ntiles);
    const int tile = (int)(item - (long long)slot * a.ntiles);
    const int rhs = a.active ? a.active[slot] : slot;
    const int row = tile * LPC + line;
    const bool valid = row < a.rows;
    V v[P::E];
    T acc = T(0);
    if (valid) {
      switch (a.mode) {
        case RF_PLAIN: rf_load<P, T, RF_PLAIN>(a, t, rhs, row, v, acc); break;
        case RF_INIT: rf_load<P, T, RF_INIT>(a, t, rhs, row, v, acc); break;
        case RF_START: rf_load<P, T, RF_START>(a, t, rhs, row, v, acc); break;
        case RF_ITER: rf_load<P, T, RF_ITER>(a, t, rhs, row, v, acc); break;
        default: rf_load<P, T, RF_S>(a, t, rhs, row, v, acc); break;
      }
    }
    __syncthreads();  // shared memory of the previous item fully consumed
    if (valid) phaseA_store<P, T>(t, v, sml, 1, 1, a.tw);
    __syncthreads();
    if (valid) {
      phaseB_load<P, T>(t, v, sml, 1, 1);
      V* out = a.plane + ((long long)rhs * a.rows + row) * P::L;
#pragma unroll
      for (int i = 0; i < P::C3; ++i) {
        const int k1 = t + i * P::TL;
        if (P::C3 * P::TL == P::R1 || k1 < P::R1) {
#pragma unroll
          for (int k2 = 0; k2 < P::R2; ++k2) out[k1 + P::R1 * k2] = v[i * P::R2 + k2];
        }
      }
    }
    if (a.mode == RF_INIT) {
      T accs[1] = {acc};
      double tot[1];
      block_sum<1>(accs, tot);
      if (threadIdx.x == 0)
        a.partial[((long long)rhs * NSLOT + 0) * a.ntiles + tile] = make_double2(tot[0], 0.0);
    }
  }
}

// --------------------------------------------------------------------------
// Row inverse pass with fused epilogues.  acc slots (complex, re/im pairs):
//   RI_V : 0 <rhat, v>
//   RI_T : 0 <t, s>, 1 <t, t>, 2 <rhat, t>, 3 <rhat, s>, 4 <s, s>
//   RI_R0: 0 <r, r>, 1 <b, b>
template <class P, typename T, int MODE>
__device__ __forceinline__ void ri_store(const RowInvArgs<T>& a, int t, int rhs,
                                         int row, const cplx<T>* v,
                                         T (&acc)[2 * NSLOT]) {
  using V = cplx<T>;
  const long long vb = (long long)rhs * a.N + (long long)row * a.nx;
  const long long mb = (long long)row * a.nx;
#pragma unroll
  for (int i = 0; i < P::C1; ++i) {
    const int n2 = t + i * P::TL;
    if (P::C1 * P::TL == P::R2 || n2 < P::R2) {
#pragma unroll
      for (int n1 = 0; n1 < P::H1; ++n1) {
        const int x = P::R2 * n1 + n2;
        const long long idx = vb + x;
        const V y = v[i * P::R1 + n1];
        if (MODE == RI_K) {
          a.out[idx] = y;
        } else if (MODE == RI_A) {
          a.out[idx] = csub(a.in[idx], y);
        } else if (MODE == RI_AH) {
          a.out[idx] = csub(a.in[idx], cconj(cmul(a.m[mb + x], y)));
        } else if (MODE == RI_V) {
          const V vv = csub(a.P[idx], y);
          a.V[idx] = vv;
          const V rh = a.RH[idx];
          acc[0] += rh.x * vv.x + rh.y * vv.y;
          acc[1] += rh.x * vv.y - rh.y * vv.x;
        } else if (MODE == RI_T) {
          const V s = a.R[idx];
          const V tt = csub(s, y);
          a.Tt[idx] = tt;
          const V rh = a.RH[idx];
          acc[0] += tt.x * s.x + tt.y * s.y;   // <t, s>
          acc[1] += tt.x * s.y - tt.y * s.x;
          acc[2] += tt.x * tt.x + tt.y * tt.y; // <t, t>
          acc[4] += rh.x * tt.x + rh.y * tt.y; // <rhat, t>
          acc[5] += rh.x * tt.y - rh.y * tt.x;
          acc[6] += rh.x * s.x + rh.y * s.y;   // <rhat, s>
          acc[7] += rh.x * s.y - rh.y * s.x;
          acc[8] += s.x * s.x + s.y * s.y;     // <s, s>
        } else {  // RI_R0: r = b - (x - K m x)
          V b = a.B[idx];
          if (a.conj_b) b = cconj(b);
          const V r = csub(b, csub(a.X[idx], y));
          a.R[idx] = r;
          a.RH[idx] = r;
          a.P[idx] = r;
          acc[0] += r.x * r.x + r.y * r.y;
          acc[2] += b.x * b.x + b.y * b.y;
        }
      }
    }
  }
}

template <class P, typename T, int LPC>
__global__ void __launch_bounds__(LPC * P::TL)
row_inv_kernel(const RowInvArgs<T> a) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  constexpr int LSTR = P::span(1) + 1;
  const int line = threadIdx.x / P::TL;
  const int t = threadIdx.x - line * P::TL;
  V* sml = sm + line * LSTR;
  const int nact = a.active ? *a.n_active : a.nb;
  const long long items = (long long)nact * a.ntiles;
  const bool dots = a.mode == RI_V || a.mode == RI_T || a.mode == RI_R0;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int slot = (int)(item / a.ntiles);
    const int tile = (int)(item - (long long)slot * a.ntiles);
    const int rhs = a.active ? a.active[slot] : slot;
    const int row = tile * LPC + line;
    const bool valid = row < a.rows;
    V v[P::E];
    if (valid) {
      const V* in = a.plane + ((long long)rhs * a.rows + row) * P::L;
#pragma unroll
      for (int i = 0; i < P::C3; ++i) {
        const int k1 = t + i * P::TL;
        if (P::C3 * P::TL == P::R1 || k1 < P::R1) {
#pragma unroll
          for (int k2 = 0; k2 < P::R2; ++k2) v[i * P::R2 + k2] = in[k1 + P::R1 * k2];
        }
      }
    }
    __syncthreads();
    if (valid) phaseC_store<P, T>(t, v, sml, 1, 1, a.tw);
    __syncthreads();
    T acc[2 * NSLOT];
#pragma unroll
    for (int k = 0; k < 2 * NSLOT; ++k) acc[k] = T(0);
    if (valid) {
      phaseD_load<P, T>(t, v, sml, 1, 1);
      switch (a.mode) {
        case RI_K: ri_store<P, T, RI_K>(a, t, rhs, row, v, acc); break;
        case RI_A: ri_store<P, T, RI_A>(a, t, rhs, row, v, acc); break;
        case RI_AH: ri_store<P, T, RI_AH>(a, t, rhs, row, v, acc); break;
        case RI_V: ri_store<P, T, RI_V>(a, t, rhs, row, v, acc); break;
        case RI_T: ri_store<P, T, RI_T>(a, t, rhs, row, v, acc); break;
        default: ri_store<P, T, RI_R0>(a, t, rhs, row, v, acc); break;
      }
    }
    if (dots) {
      double tot[2 * NSLOT];
      block_sum<2 * NSLOT>(acc, tot);
      if (threadIdx.x == 0) {
        double2* dst = a.partial + (long long)rhs * NSLOT * a.ntiles + tile;
#pragma unroll
        for (int k = 0; k < NSLOT; ++k)
          dst[(long long)k * a.ntiles] = make_double2(tot[2 * k], tot[2 * k + 1]);
      }
    }
  }
}

// --------------------------------------------------------------------------
// Column pass over tiles of TC adjacent columns; thread (c, t) handles
// column c of the tile as thread t of its line.  Shared-memory positions
// are interleaved across the tile's columns (stride TC), which keeps the
// exchange free of bank conflicts.
template <class P, typename T, int TC>
__global__ void __launch_bounds__(TC * P::TL)
col_kernel(const ColArgs<T> a) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int c = threadIdx.x % TC;
  const int t = threadIdx.x / TC;
  V* smc = sm + c;
  const int ntile = a.ncols / TC;
  const long long per_rhs = (long long)a.nplanes * ntile;
  const int nact = a.active ? *a.n_active : a.nb;
  const long long items = (long long)nact * per_rhs;
  const long long ls = a.line_stride;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int slot = (int)(item / per_rhs);
    const long long rem = item - (long long)slot * per_rhs;
    const int plane = (int)(rem / ntile);
    const int tile = (int)(rem - (long long)plane * ntile);
    const int rhs = a.active ? a.active[slot] : slot;
    const int j = tile * TC + c;
    const V* in = a.in + rhs * a.in_rhs_stride + plane * a.in_plane_stride + j;
    V* out = a.out + rhs * a.out_rhs_stride + plane * a.out_plane_stride + j;
    V v[P::E];
    if (a.mode == C_INV) {
#pragma unroll
      for (int i = 0; i < P::C3; ++i) {
        const int k1 = t + i * P::TL;
        if (P::C3 * P::TL == P::R1 || k1 < P::R1) {
#pragma unroll
          for (int k2 = 0; k2 < P::R2; ++k2)
            v[i * P::R2 + k2] = in[(long long)(k1 + P::R1 * k2) * ls];
        }
      }
    } else {
      const int nin1 = a.full ? P::R1 : P::H1;
#pragma unroll
      for (int i = 0; i < P::C1; ++i) {
        const int n2 = t + i * P::TL;
        if (P::C1 * P::TL == P::R2 || n2 < P::R2) {
#pragma unroll
          for (int n1 = 0; n1 < P::R1; ++n1)
            v[i * P::R1 + n1] = (n1 < nin1) ? in[(long long)(P::R2 * n1 + n2) * ls]
                                            : mk<T>(T(0), T(0));
        }
      }
    }
    __syncthreads();
    if (a.mode != C_INV) {
      phaseA_store<P, T>(t, v, smc, TC, 0, a.tw);
      __syncthreads();
      phaseB_load<P, T>(t, v, smc, TC, 0);
      if (a.mode == C_FWD) {
#pragma unroll
        for (int i = 0; i < P::C3; ++i) {
          const int k1 = t + i * P::TL;
          if (P::C3 * P::TL == P::R1 || k1 < P::R1) {
#pragma unroll
            for (int k2 = 0; k2 < P::R2; ++k2)
              out[(long long)(k1 + P::R1 * k2) * ls] = v[i * P::R2 + k2];
          }
        }
        continue;
      }
      const int l = a.freq_fixed >= 0 ? a.freq_fixed : (a.rhs0 + rhs) / a.n_elem;
      const V* g = a.ghat + (long long)l * a.ghat_freq_stride + j;
#pragma unroll
      for (int i = 0; i < P::C3; ++i) {
        const int k1 = t + i * P::TL;
        if (P::C3 * P::TL == P::R1 || k1 < P::R1) {
#pragma unroll
          for (int k2 = 0; k2 < P::R2; ++k2)
            v[i * P::R2 + k2] = cmul(v[i * P::R2 + k2],
                                     FWI_LDG(g + (long long)(k1 + P::R1 * k2) * a.ncols));
        }
      }
      __syncthreads();
    }
    phaseC_store<P, T>(t, v, smc, TC, 0, a.tw);
    __syncthreads();
    phaseD_load<P, T>(t, v, smc, TC, 0);
#pragma unroll
    for (int i = 0; i < P::C1; ++i) {
      const int n2 = t + i * P::TL;
      if (P::C1 * P::TL == P::R2 || n2 < P::R2) {
#pragma unroll
        for (int n1 = 0; n1 < P::H1; ++n1)
          out[(long long)(P::R2 * n1 + n2) * ls] = v[i * P::R1 + n1];
      }
    }
  }
}

// --------------------------------------------------------------------------
// Plans per transform length: L = R1 * R2 with TL threads per line.
template <int L> struct PlanFor;
template <> struct PlanFor<16> { using type = Plan<16, 4, 4, 4>; };
template <> struct PlanFor<32> { using type = Plan<32, 4, 8, 4>; };
template <> struct PlanFor<64> { using type = Plan<64, 8, 8, 8>; };
template <> struct PlanFor<128> { using type = Plan<128, 8, 16, 8>; };
template <> struct PlanFor<192> { using type = Plan<192, 12, 16, 16>; };
template <> struct PlanFor<256> { using type = Plan<256, 16, 16, 16>; };
template <> struct PlanFor<320> { using type = Plan<320, 20, 16, 20>; };
template <> struct PlanFor<384> { using type = Plan<384, 24, 16, 24>; };
template <> struct PlanFor<512> { using type = Plan<512, 16, 32, 16>; };
template <> struct PlanFor<640> { using type = Plan<640, 20, 32, 32>; };
template <> struct PlanFor<768> { using type = Plan<768, 24, 32, 32>; };
template <> struct PlanFor<1024> { using type = Plan<1024, 32, 32, 32>; };

#define FWI_FOR_EACH_L(X) \
  X(16) X(32) X(64) X(128) X(192) X(256) X(320) X(384) X(512) X(640) X(768) X(1024)

template <int L> constexpr int row_lpc() {
  constexpr int tl = PlanFor<L>::type::TL;
  return (128 / tl) > 0 ? 128 / tl : 1;
}

template <int L, typename T> constexpr size_t row_smem() {
  using P = typename PlanFor<L>::type;
  return (size_t)row_lpc<L>() * (P::span(1) + 1) * sizeof(cplx<T>);
}

// Columns per tile: 128-byte row segments for FP32 up to L = 512; eight
// columns otherwise, so that a tile is at most 256 threads.
template <int L, typename T> constexpr int col_tc() {
  return (sizeof(T) == 4 && L <= 512) ? 16 : 8;
}

template <int L, typename T> constexpr size_t col_smem() {
  return (size_t)L * col_tc<L, T>() * sizeof(cplx<T>);
}

// Persistent grid: resident CTAs per SM (occupancy) x SMs, cached per kernel.
struct GridCache { int blocks = 0; };
template <int L, typename T, int KIND> GridCache& gcache() {
  static GridCache g;
  return g;
}

template <typename K>
inline cudaError_t grid_for(K kernel, int threads, size_t smem, GridCache& gc) {
  if (gc.blocks > 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  gc.blocks = (per > 0 ? per : 1) * sms;
  return cudaSuccess;
}

// Definition of Lsop<T> for one precision; used by the instantiation units.
#define FWI_DEFINE_LSOP(TYPE)                                                         \
  template <> bool Lsop<TYPE>::supported(int L) {                                     \
    switch (L) {                                                                      \
      case 16: case 32: case 64: case 128: case 192: case 256: case 320: case 384:    \
      case 512: case 640: case 768: case 1024: return true;                           \
      default: return false;                                                          \
    }                                                                                 \
  }                                                                                   \
  template <> int Lsop<TYPE>::row_lines_per_cta(int L) {                              \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_LPC_CASE)                                                    \
      default: return 0;                                                              \
    }                                                                                 \
  }                                                                                   \
  template <> cudaError_t Lsop<TYPE>::row_fwd(int L, const RowFwdArgs<TYPE>& a,       \
                                              cudaStream_t s) {                       \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_ROWFWD_CASE)                                                 \
      default: return cudaErrorInvalidValue;                                          \
    }                                                                                 \
  }                                                                                   \
  template <> cudaError_t Lsop<TYPE>::row_inv(int L, const RowInvArgs<TYPE>& a,       \
                                              cudaStream_t s) {                       \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_ROWINV_CASE)                                                 \
      default: return cudaErrorInvalidValue;                                          \
    }                                                                                 \
  }                                                                                   \
  template <> cudaError_t Lsop<TYPE>::col(int L, const ColArgs<TYPE>& a,              \
                                          cudaStream_t s) {                           \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_COL_CASE)                                                    \
      default: return cudaErrorInvalidValue;                                          \
    }                                                                                 \
  }                                                                                   \
  template <> cudaError_t Lsop<TYPE>::prepare(int L) {                                \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_PREP_CASE)                                                   \
      default: return cudaErrorInvalidValue;                                          \
    }                                                                                 \
  }

#define FWI_LPC_CASE(LL) case LL: return row_lpc<LL>();

#define FWI_ROWFWD_CASE(LL)                                                          \
  case LL: {                                                                         \
    using P = PlanFor<LL>::type;                                                     \
    constexpr int lpc = row_lpc<LL>();                                               \
    auto k = row_fwd_kernel<P, FWI_T, lpc>;                                          \
    GridCache& gc = gcache<LL, FWI_T, 0>();                                          \
    cudaError_t e = grid_for(k, lpc * P::TL, row_smem<LL, FWI_T>(), gc);             \
    if (e != cudaSuccess) return e;                                                  \
    k<<<gc.blocks, lpc * P::TL, row_smem<LL, FWI_T>(), s>>>(a);                      \
    return cudaGetLastError();                                                       \
  }

#define FWI_ROWINV_CASE(LL)                                                          \
  case LL: {                                                                         \
    using P = PlanFor<LL>::type;                                                     \
    constexpr int lpc = row_lpc<LL>();                                               \
    auto k = row_inv_kernel<P, FWI_T, lpc>;                                          \
    GridCache& gc = gcache<LL, FWI_T, 1>();                                          \
    cudaError_t e = grid_for(k, lpc * P::TL, row_smem<LL, FWI_T>(), gc);             \
    if (e != cudaSuccess) return e;                                                  \
    k<<<gc.blocks, lpc * P::TL, row_smem<LL, FWI_T>(), s>>>(a);                      \
    return cudaGetLastError();                                                       \
  }

#define FWI_COL_CASE(LL)                                                             \
  case LL: {                                                                         \
    using P = PlanFor<LL>::type;                                                     \
    constexpr int tc = col_tc<LL, FWI_T>();                                              \
    auto k = col_kernel<P, FWI_T, tc>;                                               \
    GridCache& gc = gcache<LL, FWI_T, 2>();                                          \
    cudaError_t e = grid_for(k, tc * P::TL, col_smem<LL, FWI_T>(), gc);              \
    if (e != cudaSuccess) return e;                                                  \
    k<<<gc.blocks, tc * P::TL, col_smem<LL, FWI_T>(), s>>>(a);                       \
    return cudaGetLastError();                                                       \
  }

#define FWI_PREP_CASE(LL)                                                            \
  case LL: {                                                                         \
    using P = PlanFor<LL>::type;                                                     \
    constexpr int lpc = row_lpc<LL>();                                               \
    constexpr int tc = col_tc<LL, FWI_T>();                                              \
    cudaError_t e = grid_for(row_fwd_kernel<P, FWI_T, lpc>, lpc * P::TL,             \
                             row_smem<LL, FWI_T>(), gcache<LL, FWI_T, 0>());         \
    if (e == cudaSuccess)                                                            \
      e = grid_for(row_inv_kernel<P, FWI_T, lpc>, lpc * P::TL,                       \
                   row_smem<LL, FWI_T>(), gcache<LL, FWI_T, 1>());                   \
    if (e == cudaSuccess)                                                            \
      e = grid_for(col_kernel<P, FWI_T, tc>, tc * P::TL, col_smem<LL, FWI_T>(),      \
                   gcache<LL, FWI_T, 2>());                                          \
    return e;                                                                        \
  }

}  // namespace fwi
