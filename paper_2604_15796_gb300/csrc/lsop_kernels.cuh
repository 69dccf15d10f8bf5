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


#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc.cuh"

namespace fwi {

// Resident CTAs per SM a kernel is compiled for (its register budget per
// thread is then 65536 / (threads x blocks)).
constexpr int blocks_for_regs(int threads, int regs) {
  return (65536 / (threads * regs)) < 1 ? 1 : 65536 / (threads * regs);
}

// FP64 sum of NV (a power of two, <= 32) values over the 32 lanes of a
// warp, reduce-scatter style: at each of the first log2(NV) levels a lane
// keeps half of its values and adds the partner's copy of that half, so a
// lane performs NV - 1 + (5 - log2 NV) additions instead of 5 NV.  (FP64
// issues at a small fraction of the FP32 rate on this part.)  The pairing
// is fixed, so the result is deterministic.  On return every lane holds
// all NV sums in out[].
template <int NV>
__device__ __forceinline__ void warp_sum_scatter(double (&d)[NV], double (&out)[NV]) {
  static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV must be a power of two");
  const int lane = threadIdx.x & 31;
  int off = 16;
#pragma unroll
  for (int h = NV / 2; h >= 1; h >>= 1, off >>= 1) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double keep = hi ? d[i + h] : d[i];
      const double send = hi ? d[i] : d[i + h];
      d[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  for (; off >= 1; off >>= 1) d[0] += __shfl_xor_sync(0xffffffffu, d[0], off);
  // value k now sits in lanes k * (32 / NV) ... (k + 1) * (32 / NV) - 1
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = __shfl_sync(0xffffffffu, d[0], k * (32 / NV));
}

// Per-line fixed-order sums of NV per-thread values over the TL threads of
// each line.  The result does not depend on how many lines a CTA holds, so
// tile shapes can be tuned without changing any bit of the partial inner
// products.  32-thread lines use the warp reduce-scatter above (NV a power
// of two), 64-thread lines add the two warp results, shorter power-of-two
// lines reduce with a shuffle butterfly inside their aligned lane segment,
// other lengths use a shared-memory tree.  Every thread of the CTA must
// call it; thread t == 0 of each line receives the sums.
template <int TL, int NTHREADS, int NV, typename A>
__device__ __forceinline__ void line_sum(const A (&acc)[NV], int line, int t,
                                         double (&out)[NV]) {
  double d[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) d[k] = (double)acc[k];
  if constexpr (TL == 32 && (NV & (NV - 1)) == 0) {
    warp_sum_scatter<NV>(d, out);
  } else if constexpr (TL == 64 && (NV & (NV - 1)) == 0) {
    __shared__ double red[NTHREADS / 32][NV];
    double w[NV];
    warp_sum_scatter<NV>(d, w);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) red[warp][k] = w[k];
    __syncthreads();
    if (t == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) out[k] = red[2 * line][k] + red[2 * line + 1][k];
    __syncthreads();
  } else if constexpr ((TL & (TL - 1)) == 0 && TL <= 32) {
#pragma unroll
    for (int off = TL / 2; off > 0; off >>= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], off);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = d[k];
  } else if constexpr (TL == 64) {
    __shared__ double red[NTHREADS / 32][NV];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], off);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) red[warp][k] = d[k];
    __syncthreads();
    if (t == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) out[k] = red[2 * line][k] + red[2 * line + 1][k];
    __syncthreads();
  } else {
    // lines that are not whole warps (TL = 12, 20, 24, ...): thread k of
    // each line adds value k of its TL threads in thread order, and thread 0
    // collects the NV sums; two barriers instead of a log2(TL)-level tree.
    // The caller's next barrier precedes any rewrite of these arrays.
    static_assert(NV <= TL, "one summing thread per value");
    __shared__ double red[NTHREADS][NV];
    __shared__ double sums[NTHREADS / TL + 1][NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[threadIdx.x][k] = d[k];
    __syncthreads();
    if (t < NV) {
      const int base = threadIdx.x - t;
      double acc = 0.0;
      for (int i = 0; i < TL; ++i) acc += red[base + i][t];
      sums[line][t] = acc;
    }
    __syncthreads();
    if (t == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) out[k] = sums[line][k];
  }
  (void)line;
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
// Split plans: L = R1 * R2 where an R-point DFT with R = 32 is shared by a
// lane pair (S = 2, lanes differing by 16) so that no thread holds more
// than 16 complex values.  TL = R2 * S1 = R1 * S2 threads per line.
template <int L_, int R1_, int R2_, int S1_, int S2_> struct SPlan {
  static constexpr int L = L_, R1 = R1_, R2 = R2_, S1 = S1_, S2 = S2_;
  static constexpr int TL = R2 * S1;
  static_assert(TL == R1 * S2, "split plan thread count");
  static_assert(R1 * R2 == L, "plan factors");
  static constexpr int Q1 = R1 / S1, Q2 = R2 / S2;
  static constexpr int H1 = R1 / 2;
  static constexpr int E = Q1 > Q2 ? Q1 : Q2;
  static constexpr bool split = true;
  static constexpr int CA = 1, MA = Q1, CB = 1, MB = Q2;
  static constexpr int span(int pad) { return R2 * (R1 + pad); }
};

template <class P> struct PlanTraits {  // unsplit plans (fft_core.cuh Plan)
  static constexpr bool split = false;
  static constexpr int CA = P::C1, MA = P::R1, CB = P::C3, MB = P::R2;
};
template <int L, int R1, int R2, int S1, int S2> struct PlanTraits<SPlan<L, R1, R2, S1, S2>> {
  static constexpr bool split = true;
  static constexpr int CA = 1, MA = R1 / S1, CB = 1, MB = R2 / S2;
};

// Line-thread index g -> (index, half) for a split phase.  GP = consecutive
// g values per warp (32 for row lines, 32/TC for interleaved columns); the
// two halves of a pair sit 16 lanes apart and each half-warp reads
// consecutive shared-memory positions.
template <int S, int GP> __device__ __forceinline__ void decode(int g, int& idx, int& s) {
  if constexpr (S == 1) {
    idx = g;
    s = 0;
  } else {
    s = (g / (GP / 2)) & 1;
    idx = (g / GP) * (GP / 2) + (g % (GP / 2));
  }
}

// Phase-A slot (outer i, inner m) of thread t -> (n2, n1); false if idle.
template <class P, int GP>
__device__ __forceinline__ bool slotA(int t, int i, int m, int& n2, int& n1) {
  if constexpr (PlanTraits<P>::split) {
    int s;
    decode<P::S1, GP>(t, n2, s);
    n1 = (P::S1 == 1) ? m : 2 * m + s;
    return true;
  } else {
    n2 = t + i * P::TL;
    n1 = m;
    return P::C1 * P::TL == P::R2 || n2 < P::R2;
  }
}

// Phase-B slot (outer i, inner kp) of thread t -> (k1, k2); false if idle.
template <class P, int GP>
__device__ __forceinline__ bool slotB(int t, int i, int kp, int& k1, int& k2) {
  if constexpr (PlanTraits<P>::split) {
    int s;
    decode<P::S2, GP>(t, k1, s);
    k2 = (P::S2 == 1) ? kp : kp + P::Q2 * s;
    return true;
  } else {
    k1 = t + i * P::TL;
    k2 = kp;
    return P::C3 * P::TL == P::R1 || k1 < P::R1;
  }
}

// HALF_IN: the line's samples n1 >= R1/2 are zero (zero-padded rows and
// columns of the doubled lattice), so single-thread first DFTs skip them.
template <class P, int GP, typename T, bool HALF_IN = false, bool TWS = false>
__device__ __forceinline__ void ph_A(int t, cplx<T>* v, cplx<T>* sm, int sj, int pad,
                                     const cplx<T>* tw) {
  if constexpr (PlanTraits<P>::split) {
    int n2, s;
    decode<P::S1, GP>(t, n2, s);
    if constexpr (P::S1 == 1 && HALF_IN) DftHalfIn<P::R1, false, T>::run(v);
    else if constexpr (P::S1 == 1) Dft<P::R1, false, T>::run(v);
    else split_dft<P::Q1, false, T>(v, s);
#pragma unroll
    for (int kp = 0; kp < P::Q1; ++kp) {
      const int k1 = (P::S1 == 1) ? kp : kp + P::Q1 * s;
      cplx<T> z = v[kp];
      if (k1 > 0 && n2 > 0) z = cmul(z, tw_at<TWS>(tw + n2 * k1));
      sm[(n2 * (P::R1 + pad) + k1) * sj] = z;
    }
  } else {
    phaseA_store<P, T, HALF_IN, TWS>(t, v, sm, sj, pad, tw);
  }
}

template <class P, int GP, typename T>
__device__ __forceinline__ void ph_B(int t, cplx<T>* v, const cplx<T>* sm, int sj, int pad) {
  if constexpr (PlanTraits<P>::split) {
    int k1, s;
    decode<P::S2, GP>(t, k1, s);
#pragma unroll
    for (int m = 0; m < P::Q2; ++m) {
      const int n2 = (P::S2 == 1) ? m : 2 * m + s;
      v[m] = sm[(n2 * (P::R1 + pad) + k1) * sj];
    }
    if constexpr (P::S2 == 1) Dft<P::R2, false, T>::run(v);
    else split_dft<P::Q2, false, T>(v, s);
  } else {
    phaseB_load<P, T>(t, v, sm, sj, pad);
  }
}

template <class P, int GP, typename T, bool TWS = false>
__device__ __forceinline__ void ph_C(int t, cplx<T>* v, cplx<T>* sm, int sj, int pad,
                                     const cplx<T>* tw) {
  if constexpr (PlanTraits<P>::split) {
    int k1, s;
    decode<P::S2, GP>(t, k1, s);
    if constexpr (P::S2 == 1) Dft<P::R2, true, T>::run(v);
    else split_idft<P::Q2, true, T>(v, s);
#pragma unroll
    for (int m = 0; m < P::Q2; ++m) {
      const int n2 = (P::S2 == 1) ? m : 2 * m + s;
      cplx<T> z = v[m];
      if (k1 > 0 && n2 > 0) z = cmulc(z, tw_at<TWS>(tw + n2 * k1));
      sm[(n2 * (P::R1 + pad) + k1) * sj] = z;
    }
  } else {
    phaseC_store<P, T, TWS>(t, v, sm, sj, pad, tw);
  }
}

template <class P, int GP, typename T>
__device__ __forceinline__ void ph_D(int t, cplx<T>* v, const cplx<T>* sm, int sj, int pad) {
  if constexpr (PlanTraits<P>::split) {
    int n2, s;
    decode<P::S1, GP>(t, n2, s);
#pragma unroll
    for (int kp = 0; kp < P::Q1; ++kp) {
      const int k1 = (P::S1 == 1) ? kp : kp + P::Q1 * s;
      v[kp] = sm[(n2 * (P::R1 + pad) + k1) * sj];
    }
    // every caller keeps only the samples n1 < R1/2 (cropped output)
    if constexpr (P::S1 == 1) DftHalfOut<P::R1, true, T>::run(v);
    else split_idft<P::Q1, true, T>(v, s);
  } else {
    phaseD_load<P, T>(t, v, sm, sj, pad);
  }
}

// Lines of a row CTA span whole warps when TL >= 32 (GP = 32); shorter
// lines never use the split phases.
template <class P> constexpr int row_gp() { return 32; }

// --------------------------------------------------------------------------
// Row forward pass.  Phase-A slot (i, m) of thread t holds the sample
// x = R2*n1 + n2 of the row in v[i*MA + m].
//
// Staging slot of each array the pass reads, per mode, when a work item's
// rows are staged in shared memory (the contrast m after the mode's arrays).
template <int MODE> struct RfSlots {
  static constexpr int N = MODE == RF_ITER ? 5 : MODE == RF_S ? 2 : 1;
  static constexpr int X = 0, P = MODE == RF_ITER ? 1 : 0;
  static constexpr int R = MODE == RF_ITER ? 2 : 0, T = 3;
  static constexpr int V = MODE == RF_ITER ? 4 : 1, IN = 0, M = N;
};

// Loads of one line's samples into phase-A slots, with the mode's update
// written back to global memory.  STG: the samples come from the line's
// rows staged in shared memory (sl = the line's first sample in staging
// slot 0; slots LPC*L/2 samples apart); otherwise from the global arrays.
template <class P, typename T, int MODE, bool STG = false, int LPC = 1>
__device__ __forceinline__ void rf_load(const RowFwdArgs<T>& a, int t, int rhs, int row,
                                        cplx<T>* v, T& acc, const cplx<T>* sl = nullptr) {
  using V = cplx<T>;
  using S = RfSlots<MODE>;
  constexpr int GP = row_gp<P>();
  constexpr int SS = LPC * (P::L / 2);  // staging slot stride
  const V* __restrict__ in = a.in;
  const V* __restrict__ mm = a.m;
  V* __restrict__ X = a.X;
  V* __restrict__ R = a.R;
  V* __restrict__ RH = a.RH;
  V* __restrict__ Pp = a.P;
  const V* __restrict__ Vv = a.V;
  const V* __restrict__ Tt = a.Tt;
  const long long vb = (long long)rhs * a.N + (long long)row * a.nx;
  const long long mb = (long long)row * a.nx;
  const int nin1 = a.full ? P::R1 : P::H1;
  Coef<T> c;
  if (MODE == RF_ITER || MODE == RF_S) c = load_coef<T>(a.scal + rhs);
#pragma unroll
  for (int i = 0; i < PlanTraits<P>::CA; ++i) {
#pragma unroll
    for (int m = 0; m < PlanTraits<P>::MA; ++m) {
      int n2, n1;
      const bool ok = slotA<P, GP>(t, i, m, n2, n1);
      V w = mk<T>(T(0), T(0));
      if (ok && n1 < nin1) {
        const int x = P::R2 * n1 + n2;
        const long long idx = vb + x;
        // sample x of the array in staging slot k: staged, or in global memory
        auto ld = [&](const V* g, int k) { return STG ? sl[k * SS + x] : g[idx]; };
        V u;
        if (MODE == RF_PLAIN) {
          u = ld(in, S::IN);
          if (a.conj_in) u = cconj(u);
        } else if (MODE == RF_INIT) {
          u = ld(in, S::IN);
          if (a.conj_in) u = cconj(u);
          X[idx] = mk<T>(T(0), T(0));
          R[idx] = u;
          RH[idx] = u;
          Pp[idx] = u;
          acc += u.x * u.x + u.y * u.y;
        } else if (MODE == RF_START) {
          u = ld(Pp, S::P);
        } else if (MODE == RF_ITER) {
          // x += alpha p + omega s ; r = s - omega t ; p = r + beta (p - omega v)
          V xx = ld(X, S::X), p = ld(Pp, S::P), s = ld(R, S::R), tt = ld(Tt, S::T),
            vv = ld(Vv, S::V);
          xx = cadd(xx, cadd(cmul(c.alpha, p), cmul(c.omega, s)));
          const V r = csub(s, cmul(c.omega, tt));
          p = cadd(r, cmul(c.beta, csub(p, cmul(c.omega, vv))));
          X[idx] = xx;
          R[idx] = r;
          Pp[idx] = p;
          u = p;
        } else {  // RF_S: s = r - alpha v, stored over r
          const V s = csub(ld(R, S::R), cmul(c.alpha, ld(Vv, S::V)));
          R[idx] = s;
          u = s;
        }
        if (a.use_m) u = cmul(STG ? sl[S::M * SS + x] : mm[mb + x], u);
        w = u;
      }
      v[i * PlanTraits<P>::MA + m] = w;
    }
  }
}

// Prefetch of `bytes` at p into L2 (no registers, no completion to wait
// for; p 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The HBM rows a row pass's work item reads (its LPC lines of one
// right-hand side: contiguous in every [rhs][row][x] array), prefetched
// into L2 by one thread while the CTA transforms the previous item, so that
// the item's loads wait on L2 rather than on HBM.  Row lengths nx and
// starts row*nx are even, so every range is 16-byte aligned.
template <class P, typename T, int LPC>
__device__ __forceinline__ void rf_prefetch(const RowFwdArgs<T>& a, unsigned item,
                                            unsigned ntiles) {
  using V = cplx<T>;
  const int slot = (int)(item / ntiles);
  const int tile = (int)(item - (unsigned)slot * ntiles);
  const int rhs = a.active ? a.active[slot] : slot;
  const int row0 = tile * LPC;
  const int nr = (a.rows - row0 < LPC) ? a.rows - row0 : LPC;
  const long long off = (long long)rhs * a.N + (long long)row0 * a.nx;
  const unsigned bytes = (unsigned)(nr * a.nx * (int)sizeof(V));
  switch (a.mode) {
    case RF_PLAIN:
    case RF_INIT: l2_prefetch(a.in + off, bytes); break;
    case RF_START: l2_prefetch(a.P + off, bytes); break;
    case RF_S: l2_prefetch(a.R + off, bytes); l2_prefetch(a.V + off, bytes); break;
    default: break;
  }
  if (a.use_m) l2_prefetch(a.m + (long long)row0 * a.nx, bytes);
}

// ---- Rows staged in shared memory by bulk copies (FP32 forward pass) ----
// A work item reads LPC consecutive lines of one right-hand side, which are
// contiguous in every [rhs][row][x] array.  One thread copies the NEXT
// item's rows of every array the pass reads into a staging area with
// cp.async.bulk (one copy per array, completing on an mbarrier) as soon as
// the current item's samples are in registers, so that the HBM reads of
// item i+1 overlap the transforms of item i without holding registers; the
// threads then read their samples from shared memory.  (Staging the
// inverse pass's plane and operand rows the same way made that pass 9 %
// slower in the 3-D solve: it is held at 4 CTAs per SM by its registers,
// and it already issues its operand loads before the transforms.)
constexpr int kRowErrWait = 7;
constexpr int kRowErrDrain = 8;

// Array in staging slot k of the forward row pass (the RfSlots order; the
// contrast m after the mode's arrays), and the number of staged arrays.
template <typename T>
__device__ __forceinline__ const cplx<T>* rf_stage_src(const RowFwdArgs<T>& a, int k) {
  switch (a.mode) {
    case RF_PLAIN:
    case RF_INIT: return k == 0 ? a.in : a.m;
    case RF_START: return k == 0 ? a.P : a.m;
    case RF_ITER:
      return k == 0 ? a.X : k == 1 ? a.P : k == 2 ? a.R : k == 3 ? a.Tt : k == 4 ? a.V : a.m;
    default: return k == 0 ? a.R : k == 1 ? a.V : a.m;
  }
}
__host__ __device__ inline int rf_stage_count(int mode, int use_m) {
  const int n = mode == RF_ITER ? 5 : mode == RF_S ? 2 : 1;
  return n + (use_m ? 1 : 0);
}

// The forward row pass is latency-bound on its loads: the minimum-blocks
// bound keeps it at <= 72 registers (no spills) so that more warps are
// resident (10-14 % faster than the unconstrained 80-95 registers).  Lines
// that do not tile a warp (TL = 20, 24: the 3-D x lines) hold more samples
// per thread and get 88 (72 spilled 168 bytes per thread).
template <class P, typename T, int LPC, bool STG = false>
__global__ void __launch_bounds__(LPC * P::TL,
                                  blocks_for_regs(LPC * P::TL,
                                                  (32 % P::TL && P::TL % 32) ? 88 : 72))
row_fwd_kernel(const RowFwdArgs<T> a) {
  using V = cplx<T>;
  constexpr int GP = row_gp<P>();
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  constexpr int LSTR = P::span(1) + 1;
  constexpr int NXH = P::L / 2;  // samples per staged line (the half lattice)
  const int line = threadIdx.x / P::TL;
  const int t = threadIdx.x - line * P::TL;
  V* sml = sm + line * LSTR;
  const int nact = a.active ? *a.n_active : a.nb;
  // 32-bit item arithmetic: the context caps the batch so that every item
  // count fits (fwi_create)
  const unsigned ntiles = (unsigned)a.ntiles;
  const unsigned items = (unsigned)nact * ntiles;
  // staging (STG): after the exchange, 128-byte aligned; then the mbarrier
  // and the abort flag
  V* stg = nullptr;
  uint64_t* bar = nullptr;
  volatile int* abort_flag = nullptr;
  int nsrc = 0;
  uint32_t parity = 0;
  bool failed = false;
  int dummy_err = 0;
  int* err = nullptr;
  if constexpr (STG) {
    const uint32_t base = tc::smem_addr(smraw);
    const uint32_t ex_end = base + (uint32_t)(LPC * LSTR * sizeof(V));
    const uint32_t st0 = (ex_end + 127u) & ~127u;
    stg = reinterpret_cast<V*>(smraw + (st0 - base));
    nsrc = rf_stage_count(a.mode, a.use_m);
    bar = reinterpret_cast<uint64_t*>(stg + nsrc * LPC * NXH);
    abort_flag = reinterpret_cast<volatile int*>(bar + 1);
    err = a.err ? a.err : &dummy_err;
    if (threadIdx.x == 0) {
      tc::mbar_init(tc::smem_addr(bar), 1);
      *abort_flag = 0;
      tc::mbar_init_fence();
    }
    __syncthreads();
  }
  // bulk copies of an item's rows of every staged array (thread 0)
  auto issue = [&](unsigned it) {
    const int sl = (int)(it / ntiles);
    const int tl = (int)(it - (unsigned)sl * ntiles);
    const int rh = a.active ? a.active[sl] : sl;
    const int row0 = tl * LPC;
    const int nr = (a.rows - row0 < LPC) ? a.rows - row0 : LPC;
    const uint32_t bytes = (uint32_t)(nr * NXH * (int)sizeof(V));
    const uint32_t b = tc::smem_addr(bar);
    tc::mbar_arrive_expect_tx(b, bytes * (uint32_t)nsrc);
    for (int k = 0; k < nsrc; ++k) {
      const bool is_m = a.use_m && k == nsrc - 1;  // m: one row set for every RHS
      const long long off = is_m ? (long long)row0 * NXH
                                 : (long long)rh * a.N + (long long)row0 * NXH;
      tc::bulk_g2s(tc::smem_addr(stg + k * LPC * NXH), rf_stage_src(a, k) + off, bytes, b);
    }
  };
  if constexpr (STG) {
    if (threadIdx.x == 0 && blockIdx.x < items) issue(blockIdx.x);
  }
  for (unsigned item = blockIdx.x; item < items; item += gridDim.x) {
    const int slot = (int)(item / ntiles);
    const int tile = (int)(item - (unsigned)slot * ntiles);
    const int rhs = a.active ? a.active[slot] : slot;
    const int row = tile * LPC + line;
    const bool valid = row < a.rows;
    // (not in the BiCGSTAB update mode: its six input streams already keep
    // enough loads in flight, and the prefetch slowed it by 13 %)
    if (!STG && a.l2pf && a.mode != RF_ITER && threadIdx.x == 0 && item + gridDim.x < items)
      rf_prefetch<P, T, LPC>(a, item + gridDim.x, ntiles);
    V v[P::E];
    T acc = T(0);
    bool ok = true;
    if constexpr (STG) ok = tc::mbar_wait(tc::smem_addr(bar), parity, abort_flag, err, kRowErrWait);
    if (valid) {
      const V* sl = STG ? stg + line * NXH : nullptr;  // the line in staging slot 0
      switch (a.mode) {
        case RF_PLAIN: rf_load<P, T, RF_PLAIN, STG, LPC>(a, t, rhs, row, v, acc, sl); break;
        case RF_INIT: rf_load<P, T, RF_INIT, STG, LPC>(a, t, rhs, row, v, acc, sl); break;
        case RF_START: rf_load<P, T, RF_START, STG, LPC>(a, t, rhs, row, v, acc, sl); break;
        case RF_ITER: rf_load<P, T, RF_ITER, STG, LPC>(a, t, rhs, row, v, acc, sl); break;
        default: rf_load<P, T, RF_S, STG, LPC>(a, t, rhs, row, v, acc, sl); break;
      }
    }
    // shared memory of the previous item fully consumed (and, staged, this
    // item's rows are in registers: the staging area is free)
    if constexpr (STG) {
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      parity ^= 1u;
      if (threadIdx.x == 0 && item + gridDim.x < items) issue(item + gridDim.x);
    } else {
      __syncthreads();
    }
    // (the half-input DFT measured slower in this pass than the full one)
    if (valid) ph_A<P, GP, T, false>(t, v, sml, 1, 1, a.tw);
    __syncthreads();
    if (valid) {
      ph_B<P, GP, T>(t, v, sml, 1, 1);
      V* __restrict__ out = a.plane + ((long long)rhs * a.rows + row) * P::L;
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CB; ++i) {
#pragma unroll
        for (int kp = 0; kp < PlanTraits<P>::MB; ++kp) {
          int k1, k2;
          if (slotB<P, GP>(t, i, kp, k1, k2))
            out[k1 + P::R1 * k2] = v[i * PlanTraits<P>::MB + kp];
        }
      }
    }
    if (a.mode == RF_INIT) {
      const T accs[1] = {acc};
      double tot[1];
      line_sum<P::TL, LPC * P::TL, 1>(accs, line, t, tot);
      if (t == 0 && valid)
        a.partial[((long long)rhs * NSLOT + 0) * a.rows + row] = make_double2(tot[0], 0.0);
    }
  }
  // copies of a CTA that stopped early may still land in its shared memory
  if constexpr (STG) {
    if (failed && threadIdx.x == 0) tc::mbar_wait_drain(tc::smem_addr(bar), parity, err, kRowErrDrain);
  }
}

// --------------------------------------------------------------------------
// Row inverse pass with fused epilogues.  The epilogue operands of the
// item (p and rhat, s and rhat, ...) are loaded before the FFT phases so
// that their latency overlaps the transform.  acc slots (complex pairs):
//   RI_V : 0 <rhat, v>
//   RI_T : 0 <t, s>, 1 <t, t>, 2 <rhat, t>, 3 <rhat, s>, 4 <s, s>
//   RI_R0: 0 <r, r>, 1 <b, b>
// Phase-A slots m whose sample n1 lies in the cropped half n1 < H1: for a
// split phase A (n1 = 2m + s) these are m < H1/2, otherwise m < H1.
template <class P> constexpr int out_m() {
  if constexpr (PlanTraits<P>::split) return (P::S1 == 2) ? P::H1 / 2 : P::H1;
  else return P::H1;
}
template <class P> struct RowSlots {
  static constexpr int M = out_m<P>();
  static constexpr int N = PlanTraits<P>::CA * M;  // output samples per thread
};

template <class P, typename T, int MODE>
__device__ __forceinline__ void ri_prefetch(const RowInvArgs<T>& a, int t, int rhs, int row,
                                            cplx<T>* q0, cplx<T>* q1) {
  using V = cplx<T>;
  constexpr int GP = row_gp<P>();
  const V* __restrict__ in = a.in;
  const V* __restrict__ mm = a.m;
  const V* __restrict__ Bv = a.B;
  const V* __restrict__ X = a.X;
  const V* __restrict__ R = a.R;
  const V* __restrict__ RH = a.RH;
  const V* __restrict__ Pp = a.P;
  const long long vb = (long long)rhs * a.N + (long long)row * a.nx;
  const long long mb = (long long)row * a.nx;
#pragma unroll
  for (int i = 0; i < PlanTraits<P>::CA; ++i) {
#pragma unroll
    for (int m = 0; m < RowSlots<P>::M; ++m) {
      const int j = i * RowSlots<P>::M + m;
      int n2, n1;
      if (!slotA<P, GP>(t, i, m, n2, n1) || n1 >= P::H1) continue;
      const int x = P::R2 * n1 + n2;
      const long long idx = vb + x;
      if (MODE == RI_A) {
        q0[j] = in[idx];
      } else if (MODE == RI_AH) {
        q0[j] = in[idx];
        q1[j] = mm[mb + x];
      } else if (MODE == RI_V) {
        q0[j] = Pp[idx];
        q1[j] = RH[idx];
      } else if (MODE == RI_T) {
        q0[j] = R[idx];
        q1[j] = RH[idx];
      } else if (MODE == RI_R0) {
        q0[j] = X[idx];
        q1[j] = Bv[idx];
      }
    }
  }
}

template <class P, typename T, int MODE>
__device__ __forceinline__ void ri_store(const RowInvArgs<T>& a, int t, int rhs, int row,
                                         const cplx<T>* v, const cplx<T>* q0,
                                         const cplx<T>* q1, T (&acc)[2 * NSLOT]) {
  using V = cplx<T>;
  constexpr int GP = row_gp<P>();
  V* __restrict__ out = a.out;
  V* __restrict__ R = a.R;
  V* __restrict__ RH = a.RH;
  V* __restrict__ Pp = a.P;
  V* __restrict__ Vv = a.V;
  V* __restrict__ Tt = a.Tt;
  const long long vb = (long long)rhs * a.N + (long long)row * a.nx;
#pragma unroll
  for (int i = 0; i < PlanTraits<P>::CA; ++i) {
#pragma unroll
    for (int m = 0; m < RowSlots<P>::M; ++m) {
      const int j = i * RowSlots<P>::M + m;
      int n2, n1;
      if (!slotA<P, GP>(t, i, m, n2, n1) || n1 >= P::H1) continue;
      const long long idx = vb + P::R2 * n1 + n2;
      // phase-D output slot of sample n1 (< H1): same position as in phase A
      const V y = v[i * PlanTraits<P>::MA + m];
      if (MODE == RI_K) {
        out[idx] = y;
      } else if (MODE == RI_A) {
        out[idx] = csub(q0[j], y);
      } else if (MODE == RI_AH) {
        out[idx] = csub(q0[j], cconj(cmul(q1[j], y)));
      } else if (MODE == RI_V) {
        const V vv = csub(q0[j], y);
        Vv[idx] = vv;
        const V rh = q1[j];
        acc[0] += rh.x * vv.x + rh.y * vv.y;
        acc[1] += rh.x * vv.y - rh.y * vv.x;
      } else if (MODE == RI_T) {
        const V s = q0[j];
        const V tt = csub(s, y);
        Tt[idx] = tt;
        const V rh = q1[j];
        acc[0] += tt.x * s.x + tt.y * s.y;    // <t, s>
        acc[1] += tt.x * s.y - tt.y * s.x;
        acc[2] += tt.x * tt.x + tt.y * tt.y;  // <t, t>
        acc[4] += rh.x * tt.x + rh.y * tt.y;  // <rhat, t>
        acc[5] += rh.x * tt.y - rh.y * tt.x;
        acc[6] += rh.x * s.x + rh.y * s.y;    // <rhat, s>
        acc[7] += rh.x * s.y - rh.y * s.x;
        acc[8] += s.x * s.x + s.y * s.y;      // <s, s>
      } else {  // RI_R0: r = b - (x - K m x)
        V b = q1[j];
        if (a.conj_b) b = cconj(b);
        const V r = csub(b, csub(q0[j], y));
        R[idx] = r;
        RH[idx] = r;
        Pp[idx] = r;
        acc[0] += r.x * r.x + r.y * r.y;
        acc[2] += b.x * b.x + b.y * b.y;
      }
    }
  }
}

template <class P, typename T, int LPC, int MODE>
__device__ __forceinline__ void ri_prefetch_l2(const RowInvArgs<T>& a, unsigned item,
                                               unsigned ntiles) {
  using V = cplx<T>;
  const int slot = (int)(item / ntiles);
  const int tile = (int)(item - (unsigned)slot * ntiles);
  const int rhs = a.active ? a.active[slot] : slot;
  const int row0 = tile * LPC;
  const int nr = (a.rows - row0 < LPC) ? a.rows - row0 : LPC;
  l2_prefetch(a.plane + ((long long)rhs * a.rows + row0) * P::L,
              (unsigned)(nr * P::L * (int)sizeof(V)));
  const long long off = (long long)rhs * a.N + (long long)row0 * a.nx;
  const unsigned bytes = (unsigned)(nr * a.nx * (int)sizeof(V));
  if (MODE == RI_A || MODE == RI_AH) l2_prefetch(a.in + off, bytes);
  if (MODE == RI_AH) l2_prefetch(a.m + (long long)row0 * a.nx, bytes);
  if (MODE == RI_V) { l2_prefetch(a.P + off, bytes); l2_prefetch(a.RH + off, bytes); }
  if (MODE == RI_T) { l2_prefetch(a.R + off, bytes); l2_prefetch(a.RH + off, bytes); }
  if (MODE == RI_R0) { l2_prefetch(a.X + off, bytes); l2_prefetch(a.B + off, bytes); }
}

template <class P, typename T, int LPC, int MODE>
__device__ __forceinline__ void row_inv_items(const RowInvArgs<T>& a, cplx<T>* sml, int line,
                                              int t) {
  using V = cplx<T>;
  constexpr int GP = row_gp<P>();
  constexpr bool dots = MODE == RI_V || MODE == RI_T || MODE == RI_R0;
  constexpr int NS = RowSlots<P>::N;
  const int nact = a.active ? *a.n_active : a.nb;
  // 32-bit item arithmetic: the context caps the batch so that every item
  // count fits (fwi_create)
  const unsigned ntiles = (unsigned)a.ntiles;
  const unsigned items = (unsigned)nact * ntiles;
  for (unsigned item = blockIdx.x; item < items; item += gridDim.x) {
    const int slot = (int)(item / ntiles);
    const int tile = (int)(item - (unsigned)slot * ntiles);
    const int rhs = a.active ? a.active[slot] : slot;
    const int row = tile * LPC + line;
    const bool valid = row < a.rows;
    if (a.l2pf && threadIdx.x == 0 && item + gridDim.x < items)
      ri_prefetch_l2<P, T, LPC, MODE>(a, item + gridDim.x, ntiles);
    V v[P::E];
    V q0[NS], q1[NS];
    if (valid) {
      const V* __restrict__ in = a.plane + ((long long)rhs * a.rows + row) * P::L;
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CB; ++i) {
#pragma unroll
        for (int kp = 0; kp < PlanTraits<P>::MB; ++kp) {
          int k1, k2;
          if (slotB<P, GP>(t, i, kp, k1, k2))
            v[i * PlanTraits<P>::MB + kp] = in[k1 + P::R1 * k2];
        }
      }
      ri_prefetch<P, T, MODE>(a, t, rhs, row, q0, q1);
    }
    __syncthreads();
    if (valid) ph_C<P, GP, T>(t, v, sml, 1, 1, a.tw);
    __syncthreads();
    T acc[2 * NSLOT];
#pragma unroll
    for (int k = 0; k < 2 * NSLOT; ++k) acc[k] = T(0);
    if (valid) {
      ph_D<P, GP, T>(t, v, sml, 1, 1);
      ri_store<P, T, MODE>(a, t, rhs, row, v, q0, q1, acc);
    }
    if (dots) {
      // only the live accumulators enter the FP64 line sum
      constexpr int NV = MODE == RI_T ? 8 : 2;
      T live[NV];
      if constexpr (MODE == RI_T) {
        const int src[8] = {0, 1, 2, 4, 5, 6, 7, 8};
#pragma unroll
        for (int k = 0; k < 8; ++k) live[k] = acc[src[k]];
      } else if constexpr (MODE == RI_V) {
        live[0] = acc[0];
        live[1] = acc[1];
      } else {
        live[0] = acc[0];
        live[1] = acc[2];
      }
      double tot[NV];
      line_sum<P::TL, LPC * P::TL, NV>(live, line, t, tot);
      if (t == 0 && valid) {
        double full[2 * NSLOT];
#pragma unroll
        for (int k = 0; k < 2 * NSLOT; ++k) full[k] = 0.0;
        if constexpr (MODE == RI_T) {
          const int dst_k[8] = {0, 1, 2, 4, 5, 6, 7, 8};
#pragma unroll
          for (int k = 0; k < 8; ++k) full[dst_k[k]] = tot[k];
        } else if constexpr (MODE == RI_V) {
          full[0] = tot[0];
          full[1] = tot[1];
        } else {
          full[0] = tot[0];
          full[2] = tot[1];
        }
        double2* dst = a.partial + (long long)rhs * NSLOT * a.rows + row;
#pragma unroll
        for (int k = 0; k < NSLOT; ++k)
          dst[(long long)k * a.rows] = make_double2(full[2 * k], full[2 * k + 1]);
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
  switch (a.mode) {
    case RI_K: row_inv_items<P, T, LPC, RI_K>(a, sml, line, t); break;
    case RI_A: row_inv_items<P, T, LPC, RI_A>(a, sml, line, t); break;
    case RI_AH: row_inv_items<P, T, LPC, RI_AH>(a, sml, line, t); break;
    case RI_V: row_inv_items<P, T, LPC, RI_V>(a, sml, line, t); break;
    case RI_T: row_inv_items<P, T, LPC, RI_T>(a, sml, line, t); break;
    default: row_inv_items<P, T, LPC, RI_R0>(a, sml, line, t); break;
  }
}

// --------------------------------------------------------------------------
// Work item of a column pass -> (RHS slot, plane, column tile).  The
// convolution sweeps all right-hand sides of a group of kConvTileGroup
// adjacent column tiles together (tile fastest within the group, then the
// slot), so that each tile of the kernel spectrum is read from HBM once per
// frequency and served from L2 for the other right-hand sides (in 3-D one
// frequency's spectrum, lz*ly*lx*8 bytes, exceeds L2), while each right-
// hand side's rows are read as kConvTileGroup * 128-byte runs rather than
// single 128-byte segments of as many different volumes as there are CTAs.
// The other passes go right-hand side by right-hand side.
constexpr int kConvTileGroup = 8;
struct ColItem { int slot, plane, tile; };
__device__ __forceinline__ ColItem col_item(unsigned item, unsigned nact, unsigned per_rhs,
                                            unsigned ntile, int nplanes, bool slot_fast) {
  ColItem it;
  unsigned rem;
  if (slot_fast) {
    // plane, then tile group, then slot, then tile; the last group of a
    // plane may be short
    const unsigned per_plane = nact * ntile;
    const unsigned pl = (nplanes == 1) ? 0u : item / per_plane;
    const unsigned ri = item - pl * per_plane;
    const unsigned gsz = nact * (unsigned)kConvTileGroup;
    const unsigned g0 = ri / gsz * (unsigned)kConvTileGroup;  // first tile of the group
    const unsigned r = ri - g0 * nact;
    const unsigned k = (ntile - g0 < (unsigned)kConvTileGroup) ? ntile - g0
                                                               : (unsigned)kConvTileGroup;
    it.slot = (int)(r / k);
    it.plane = (int)pl;
    it.tile = (int)(g0 + (r - (unsigned)it.slot * k));
    return it;
  }
  it.slot = (int)(item / per_rhs);
  rem = item - (unsigned)it.slot * per_rhs;
  it.plane = (nplanes == 1) ? 0 : (int)(rem / ntile);
  it.tile = (int)(rem - (unsigned)it.plane * ntile);
  return it;
}

// The transforms of one column item after its samples are in registers
// (phase-A slots for the forward and convolution modes, phase-B slots for
// the inverse) and the exchange buffer is free: forward FFT along the
// column, product with the kernel spectrum, inverse FFT, cropped store
// (C_CONV); forward FFT and store of every frequency sample (C_FWD);
// inverse FFT and cropped store (C_INV).  `out` points at the item's first
// output sample of column j.  TWS: the twiddle table `tw` is in shared
// memory.  gs: the item's kernel-spectrum tile staged in shared memory,
// offset to this thread's column (rows 0..L/2 of the TC columns, row
// stride TC; row k > L/2 is row L - k: the spectrum of the lattice kernel,
// even in each offset, is even in the frequency index), or NULL to read the
// spectrum from global memory.  hook.wait_spectrum() is called by thread 0
// before the barrier that precedes the product (and returns false if the
// staging failed), hook.spectrum_done() by every thread after the barrier
// that follows it (every thread is then done with gs).
struct NoColHook {
  __device__ bool wait_spectrum() const { return true; }
  __device__ void spectrum_done() const {}
};

// Spectrum row of frequency k = k1 + R1 k2 (k1 < R1), folded onto 0..L/2
// (the spectrum is even in k).  For unsplit plans with R1 | L/2 the fold is
// known from the slot alone: k <= L/2 exactly when k2 < L/(2 R1) (k = L/2
// at k2 = L/(2 R1), k1 = 0 folds onto itself), so no per-element compare.
template <class P>
__device__ __forceinline__ int spectrum_row(int k1, int k2, int kp) {
  const int k = k1 + P::R1 * k2;
  if constexpr (!PlanTraits<P>::split && (P::L / 2) % P::R1 == 0) {
    return (kp < P::L / (2 * P::R1)) ? k : P::L - k;
  } else {
    return (k <= P::L / 2) ? k : P::L - k;
  }
}

template <class P, typename T, int TC, bool TWS = false, class Hook = NoColHook>
__device__ __forceinline__ bool col_transform_store(const ColArgs<T>& a, int t, cplx<T>* smc,
                                                    cplx<T>* v, int rhs, int j,
                                                    cplx<T>* __restrict__ out,
                                                    const cplx<T>* tw,
                                                    const cplx<T>* gs = nullptr,
                                                    const Hook& hook = Hook()) {
  using V = cplx<T>;
  constexpr int GP = 32 / TC;
  const long long ls = a.line_stride;
  bool ok = true;
  if (a.mode != C_INV) {
    if (a.full) ph_A<P, GP, T, false, TWS>(t, v, smc, TC, 0, tw);
    else ph_A<P, GP, T, true, TWS>(t, v, smc, TC, 0, tw);
    // one thread waits for the staged spectrum; the barrier hands its
    // completion (and the copied data) to the others
    if (gs && a.mode == C_CONV && threadIdx.x == 0) ok = hook.wait_spectrum();
    __syncthreads();
    ph_B<P, GP, T>(t, v, smc, TC, 0);
    if (a.mode == C_FWD) {
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CB; ++i) {
#pragma unroll
        for (int kp = 0; kp < PlanTraits<P>::MB; ++kp) {
          int k1, k2;
          if (slotB<P, GP>(t, i, kp, k1, k2))
            out[(long long)(k1 + P::R1 * k2) * ls] = v[i * PlanTraits<P>::MB + kp];
        }
      }
      return ok;
    }
    if (gs) {
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CB; ++i) {
#pragma unroll
        for (int kp = 0; kp < PlanTraits<P>::MB; ++kp) {
          int k1, k2;
          if (slotB<P, GP>(t, i, kp, k1, k2)) {
            const int r = i * PlanTraits<P>::MB + kp;
            v[r] = cmul(v[r], gs[spectrum_row<P>(k1, k2, kp) * TC]);
          }
        }
      }
    } else {
      const int l = a.freq_fixed >= 0 ? a.freq_fixed : (a.rhs0 + rhs) / a.n_elem;
      const V* __restrict__ g = a.ghat + (long long)l * a.ghat_freq_stride + j;
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CB; ++i) {
#pragma unroll
        for (int kp = 0; kp < PlanTraits<P>::MB; ++kp) {
          int k1, k2;
          if (slotB<P, GP>(t, i, kp, k1, k2)) {
            const int r = i * PlanTraits<P>::MB + kp;
            // the same rows as the staged tile
            v[r] = cmul(v[r], FWI_LDG(g + (long long)spectrum_row<P>(k1, k2, kp) * a.ncols));
          }
        }
      }
    }
    __syncthreads();
    if (gs) hook.spectrum_done();
  }
  ph_C<P, GP, T, TWS>(t, v, smc, TC, 0, tw);
  __syncthreads();
  ph_D<P, GP, T>(t, v, smc, TC, 0);
#pragma unroll
  for (int i = 0; i < PlanTraits<P>::CA; ++i) {
#pragma unroll
    for (int m = 0; m < PlanTraits<P>::MA; ++m) {
      int n2, n1;
      if (slotA<P, GP>(t, i, m, n2, n1) && n1 < P::H1)
        out[(long long)(P::R2 * n1 + n2) * ls] = v[i * PlanTraits<P>::MA + m];
    }
  }
  return ok;
}

// Column passes: 512-thread tiles at 64 registers (two CTAs per SM), the
// smaller tiles at 80 (three 256-thread CTAs per SM: more warps to hide
// the staging and kernel-spectrum loads; measured on the 160 x 160 x 128
// volume, 1.94 -> 1.88 s per step against two CTAs at 128 registers).
constexpr int col_regs(int threads) { return threads >= 512 ? 64 : 80; }

template <class P, typename T, int TC>
__global__ void __launch_bounds__(TC * P::TL, blocks_for_regs(TC * P::TL, col_regs(TC * P::TL)))
col_kernel(const ColArgs<T> a) {
  using V = cplx<T>;
  constexpr int GP = 32 / TC;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int c = threadIdx.x % TC;
  const int t = threadIdx.x / TC;
  V* smc = sm + c;
  const unsigned ntile = (unsigned)(a.ncols / TC);
  const unsigned per_rhs = (unsigned)a.nplanes * ntile;
  const int nact = a.active ? *a.n_active : a.nb;
  const unsigned items = (unsigned)nact * per_rhs;  // < 2^31 (fwi_create caps the batch)
  const long long ls = a.line_stride;
  const bool slot_fast = a.mode == C_CONV;
  for (unsigned item = blockIdx.x; item < items; item += gridDim.x) {
    const ColItem it = col_item(item, (unsigned)nact, per_rhs, ntile, a.nplanes, slot_fast);
    const int plane = it.plane, tile = it.tile;
    const int rhs = a.active ? a.active[it.slot] : it.slot;
    const int j = tile * TC + c;
    const V* __restrict__ in = a.in + rhs * a.in_rhs_stride + plane * a.in_plane_stride + j;
    V* __restrict__ out = a.out + rhs * a.out_rhs_stride + plane * a.out_plane_stride + j;
    V v[P::E];
    if (a.mode == C_INV) {
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CB; ++i) {
#pragma unroll
        for (int kp = 0; kp < PlanTraits<P>::MB; ++kp) {
          int k1, k2;
          if (slotB<P, GP>(t, i, kp, k1, k2))
            v[i * PlanTraits<P>::MB + kp] = in[(long long)(k1 + P::R1 * k2) * ls];
        }
      }
    } else {
      const int nin1 = a.full ? P::R1 : P::H1;
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CA; ++i) {
#pragma unroll
        for (int m = 0; m < PlanTraits<P>::MA; ++m) {
          int n2, n1;
          const bool ok = slotA<P, GP>(t, i, m, n2, n1);
          v[i * PlanTraits<P>::MA + m] = (ok && n1 < nin1)
                                             ? in[(long long)(P::R2 * n1 + n2) * ls]
                                             : mk<T>(T(0), T(0));
        }
      }
    }
    __syncthreads();
    col_transform_store<P, T, TC>(a, t, smc, v, rhs, j, out, a.tw);
  }
}

// --------------------------------------------------------------------------
// Column pass with the input tiles staged by the tensor memory accelerator
// (FP32, zero-padded or inverse input).  One thread of the CTA issues the
// TMA copy of the NEXT work item's input tile (TC columns x the line's
// nonzero rows, one 3-D box per <= 256 rows) into a staging buffer as soon
// as every thread has moved the current tile into registers, so the HBM
// read of item i+1 overlaps the transforms of item i.  The staging buffer
// is a separate region of shared memory from the transform exchange.  The
// wait on the copy's mbarrier is bounded (1 s): on a timeout the CTA
// records the code in a.err, waits (bounded) for its copy in flight and
// stops; the entry points report the code.
//
// Tensor map: 3-D, innermost the columns (as 2 floats each), then the
// line's rows (stride line_stride), then (RHS, plane) pairs (stride
// in_rhs_stride / nplanes); box {2 TC, rows_in / nbox, 1}.
constexpr int kColErrWait = 5;
constexpr int kColErrDrain = 6;

// Shared-memory layout of col_tma_kernel (offsets in float2 from the
// 128-byte aligned base): exchange L x TC | input staging rows_in x TC |
// kernel-spectrum staging (L/2 + 1) x TC (convolution with gmap only) |
// twiddle table L | two mbarriers and the abort flag.
template <int L, int TC> struct ColTmaSmem {
  static constexpr int G_ROWS = L / 2 + 1;
  static constexpr size_t bytes(int rows_in, bool gstage) {
    return ((size_t)L * TC + (size_t)rows_in * TC + (gstage ? (size_t)G_ROWS * TC : 0) +
            (size_t)L) * sizeof(float2) + 32 + 128;
  }
};

template <class P, int TC, bool GSTAGE>
__global__ void __launch_bounds__(TC * P::TL, blocks_for_regs(TC * P::TL, col_regs(TC * P::TL)))
col_tma_kernel(const ColArgs<float> a, const __grid_constant__ CUtensorMap map,
               const __grid_constant__ CUtensorMap gmap, int rows_in, int nbox) {
  using V = float2;
  constexpr int GP = 32 / TC;
  constexpr int G_ROWS = ColTmaSmem<P::L, TC>::G_ROWS;
  extern __shared__ __align__(16) unsigned char smraw[];
  // TMA destinations 128-byte aligned (the launch adds 128 bytes of slack)
  const uint32_t base_pad = (128u - (tc::smem_addr(smraw) & 127u)) & 127u;
  V* sm = reinterpret_cast<V*>(smraw + base_pad);            // exchange, L x TC
  V* stg = sm + P::L * TC;                                   // input staging, rows_in x TC
  V* gst = stg + rows_in * TC;                               // spectrum staging
  V* tws = gst + (GSTAGE ? G_ROWS * TC : 0);                 // twiddles, L
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + P::L);   // [0] input, [1] spectrum
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 2);
  const uint32_t bar_in = tc::smem_addr(bar), bar_g = tc::smem_addr(bar + 1);
  const uint32_t stg_a = tc::smem_addr(stg), gst_a = tc::smem_addr(gst);
  const int c = threadIdx.x % TC;
  const int t = threadIdx.x / TC;
  V* smc = sm + c;
  const unsigned ntile = (unsigned)(a.ncols / TC);
  const unsigned per_rhs = (unsigned)a.nplanes * ntile;
  const int nact = a.active ? *a.n_active : a.nb;
  const unsigned items = (unsigned)nact * per_rhs;  // < 2^31 (fwi_create caps the batch)
  const bool slot_fast = a.mode == C_CONV;
  const bool use_g = GSTAGE && a.mode == C_CONV;
  const int box_rows = rows_in / nbox;
  const uint32_t tile_bytes = (uint32_t)(rows_in * TC * sizeof(V));
  const uint32_t g_bytes = (uint32_t)(G_ROWS * TC * sizeof(V));
  int dummy_err = 0;
  int* err = a.err ? a.err : &dummy_err;

  auto rhs_of = [&](const ColItem& it) { return a.active ? a.active[it.slot] : it.slot; };
  auto issue_input = [&](unsigned item) {
    const ColItem it = col_item(item, (unsigned)nact, per_rhs, ntile, a.nplanes, slot_fast);
    tc::mbar_arrive_expect_tx(bar_in, tile_bytes);
    for (int b = 0; b < nbox; ++b)
      tc::tma_load_3d(stg_a + (uint32_t)(b * box_rows * TC * sizeof(V)), &map, 2 * it.tile * TC,
                  b * box_rows, rhs_of(it) * a.nplanes + it.plane, bar_in);
  };
  auto issue_spectrum = [&](unsigned item) {
    const ColItem it = col_item(item, (unsigned)nact, per_rhs, ntile, a.nplanes, slot_fast);
    const int l = a.freq_fixed >= 0 ? a.freq_fixed : (a.rhs0 + rhs_of(it)) / a.n_elem;
    tc::mbar_arrive_expect_tx(bar_g, g_bytes);
    tc::tma_load_3d(gst_a, &gmap, 2 * it.tile * TC, 0, l, bar_g);
  };

  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map)) : "memory");
    tc::mbar_init(bar_in, 1);
    tc::mbar_init(bar_g, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  for (int i = threadIdx.x; i < P::L; i += blockDim.x) tws[i] = a.tw[i];
  __syncthreads();
  if (threadIdx.x == 0 && blockIdx.x < items) {
    issue_input(blockIdx.x);
    if (use_g) issue_spectrum(blockIdx.x);
  }
  uint32_t par_in = 0, par_g = 0;
  bool failed = false, bad = false;
  // the spectrum wait and the issue of the next item's spectrum, called
  // from the transforms around their use of the staged tile
  struct Hook {
    uint32_t bar; uint32_t* par; volatile int* abort; int* err; bool* bad;
    unsigned next, items; const decltype(issue_spectrum)* issue;
    __device__ bool wait_spectrum() const {
      const bool ok = tc::mbar_wait(bar, *par, abort, err, kColErrWait);
      if (!ok) *bad = true;
      return ok;
    }
    __device__ void spectrum_done() const {
      *par ^= 1u;
      if (threadIdx.x == 0 && next < items && !*abort) (*issue)(next);
    }
  };
  for (unsigned item = blockIdx.x; item < items; item += gridDim.x) {
    const ColItem it = col_item(item, (unsigned)nact, per_rhs, ntile, a.nplanes, slot_fast);
    const int rhs = rhs_of(it);
    const int j = it.tile * TC + c;
    const bool ok = tc::mbar_wait(bar_in, par_in, abort_flag, err, kColErrWait);
    V v[P::E];
    if (a.mode == C_INV) {
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CB; ++i) {
#pragma unroll
        for (int kp = 0; kp < PlanTraits<P>::MB; ++kp) {
          int k1, k2;
          if (slotB<P, GP>(t, i, kp, k1, k2))
            v[i * PlanTraits<P>::MB + kp] = stg[(k1 + P::R1 * k2) * TC + c];
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < PlanTraits<P>::CA; ++i) {
#pragma unroll
        for (int m = 0; m < PlanTraits<P>::MA; ++m) {
          int n2, n1;
          const bool in = slotA<P, GP>(t, i, m, n2, n1);
          v[i * PlanTraits<P>::MA + m] =
              (in && n1 < P::H1) ? stg[(P::R2 * n1 + n2) * TC + c] : mk<float>(0.f, 0.f);
        }
      }
    }
    // every thread holds its samples (the input staging is free) and is
    // done with the previous item's exchange; a failed wait (this item's
    // input, or the previous item's spectrum) stops the CTA
    if (__syncthreads_or(!ok || bad)) {
      failed = true;
      break;
    }
    par_in ^= 1u;
    const unsigned next = item + gridDim.x;
    if (threadIdx.x == 0 && next < items) issue_input(next);
    V* __restrict__ out = a.out + rhs * a.out_rhs_stride + it.plane * a.out_plane_stride + j;
    if constexpr (GSTAGE) {
      const Hook hook{bar_g, &par_g, abort_flag, err, &bad, next, items, &issue_spectrum};
      col_transform_store<P, float, TC, true, Hook>(a, t, smc, v, rhs, j, out, tws,
                                                    use_g ? gst + c : nullptr, hook);
    } else {
      col_transform_store<P, float, TC, true>(a, t, smc, v, rhs, j, out, tws);
    }
  }
  // copies of a CTA that stopped early may still land in its shared memory
  if (failed && threadIdx.x == 0) {
    tc::mbar_wait_drain(bar_in, par_in, err, kColErrDrain);
    if (use_g) tc::mbar_wait_drain(bar_g, par_g, err, kColErrDrain);
  }
}

}  // namespace fwi

#include "col_pair.cuh"

namespace fwi {

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
template <> struct PlanFor<512> { using type = SPlan<512, 16, 32, 1, 2>; };
template <> struct PlanFor<640> { using type = Plan<640, 20, 32, 32>; };
template <> struct PlanFor<768> { using type = Plan<768, 24, 32, 32>; };
template <> struct PlanFor<1024> { using type = SPlan<1024, 32, 32, 2, 2>; };

#define FWI_FOR_EACH_L(X) \
  X(16) X(32) X(64) X(128) X(192) X(256) X(320) X(384) X(512) X(640) X(768) X(1024)

// Tile-shape variants (autotuned per context; results are identical for
// every variant): row passes with 128 / 64 / 256 threads per CTA, column
// passes with the default column-tile width or half of it.  Only the
// lengths of the benchmark grids carry the extra variants.
constexpr int kRowVariants = 3;
constexpr int kColVariants = 2;
template <int L> constexpr bool tuned_len() { return L == 256 || L == 320 || L == 512 || L == 1024; }

template <int L, int VAR> constexpr int row_lpc_v() {
  constexpr int tl = PlanFor<L>::type::TL;
  constexpr int threads = (VAR == 1) ? 64 : (VAR == 2) ? 256 : 128;
  return (threads / tl) > 0 ? threads / tl : 1;
}
template <int L> constexpr int row_lpc() { return row_lpc_v<L, 0>(); }

template <int L, typename T, int VAR> constexpr size_t row_smem_v() {
  using P = typename PlanFor<L>::type;
  return (size_t)row_lpc_v<L, VAR>() * (P::span(1) + 1) * sizeof(cplx<T>);
}

// Columns per tile: 128-byte row segments for FP32 up to L = 512; eight
// columns otherwise (at most 512 threads per tile); variant 1 halves it.
template <int L, typename T, int VAR> constexpr int col_tc_v() {
  constexpr int base = (sizeof(T) == 4 && L <= 512) ? 16 : 8;
  return VAR == 1 ? base / 2 : base;
}
template <int L, typename T> constexpr int col_tc() { return col_tc_v<L, T, 0>(); }

template <int L, typename T, int VAR> constexpr size_t col_smem_v() {
  return (size_t)L * col_tc_v<L, T, VAR>() * sizeof(cplx<T>);
}

// Persistent grid: resident CTAs per SM (occupancy) x SMs, cached per kernel
// (initialised once, thread-safe: contexts may run on several host threads).
struct GridCache { std::atomic<int> blocks{0}; };
inline std::mutex& grid_mutex() {
  static std::mutex m;
  return m;
}
template <int L, typename T, int KIND, int VAR> GridCache& gcache() {
  static GridCache g;
  return g;
}

// attr_smem: the kernel's dynamic shared-memory limit to set (at least
// smem; a kernel launched with several sizes gets the largest).
template <typename K>
inline cudaError_t grid_for(K kernel, int threads, size_t smem, GridCache& gc,
                            size_t attr_smem = 0) {
  if (gc.blocks.load(std::memory_order_acquire) > 0) return cudaSuccess;
  std::lock_guard<std::mutex> lock(grid_mutex());
  if (gc.blocks.load(std::memory_order_relaxed) > 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(attr_smem > smem ? attr_smem : smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  gc.blocks.store((per > 0 ? per : 1) * sms, std::memory_order_release);
  return cudaSuccess;
}

// Bulk copies start on 16-byte boundaries: every array the staged pass
// copies from must be 16-byte aligned (row starts row*nx and right-hand-side
// starts rhs*N are, since nx is even); otherwise the plain pass runs, as it
// does when the rows are not the half lattice (nx = L/2) the staging holds.
inline bool al16(const void* p) { return ((uintptr_t)p & 15) == 0; }
template <typename T> bool rf_stage_aligned(const RowFwdArgs<T>& a) {
  const bool ok = (a.N * (long long)sizeof(cplx<T>)) % 16 == 0 && (!a.use_m || al16(a.m));
  switch (a.mode) {
    case RF_PLAIN: case RF_INIT: return ok && al16(a.in);
    case RF_START: return ok && al16(a.P);
    case RF_ITER: return ok && al16(a.X) && al16(a.P) && al16(a.R) && al16(a.Tt) && al16(a.V);
    default: return ok && al16(a.R) && al16(a.V);
  }
}

// Dynamic shared memory of the staged forward row pass: exchange, 128-byte
// alignment slack, nsrc staged arrays of lpc lines of L/2 samples, mbarrier
// and abort flag.
template <int L, typename T, int VAR> constexpr size_t row_fwd_stage_smem(int nsrc) {
  return row_smem_v<L, T, VAR>() + 128 +
         (size_t)nsrc * row_lpc_v<L, VAR>() * (L / 2) * sizeof(cplx<T>) + 16;
}

// Staging pays while at least three CTAs fit per SM: the BiCGSTAB update
// mode's six arrays of 768-sample rows (about 100 KB) left two and made that
// pass 13 % slower than its plain loads, every other measured case is faster.
constexpr size_t kRowStageMaxSmem = 80 * 1024;

template <int L, typename T, int VAR>
cudaError_t launch_row_fwd(const RowFwdArgs<T>& a, cudaStream_t s) {
  using P = typename PlanFor<L>::type;
  constexpr int lpc = row_lpc_v<L, VAR>();
  if constexpr (sizeof(T) == 4) {
    const int nsrc = rf_stage_count(a.mode, a.use_m);
    if (a.stage && !a.full && 2 * a.nx == L && rf_stage_aligned(a) &&
        row_fwd_stage_smem<L, T, VAR>(nsrc) <= kRowStageMaxSmem) {
      auto k = row_fwd_kernel<P, T, lpc, true>;
      const size_t smem = row_fwd_stage_smem<L, T, VAR>(nsrc);
      // one occupancy per staged-array count (the modes differ in smem)
      GridCache& gc = nsrc <= 1 ? gcache<L, T, 11, VAR>()
                    : nsrc == 2 ? gcache<L, T, 12, VAR>()
                    : nsrc == 3 ? gcache<L, T, 13, VAR>()
                    : nsrc == 5 ? gcache<L, T, 15, VAR>()
                                : gcache<L, T, 16, VAR>();
      cudaError_t e = grid_for(k, lpc * P::TL, smem, gc, row_fwd_stage_smem<L, T, VAR>(6));
      if (e != cudaSuccess) return e;
      k<<<gc.blocks.load(), lpc * P::TL, smem, s>>>(a);
      return cudaGetLastError();
    }
  }
  auto k = row_fwd_kernel<P, T, lpc>;
  GridCache& gc = gcache<L, T, 0, VAR>();
  cudaError_t e = grid_for(k, lpc * P::TL, row_smem_v<L, T, VAR>(), gc);
  if (e != cudaSuccess) return e;
  k<<<gc.blocks.load(), lpc * P::TL, row_smem_v<L, T, VAR>(), s>>>(a);
  return cudaGetLastError();
}

template <int L, typename T, int VAR>
cudaError_t launch_row_inv(const RowInvArgs<T>& a, cudaStream_t s) {
  using P = typename PlanFor<L>::type;
  constexpr int lpc = row_lpc_v<L, VAR>();
  auto k = row_inv_kernel<P, T, lpc>;
  GridCache& gc = gcache<L, T, 1, VAR>();
  cudaError_t e = grid_for(k, lpc * P::TL, row_smem_v<L, T, VAR>(), gc);
  if (e != cudaSuccess) return e;
  k<<<gc.blocks.load(), lpc * P::TL, row_smem_v<L, T, VAR>(), s>>>(a);
  return cudaGetLastError();
}

// Tensor map of the kernel spectrum for the convolution's staging: rows
// 0..L/2 of TC columns of one frequency per box.  False when the box does
// not fit (L/2 + 1 > 256 rows) or the staging would cost occupancy.
template <int L, int TC>
bool col_spectrum_map(const ColArgs<float>& a, int rows_in, CUtensorMap* map) {
  if (!a.gstage || a.mode != C_CONV || !a.ghat || a.n_freq < 1) return false;
  if (L / 2 + 1 > 256 || ColTmaSmem<L, TC>::bytes(rows_in, true) > 76 * 1024) return false;
  tc::TensorMapEncodeFn enc = tc::tensor_map_encoder();
  if (!enc || ((uintptr_t)a.ghat & 15) || (a.ncols * 8) % 16 || (a.ghat_freq_stride * 8) % 16)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * a.ncols, (cuuint64_t)L, (cuuint64_t)a.n_freq};
  const cuuint64_t strides[2] = {(cuuint64_t)a.ncols * 8, (cuuint64_t)a.ghat_freq_stride * 8};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * TC), (cuuint32_t)(L / 2 + 1), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(a.ghat), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Tensor map of a column pass's input (see col_tma_kernel).  False when the
// pass does not fit the TMA path (then the plain kernel runs).
template <int L, int TC>
bool col_tensor_map(const ColArgs<float>& a, CUtensorMap* map, int* rows_in, int* nbox) {
  if (!a.tma || a.full) return false;
  tc::TensorMapEncodeFn enc = tc::tensor_map_encoder();
  if (!enc || a.nplanes < 1 || a.nb < 1 || a.ncols % TC) return false;
  const int rin = (a.mode == C_INV) ? L : L / 2;
  const int nb = (rin + 255) / 256;
  if (rin % nb) return false;
  if (a.in_rhs_stride % a.nplanes) return false;
  const long long pstride = a.in_rhs_stride / a.nplanes;
  if (a.nplanes > 1 && pstride != a.in_plane_stride) return false;
  if (((uintptr_t)a.in & 15) || (a.line_stride * 8) % 16 || (pstride * 8) % 16) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * a.ncols, (cuuint64_t)rin,
                              (cuuint64_t)a.nb * a.nplanes};
  const cuuint64_t strides[2] = {(cuuint64_t)a.line_stride * 8, (cuuint64_t)pstride * 8};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * TC), (cuuint32_t)(rin / nb), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(a.in), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  *rows_in = rin;
  *nbox = nb;
  return true;
}

// The two-column convolution stores 16-byte column pairs.
template <typename T> bool col_pair_ok(const ColArgs<T>& a) {
  return a.mode == C_CONV && a.pairs && a.ghat && ((uintptr_t)a.out & 15) == 0 &&
         a.out_rhs_stride % 2 == 0 && a.line_stride % 2 == 0 &&
         (a.nplanes == 1 || a.out_plane_stride % 2 == 0);
}

template <int L, typename T, int VAR>
cudaError_t launch_col(const ColArgs<T>& a, cudaStream_t s) {
  using P = typename PlanFor<L>::type;
  constexpr int tc = col_tc_v<L, T, VAR>();
  if constexpr (sizeof(T) == 4) {
    CUtensorMap map, gmap;
    int rows_in = 0, nbox = 0;
    if (col_tensor_map<L, tc>(a, &map, &rows_in, &nbox)) {
      using SM = ColTmaSmem<L, tc>;
      if constexpr (L / 2 + 1 <= 256) {
        if (col_spectrum_map<L, tc>(a, rows_in, &gmap)) {
          if constexpr (pair_plan<P>() && tc % 2 == 0) {
            if (col_pair_ok(a)) {
              auto k = col_pair_kernel<P, tc, true>;
              const size_t smem = ColPairSmem<L, tc>::bytes(rows_in, true);
              GridCache& gc = gcache<L, T, 6, VAR>();
              cudaError_t e = grid_for(k, tc / 2 * P::TL, smem, gc);
              if (e != cudaSuccess) return e;
              k<<<gc.blocks.load(), tc / 2 * P::TL, smem, s>>>(a, map, gmap, rows_in, nbox);
              return cudaGetLastError();
            }
          }
          auto k = col_tma_kernel<P, tc, true>;
          const size_t smem = SM::bytes(rows_in, true);
          GridCache& gc = gcache<L, T, 5, VAR>();
          cudaError_t e = grid_for(k, tc * P::TL, smem, gc);
          if (e != cudaSuccess) return e;
          k<<<gc.blocks.load(), tc * P::TL, smem, s>>>(a, map, gmap, rows_in, nbox);
          return cudaGetLastError();
        }
      }
      std::memset(&gmap, 0, sizeof(gmap));
      // The plain kernel's residency: the TMA kernel below runs only where
      // its staging buffer keeps at least as many CTAs per SM (the 768-point
      // columns' staging left two of three, and the pass ran 20 % slower).
      auto kp = col_kernel<P, T, tc>;
      GridCache& gcp = gcache<L, T, 2, VAR>();
      {
        cudaError_t e = grid_for(kp, tc * P::TL, col_smem_v<L, T, VAR>(), gcp);
        if (e != cudaSuccess) return e;
      }
      if constexpr (pair_plan<P>() && tc % 2 == 0) {
        // the spectrum from global memory (16-byte column pairs)
        if (col_pair_ok(a) && ((uintptr_t)a.ghat & 15) == 0 && a.ncols % 2 == 0 &&
            a.ghat_freq_stride % 2 == 0) {
          auto k = col_pair_kernel<P, tc, false>;
          const size_t smem = ColPairSmem<L, tc>::bytes(rows_in, false);
          GridCache& gc = gcache<L, T, 7, VAR>();
          cudaError_t e = grid_for(k, tc / 2 * P::TL, smem, gc);
          if (e != cudaSuccess) return e;
          k<<<gc.blocks.load(), tc / 2 * P::TL, smem, s>>>(a, map, gmap, rows_in, nbox);
          return cudaGetLastError();
        }
      }
      auto k = col_tma_kernel<P, tc, false>;
      const size_t smem = SM::bytes(rows_in, false);
      const size_t smem_max = SM::bytes(L, false);  // inverse mode: all L rows staged
      GridCache& gc = (a.mode == C_INV) ? gcache<L, T, 4, VAR>() : gcache<L, T, 3, VAR>();
      cudaError_t e = grid_for(k, tc * P::TL, smem, gc, smem_max);
      if (e != cudaSuccess) return e;
      if (gc.blocks.load() >= gcp.blocks.load()) {
        k<<<gc.blocks.load(), tc * P::TL, smem, s>>>(a, map, gmap, rows_in, nbox);
        return cudaGetLastError();
      }
    }
  }
  auto k = col_kernel<P, T, tc>;
  GridCache& gc = gcache<L, T, 2, VAR>();
  cudaError_t e = grid_for(k, tc * P::TL, col_smem_v<L, T, VAR>(), gc);
  if (e != cudaSuccess) return e;
  k<<<gc.blocks.load(), tc * P::TL, col_smem_v<L, T, VAR>(), s>>>(a);
  return cudaGetLastError();
}

// Variant dispatch: tuned lengths of the FP32 path carry every variant, all
// other (length, precision) pairs only the default.
template <int L, typename T> constexpr bool has_variants() {
  return tuned_len<L>() && sizeof(T) == 4;
}

template <int L, typename T>
cudaError_t row_fwd_v(int var, const RowFwdArgs<T>& a, cudaStream_t s) {
  if constexpr (has_variants<L, T>()) {
    if (var == 1) return launch_row_fwd<L, T, 1>(a, s);
    if (var == 2) return launch_row_fwd<L, T, 2>(a, s);
  }
  return launch_row_fwd<L, T, 0>(a, s);
}
template <int L, typename T>
cudaError_t row_inv_v(int var, const RowInvArgs<T>& a, cudaStream_t s) {
  if constexpr (has_variants<L, T>()) {
    if (var == 1) return launch_row_inv<L, T, 1>(a, s);
    if (var == 2) return launch_row_inv<L, T, 2>(a, s);
  }
  return launch_row_inv<L, T, 0>(a, s);
}
template <int L, typename T>
cudaError_t col_v(int var, const ColArgs<T>& a, cudaStream_t s) {
  if constexpr (has_variants<L, T>()) {
    if (var == 1) return launch_col<L, T, 1>(a, s);
  }
  return launch_col<L, T, 0>(a, s);
}
template <int L, typename T> int row_lpc_of(int var) {
  if constexpr (has_variants<L, T>()) {
    if (var == 1) return row_lpc_v<L, 1>();
    if (var == 2) return row_lpc_v<L, 2>();
  }
  return row_lpc_v<L, 0>();
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
  template <> int Lsop<TYPE>::variants(int L, int kind) {                             \
    const bool t = (sizeof(TYPE) == 4) &&                                             \
                   (L == 256 || L == 320 || L == 512 || L == 1024);                   \
    return t ? (kind == 2 ? kColVariants : kRowVariants) : 1;                         \
  }                                                                                   \
  template <> int Lsop<TYPE>::row_lines_per_cta(int L, int var) {                     \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_LPC_CASE)                                                    \
      default: return 0;                                                              \
    }                                                                                 \
  }                                                                                   \
  template <> cudaError_t Lsop<TYPE>::row_fwd(int L, const RowFwdArgs<TYPE>& a,       \
                                              cudaStream_t s, int var) {              \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_ROWFWD_CASE)                                                 \
      default: return cudaErrorInvalidValue;                                          \
    }                                                                                 \
  }                                                                                   \
  template <> cudaError_t Lsop<TYPE>::row_inv(int L, const RowInvArgs<TYPE>& a,       \
                                              cudaStream_t s, int var) {              \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_ROWINV_CASE)                                                 \
      default: return cudaErrorInvalidValue;                                          \
    }                                                                                 \
  }                                                                                   \
  template <> cudaError_t Lsop<TYPE>::col(int L, const ColArgs<TYPE>& a,              \
                                          cudaStream_t s, int var) {                  \
    switch (L) {                                                                      \
      FWI_FOR_EACH_L(FWI_COL_CASE)                                                    \
      default: return cudaErrorInvalidValue;                                          \
    }                                                                                 \
  }

#define FWI_LPC_CASE(LL) case LL: return row_lpc_of<LL, FWI_T>(var);
#define FWI_ROWFWD_CASE(LL) case LL: return row_fwd_v<LL, FWI_T>(var, a, s);
#define FWI_ROWINV_CASE(LL) case LL: return row_inv_v<LL, FWI_T>(var, a, s);
#define FWI_COL_CASE(LL) case LL: return col_v<LL, FWI_T>(var, a, s);

}  // namespace fwi
