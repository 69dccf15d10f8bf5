// Convolution pass with two columns per thread (FP32; plans listed at
// pair_plan: power-of-two DFTs, whole first DFTs per thread).
//
// The transforms are the four-step FFT of fft_core.cuh (forward FFT along
// the column with the zero-padded half pruned, product with the kernel
// spectrum, inverse FFT with the cropped half pruned; Eq. 5, Sec. IV-A),
// computed for the columns 2p and 2p + 1 of a tile together: a value pair
// PC holds the two columns' real parts in one f32x2 register pair and their
// imaginary parts in another.  Every butterfly is then a packed
// add.rn.f32x2 / sub.rn.f32x2 on operands that already sit in register
// pairs, and a product by a twiddle (the same for both columns) is four or
// five packed multiplies and adds instead of eight scalar ones; the
// shared-memory exchange moves 16 bytes per access.  Rounding: every packed
// operation rounds each lane exactly as the scalar operation would; the
// products are formed as re*c - im*s with one rounding per product and per
// sum, so results agree with the one-column kernel to FP32 rounding.
//
// The rest follows col_tma_kernel: persistent CTAs over the slot-fast item
// order, the next item's input tile (and, where it fits, its kernel-spectrum
// tile) staged by TMA into shared memory while the current item transforms,
// bounded mbarrier waits with the same error codes.  Split plans share their
// second DFTs over a lane pair, exchanging column pairs by warp shuffles.
#pragma once

namespace fwi {
namespace pair {

using u64 = unsigned long long;
// Two complex values (columns a and b): re = (re_a, re_b), im = (im_a, im_b).
struct PC {
  u64 re, im;
};

__device__ __forceinline__ u64 pk(float x, float y) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void upk(u64 v, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}
__device__ __forceinline__ u64 f2add(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 f2sub(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 f2mul(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// a * b + c
__device__ __forceinline__ u64 f2fma(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ u64 f2neg(u64 a) { return f2mul(a, pk(-1.f, -1.f)); }

__device__ __forceinline__ PC padd(PC a, PC b) { return {f2add(a.re, b.re), f2add(a.im, b.im)}; }
__device__ __forceinline__ PC psub(PC a, PC b) { return {f2sub(a.re, b.re), f2sub(a.im, b.im)}; }

// 16-byte shared-memory access of a pair stored as (re_a, re_b, im_a, im_b)
__device__ __forceinline__ PC lds_pc(const float4* p) {
  PC v;
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];"
               : "=l"(v.re), "=l"(v.im)
               : "r"(tc::smem_addr(p)));
  return v;
}
__device__ __forceinline__ void sts_pc(float4* p, PC v) {
  asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(tc::smem_addr(p)), "l"(v.re), "l"(v.im)
               : "memory");
}
// Two interleaved complex values (re_a, im_a, re_b, im_b) -> pair
__device__ __forceinline__ PC from_interleaved(float4 q) { return {pk(q.x, q.z), pk(q.y, q.w)}; }
__device__ __forceinline__ float4 to_interleaved(PC v) {
  float4 q;
  upk(v.re, q.x, q.z);
  upk(v.im, q.y, q.w);
  return q;
}

// z * w_R^J (forward) or z * conj(w_R^J) (inverse), J known at compile time.
template <int J, int R, bool INV> __device__ __forceinline__ PC ptw_ct(PC z) {
  constexpr int q = tw_quarter(J, R);
  if constexpr (q == 0) {
    return z;
  } else if constexpr (q == 2) {
    return {f2neg(z.re), f2neg(z.im)};
  } else if constexpr ((q == 1) != INV && (q == 1 || q == 3)) {
    return {z.im, f2neg(z.re)};  // * (-i)
  } else if constexpr (q == 1 || q == 3) {
    return {f2neg(z.im), z.re};  // * (+i)
  } else {
    constexpr float c = (float)tw_re(J, R);
    constexpr float s = INV ? (float)-tw_im(J, R) : (float)tw_im(J, R);
    // (re c - im s, re s + im c)
    return {f2fma(z.re, pk(c, c), f2mul(z.im, pk(-s, -s))),
            f2fma(z.re, pk(s, s), f2mul(z.im, pk(c, c)))};
  }
}
// z * (c + i s), the same twiddle for both columns, from the pair table
__device__ __forceinline__ PC ptw_tab(PC z, u64 cc, u64 ss) {
  return {f2sub(f2mul(z.re, cc), f2mul(z.im, ss)), f2fma(z.re, ss, f2mul(z.im, cc))};
}
// z * (c - i s)
__device__ __forceinline__ PC ptw_tab_conj(PC z, u64 cc, u64 ss) {
  return {f2fma(z.im, ss, f2mul(z.re, cc)), f2sub(f2mul(z.im, cc), f2mul(z.re, ss))};
}
// z * g with a different g per column: gr = (gr_a, gr_b), gi = (gi_a, gi_b)
__device__ __forceinline__ PC pmul(PC z, u64 gr, u64 gi) {
  return {f2sub(f2mul(z.re, gr), f2mul(z.im, gi)), f2fma(z.re, gi, f2mul(z.im, gr))};
}

// In-register DFT of size R (a power of two), natural order, in place.
template <int R, bool INV> struct PDft;
template <bool INV> struct PDft<1, INV> {
  static __device__ __forceinline__ void run(PC*) {}
};
template <bool INV> struct PDft<2, INV> {
  static __device__ __forceinline__ void run(PC* x) {
    const PC a = x[0], b = x[1];
    x[0] = padd(a, b);
    x[1] = psub(a, b);
  }
};
template <bool INV> struct PDft<4, INV> {
  static __device__ __forceinline__ void run(PC* x) {
    const PC a0 = padd(x[0], x[2]), a1 = psub(x[0], x[2]);
    const PC b0 = padd(x[1], x[3]), d = psub(x[1], x[3]);
    x[0] = padd(a0, b0);
    x[2] = psub(a0, b0);
    // X1 = a1 + w d, X3 = a1 - w d with w = -i (forward) or +i (inverse)
    if constexpr (!INV) {
      x[1] = {f2add(a1.re, d.im), f2sub(a1.im, d.re)};
      x[3] = {f2sub(a1.re, d.im), f2add(a1.im, d.re)};
    } else {
      x[1] = {f2sub(a1.re, d.im), f2add(a1.im, d.re)};
      x[3] = {f2add(a1.re, d.im), f2sub(a1.im, d.re)};
    }
  }
};
// R = A * B: A-point DFTs over n1 (n = B n1 + n2), twiddle w_R^{n2 k1},
// B-point DFTs over n2; output index k = k1 + A k2.
template <int R, bool INV> struct PDft {
  static constexpr int A = first_factor(R);
  static constexpr int B = R / A;
  static_assert((R & (R - 1)) == 0 && A * B == R && B > 1, "power-of-two sizes only");
  static __device__ __forceinline__ void run(PC* x) {
    PC y[R];
    SFor<B>::run([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      PC t[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n1] = x[B * n1 + n2];
      PDft<A, INV>::run(t);
      SFor<A>::run([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        y[n2 * A + k1] = ptw_ct<(n2 * k1) % R, R, INV>(t[k1]);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      PC u[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) u[n2] = y[n2 * A + k1];
      PDft<B, INV>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = u[k2];
    }
  }
};
// R-point DFT whose inputs x[R/2 .. R) are zero.
template <int R, bool INV> struct PDftHalfIn {
  static __device__ __forceinline__ void run(PC* x) {
    constexpr int H = R / 2;
    PC a[H], b[H];
    SFor<H>::run([&](auto nc) {
      constexpr int n = decltype(nc)::value;
      a[n] = x[n];
      b[n] = ptw_ct<n, R, INV>(x[n]);
    });
    PDft<H, INV>::run(a);
    PDft<H, INV>::run(b);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      x[2 * k] = a[k];
      x[2 * k + 1] = b[k];
    }
  }
};
// R-point DFT of which only the outputs x[0 .. R/2) are formed.
template <int R, bool INV> struct PDftHalfOut {
  static __device__ __forceinline__ void run(PC* x) {
    constexpr int H = R / 2;
    PC a[H], b[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      a[k] = x[2 * k];
      b[k] = x[2 * k + 1];
    }
    PDft<H, INV>::run(a);
    PDft<H, INV>::run(b);
    SFor<H>::run([&](auto nc) {
      constexpr int n = decltype(nc)::value;
      x[n] = padd(a[n], ptw_ct<n, R, INV>(b[n]));
    });
  }
};

// Exchange of a pair with the partner lane of a split DFT (16 lanes away).
__device__ __forceinline__ PC shfl_pc(PC a) {
  float x0, x1, y0, y1;
  upk(a.re, x0, x1);
  upk(a.im, y0, y1);
  x0 = __shfl_xor_sync(0xffffffffu, x0, 16);
  x1 = __shfl_xor_sync(0xffffffffu, x1, 16);
  y0 = __shfl_xor_sync(0xffffffffu, y0, 16);
  y1 = __shfl_xor_sync(0xffffffffu, y1, 16);
  return {pk(x0, x1), pk(y0, y1)};
}
// z * (h w + (1 - h)) with w = w_R^J (conjugated for INV): lane h = 0 keeps
// z, lane 1 gets z w (hf = h, hc = 1 - h are exactly 0 or 1)
template <int J, int R, bool INV>
__device__ __forceinline__ PC plane_twiddle(PC z, float hf, float hc) {
  constexpr int q = tw_quarter(J, R);
  if constexpr (q == 0) {
    return z;
  } else {
    constexpr double wr = q == 2 ? -1.0 : (q == 1 || q == 3) ? 0.0 : tw_re(J, R);
    constexpr double wf = q == 1 ? -1.0 : q == 3 ? 1.0 : q == 2 ? 0.0 : tw_im(J, R);
    constexpr double wi = INV ? -wf : wf;
    const float av = hf * (float)wr + hc;
    const float bv = hf * (float)wi;
    return ptw_tab(z, pk(av, av), pk(bv, bv));
  }
}
// R = 2Q point DFT over a lane pair (lanes 16 apart).  split: lane h holds
// x[2m + h] (m < Q) and ends with X[k + Q h] (k < Q).  isplit: lane h holds
// X[k + Q h] and ends with x[2m + h] (unnormalised).
template <int Q, bool INV> __device__ __forceinline__ void psplit_dft(PC* u, int h) {
  PDft<Q, INV>::run(u);
  const float hf = (float)h, hc = (float)(1 - h), sg = (float)(1 - 2 * h);
  const u64 sgp = pk(sg, sg);
  SFor<Q>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const PC v = plane_twiddle<k, 2 * Q, INV>(u[k], hf, hc);
    const PC o = shfl_pc(v);
    u[k] = {f2fma(sgp, v.re, o.re), f2fma(sgp, v.im, o.im)};
  });
}
template <int Q, bool INV> __device__ __forceinline__ void psplit_idft(PC* u, int h) {
  const float hf = (float)h, hc = (float)(1 - h), sg = (float)(1 - 2 * h);
  const u64 sgp = pk(sg, sg);
  SFor<Q>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const PC own = u[k];
    const PC o = shfl_pc(own);
    const PC z = {f2fma(sgp, own.re, o.re), f2fma(sgp, own.im, o.im)};
    u[k] = plane_twiddle<k, 2 * Q, INV>(z, hf, hc);
  });
  PDft<Q, INV>::run(u);
}

}  // namespace pair

constexpr bool pow2_at_least(int r, int m) { return r >= m && (r & (r - 1)) == 0; }

// Plans the two-column kernel covers: unsplit plans with one thread per n2
// and per k1 (R1 = R2 = TL), and split plans whose first DFTs are whole
// (S1 = 1) and whose second DFTs are shared by a lane pair (S2 = 2); all
// DFT sizes powers of two.
template <class P> constexpr bool pair_plan() {
  if constexpr (PlanTraits<P>::split) {
    return P::S1 == 1 && P::S2 == 2 && pow2_at_least(P::R1, 4) && pow2_at_least(P::Q2, 2);
  } else {
    return P::R1 == P::TL && P::R2 == P::TL && pow2_at_least(P::R1, 4);
  }
}

// Shared memory (bytes from the 128-byte aligned base): exchange L x TC/2
// pairs (16 bytes each) | input staging rows_in x TC | spectrum staging
// (L/2 + 1) x TC (GS only) | pair twiddle table L x (c, c, s, s) | two
// mbarriers and the abort flag.
template <int L, int TC> struct ColPairSmem {
  static constexpr int G_ROWS = L / 2 + 1;
  static constexpr size_t bytes(int rows_in, bool gs) {
    return ((size_t)L * TC + (size_t)rows_in * TC + (gs ? (size_t)G_ROWS * TC : 0)) *
               sizeof(float2) +
           (size_t)L * sizeof(float4) + 32 + 128;
  }
};

// GS: the kernel spectrum tile of each item is staged by TMA (rows 0..L/2);
// otherwise each thread reads its spectrum pairs from global memory (L2).
// Registers: 168 keeps three 128-thread CTAs per SM (the shared memory of
// the 256-point convolution holds three as well); 256-thread CTAs get 128
// (two per SM).
constexpr int pair_regs(int threads) { return threads > 128 ? 128 : 168; }
template <class P, int TC, bool GS>
__global__ void __launch_bounds__(TC / 2 * P::TL,
                                  blocks_for_regs(TC / 2 * P::TL, pair_regs(TC / 2 * P::TL)))
col_pair_kernel(const ColArgs<float> a, const __grid_constant__ CUtensorMap map,
                const __grid_constant__ CUtensorMap gmap, int rows_in, int nbox) {
  using namespace pair;
  static_assert(pair_plan<P>(), "two-column plan");
  constexpr bool SPLIT = PlanTraits<P>::split;
  constexpr int NP = TC / 2;  // column pairs per tile
  constexpr int GP = 32 / NP;  // consecutive line threads per warp
  constexpr int R1 = P::R1, R2 = P::R2, H1 = P::H1;
  constexpr int NB = PlanTraits<P>::MB;  // phase-B values per thread (R2, or Q2 split)
  constexpr int G_ROWS = ColPairSmem<P::L, TC>::G_ROWS;
  extern __shared__ __align__(16) unsigned char smraw[];
  const uint32_t base_pad = (128u - (tc::smem_addr(smraw) & 127u)) & 127u;
  float4* ex = reinterpret_cast<float4*>(smraw + base_pad);        // exchange, L x NP
  float2* stg = reinterpret_cast<float2*>(ex + P::L * NP);         // input staging
  float2* gst = stg + rows_in * TC;                                // spectrum staging
  float4* twp = reinterpret_cast<float4*>(gst + (GS ? G_ROWS * TC : 0));  // pair twiddles
  uint64_t* bar = reinterpret_cast<uint64_t*>(twp + P::L);         // [0] input, [1] spectrum
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 2);
  const uint32_t bar_in = tc::smem_addr(bar), bar_g = tc::smem_addr(bar + 1);
  const uint32_t stg_a = tc::smem_addr(stg), gst_a = tc::smem_addr(gst);
  const float4* stg4 = reinterpret_cast<const float4*>(stg);
  const float4* gst4 = reinterpret_cast<const float4*>(gst);
  const int cp = threadIdx.x % NP;  // column pair 2cp, 2cp + 1 of the tile
  const int t = threadIdx.x / NP;   // thread of the line (owns n2 = t in phases A, D)
  // phases B, C: this thread's k1 and, split, its half h of the lane pair
  int kb, h = 0;
  if constexpr (SPLIT) decode<2, GP>(t, kb, h);
  else kb = t;
  const unsigned ntile = (unsigned)(a.ncols / TC);
  const unsigned per_rhs = (unsigned)a.nplanes * ntile;
  const int nact = a.active ? *a.n_active : a.nb;
  const unsigned items = (unsigned)nact * per_rhs;  // < 2^31 (fwi_create caps the batch)
  const int box_rows = rows_in / nbox;
  const uint32_t tile_bytes = (uint32_t)(rows_in * TC * sizeof(float2));
  const uint32_t g_bytes = (uint32_t)(G_ROWS * TC * sizeof(float2));
  const long long ls = a.line_stride;
  int dummy_err = 0;
  int* err = a.err ? a.err : &dummy_err;

  auto rhs_of = [&](const ColItem& it) { return a.active ? a.active[it.slot] : it.slot; };
  auto issue_input = [&](unsigned item) {
    const ColItem it = col_item(item, (unsigned)nact, per_rhs, ntile, a.nplanes, true);
    tc::mbar_arrive_expect_tx(bar_in, tile_bytes);
    for (int b = 0; b < nbox; ++b)
      tc::tma_load_3d(stg_a + (uint32_t)(b * box_rows * TC * sizeof(float2)), &map,
                      2 * it.tile * TC, b * box_rows, rhs_of(it) * a.nplanes + it.plane, bar_in);
  };
  auto issue_spectrum = [&](unsigned item) {
    const ColItem it = col_item(item, (unsigned)nact, per_rhs, ntile, a.nplanes, true);
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
  for (int i = threadIdx.x; i < P::L; i += blockDim.x) {
    const float2 w = a.tw[i];
    twp[i] = make_float4(w.x, w.x, w.y, w.y);
  }
  __syncthreads();
  if (threadIdx.x == 0 && blockIdx.x < items) {
    issue_input(blockIdx.x);
    if (GS) issue_spectrum(blockIdx.x);
  }
  uint32_t par_in = 0, par_g = 0;
  bool failed = false, bad = false;
  for (unsigned item = blockIdx.x; item < items; item += gridDim.x) {
    const ColItem it = col_item(item, (unsigned)nact, per_rhs, ntile, a.nplanes, true);
    const int j = it.tile * TC + 2 * cp;
    const bool ok = tc::mbar_wait(bar_in, par_in, abort_flag, err, kColErrWait);
    PC v[P::E];
    const u64 zero = pk(0.f, 0.f);
    // phase-A samples x[R2 n1 + t] (n1 < R1/2; the rest is the zero padding)
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1)
      v[n1] = (n1 < H1) ? from_interleaved(stg4[(R2 * n1 + t) * NP + cp]) : PC{zero, zero};
    // every thread holds its samples (the input staging is free) and is done
    // with the previous item's exchange; a failed wait (this item's input,
    // or the previous item's spectrum) stops the CTA
    if (__syncthreads_or(!ok || bad)) {
      failed = true;
      break;
    }
    par_in ^= 1u;
    const unsigned next = item + gridDim.x;
    if (threadIdx.x == 0 && next < items) issue_input(next);
    float2* __restrict__ out =
        a.out + rhs_of(it) * a.out_rhs_stride + it.plane * a.out_plane_stride + j;

    // phase A: R1-point DFTs, twiddle w_L^{t k1}, y[t][k1] to the exchange
    PDftHalfIn<R1, false>::run(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      PC z = v[k1];
      if (k1 > 0 && t > 0) {
        const float4 w = twp[t * k1];
        z = ptw_tab(z, pk(w.x, w.y), pk(w.z, w.w));
      }
      sts_pc(ex + (t * R1 + k1) * NP + cp, z);
    }
    // one thread waits for the staged spectrum; the barrier hands its
    // completion (and the copied data) to the others
    if (GS && threadIdx.x == 0 && !tc::mbar_wait(bar_g, par_g, abort_flag, err, kColErrWait))
      bad = true;
    __syncthreads();
    // phase B: R2-point DFTs over n2 (split: over the lane pair, n2 = 2m + h);
    // v[kp] = X[kb + R1 k2] with k2 = kp (split: kp + Q2 h)
#pragma unroll
    for (int m = 0; m < NB; ++m) {
      const int n2 = SPLIT ? 2 * m + h : m;
      v[m] = lds_pc(ex + (n2 * R1 + kb) * NP + cp);
    }
    if constexpr (SPLIT) psplit_dft<NB, false>(v, h);
    else PDft<R2, false>::run(v);
    // product with the kernel spectrum (rows folded onto 0..L/2): the
    // staged tile, or the columns (j, j + 1) of this item's frequency
    const float4* __restrict__ gg = nullptr;
    if constexpr (!GS) {
      const int l = a.freq_fixed >= 0 ? a.freq_fixed : (a.rhs0 + rhs_of(it)) / a.n_elem;
      gg = reinterpret_cast<const float4*>(a.ghat + (long long)l * a.ghat_freq_stride + j);
    }
#pragma unroll
    for (int kp = 0; kp < NB; ++kp) {
      const int row = spectrum_row<P>(kb, SPLIT ? kp + NB * h : kp, kp);
      float4 g;
      if constexpr (GS) g = gst4[row * NP + cp];
      else g = __ldg(gg + (long long)row * (a.ncols / 2));
      v[kp] = pmul(v[kp], pk(g.x, g.z), pk(g.y, g.w));
    }
    if constexpr (GS) {
      __syncthreads();
      // every thread is done with the staged spectrum: stage the next one
      par_g ^= 1u;
      if (threadIdx.x == 0 && next < items && !*abort_flag) issue_spectrum(next);
    } else {
      __syncthreads();  // every thread has read its phase-B values
    }
    // phase C: inverse DFTs over k2, twiddle w_L^{-n2 kb}, y[n2][kb]
    if constexpr (SPLIT) psplit_idft<NB, true>(v, h);
    else PDft<R2, true>::run(v);
#pragma unroll
    for (int m = 0; m < NB; ++m) {
      const int n2 = SPLIT ? 2 * m + h : m;
      PC z = v[m];
      if (n2 > 0 && kb > 0) {
        const float4 w = twp[n2 * kb];
        z = ptw_tab_conj(z, pk(w.x, w.y), pk(w.z, w.w));
      }
      sts_pc(ex + (n2 * R1 + kb) * NP + cp, z);
    }
    __syncthreads();
    // phase D: inverse R1-point DFTs of which the cropped half is formed
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = lds_pc(ex + (t * R1 + k1) * NP + cp);
    PDftHalfOut<R1, true>::run(v);
#pragma unroll
    for (int n1 = 0; n1 < H1; ++n1)
      *reinterpret_cast<float4*>(out + (long long)(R2 * n1 + t) * ls) = to_interleaved(v[n1]);
  }
  // copies of a CTA that stopped early may still land in its shared memory
  if (failed && threadIdx.x == 0) {
    tc::mbar_wait_drain(bar_in, par_in, err, kColErrDrain);
    if (GS) tc::mbar_wait_drain(bar_g, par_g, err, kColErrDrain);
  }
}

}  // namespace fwi
