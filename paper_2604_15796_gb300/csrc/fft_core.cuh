// Register/shared-memory FFT building blocks for the Lippmann-Schwinger
// convolution of Sec. IV-A (K w = IFFT(Ghat_hat . FFT(pad(w))), cropped).
//
// One transform line of length L = R1 * R2 is computed with the four-step
// factorisation (index n = R2*n1 + n2, frequency k = k1 + R1*k2):
//
//   X[k1 + R1 k2] = sum_{n2} w_R2^{n2 k2} w_L^{n2 k1} sum_{n1} x[R2 n1 + n2] w_R1^{n1 k1}
//
// phase A: each thread owns columns n2 and does the R1-point DFTs in
//          registers, multiplies by w_L^{n2 k1} and writes the result to
//          shared memory;
// phase B: each thread owns rows k1, reads them back and does the R2-point
//          DFTs in registers; X[k1 + R1 k2] then sits in the registers of
//          the thread owning k1.
// The inverse runs the two phases in the opposite order with conjugate
// twiddles (phase C then phase D), without the 1/L factor.  Input and
// output are in natural order, and the global-memory side of each phase is
// coalesced: consecutive threads own consecutive n2 (or k1).
//
// Zero padding and cropping of the doubled lattice (inputs x[n] = 0 for
// n >= L/2, outputs needed only for n < L/2) are exploited in phases A and
// D: only n1 < R1/2 is loaded and only n1 < R1/2 is produced.
//
// The code is plain arithmetic on arrays (no intrinsics) so that it also
// compiles as host C++ for index-logic unit tests.
#pragma once

#include <vector_types.h>

#if defined(__CUDACC__)
#define FWI_HD __host__ __device__ __forceinline__
#else
#define FWI_HD inline
#endif

// Read-only (texture-path) load on the device, plain load on the host.
#if defined(__CUDA_ARCH__)
#define FWI_LDG(p) __ldg(p)
#else
#define FWI_LDG(p) (*(p))
#endif

namespace fwi {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename T> FWI_HD cplx<T> mk(T re, T im) { cplx<T> z; z.x = re; z.y = im; return z; }
template <typename V> FWI_HD V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> FWI_HD V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
#if defined(__CUDA_ARCH__)
// FP32 complex add / subtract as one packed f32x2 instruction (sm_100+):
// both lanes are rounded exactly as the two scalar operations would be.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  unsigned long long ua, ub, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ua) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(ub) : "f"(b.x), "f"(b.y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(ua), "l"(ub));
  float2 o;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
  return o;
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  unsigned long long ua, ub, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ua) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(ub) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(ua), "l"(ub));
  float2 o;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
  return o;
}
#endif
template <typename V> FWI_HD V cmul(V a, V b) {
  V z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// a * conj(b)
template <typename V> FWI_HD V cmulc(V a, V b) {
  V z; z.x = a.x * b.x + a.y * b.y; z.y = a.y * b.x - a.x * b.y; return z;
}
template <typename V> FWI_HD V cconj(V a) { a.y = -a.y; return a; }
// Twiddle-table element: from shared memory (TWS) or through the read-only
// path from global memory.
template <bool TWS, typename V> FWI_HD V tw_at(const V* p) {
  if constexpr (TWS) return *p;
  else return FWI_LDG(p);
}
template <typename V, typename S> FWI_HD V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> FWI_HD V mul_mi(V a) {
  V z;
  if (INV) { z.x = -a.y; z.y = a.x; } else { z.x = a.y; z.y = -a.x; }
  return z;
}

// ---------------------------------------------------------------------------
// Compile-time twiddles w_R^j = exp(-2 pi i j / R) for the in-register DFTs.
// Evaluated by a Taylor series after reduction of the angle to [-pi, pi];
// multiples of pi/2 are exact.  Only ever evaluated in constant expressions.
constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double ct_sin(double x) {
  double term = x, sum = x;
  for (int n = 1; n < 22; ++n) {
    term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double ct_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 22; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
// angle of exp(-2 pi i j / R) reduced to (-pi, pi]
constexpr double ct_angle(int j, int R) {
  int a = ((j % R) + R) % R;
  double t = -2.0 * kPi * (double)a / (double)R;
  if (2 * a > R) t += 2.0 * kPi;
  return t;
}
constexpr double tw_re(int j, int R) { return ct_cos(ct_angle(j, R)); }
constexpr double tw_im(int j, int R) { return ct_sin(ct_angle(j, R)); }
// quarter-turn index of w_R^j if it is one of 1, -i, -1, +i, else -1
constexpr int tw_quarter(int j, int R) {
  return ((4 * j) % R == 0) ? ((4 * j / R) % 4) : -1;
}

template <int V> struct IC { static constexpr int value = V; };
// Compile-time loop: f(IC<0>{}), ..., f(IC<N-1>{}).
template <int N> struct SFor {
  template <int I = 0, class F> static FWI_HD void run(const F& f) {
    if constexpr (I < N) {
      f(IC<I>{});
      run<I + 1>(f);
    }
  }
};

// z * w_R^J (forward) or z * conj(w_R^J) (inverse), J known at compile time.
template <int J, int R, bool INV, typename V> FWI_HD V twiddle_ct(V z) {
  constexpr int q = tw_quarter(J, R);
  if constexpr (q == 0) {
    return z;
  } else if constexpr (q == 2) {
    z.x = -z.x; z.y = -z.y; return z;
  } else if constexpr (q == 1) {
    return mul_mi<INV>(z);
  } else if constexpr (q == 3) {
    return mul_mi<!INV>(z);
  } else {
    using S = decltype(z.x);
    constexpr double wr = tw_re(J, R);
    constexpr double wi = INV ? -tw_im(J, R) : tw_im(J, R);
    V w; w.x = S(wr); w.y = S(wi);
    return cmul(z, w);
  }
}

// ---------------------------------------------------------------------------
// In-register DFT of compile-time size R, natural order in and out, in place.
// INV selects exp(+2 pi i jk / R) (unnormalised).
template <int R, bool INV, typename T> struct Dft;

template <bool INV, typename T> struct Dft<1, INV, T> {
  static FWI_HD void run(cplx<T>*) {}
};
template <bool INV, typename T> struct Dft<2, INV, T> {
  static FWI_HD void run(cplx<T>* x) {
    cplx<T> a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};
template <bool INV, typename T> struct Dft<3, INV, T> {
  static FWI_HD void run(cplx<T>* x) {
    const T c1 = T(-0.5);
    const T s1 = T(INV ? 0.86602540378443864676 : -0.86602540378443864676);
    cplx<T> a = x[0], b = x[1], c = x[2];
    cplx<T> sp = cadd(b, c), sm = csub(b, c);
    x[0] = cadd(a, sp);
    cplx<T> t = mk<T>(a.x + c1 * sp.x, a.y + c1 * sp.y);
    // s1 * i * sm
    cplx<T> u = mk<T>(-s1 * sm.y, s1 * sm.x);
    x[1] = cadd(t, u);
    x[2] = csub(t, u);
  }
};
template <bool INV, typename T> struct Dft<4, INV, T> {
  static FWI_HD void run(cplx<T>* x) {
    cplx<T> a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
    cplx<T> b0 = cadd(x[1], x[3]), b1 = mul_mi<INV>(csub(x[1], x[3]));
    x[0] = cadd(a0, b0);
    x[2] = csub(a0, b0);
    x[1] = cadd(a1, b1);
    x[3] = csub(a1, b1);
  }
};
template <bool INV, typename T> struct Dft<5, INV, T> {
  static FWI_HD void run(cplx<T>* x) {
    // direct evaluation with cos/sin of 2 pi/5 and 4 pi/5
    const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);
    const T s1 = T(INV ? 0.95105651629515357212 : -0.95105651629515357212);
    const T s2 = T(INV ? 0.58778525229247312917 : -0.58778525229247312917);
    cplx<T> a = x[0];
    cplx<T> p1 = cadd(x[1], x[4]), m1 = csub(x[1], x[4]);
    cplx<T> p2 = cadd(x[2], x[3]), m2 = csub(x[2], x[3]);
    x[0] = cadd(a, cadd(p1, p2));
    cplx<T> t1 = mk<T>(a.x + c1 * p1.x + c2 * p2.x, a.y + c1 * p1.y + c2 * p2.y);
    cplx<T> t2 = mk<T>(a.x + c2 * p1.x + c1 * p2.x, a.y + c2 * p1.y + c1 * p2.y);
    // i * (s1 m1 + s2 m2), i * (s2 m1 - s1 m2)
    cplx<T> u1 = mk<T>(-(s1 * m1.y + s2 * m2.y), s1 * m1.x + s2 * m2.x);
    cplx<T> u2 = mk<T>(-(s2 * m1.y - s1 * m2.y), s2 * m1.x - s1 * m2.x);
    x[1] = cadd(t1, u1);
    x[4] = csub(t1, u1);
    x[2] = cadd(t2, u2);
    x[3] = csub(t2, u2);
  }
};

constexpr int first_factor(int R) {
  return (R % 4 == 0 && R != 4) ? 4 : (R % 2 == 0 ? 2 : (R % 3 == 0 ? 3 : 5));
}

// Composite R = A * B: A-point DFTs over n1 (n = B n1 + n2), twiddle
// w_R^{n2 k1}, B-point DFTs over n2; output index k = k1 + A k2.
template <int R, bool INV, typename T> struct Dft {
  static constexpr int A = first_factor(R);
  static constexpr int B = R / A;
  static_assert(A * B == R && B > 1, "unsupported DFT size");
  static FWI_HD void run(cplx<T>* x) {
    cplx<T> y[R];
    SFor<B>::run([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      cplx<T> t[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n1] = x[B * n1 + n2];
      Dft<A, INV, T>::run(t);
      SFor<A>::run([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        y[n2 * A + k1] = twiddle_ct<(n2 * k1) % R, R, INV>(t[k1]);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      cplx<T> u[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) u[n2] = y[n2 * A + k1];
      Dft<B, INV, T>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = u[k2];
    }
  }
};

// R-point DFT whose inputs x[R/2 .. R) are zero (a zero-padded half):
// X[2k] = DFT_{R/2}(x)[k], X[2k+1] = DFT_{R/2}(w_R^n x[n])[k].
template <int R, bool INV, typename T> struct DftHalfIn {
  static_assert(R % 2 == 0, "even size");
  static FWI_HD void run(cplx<T>* x) {
    constexpr int H = R / 2;
    cplx<T> a[H], b[H];
    SFor<H>::run([&](auto nc) {
      constexpr int n = decltype(nc)::value;
      a[n] = x[n];
      b[n] = twiddle_ct<n, R, INV>(x[n]);
    });
    Dft<H, INV, T>::run(a);
    Dft<H, INV, T>::run(b);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      x[2 * k] = a[k];
      x[2 * k + 1] = b[k];
    }
  }
};

// R-point DFT of which only the outputs x[0 .. R/2) are wanted (a cropped
// half): x[n] = DFT_{R/2}(X_even)[n] + w_R^n DFT_{R/2}(X_odd)[n].  The
// entries x[R/2 .. R) are left undefined.
template <int R, bool INV, typename T> struct DftHalfOut {
  static_assert(R % 2 == 0, "even size");
  static FWI_HD void run(cplx<T>* x) {
    constexpr int H = R / 2;
    cplx<T> a[H], b[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
      a[k] = x[2 * k];
      b[k] = x[2 * k + 1];
    }
    Dft<H, INV, T>::run(a);
    Dft<H, INV, T>::run(b);
    SFor<H>::run([&](auto nc) {
      constexpr int n = decltype(nc)::value;
      x[n] = cadd(a[n], twiddle_ct<n, R, INV>(b[n]));
    });
  }
};

// ---------------------------------------------------------------------------
// Line plan: L = R1 * R2 handled by TL threads.  Thread t owns columns
// n2 = t + i*TL (i < C1) in phases A/D and rows k1 = t + i*TL (i < C3) in
// phases B/C.  Shared-memory position of y[n2][k1] is
//   (n2 * (R1 + PAD) + k1) * SJ
// relative to the line's base, with SJ the stride between consecutive
// positions (1 for row-major lines, the tile width for interleaved columns).
template <int L_, int R1_, int R2_, int TL_> struct Plan {
  static constexpr int L = L_, R1 = R1_, R2 = R2_, TL = TL_;
  static_assert(R1 * R2 == L, "plan factors");
  static_assert(R1 % 2 == 0, "R1 must be even for the half-lattice pruning");
  static constexpr int C1 = (R2 + TL - 1) / TL;
  static constexpr int C3 = (R1 + TL - 1) / TL;
  static constexpr int E1 = C1 * R1;
  static constexpr int E3 = C3 * R2;
  static constexpr int E = E1 > E3 ? E1 : E3;
  static constexpr int H1 = R1 / 2;  // nonzero / needed n1 under pruning
  // positions used by one line in shared memory (before the SJ stride)
  static constexpr int span(int pad) { return R2 * (R1 + pad); }
};

// Phase A (forward): registers v hold, for each owned n2, the R1 input
// samples x[R2 n1 + n2] at v[i*R1 + n1] (loaded by the caller; entries with
// n1 >= NIN1 must be zero).  Computes the R1-point DFTs, applies the
// four-step twiddle w_L^{n2 k1} (table tw of L entries, forward sign), and
// stores y[n2][k1] into shared memory.  HALF_IN: the samples n1 >= R1/2 are
// zero (a zero-padded line) and the DFTs skip them.
template <class P, typename T, bool HALF_IN = false, bool TWS = false>
FWI_HD void phaseA_store(int t, cplx<T>* v, cplx<T>* sm, int sj, int pad,
                         const cplx<T>* tw) {
#pragma unroll
  for (int i = 0; i < P::C1; ++i) {
    const int n2 = t + i * P::TL;
    if (P::C1 * P::TL == P::R2 || n2 < P::R2) {
      if constexpr (HALF_IN) DftHalfIn<P::R1, false, T>::run(v + i * P::R1);
      else Dft<P::R1, false, T>::run(v + i * P::R1);
#pragma unroll
      for (int k1 = 0; k1 < P::R1; ++k1) {
        cplx<T> z = v[i * P::R1 + k1];
        if (k1 > 0 && n2 > 0) z = cmul(z, tw_at<TWS>(tw + n2 * k1));
        sm[(n2 * (P::R1 + pad) + k1) * sj] = z;
      }
    }
  }
}

// Phase B (forward): reads y[n2][k1] for each owned k1 and all n2, does the
// R2-point DFTs.  On return v[i*R2 + k2] = X[k1 + R1 k2] with k1 = t + i*TL.
template <class P, typename T>
FWI_HD void phaseB_load(int t, cplx<T>* v, const cplx<T>* sm, int sj, int pad) {
#pragma unroll
  for (int i = 0; i < P::C3; ++i) {
    const int k1 = t + i * P::TL;
    if (P::C3 * P::TL == P::R1 || k1 < P::R1) {
#pragma unroll
      for (int n2 = 0; n2 < P::R2; ++n2)
        v[i * P::R2 + n2] = sm[(n2 * (P::R1 + pad) + k1) * sj];
      Dft<P::R2, false, T>::run(v + i * P::R2);
    }
  }
}

// Phase C (inverse): v[i*R2 + k2] holds X[k1 + R1 k2] for each owned k1.
// Inverse R2-point DFTs over k2, conjugate twiddle w_L^{-n2 k1}, store
// y[n2][k1] to shared memory.
template <class P, typename T, bool TWS = false>
FWI_HD void phaseC_store(int t, cplx<T>* v, cplx<T>* sm, int sj, int pad,
                         const cplx<T>* tw) {
#pragma unroll
  for (int i = 0; i < P::C3; ++i) {
    const int k1 = t + i * P::TL;
    if (P::C3 * P::TL == P::R1 || k1 < P::R1) {
      Dft<P::R2, true, T>::run(v + i * P::R2);
#pragma unroll
      for (int n2 = 0; n2 < P::R2; ++n2) {
        cplx<T> z = v[i * P::R2 + n2];
        if (k1 > 0 && n2 > 0) z = cmulc(z, tw_at<TWS>(tw + n2 * k1));
        sm[(n2 * (P::R1 + pad) + k1) * sj] = z;
      }
    }
  }
}

// Phase D (inverse): reads y[n2][k1] for each owned n2 and all k1, inverse
// R1-point DFTs of which only the cropped half is formed.  On return
// v[i*R1 + n1] = x[R2 n1 + n2] (unnormalised) for n1 < R1/2; the entries
// n1 >= R1/2 are undefined (every caller keeps the cropped half only).
template <class P, typename T>
FWI_HD void phaseD_load(int t, cplx<T>* v, const cplx<T>* sm, int sj, int pad) {
#pragma unroll
  for (int i = 0; i < P::C1; ++i) {
    const int n2 = t + i * P::TL;
    if (P::C1 * P::TL == P::R2 || n2 < P::R2) {
#pragma unroll
      for (int k1 = 0; k1 < P::R1; ++k1)
        v[i * P::R1 + k1] = sm[(n2 * (P::R1 + pad) + k1) * sj];
      DftHalfOut<P::R1, true, T>::run(v + i * P::R1);
    }
  }
}

// ---------------------------------------------------------------------------
// Radix-2 split of an R = 2Q point DFT over a pair of lanes that differ by 16
// (device only: the pair exchanges values with warp shuffles).
//
// split_dft : lane h holds x[2m + h] (m < Q); on return it holds
//             X[k + Q h] (k < Q) of the direction INV.
// split_idft: lane h holds X[k + Q h]; on return it holds x[2m + h] of the
//             direction INV (unnormalised).
#if defined(__CUDACC__)
template <typename V> __device__ __forceinline__ V shfl_pair(V a) {
  V o;
  o.x = __shfl_xor_sync(0xffffffffu, a.x, 16);
  o.y = __shfl_xor_sync(0xffffffffu, a.y, 16);
  return o;
}

// Twiddle applied only on lane h = 1 of a pair, without selects:
// z * (h w + (1 - h)) with w = w_R^J (conjugated for INV) and hf = h,
// hc = 1 - h exactly 0 or 1, so lane 0 gets z and lane 1 gets z w exactly
// as the plain product.
template <int J, int R, bool INV, typename V, typename S>
__device__ __forceinline__ V lane_twiddle(V z, S hf, S hc) {
  constexpr int q = tw_quarter(J, R);
  if constexpr (q == 0) {
    return z;
  } else {
    // exact quarter turns; otherwise the compile-time cosine / sine
    constexpr double wr = q == 2 ? -1.0 : (q == 1 || q == 3) ? 0.0 : tw_re(J, R);
    constexpr double wf = q == 1 ? -1.0 : q == 3 ? 1.0 : q == 2 ? 0.0 : tw_im(J, R);
    constexpr double wi = INV ? -wf : wf;
    const S a = hf * S(wr) + hc;  // h wr + (1 - h)
    const S b = hf * S(wi);       // h wi
    V o;
    o.x = z.x * a - z.y * b;
    o.y = z.x * b + z.y * a;
    return o;
  }
}

// Lane h = 0 holds E, lane 1 holds O (the DFT_Q of the even / odd samples):
// lane 1 sends w^k O, lane 0 sends E, and each lane forms
// (1 - 2h) v + received, i.e. E + w^k O on lane 0 and E - w^k O on lane 1.
template <int Q, bool INV, typename T>
__device__ __forceinline__ void split_dft(cplx<T>* u, int h) {
  Dft<Q, INV, T>::run(u);
  const T hf = T(h), hc = T(1 - h), sg = T(1 - 2 * h);
  SFor<Q>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const cplx<T> v = lane_twiddle<k, 2 * Q, INV>(u[k], hf, hc);
    const cplx<T> o = shfl_pair(v);
    u[k] = mk<T>(sg * v.x + o.x, sg * v.y + o.y);
  });
}

// Lane 0 holds X[k], lane 1 holds X[k + Q]: lane 0 forms X[k] + X[k + Q],
// lane 1 (X[k] - X[k + Q]) w^k, then each lane's inverse DFT_Q.
template <int Q, bool INV, typename T>
__device__ __forceinline__ void split_idft(cplx<T>* u, int h) {
  const T hf = T(h), hc = T(1 - h), sg = T(1 - 2 * h);
  SFor<Q>::run([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const cplx<T> own = u[k];
    const cplx<T> o = shfl_pair(own);
    const cplx<T> z = mk<T>(sg * own.x + o.x, sg * own.y + o.y);
    u[k] = lane_twiddle<k, 2 * Q, INV>(z, hf, hc);
  });
  Dft<Q, INV, T>::run(u);
}
#endif

}  // namespace fwi
