// Tensor-core (tcgen05, TF32) versions of the two FP32 pixel contractions
// of the data equation and the implicit Jacobian (Eq. 4, 15-17; Sec. IV-B,
// IV-C):
//
//  contract : Y_l[e][j] = sum_n X_l[e][n] (a[n] Q_l[j][n])       (data, J a)
//  J^H      : z_l[n]    = s_l sum_e conj(X_l[e][n]) W_l[e][n],
//             W_l[e][n] = sum_j B_l[e][j] conj(X_l[j][n])           (J^H b)
//
// Both are complex GEMMs with one dimension of 128 array elements per tile
// and the pixels as the long dimension (K for the contraction, M for J^H).
// A complex product is four real products; in the 128 x 256 accumulator
// [Re | Im] they are two MMAs per k-step,
//     D += Ar [Br; Bi]^T   and   D += Ai [-Bi; Br]^T,
// with the B rows kept once as the stack [-Bi | Br | Bi].  Each real
// operand is split into TF32 hi + lo parts and a b is taken as
// ah bh + ah bl + al bh (3xTF32), which keeps the products at FP32
// accuracy; accumulation is FP32 in TMEM and partial sums over CTAs are
// combined in FP64 by the callers' reduction kernels.
//
// Pipelines: raw FP32 operand tiles arrive several stages ahead, by TMA
// tensor copies that one producer thread issues (or, without TMA, by the
// producers' own cp.async); four producer warps split them into the TF32
// operand planes of a shared-memory stage and signal an mbarrier; one warp
// issues the MMAs and
// releases the stage with tcgen05.commit; two TMEM accumulators alternate so
// that four more warps read one out while the MMAs fill the other.  Every
// wait is bounded (tc.cuh).
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "ctx.cuh"
#include "prof.cuh"
#include "tc.cuh"

namespace fwi {

namespace {

using tc::smem_addr;

constexpr int ROWS = 128;             // MMA M, rows of an operand tile
constexpr int KS = 8;                 // complex values per k-step (TF32 K = 8)
constexpr int PLANE = ROWS * 32;      // one 128-row operand block of a k-step
constexpr int BROWS = 3 * ROWS;       // B stack [-Bi | Br | Bi]
constexpr int BPLANE = BROWS * 32;
constexpr uint32_t LBO_A = 16 * ROWS, LBO_B = 16 * BROWS, SBO = 128;
constexpr uint32_t IDESC = tc::idesc_tf32(128, 256, false);
// 4 producer warps, 1 MMA warp, 4 accumulator warps (drain / epilogue)
constexpr int C_THREADS = 288;
constexpr int C_TILE_STRIDE = 17;     // drain transpose tile: [32 rows][16 + 1] float2
constexpr int C_TILE_BYTES = 32 * C_TILE_STRIDE * 8;

// Operand planes inside a conversion stage: A = {Ar hi, Ar lo, Ai hi, Ai lo}
// (one 128-row block each), then B hi and B lo (384 rows each).
__device__ __forceinline__ void issue_kstep(uint32_t tmem, uint32_t a_base, uint32_t b_base,
                                           uint32_t first) {
  using namespace tc;
  const uint64_t ar_h = sdesc(a_base + 0 * PLANE, LBO_A, SBO);
  const uint64_t ar_l = sdesc(a_base + 1 * PLANE, LBO_A, SBO);
  const uint64_t ai_h = sdesc(a_base + 2 * PLANE, LBO_A, SBO);
  const uint64_t ai_l = sdesc(a_base + 3 * PLANE, LBO_A, SBO);
  // [Br; Bi] starts at row 128 of the stack, [-Bi; Br] at row 0
  const uint64_t b1_h = sdesc(b_base + 16 * ROWS, LBO_B, SBO);
  const uint64_t b1_l = sdesc(b_base + BPLANE + 16 * ROWS, LBO_B, SBO);
  const uint64_t b2_h = sdesc(b_base, LBO_B, SBO);
  const uint64_t b2_l = sdesc(b_base + BPLANE, LBO_B, SBO);
  mma_tf32(tmem, ar_h, b1_h, IDESC, first ? 0u : 1u);
  mma_tf32(tmem, ar_h, b1_l, IDESC, 1u);
  mma_tf32(tmem, ar_l, b1_h, IDESC, 1u);
  mma_tf32(tmem, ai_h, b2_h, IDESC, 1u);
  mma_tf32(tmem, ai_h, b2_l, IDESC, 1u);
  mma_tf32(tmem, ai_l, b2_h, IDESC, 1u);
}

// Store 4 consecutive-k values of operand row `row` (hi and lo planes).
__device__ __forceinline__ void put_a(uint32_t plane_hi, uint32_t plane_lo, int half, int row,
                                      const float (&v)[4]) {
  float h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) tc::split_tf32(v[i], h[i], l[i]);
  const uint32_t off = (uint32_t)(half * 16 * ROWS + 16 * row);
  tc::sts128(plane_hi + off, h[0], h[1], h[2], h[3]);
  tc::sts128(plane_lo + off, l[0], l[1], l[2], l[3]);
}

// B row `row`: re and im parts into the [-Bi | Br | Bi] stack.
__device__ __forceinline__ void put_b(uint32_t bhi, uint32_t blo, int half, int row,
                                      const float (&re)[4], const float (&im)[4]) {
  float rh[4], rl[4], ih[4], il[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    tc::split_tf32(re[i], rh[i], rl[i]);
    tc::split_tf32(im[i], ih[i], il[i]);
  }
  const uint32_t o = (uint32_t)(half * 16 * BROWS + 16 * row);
  tc::sts128(bhi + o, -ih[0], -ih[1], -ih[2], -ih[3]);
  tc::sts128(bhi + o + 16 * ROWS, rh[0], rh[1], rh[2], rh[3]);
  tc::sts128(bhi + o + 32 * ROWS, ih[0], ih[1], ih[2], ih[3]);
  tc::sts128(blo + o, -il[0], -il[1], -il[2], -il[3]);
  tc::sts128(blo + o + 16 * ROWS, rl[0], rl[1], rl[2], rl[3]);
  tc::sts128(blo + o + 32 * ROWS, il[0], il[1], il[2], il[3]);
}

__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts64(uint32_t addr, float a, float b) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ float2 lds64(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}

// ---------------------------------------------------------------------------
// Contraction: one CTA per (pixel chunk s, tile pair (eb, jb), frequency l);
// accumulator D[e][j] (128 x [128 Re | 128 Im]) over its pixel chunk,
// written as FP32 partials part[s][l][e][j].
// Raw stages: 128 rows of X (and of Q unless the two share rows) plus the
// 8 weights a[n]; SHARED (X == Q, one element tile) keeps 8 stages in
// flight, the general case 4; after them come the four drain warps'
// transpose tiles.
constexpr int C_CONV = 3;
constexpr int C_RAWROW = 80;  // 8 complex (64 bytes) + 16 bytes of padding
constexpr int C_CONV_BYTES = 4 * PLANE + 2 * BPLANE;
template <bool SHARED> struct CRaw {
  static constexpr int N = SHARED ? 8 : 4;
  static constexpr int X = 0, Q = ROWS * C_RAWROW;
  static constexpr int A = (SHARED ? 1 : 2) * ROWS * C_RAWROW;
  static constexpr int BYTES = A + 64;
  static constexpr int TILES = C_CONV * C_CONV_BYTES + N * BYTES;
  static constexpr int SMEM = TILES + 4 * C_TILE_BYTES;
};
// Raw stages filled by TMA: rows of 64 bytes without padding, written with
// the 64-byte swizzle (16-byte chunk q of row r lands at chunk q ^ ((r / 2)
// mod 4)), which keeps the producers' 16-byte row reads free of bank
// conflicts; stages 1024-byte aligned for the swizzle pattern.
template <bool SHARED> struct CRawT {
  static constexpr int N = SHARED ? 8 : 4;
  static constexpr int TILE = ROWS * 64;  // one operand's box
  static constexpr int X = 0, Q = TILE;
  static constexpr int A = (SHARED ? 1 : 2) * TILE;
  static constexpr int BYTES = ((A + 64 + 1023) / 1024) * 1024;
  static constexpr int TX = (SHARED ? 1 : 2) * TILE;  // bytes the TMA copies deliver
  static constexpr int TILES = C_CONV * C_CONV_BYTES + N * BYTES;
  static constexpr int SMEM = TILES + 4 * C_TILE_BYTES;
};
// Byte offset of 16-byte chunk q of row r in a swizzled 64-byte-row tile.
__device__ __forceinline__ uint32_t swz64(int r, int q) {
  return (uint32_t)(r * 64 + ((q ^ ((r >> 1) & 3)) << 4));
}

struct ContractArgs {
  const float2* X;
  const float2* Q;
  const float2* a;  // may be NULL
  float2* part;
  int* err;
  long long N, chunk;
  int NE, n_freq;
  int sub_ks;       // k-steps per accumulation sub-chunk
  int stall;        // test of the failure path: withhold the first stage
};

// Two accumulators (TMEM columns 0-255 and 256-511) alternate between
// sub-chunks: while the MMA warp accumulates sub-chunk s into buffer s % 2,
// four drain warps add buffer (s - 1) % 2 into the CTA's FP32 partial.  A
// drain warp owns the 32 TMEM lanes of its quadrant (32 rows e) and moves
// 16 columns at a time through a shared transpose tile, so that its global
// read-modify-write covers two 128-byte row segments per instruction.
// XTMA: the raw X (and Q) tiles arrive by TMA tensor copies (64-byte
// swizzle) issued by one producer thread and completing on bar_raw; the
// weights a still come by cp.async.  Otherwise every producer copies its
// rows with cp.async.
template <bool SHARED, bool XTMA>
__global__ void __launch_bounds__(C_THREADS, 1) tc_contract_kernel(
    ContractArgs p, const __grid_constant__ CUtensorMap xmap,
    const __grid_constant__ CUtensorMap qmap) {
  using namespace tc;
  using RW = typename std::conditional<XTMA, CRawT<SHARED>, CRaw<SHARED>>::type;
  constexpr int C_RAW = RW::N, C_RAW_BYTES = RW::BYTES;
  constexpr int C_RAW_X = RW::X, C_RAW_Q = RW::Q, C_RAW_A = RW::A;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full[C_CONV], bar_empty[C_CONV], bar_done[2],
      bar_freed[2], bar_final, bar_raw[C_RAW];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = blockIdx.x, l = blockIdx.z;
  const int nbe = (p.NE + ROWS - 1) / ROWS;
  const int eb = blockIdx.y % nbe, jb = blockIdx.y / nbe;
  const long long n_begin = (long long)s * p.chunk;
  const long long n_end = (n_begin + p.chunk < p.N) ? n_begin + p.chunk : p.N;
  const int nch = (n_begin < p.N) ? (int)((n_end - n_begin + KS - 1) / KS) : 0;
  const float2* Xl = p.X + (long long)l * p.NE * p.N;
  const float2* Ql = p.Q + (long long)l * p.NE * p.N;
  constexpr bool same_rows = SHARED;
  const bool has_a = p.a != nullptr;

  if (tid == 0) {
    for (int i = 0; i < C_CONV; ++i) {
      mbar_init(smem_addr(&bar_full[i]), 128);
      mbar_init(smem_addr(&bar_empty[i]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_addr(&bar_done[b]), 1);
      mbar_init(smem_addr(&bar_freed[b]), 128);
    }
    mbar_init(smem_addr(&bar_final), 1);
    if (XTMA)
      for (int i = 0; i < C_RAW; ++i) mbar_init(smem_addr(&bar_raw[i]), 1);
    abort_flag = 0;
    mbar_init_fence();
    if (XTMA) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap))
                   : "memory");
      if (!same_rows)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&qmap))
                     : "memory");
    }
  }
  if (warp == 0) tmem_alloc(smem_addr(&tmem_base), 512);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t sbase = smem_addr(smem);
  const uint32_t raw0 = sbase + C_CONV * C_CONV_BYTES;
  const int nsub = (nch + p.sub_ks - 1) / p.sub_ks;

  if (warp >= 5) {
    const int q = warp & 3;             // TMEM lane quadrant: rows 32q .. 32q + 31
    const uint32_t tile = sbase + RW::TILES + q * C_TILE_BYTES;
    const int e0 = eb * ROWS + 32 * q;  // first row of the quadrant
    float2* part = p.part + ((long long)s * p.n_freq + l) * p.NE * p.NE;
    const int rsub = lane >> 4, csub = lane & 15;  // read-back position in a tile
    for (int sub = 0; sub < nsub; ++sub) {
      const int b = sub & 1;
      const bool ok = mbar_wait(smem_addr(&bar_done[b]), (sub >> 1) & 1, &abort_flag, p.err,
                                kErrWaitDone);
      fence_after_sync();
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16) + 256u * b;
#pragma unroll 1
      for (int cb = 0; cb < ROWS / 16; ++cb) {
        uint32_t re[16], im[16];
        tmem_ld16(lane_addr + 16 * cb, re);
        tmem_ld16(lane_addr + ROWS + 16 * cb, im);
        tmem_wait_ld();
        // this lane's row (32q + lane), columns 16 cb .. 16 cb + 15
#pragma unroll
        for (int k = 0; k < 16; ++k)
          sts64(tile + (uint32_t)((lane * C_TILE_STRIDE + k) * 8), __uint_as_float(re[k]),
                __uint_as_float(im[k]));
        __syncwarp();
        const int jj = jb * ROWS + 16 * cb + csub;
#pragma unroll 4
        for (int ii = 0; ii < 16; ++ii) {
          const int rr = 2 * ii + rsub;
          const int e = e0 + rr;
          const float2 t = lds64(tile + (uint32_t)((rr * C_TILE_STRIDE + csub) * 8));
          if (e < p.NE && jj < p.NE) {
            float2* dst = part + (long long)e * p.NE + jj;
            float2 v = ok ? t : make_float2(0.f, 0.f);
            if (sub > 0) {
              const float2 o = *dst;
              v.x += o.x;
              v.y += o.y;
            }
            *dst = v;
          }
        }
        __syncwarp();
      }
      fence_before_sync();  // the TMEM reads precede the buffer's next MMAs
      mbar_arrive(smem_addr(&bar_freed[b]));
    }
    if (nch == 0) {
      for (int rr = 0; rr < 32; ++rr) {
        const int e = e0 + rr;
        for (int jj = jb * ROWS + lane; jj < jb * ROWS + ROWS; jj += 32)
          if (e < p.NE && jj < p.NE) part[(long long)e * p.NE + jj] = make_float2(0.f, 0.f);
      }
    }
  } else if (warp < 4) {
    const int r = tid;
    // raw fill: four lanes copy one row's 64-byte segment, so each warp
    // instruction reads eight rows in whole 32-byte sectors
    const int fq = r & 3;   // 16-byte piece of the segment
    const int fr = r >> 2;  // first row of this thread (rows fr + 32 k)
    auto issue = [&](int g) {
      if (g < nch) {
        const long long n0 = n_begin + (long long)g * KS;
        const uint32_t rb = raw0 + (uint32_t)((g % C_RAW) * C_RAW_BYTES);
        if (XTMA) {
          // k-steps never straddle a chunk end (chunks are whole k-steps);
          // rows e >= NE and pixels n >= N are outside the tensor: zero fill
          if (r == 0) {
            const uint32_t bar = smem_addr(&bar_raw[g % C_RAW]);
            mbar_arrive_expect_tx(bar, (uint32_t)CRawT<SHARED>::TX);
            tma_load_3d(rb + C_RAW_X, &xmap, (int)(2 * n0), eb * ROWS, l, bar);
            if (!same_rows) tma_load_3d(rb + C_RAW_Q, &qmap, (int)(2 * n0), jb * ROWS, l, bar);
          }
        } else {
          const long long n = n0 + 2 * fq;
          const bool okn = n < n_end;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int rr = fr + 32 * k;
            const int er = eb * ROWS + rr, jr = jb * ROWS + rr;
            const bool okx = okn && er < p.NE, okq = okn && jr < p.NE;
            cp_async16(rb + C_RAW_X + rr * C_RAWROW + 16 * fq,
                       okx ? Xl + (long long)er * p.N + n : Xl, okx ? 16u : 0u);
            if (!same_rows)
              cp_async16(rb + C_RAW_Q + rr * C_RAWROW + 16 * fq,
                         okq ? Ql + (long long)jr * p.N + n : Ql, okq ? 16u : 0u);
          }
        }
        if (has_a && r < 4) {
          const long long n = n0 + 2 * r;
          const bool ok = n < n_end;
          cp_async16(rb + C_RAW_A + 16 * r, ok ? p.a + n : p.a, ok ? 16u : 0u);
        }
      }
      cp_async_commit();
    };
#pragma unroll
    for (int g = 0; g < C_RAW - 1; ++g) issue(g);
    for (int g = 0; g < nch; ++g) {
      if (XTMA)
        mbar_wait(smem_addr(&bar_raw[g % C_RAW]), (g / C_RAW) & 1, &abort_flag, p.err,
                  kErrWaitFull);
      cp_async_wait<C_RAW - 2>();
      bar_sync(1, 128);  // chunk g visible to all; everyone done with chunk g-1
      issue(g + C_RAW - 1);
      const int cs = g % C_CONV;
      mbar_wait(smem_addr(&bar_empty[cs]), ((g / C_CONV) & 1) ^ 1, &abort_flag, p.err,
                kErrWaitEmpty);
      const uint32_t rb = raw0 + (uint32_t)((g % C_RAW) * C_RAW_BYTES);
      const uint32_t cb = sbase + (uint32_t)(cs * C_CONV_BYTES);
      const uint32_t bhi = cb + 4 * PLANE, blo = bhi + BPLANE;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float2 x[4], q[4];
        // chunks 2 half and 2 half + 1 of row r (swizzled when TMA filled)
        const uint32_t o0 = XTMA ? swz64(r, 2 * half) : (uint32_t)(r * C_RAWROW + 32 * half);
        const uint32_t o1 = XTMA ? swz64(r, 2 * half + 1) : o0 + 16;
        {
          const float4 u0 = lds128(rb + C_RAW_X + o0);
          const float4 u1 = lds128(rb + C_RAW_X + o1);
          x[0] = make_float2(u0.x, u0.y); x[1] = make_float2(u0.z, u0.w);
          x[2] = make_float2(u1.x, u1.y); x[3] = make_float2(u1.z, u1.w);
        }
        if (same_rows) {
#pragma unroll
          for (int i = 0; i < 4; ++i) q[i] = x[i];
        } else {
          const float4 u0 = lds128(rb + C_RAW_Q + o0);
          const float4 u1 = lds128(rb + C_RAW_Q + o1);
          q[0] = make_float2(u0.x, u0.y); q[1] = make_float2(u0.z, u0.w);
          q[2] = make_float2(u1.x, u1.y); q[3] = make_float2(u1.z, u1.w);
        }
        if (has_a) {
          const float4 u0 = lds128(rb + C_RAW_A + 32 * half);
          const float4 u1 = lds128(rb + C_RAW_A + 32 * half + 16);
          const float2 av[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w),
                                make_float2(u1.x, u1.y), make_float2(u1.z, u1.w)};
#pragma unroll
          for (int i = 0; i < 4; ++i)
            q[i] = make_float2(q[i].x * av[i].x - q[i].y * av[i].y,
                               q[i].x * av[i].y + q[i].y * av[i].x);
        }
        const float xr[4] = {x[0].x, x[1].x, x[2].x, x[3].x};
        const float xi[4] = {x[0].y, x[1].y, x[2].y, x[3].y};
        const float qr[4] = {q[0].x, q[1].x, q[2].x, q[3].x};
        const float qi[4] = {q[0].y, q[1].y, q[2].y, q[3].y};
        put_a(cb + 0 * PLANE, cb + 1 * PLANE, half, r, xr);
        put_a(cb + 2 * PLANE, cb + 3 * PLANE, half, r, xi);
        put_b(bhi, blo, half, r, qr, qi);
      }
      fence_proxy_async();
      if (!(p.stall && g == 0)) mbar_arrive(smem_addr(&bar_full[cs]));
    }
    cp_async_wait<0>();
    if (XTMA && r == 0 && abort_flag) {
      // copies issued before a wait gave up may still land in this CTA's
      // shared memory: wait (bounded) for the last one of every raw stage
      for (int i = 0; i < C_RAW && i < nch; ++i) {
        const int g = nch - 1 - ((nch - 1 - i) % C_RAW);
        mbar_wait_drain(smem_addr(&bar_raw[g % C_RAW]), (g / C_RAW) & 1, p.err, kErrWaitDrain);
      }
    }
  } else {
    for (int g = 0; g < nch; ++g) {
      const int cs = g % C_CONV;
      const int sub = g / p.sub_ks, b = sub & 1;
      if (g % p.sub_ks == 0 && sub >= 2) {
        // buffer b is free once sub-chunk sub - 2 has been drained
        mbar_wait(smem_addr(&bar_freed[b]), ((sub - 2) >> 1) & 1, &abort_flag, p.err,
                  kErrWaitEmpty);
        fence_after_sync();
      }
      const bool ok = mbar_wait(smem_addr(&bar_full[cs]), (g / C_CONV) & 1, &abort_flag,
                                p.err, kErrWaitFull);
      fence_after_sync();
      if (lane == 0 && ok) {
        const uint32_t cb = sbase + (uint32_t)(cs * C_CONV_BYTES);
        issue_kstep(tmem + 256u * b, cb, cb + 4 * PLANE, g % p.sub_ks == 0);
        commit(smem_addr(&bar_empty[cs]));
      }
      if (lane == 0 && ((g + 1) % p.sub_ks == 0 || g == nch - 1))
        commit(smem_addr(&bar_done[b]));
      __syncwarp();
    }
    if (lane == 0) commit(smem_addr(&bar_final));  // after every MMA of this CTA
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    // no MMA of this CTA may still write the columns being freed (also when
    // a wait gave up)
    if (lane == 0) mbar_wait_drain(smem_addr(&bar_final), 0, p.err, kErrWaitDrain);
    __syncwarp();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// J^H: persistent CTAs over units (frequency l, element tile eb, tile of 128
// pixels).  Per unit the accumulator holds W[n][e] (128 pixels x [128 Re |
// 128 Im]); two accumulators alternate between units, and four epilogue
// warps form s_l sum_e conj(X[e][n]) W[e][n] into zpart[l][eb][n] (FUSED) or
// write W itself while the MMAs of the next unit proceed.
constexpr int M_CONV = 3, M_RAW = 6;
constexpr int M_RAW_BYTES = KS * ROWS * 8;               // [8 j][128 n] complex
constexpr int M_A_BYTES = 4 * PLANE;
constexpr int M_B_BYTES = 2 * BPLANE;                    // one k-step of B hi + lo
constexpr int M_CONV_BYTES = M_A_BYTES + M_B_BYTES;
constexpr int M_SMEM = M_CONV * M_CONV_BYTES + M_RAW * M_RAW_BYTES;

struct JhArgs {
  const float2* X;     // [n_freq][NE][N] mixed operand (rows j)
  const float2* Xe;    // [n_freq][NE][N] FUSED: epilogue operand (rows e)
  const float* bops;   // [n_freq][nbe][nks] k-step blocks of the B stack (hi, lo)
  const double* scale; // [n_freq]
  float2* zpart;       // FUSED: [n_freq][nbe][N]; else W itself, [n_freq][NE][N]
  int* err;
  long long N;
  int NE, n_freq, nbe, nks, npb, units;
  int conj_x;          // A = conj(X)^T (J^H) or X^T (adjoint sources)
};

// FUSED: z_l[n] = s_l sum_e conj(X[e][n]) W[e][n] (J^H b); otherwise the
// mix W_l[e][n] = s_l sum_j B[e][j] X'[j][n] itself is written (adjoint
// sources conj(s_e) = k^2 dV sum_j p0_j conj(r_ej)).
// XTMA: the raw tiles of the mixed operand (8 rows j x 128 pixels, one box)
// arrive by TMA tensor copies issued by one producer thread and completing
// on bar_raw; otherwise every producer copies its part with cp.async.
template <bool FUSED, bool XTMA>
__global__ void __launch_bounds__(C_THREADS, 1) tc_jh_kernel(JhArgs p,
                                                             const __grid_constant__ CUtensorMap xmap) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full[M_CONV], bar_empty[M_CONV], bar_done[2],
      bar_freed[2], bar_final, bar_raw[M_RAW];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int my_units = (blockIdx.x < p.units)
                           ? (p.units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                           : 0;
  const int nchunks = my_units * p.nks;

  if (tid == 0) {
    for (int i = 0; i < M_CONV; ++i) {
      mbar_init(smem_addr(&bar_full[i]), 129);  // 128 producers + expect_tx
      mbar_init(smem_addr(&bar_empty[i]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_addr(&bar_done[b]), 1);
      mbar_init(smem_addr(&bar_freed[b]), 128);
    }
    mbar_init(smem_addr(&bar_final), 1);
    if (XTMA)
      for (int i = 0; i < M_RAW; ++i) mbar_init(smem_addr(&bar_raw[i]), 1);
    abort_flag = 0;
    mbar_init_fence();
    if (XTMA)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap))
                   : "memory");
  }
  if (warp == 0) tmem_alloc(smem_addr(&tmem_base), 512);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t sbase = smem_addr(smem);
  const uint32_t raw0 = sbase + M_CONV * M_CONV_BYTES;

  // unit index -> (l, eb, pixel tile)
  auto unit_of = [&](int k, int& l, int& eb, int& pb) {
    const int u = (int)blockIdx.x + k * (int)gridDim.x;
    pb = u % p.npb;
    eb = (u / p.npb) % p.nbe;
    l = u / (p.npb * p.nbe);
  };

  if (warp >= 5) {
    // epilogue warps: TMEM lane = pixel 32 q + lane of the unit's tile
    const int q = warp & 3;
    const int r = 32 * q + lane;
    for (int k = 0; k < my_units; ++k) {
      int l, eb, pb;
      unit_of(k, l, eb, pb);
      const int b = k & 1;
      const bool ok = mbar_wait(smem_addr(&bar_done[b]), (k >> 1) & 1, &abort_flag, p.err,
                                kErrWaitDone);
      fence_after_sync();
      const float2* Xl = p.Xe + (long long)l * p.NE * p.N;
      const float sc = (float)p.scale[l];
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16) + 256u * b;
      const long long n = (long long)pb * ROWS + r;
      const bool nv = n < p.N;
      float zx = 0.f, zy = 0.f;
#pragma unroll 1
      for (int ec = 0; ec < ROWS / 32; ++ec) {
        uint32_t wr[32], wi[32];
        tmem_ld32(lane_addr + (uint32_t)(32 * ec), wr);
        tmem_ld32(lane_addr + (uint32_t)(ROWS + 32 * ec), wi);
        tmem_wait_ld();
        if constexpr (FUSED) {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int e = eb * ROWS + 32 * ec + i;
            if (nv && e < p.NE) {
              const float2 x = __ldg(Xl + (long long)e * p.N + n);
              const float a = __uint_as_float(wr[i]), bb = __uint_as_float(wi[i]);
              zx += x.x * a + x.y * bb;
              zy += x.x * bb - x.y * a;
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int e = eb * ROWS + 32 * ec + i;
            if (nv && e < p.NE)
              p.zpart[((long long)l * p.NE + e) * p.N + n] =
                  ok ? make_float2(__uint_as_float(wr[i]) * sc, __uint_as_float(wi[i]) * sc)
                     : make_float2(0.f, 0.f);
          }
        }
      }
      if constexpr (FUSED) {
        if (nv)
          p.zpart[((long long)l * p.nbe + eb) * p.N + n] =
              ok ? make_float2(zx * sc, zy * sc) : make_float2(0.f, 0.f);
      }
      fence_before_sync();  // the TMEM reads precede the buffer's next MMAs
      mbar_arrive(smem_addr(&bar_freed[b]));
    }
  } else if (warp < 4) {
    const int r = tid;
    auto issue = [&](int g) {
      if (g < nchunks) {
        int l, eb, pb;
        unit_of(g / p.nks, l, eb, pb);
        const int ks = g % p.nks;
        const uint32_t rb = raw0 + (uint32_t)((g % M_RAW) * M_RAW_BYTES);
        if (XTMA) {
          // rows j >= NE and pixels n >= N are outside the tensor: zero fill
          if (r == 0) {
            const uint32_t bar = smem_addr(&bar_raw[g % M_RAW]);
            mbar_arrive_expect_tx(bar, M_RAW_BYTES);
            tma_load_3d(rb, &xmap, 2 * pb * ROWS, ks * KS, l, bar);
          }
        } else {
          const float2* Xl = p.X + (long long)l * p.NE * p.N;
#pragma unroll
          for (int k = 0; k < (KS * ROWS / 2) / 128; ++k) {
            const int i = r + 128 * k;
            const int jj = i / (ROWS / 2), pr = i % (ROWS / 2);
            const int jrow = ks * KS + jj;
            const long long n = (long long)pb * ROWS + 2 * pr;
            const bool ok = (jrow < p.NE) && (n < p.N);
            cp_async16(rb + (uint32_t)(jj * ROWS * 8 + 16 * pr),
                       ok ? Xl + (long long)jrow * p.N + n : p.X, ok ? 16u : 0u);
          }
        }
      }
      if (!XTMA) cp_async_commit();
    };
#pragma unroll
    for (int g = 0; g < M_RAW - 1; ++g) issue(g);
    for (int g = 0; g < nchunks; ++g) {
      if (XTMA)
        mbar_wait(smem_addr(&bar_raw[g % M_RAW]), (g / M_RAW) & 1, &abort_flag, p.err,
                  kErrWaitFull);
      else
        cp_async_wait<M_RAW - 2>();
      bar_sync(1, 128);
      issue(g + M_RAW - 1);
      const int kunit = g / p.nks, ks = g % p.nks;
      int l, eb, pb;
      unit_of(kunit, l, eb, pb);
      const int cs = g % M_CONV;
      mbar_wait(smem_addr(&bar_empty[cs]), ((g / M_CONV) & 1) ^ 1, &abort_flag, p.err,
                kErrWaitEmpty);
      const uint32_t cb = sbase + (uint32_t)(cs * M_CONV_BYTES);
      if (r == 0) {
        const uint32_t fb = smem_addr(&bar_full[cs]);
        mbar_arrive_expect_tx(fb, M_B_BYTES);
        const float* src =
            p.bops + ((((long long)l * p.nbe + eb) * p.nks + ks) * (long long)(M_B_BYTES / 4));
        bulk_g2s(cb + M_A_BYTES, src, M_B_BYTES, fb);
      }
      const uint32_t rb = raw0 + (uint32_t)((g % M_RAW) * M_RAW_BYTES);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float re[4], im[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 v = lds64(rb + (uint32_t)((4 * half + i) * ROWS * 8 + 8 * r));
          re[i] = v.x;
          im[i] = p.conj_x ? -v.y : v.y;
        }
        put_a(cb + 0 * PLANE, cb + 1 * PLANE, half, r, re);
        put_a(cb + 2 * PLANE, cb + 3 * PLANE, half, r, im);
      }
      fence_proxy_async();
      mbar_arrive(smem_addr(&bar_full[cs]));
    }
    if (!XTMA) {
      cp_async_wait<0>();
    } else if (r == 0 && abort_flag) {
      // copies issued before a wait gave up may still land in this CTA's
      // shared memory: wait (bounded) for the last one of every raw stage
      for (int i = 0; i < M_RAW && i < nchunks; ++i) {
        const int g = nchunks - 1 - ((nchunks - 1 - i) % M_RAW);
        mbar_wait_drain(smem_addr(&bar_raw[g % M_RAW]), (g / M_RAW) & 1, p.err, kErrWaitDrain);
      }
    }
  } else {
    for (int g = 0; g < nchunks; ++g) {
      const int cs = g % M_CONV, ks = g % p.nks, kunit = g / p.nks, b = kunit & 1;
      if (ks == 0 && kunit >= 2) {
        // buffer b is free once unit kunit - 2 has been read out
        mbar_wait(smem_addr(&bar_freed[b]), ((kunit - 2) >> 1) & 1, &abort_flag, p.err,
                  kErrWaitEmpty);
        fence_after_sync();
      }
      const bool ok = mbar_wait(smem_addr(&bar_full[cs]), (g / M_CONV) & 1, &abort_flag,
                                p.err, kErrWaitFull);
      fence_after_sync();
      if (lane == 0 && ok) {
        const uint32_t cb = sbase + (uint32_t)(cs * M_CONV_BYTES);
        issue_kstep(tmem + 256u * b, cb, cb + M_A_BYTES, ks == 0);
        commit(smem_addr(&bar_empty[cs]));
      }
      if (lane == 0 && ks == p.nks - 1) commit(smem_addr(&bar_done[b]));
      __syncwarp();
    }
    if (lane == 0) commit(smem_addr(&bar_final));  // after every MMA of this CTA
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    if (lane == 0) mbar_wait_drain(smem_addr(&bar_final), 0, p.err, kErrWaitDrain);
    __syncwarp();
    tmem_dealloc(tmem, 512);
  }
}

// B operand of J^H: per (l, eb, k-step) the stack [-Bi | Br | Bi] of
// B = y_l[e][j] (e in tile eb, j in the k-step) as TF32 hi and lo planes,
// laid out exactly as one shared-memory stage.
template <typename V>
__global__ void tc_jh_bops_kernel(const V* __restrict__ y, float* __restrict__ bops,
                                  int NE, int nbe, int nks, long long nseg) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nseg;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long blk = idx / (2 * 2 * BROWS);
    const int rem = (int)(idx % (2 * 2 * BROWS));
    const int hl = rem / (2 * BROWS), half = (rem / BROWS) % 2, row = rem % BROWS;
    const int ks = (int)(blk % nks), eb = (int)((blk / nks) % nbe);
    const long long l = blk / ((long long)nks * nbe);
    const int e = eb * ROWS + row % ROWS, part = row / ROWS;
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = ks * KS + 4 * half + k;
      double x = 0.0;
      if (e < NE && j < NE) {
        const V b = y[(l * NE + e) * NE + j];
        x = part == 0 ? -(double)b.y : (part == 1 ? (double)b.x : (double)b.y);
      }
      const float hi = tc::to_tf32((float)x);
      v[k] = hl == 0 ? hi : tc::to_tf32((float)(x - (double)hi));
    }
    float4* dst = (float4*)(bops + blk * (M_B_BYTES / 4) + hl * (BPLANE / 4) +
                            half * (16 * BROWS / 4) + 4 * row);
    *dst = make_float4(v[0], v[1], v[2], v[3]);
  }
}

int blocks_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// A field array [n_freq][NE][N] (complex FP32) as a 3-D tensor of floats
// (innermost the 2 N floats of a row) with boxes of box_x floats x box_rows
// rows of one frequency; swz64: 64-byte swizzle (box rows of 64 bytes).
bool field_tensor_map(const fwi_ctx* c, const float2* base, int box_x, int box_rows,
                      bool swz64, CUtensorMap* map) {
  tc::TensorMapEncodeFn enc = tc::tensor_map_encoder();
  if (!enc || ((uintptr_t)base & 15) || (c->N * 8) % 16) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * c->N, (cuuint64_t)c->n_elem,
                              (cuuint64_t)c->n_freq};
  const cuuint64_t strides[2] = {(cuuint64_t)c->N * 8, (cuuint64_t)c->n_elem * c->N * 8};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             swz64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;

cudaError_t set_attrs() {
  std::call_once(g_attr_once, [] {
    g_attr_err = cudaFuncSetAttribute(tc_contract_kernel<true, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      CRaw<true>::SMEM);
    if (g_attr_err == cudaSuccess)
      g_attr_err = cudaFuncSetAttribute(tc_contract_kernel<false, false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        CRaw<false>::SMEM);
    if (g_attr_err == cudaSuccess)
      g_attr_err = cudaFuncSetAttribute(tc_contract_kernel<true, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        CRawT<true>::SMEM);
    if (g_attr_err == cudaSuccess)
      g_attr_err = cudaFuncSetAttribute(tc_contract_kernel<false, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        CRawT<false>::SMEM);
    if (g_attr_err == cudaSuccess)
      g_attr_err = cudaFuncSetAttribute(tc_jh_kernel<true, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, M_SMEM);
    if (g_attr_err == cudaSuccess)
      g_attr_err = cudaFuncSetAttribute(tc_jh_kernel<false, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, M_SMEM);
    if (g_attr_err == cudaSuccess)
      g_attr_err = cudaFuncSetAttribute(tc_jh_kernel<true, false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, M_SMEM);
    if (g_attr_err == cudaSuccess)
      g_attr_err = cudaFuncSetAttribute(tc_jh_kernel<false, false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, M_SMEM);
  });
  return g_attr_err;
}

// Shared launcher of the two mixes; B is [n_freq][NE][NE] (double2 for
// J^H, float2 for the adjoint sources).
template <bool FUSED, typename V>
int tc_mix(fwi_ctx* c, const V* B, const float2* X, int conj_x, float2* out, int kclass,
           double bytes, double flops);

}  // namespace

bool tc_usable(const fwi_ctx* c) {
  return !c->fp64 && c->use_tc && (c->N % 2 == 0) && c->tc_bops != nullptr;
}

size_t tc_bops_bytes(int n_elem, int n_freq) {
  const size_t nbe = (size_t)(n_elem + ROWS - 1) / ROWS;
  const size_t nks = (size_t)(n_elem + KS - 1) / KS;
  return (size_t)n_freq * nbe * nks * M_B_BYTES;
}

int tc_contract_partials(fwi_ctx* c, const float2* X, const float2* a, const float2* Q,
                         float2* part) {
  cudaError_t e = set_attrs();
  if (e != cudaSuccess) {
    cuda_fail(c, e, "tc_contract attributes");
    return -1;
  }
  const int nbe = (c->n_elem + ROWS - 1) / ROWS;
  const int tiles = nbe * nbe * c->n_freq;
  int split = c->n_sm / tiles;
  if (split > c->jsplit_n) split = c->jsplit_n;
  if (split < 1) split = 1;
  long long chunk = (c->N + split - 1) / split;
  chunk = ((chunk + KS - 1) / KS) * KS;
  split = (int)((c->N + chunk - 1) / chunk);
  // Balanced sub-chunks of at most 512 pixels bound the FP32 accumulation
  // chain in TMEM (drained by separate warps while the MMAs continue); the
  // partial of a CTA collects its sub-chunks in order.
  const long long chunk_ks = chunk / KS;
  const long long nsub = (chunk_ks + 63) / 64;
  const int sub_ks = (int)((chunk_ks + nsub - 1) / nsub);
  ContractArgs args{X, Q, a, part, c->tc_err, c->N, chunk, c->n_elem, c->n_freq, sub_ks,
                    c->tc_stall};
  c->tc_stall = 0;  // one launch
  dim3 grid(split, nbe * nbe, c->n_freq);
  const double fe = (double)c->n_freq * c->n_elem * c->N;
  const bool shared_rows = X == Q && nbe == 1;
  CUtensorMap xmap, qmap;
  const bool xtma = c->jac_tma && field_tensor_map(c, X, 2 * KS, ROWS, true, &xmap) &&
                    (shared_rows || field_tensor_map(c, Q, 2 * KS, ROWS, true, &qmap));
  if (!xtma) std::memset(&xmap, 0, sizeof(xmap));
  if (!xtma || shared_rows) std::memset(&qmap, 0, sizeof(qmap));
  {
    Prof pf(c, KC_CONTRACT, (2.0 * fe + (a ? c->N : 0)) * sizeof(float2),
            8.0 * fe * c->n_elem);
    if (shared_rows && xtma)
      tc_contract_kernel<true, true><<<grid, C_THREADS, CRawT<true>::SMEM, c->stream>>>(
          args, xmap, qmap);
    else if (xtma)
      tc_contract_kernel<false, true><<<grid, C_THREADS, CRawT<false>::SMEM, c->stream>>>(
          args, xmap, qmap);
    else if (shared_rows)
      tc_contract_kernel<true, false><<<grid, C_THREADS, CRaw<true>::SMEM, c->stream>>>(
          args, xmap, qmap);
    else
      tc_contract_kernel<false, false><<<grid, C_THREADS, CRaw<false>::SMEM, c->stream>>>(
          args, xmap, qmap);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_fail(c, e, "tc_contract_kernel");
    return -1;
  }
  return split;
}

namespace {

template <bool FUSED, typename V>
int tc_mix(fwi_ctx* c, const V* B, const float2* X, const float2* Xe, int conj_x, float2* out,
           int kclass, double bytes, double flops) {
  cudaError_t e = set_attrs();
  if (e != cudaSuccess) {
    cuda_fail(c, e, "tc_mix attributes");
    return -1;
  }
  const int nbe = (c->n_elem + ROWS - 1) / ROWS;
  const int nks = (c->n_elem + KS - 1) / KS;
  const long long nseg = (long long)c->n_freq * nbe * nks * 2 * 2 * BROWS;
  {
    Prof pf(c, KC_MISC);
    tc_jh_bops_kernel<V><<<blocks_for(nseg, 256, c->n_sm * 8), 256, 0, c->stream>>>(
        B, (float*)c->tc_bops, c->n_elem, nbe, nks, nseg);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_fail(c, e, "tc_jh_bops_kernel");
    return -1;
  }
  const int npb = (int)((c->N + ROWS - 1) / ROWS);
  const int units = c->n_freq * nbe * npb;
  const int grid = units < c->n_sm ? units : c->n_sm;
  JhArgs args{X, Xe, (const float*)c->tc_bops, c->red, out, c->tc_err, c->N,
              c->n_elem, c->n_freq, nbe, nks, npb, units, conj_x};
  // the mixed operand [n_freq][NE][N] as a 3-D tensor of floats, box 8 rows
  // (one k-step of j) x 128 pixels
  CUtensorMap xmap;
  const bool xtma = c->jac_tma && field_tensor_map(c, X, 2 * ROWS, KS, false, &xmap);
  if (!xtma) std::memset(&xmap, 0, sizeof(xmap));
  {
    Prof pf(c, kclass, bytes, flops);
    if (xtma)
      tc_jh_kernel<FUSED, true><<<grid, C_THREADS, M_SMEM, c->stream>>>(args, xmap);
    else
      tc_jh_kernel<FUSED, false><<<grid, C_THREADS, M_SMEM, c->stream>>>(args, xmap);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_fail(c, e, "tc_jh_kernel");
    return -1;
  }
  return c->n_freq * nbe;
}

}  // namespace

// z_l[n] = s_l sum_e conj(X[e][n]) sum_j y[e][j] conj(Q[j][n]): Q the
// receiver fields (mixed by the MMAs), X the transmit fields (epilogue).
int tc_jh_partials(fwi_ctx* c, const double2* y, const float2* Q, const float2* X,
                   float2* zpart) {
  const double fe = (double)c->n_freq * c->n_elem * c->N;
  return tc_mix<true>(c, y, Q, X, 1, zpart, KC_MIX_JH, 2.0 * fe * sizeof(float2),
                      8.0 * fe * c->n_elem + 8.0 * fe);
}

int tc_adjoint_sources(fwi_ctx* c, const float2* B, const float2* Q, float2* out) {
  const double fe = (double)c->n_freq * c->n_elem * c->N;
  return tc_mix<false>(c, B, Q, nullptr, 0, out, KC_MIX_SOURCES, 2.0 * fe * sizeof(float2),
                       8.0 * fe * c->n_elem);
}

// The error word is read back with the callers' final synchronisation:
// tc_err_fetch enqueues the copy, tc_err_check inspects it after the sync.
void tc_err_fetch(fwi_ctx* c) {
  if (c->tc_err && c->h_tc_err)
    cudaMemcpyAsync(c->h_tc_err, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
}

fwi_status tc_err_check(fwi_ctx* c) {
  if (!c->h_tc_err || *c->h_tc_err == 0) return FWI_OK;
  const int code = *c->h_tc_err;
  *c->h_tc_err = 0;
  cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream);
  // codes 1-4: tensor-core contractions; 5-6: TMA staging of the column
  // passes; 7-8: bulk-copy staging of the row passes
  const char* where = code <= 4   ? "tensor-core contraction"
                      : code <= 6 ? "column pass TMA staging"
                                  : "row pass bulk-copy staging";
  return fail(c, FWI_ERR_CUDA, std::string(where) + ": pipeline wait timed out (code " +
                                   std::to_string(code) + ")");
}

}  // namespace fwi
