// Batched BiCGSTAB for the Lippmann-Schwinger systems A_l p = b,
// A_l = I - K_l diag(m) (Eq. 5; the paper solves them with a Krylov method,
// Sec. IV-A).  All right-hand sides of a batch iterate together in one
// persistent launch per pass; fields and operator applications are in the
// field precision, inner products, step scalars and the stopping test in
// FP64.  One iteration (van der Vorst's BiCGSTAB) is the pass sequence
//
//   col(conv) -> row_inv[v = p - K m p, <rhat,v>] -> S1 (alpha)
//   row_fwd[s = r - alpha v] -> col(conv) -> row_inv[t = s - K m s, dots]
//   S2 (omega, rho, beta, ||r||, convergence) -> compact
//   row_fwd[x += alpha p + omega s; r = s - omega t; p = r + beta (p - omega v)]
//
// captured once in a CUDA graph and replayed; the host reads the number of
// active right-hand sides between replays.  ||r_new||^2 = ||s||^2 -
// |<t,s>|^2/||t||^2 and rho_new = <rhat,s> - omega <rhat,t> come from the
// partial sums of the t-pass, so the x/r/p update fuses into the next
// forward row pass.  The last update of each finished RHS is applied by a
// final elementwise pass.
#include <sys/stat.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "ctx.cuh"
#include "prof.cuh"

namespace fwi {

namespace {

__device__ inline double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ inline double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ inline double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ inline double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ inline double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ inline bool zfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Warp-cooperative fixed-order sum of one slot's per-row partials.
__device__ inline double2 warp_slot_sum(const double2* part, int nparts, int lane) {
  double2 s = make_double2(0.0, 0.0);
  for (int i = lane; i < nparts; i += 32) s = zadd(s, part[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
  }
  return s;
}

// S0: initial state from the INIT (slot 0 = ||b||^2) or R0 (slot 0 =
// ||r0||^2, slot 1 = ||b||^2) partials.
__global__ void s0_kernel(Scal* scal, const double2* partial, int nparts, int nb,
                          int from_r0, double tol2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nb) return;
  const double2* p = partial + (long long)warp * NSLOT * nparts;
  const double r2 = warp_slot_sum(p, nparts, lane).x;
  const double b2 = from_r0 ? warp_slot_sum(p + nparts, nparts, lane).x : r2;
  if (lane == 0) {
    Scal s;
    s.rho = make_double2(r2, 0.0);
    s.alpha = make_double2(0.0, 0.0);
    s.omega = make_double2(0.0, 0.0);
    s.beta = make_double2(0.0, 0.0);
    s.bnorm2 = b2;
    s.rnorm2 = r2;
    s.iters = 0;
    s.pending = 0;
    const bool fin = isfinite(r2) && isfinite(b2);
    s.status = fin ? FWI_OK : FWI_ERR_NONFINITE;
    s.active = (fin && b2 > 0.0 && r2 > tol2 * b2) ? 1 : 0;
    scal[warp] = s;
  }
}

// S1: alpha = rho / <rhat, v>.
__global__ void s1_kernel(Scal* scal, const double2* partial, int nparts,
                          const int* active, const int* n_active) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= *n_active) return;
  const int rhs = active[warp];
  const double2 rv = warp_slot_sum(partial + (long long)rhs * NSLOT * nparts, nparts, lane);
  if (lane == 0) {
    Scal& s = scal[rhs];
    if (!zfinite(rv)) {
      s.status = FWI_ERR_NONFINITE;
      s.alpha = make_double2(0.0, 0.0);
    } else if (zabs2(rv) == 0.0) {
      s.status = FWI_ERR_BREAKDOWN;
      s.alpha = make_double2(0.0, 0.0);
    } else {
      s.alpha = zdiv(s.rho, rv);
    }
  }
}

// S2: omega, rho_new, ||r_new||^2, stopping test, beta.
__global__ void s2_kernel(Scal* scal, const double2* partial, int nparts,
                          const int* active, const int* n_active, double tol2,
                          int max_it) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= *n_active) return;
  const int rhs = active[warp];
  const double2* p = partial + (long long)rhs * NSLOT * nparts;
  const double2 ts = warp_slot_sum(p, nparts, lane);
  const double tt = warp_slot_sum(p + nparts, nparts, lane).x;
  const double2 rt = warp_slot_sum(p + 2 * nparts, nparts, lane);
  const double2 rs = warp_slot_sum(p + 3 * nparts, nparts, lane);
  const double ss = warp_slot_sum(p + 4 * nparts, nparts, lane).x;
  if (lane != 0) return;
  Scal& s = scal[rhs];
  s.iters += 1;
  if (s.status != FWI_OK) {  // breakdown / non-finite flagged in S1
    s.omega = make_double2(0.0, 0.0);
    s.active = 0;
    s.pending = (s.status == FWI_ERR_BREAKDOWN) ? 1 : 0;
    return;
  }
  if (!(zfinite(ts) && isfinite(tt) && zfinite(rt) && zfinite(rs) && isfinite(ss))) {
    s.status = FWI_ERR_NONFINITE;
    s.active = 0;
    s.pending = 0;
    return;
  }
  double2 omega = make_double2(0.0, 0.0);
  double rn2 = ss;
  if (tt > 0.0) {
    omega = make_double2(ts.x / tt, ts.y / tt);
    rn2 = ss - zabs2(ts) / tt;
    if (rn2 < 0.0) rn2 = 0.0;
  }
  const double2 rho_new = zsub(rs, zmul(omega, rt));
  s.omega = omega;
  s.rnorm2 = rn2;
  s.pending = 1;
  if (rn2 <= tol2 * s.bnorm2) {
    s.active = 0;
  } else if (s.iters >= max_it) {
    s.status = FWI_ERR_NOT_CONVERGED;
    s.active = 0;
  } else if (zabs2(omega) == 0.0 || zabs2(s.rho) == 0.0 || zabs2(rho_new) == 0.0) {
    s.status = FWI_ERR_BREAKDOWN;
    s.active = 0;
  } else {
    s.beta = zmul(zdiv(rho_new, s.rho), zdiv(s.alpha, omega));
    s.rho = rho_new;
    s.pending = 0;  // the update is fused into the next forward row pass
  }
}

// Active-list compaction in RHS order (one block).
__global__ void compact_kernel(const Scal* scal, int nb, int* active, int* n_active) {
  __shared__ int warp_tot[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int start = 0; start < nb; start += blockDim.x) {
    const int i = start + threadIdx.x;
    const int f = (i < nb && scal[i].active) ? 1 : 0;
    int incl = f;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int nw = blockDim.x >> 5;
      int v = (lane < nw) ? warp_tot[lane] : 0;
      int inc = v;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
      }
      if (lane < nw) warp_tot[lane] = inc - v;  // exclusive
    }
    __syncthreads();
    if (f) active[base + warp_tot[warp] + incl - 1] = i;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) base += warp_tot[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_active = base;
}

// Final update x += alpha p + omega s for every RHS with a pending update.
template <typename T>
__global__ void finalize_kernel(cplx<T>* X, const cplx<T>* P, const cplx<T>* S,
                                Scal* scal, int nb, long long N) {
  const long long total = N * nb;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(id / N);
    const Scal& s = scal[rhs];
    if (!s.pending) continue;
    const cplx<T> a = mk<T>((T)s.alpha.x, (T)s.alpha.y);
    const cplx<T> w = mk<T>((T)s.omega.x, (T)s.omega.y);
    X[id] = cadd(X[id], cadd(cmul(a, P[id]), cmul(w, S[id])));
  }
}

template <typename T>
__global__ void copy_conj_kernel(cplx<T>* dst, const cplx<T>* src, long long n, int conj) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    cplx<T> v = src[i];
    if (conj) v.y = -v.y;
    dst[i] = v;
  }
}

inline int blocks_for(long long n, int threads, int cap) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// Argument bundles for one batch, or for one half of a batch: the views
// of the per-RHS state (Krylov vectors, planes, scalars, partial sums,
// active list) start at slot `off` of the context's batch buffers, the
// half's active count lives in n_active[half], and its work goes to
// stream `st`.
template <typename T> struct Batch {
  fwi_ctx* c;
  int rhs0, nb;
  cplx<T>* X;
  cudaStream_t st;
  Scal* scal;
  double2* partial;
  int* active;
  int* n_active;
  RowFwdArgs<T> rf;
  RowInvArgs<T> ri;
  ColArgs<T> cz, cy_fwd, cy_inv;
};

template <typename T>
Batch<T> make_batch(fwi_ctx* c, cplx<T>* X, int rhs0, int nb, int off = 0, int half = 0,
                    cudaStream_t st = nullptr) {
  Batch<T> b{};
  b.c = c; b.rhs0 = rhs0; b.nb = nb; b.X = X;
  b.st = st ? st : c->stream;
  b.scal = c->scal + off;
  b.partial = c->partial + (long long)off * NSLOT * c->rows;
  b.active = c->active + off;
  b.n_active = c->n_active + half;
  const long long vo = (long long)off * c->N;
  cplx<T>* R = (cplx<T>*)c->kv[0] + vo;
  cplx<T>* RH = (cplx<T>*)c->kv[1] + vo;
  cplx<T>* P = (cplx<T>*)c->kv[2] + vo;
  cplx<T>* V = (cplx<T>*)c->kv[3] + vo;
  cplx<T>* Tt = (cplx<T>*)c->kv[4] + vo;
  cplx<T>* plane1 = (cplx<T>*)c->plane1 + (long long)off * c->rows * c->lx;
  cplx<T>* plane2 = c->plane2 ? (cplx<T>*)c->plane2 + (long long)off * c->nz * c->ly * c->lx
                              : nullptr;
  RowFwdArgs<T>& r = b.rf;
  r.m = (const cplx<T>*)c->mF; r.use_m = 1;
  r.X = X; r.R = R; r.RH = RH; r.P = P; r.V = V; r.Tt = Tt;
  r.plane = plane1; r.tw = (const cplx<T>*)c->tw_x;
  r.active = b.active; r.n_active = b.n_active; r.nb = nb;
  r.scal = b.scal; r.partial = b.partial;
  r.nx = c->nx; r.rows = c->rows; r.N = c->N; r.l2pf = c->row_l2pf;
  r.stage = c->row_stage; r.err = c->tc_err;
  {
    const int lpc = Lsop<T>::row_lines_per_cta(c->lx, c->var_rf);
    r.ntiles = (c->rows + lpc - 1) / lpc;
  }
  RowInvArgs<T>& q = b.ri;
  q.plane = plane1; q.m = (const cplx<T>*)c->mF;
  q.X = X; q.R = R; q.RH = RH; q.P = P; q.V = V; q.Tt = Tt;
  q.tw = (const cplx<T>*)c->tw_x;
  q.active = b.active; q.n_active = b.n_active; q.nb = nb;
  q.partial = b.partial; q.nx = c->nx; q.rows = c->rows; q.N = c->N; q.l2pf = c->row_l2pf;
  {
    const int lpc = Lsop<T>::row_lines_per_cta(c->lx, c->var_ri);
    q.ntiles = (c->rows + lpc - 1) / lpc;
  }
  const long long lyx = (long long)c->ly * c->lx;
  if (c->dim == 2) {
    ColArgs<T>& z = b.cz;
    z.mode = C_CONV; z.in = plane1; z.out = plane1;
    z.in_rhs_stride = z.out_rhs_stride = (long long)c->rows * c->lx;
    z.line_stride = c->lx; z.ncols = c->lx; z.nplanes = 1;
  } else {
    ColArgs<T>& y = b.cy_fwd;
    y.mode = C_FWD; y.in = plane1; y.out = plane2;
    y.in_rhs_stride = (long long)c->rows * c->lx;
    y.out_rhs_stride = (long long)c->nz * lyx;
    y.in_plane_stride = (long long)c->ny * c->lx; y.out_plane_stride = lyx;
    y.line_stride = c->lx; y.ncols = c->lx; y.nplanes = c->nz;
    y.tw = (const cplx<T>*)c->tw_y;
    ColArgs<T>& w = b.cy_inv;
    w = y;
    w.mode = C_INV; w.in = plane2; w.out = plane1;
    w.in_rhs_stride = y.out_rhs_stride; w.out_rhs_stride = y.in_rhs_stride;
    w.in_plane_stride = lyx; w.out_plane_stride = (long long)c->ny * c->lx;
    ColArgs<T>& z = b.cz;
    z.mode = C_CONV; z.in = plane2; z.out = plane2;
    z.in_rhs_stride = z.out_rhs_stride = (long long)c->nz * lyx;
    z.line_stride = lyx; z.ncols = (int)lyx; z.nplanes = 1;
  }
  for (ColArgs<T>* a : {&b.cz, &b.cy_fwd, &b.cy_inv}) {
    a->active = b.active; a->n_active = b.n_active; a->nb = nb;
    a->rhs0 = rhs0; a->n_elem = c->n_elem; a->freq_fixed = -1;
    a->tma = c->col_tma; a->gstage = c->col_gstage; a->pairs = c->col_pairs;
    a->err = c->tc_err;
  }
  b.cz.tw = (const cplx<T>*)c->tw_z;
  b.cz.ghat = (const cplx<T>*)c->ghat;
  b.cz.ghat_freq_stride = (long long)c->lz * lyx;
  b.cz.n_freq = c->n_freq;
  return b;
}

// Algorithmic HBM bytes of one pass for one right-hand side: every vector
// and plane element the pass must read or write once.
template <typename T> double pass_bytes(const fwi_ctx* c, int kind) {
  const double N = (double)c->N, e = (double)sizeof(cplx<T>);
  const double p1 = (double)c->rows * c->lx;
  const double p2 = (c->dim == 3) ? (double)c->nz * c->ly * c->lx : 0.0;
  switch (kind) {
    case KC_ROW_FWD_INIT: return (5 * N + p1) * e;   // b -> x, r, rhat, p; plane
    case KC_ROW_FWD_ITER: return (8 * N + p1) * e;   // x p s t v -> x r p; plane
    case KC_ROW_FWD_S: return (3 * N + p1) * e;      // r v -> s; plane
    case KC_ROW_FWD_PLAIN: return (N + p1) * e;
    case KC_COL_CONV: return (c->dim == 2 ? 2 * p1 : 2 * p2) * e;
    case KC_COL_FWD:
    case KC_COL_INV: return (p1 + p2) * e;
    case KC_ROW_INV_V:                               // plane p rhat -> v
    case KC_ROW_INV_T: return (3 * N + p1) * e;      // plane s rhat -> t
    default: return 0.0;
  }
}

// Nominal FFT flops of one column pass for one right-hand side: 5 L log2 L
// per complex L-point transform (forward and inverse along the column for
// the convolution, one transform for the 3-D y passes) plus 6 flops per
// spectrum multiply.
template <typename T> double pass_flops(const fwi_ctx* c, int kind) {
  auto fft = [](double L) { return 5.0 * L * std::log2(L); };
  const double lx = c->lx, ly = c->ly, lz = c->lz;
  switch (kind) {
    case KC_COL_CONV: return lx * ly * (2.0 * fft(lz) + 6.0 * lz);
    case KC_COL_FWD:
    case KC_COL_INV: return lx * (double)c->nz * fft(ly);
    default: return 0.0;
  }
}

// Ghat reads of one convolution launch (once per frequency).
template <typename T> double ghat_bytes(const fwi_ctx* c) {
  return (double)c->n_freq * c->lx * c->ly * c->lz * sizeof(cplx<T>);
}

// The column part of one operator application (between the row passes).
// `units`: right-hand sides the launch processes (for the byte count).
template <typename T> cudaError_t columns(const Batch<T>& b, bool use_list, double units) {
  fwi_ctx* c = b.c;
  ColArgs<T> z = b.cz;
  if (!use_list) z.active = nullptr;
  if (c->dim == 2) {
    Prof p(c, KC_COL_CONV, units * pass_bytes<T>(c, KC_COL_CONV) + ghat_bytes<T>(c),
           units * pass_flops<T>(c, KC_COL_CONV));
    return Lsop<T>::col(c->lz, z, b.st, c->var_cz);
  }
  ColArgs<T> y = b.cy_fwd, w = b.cy_inv;
  if (!use_list) { y.active = nullptr; w.active = nullptr; }
  cudaError_t e;
  {
    Prof p(c, KC_COL_FWD, units * pass_bytes<T>(c, KC_COL_FWD),
           units * pass_flops<T>(c, KC_COL_FWD));
    e = Lsop<T>::col(c->ly, y, b.st, c->var_cy);
  }
  if (e == cudaSuccess) {
    Prof p(c, KC_COL_CONV, units * pass_bytes<T>(c, KC_COL_CONV) + ghat_bytes<T>(c),
           units * pass_flops<T>(c, KC_COL_CONV));
    e = Lsop<T>::col(c->lz, z, b.st, c->var_cz);
  }
  if (e == cudaSuccess) {
    Prof p(c, KC_COL_INV, units * pass_bytes<T>(c, KC_COL_INV),
           units * pass_flops<T>(c, KC_COL_INV));
    e = Lsop<T>::col(c->ly, w, b.st, c->var_cy);
  }
  return e;
}

template <typename T> cudaError_t row_fwd(const Batch<T>& b, int mode, bool use_list,
                                          double units, const cplx<T>* in = nullptr,
                                          int conj_in = 0, int use_m = 1) {
  RowFwdArgs<T> r = b.rf;
  r.mode = mode; r.in = in; r.conj_in = conj_in; r.use_m = use_m;
  if (!use_list) r.active = nullptr;
  const int k = mode == RF_INIT ? KC_ROW_FWD_INIT : mode == RF_ITER ? KC_ROW_FWD_ITER
              : mode == RF_S ? KC_ROW_FWD_S : KC_ROW_FWD_PLAIN;
  Prof p(b.c, k, units * pass_bytes<T>(b.c, k));
  return Lsop<T>::row_fwd(b.c->lx, r, b.st, b.c->var_rf);
}

template <typename T> cudaError_t row_inv(const Batch<T>& b, int mode, bool use_list,
                                          double units, const cplx<T>* in = nullptr,
                                          cplx<T>* out = nullptr, const cplx<T>* B = nullptr,
                                          int conj_b = 0) {
  RowInvArgs<T> q = b.ri;
  q.mode = mode; q.in = in; q.out = out; q.B = B; q.conj_b = conj_b;
  if (!use_list) q.active = nullptr;
  const int k = mode == RI_V ? KC_ROW_INV_V : mode == RI_T ? KC_ROW_INV_T : KC_ROW_INV_OTHER;
  Prof p(b.c, k, units * pass_bytes<T>(b.c, k));
  return Lsop<T>::row_inv(b.c->lx, q, b.st, b.c->var_ri);
}

// Host copy of the active count (profiling mode only: synchronises).
inline int read_active(fwi_ctx* c, const int* n_active = nullptr) {
  if (cudaMemcpyAsync(c->h_n_active, n_active ? n_active : c->n_active, sizeof(int),
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return 0;
  cudaStreamSynchronize(c->stream);
  return *c->h_n_active;
}

// One BiCGSTAB iteration body (from the column pass of the first
// operator application to the fused update of the next iteration).
// `units`: active right-hand sides (byte accounting in profiling mode).
// `after_col`: if given, recorded on the batch's stream after the first
// column pass (used to start a second chain one pass behind).
template <typename T>
cudaError_t iteration(const Batch<T>& b, double units, cudaEvent_t after_col = nullptr) {
  fwi_ctx* c = b.c;
  const int wb = blocks_for((long long)b.nb * 32, 256, 1 << 30);
  const double tol2 = c->tol * c->tol;
  cudaError_t e = columns(b, true, units);
  if (e == cudaSuccess && after_col) e = cudaEventRecord(after_col, b.st);
  if (e == cudaSuccess) e = row_inv(b, RI_V, true, units);
  if (e == cudaSuccess) {
    Prof p(c, KC_KRYLOV_SCALAR);
    s1_kernel<<<wb, 256, 0, b.st>>>(b.scal, b.partial, c->rows, b.active, b.n_active);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = row_fwd(b, RF_S, true, units);
  if (e == cudaSuccess) e = columns(b, true, units);
  if (e == cudaSuccess) e = row_inv(b, RI_T, true, units);
  if (e == cudaSuccess) {
    Prof p(c, KC_KRYLOV_SCALAR);
    s2_kernel<<<wb, 256, 0, b.st>>>(b.scal, b.partial, c->rows, b.active, b.n_active, tol2,
                                   c->max_it);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    Prof p(c, KC_KRYLOV_SCALAR);
    compact_kernel<<<1, 1024, 0, b.st>>>(b.scal, b.nb, b.active, b.n_active);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const double u2 =
        (c->profiling && !c->capturing) ? (double)read_active(c, b.n_active) : units;
    e = row_fwd(b, RF_ITER, true, u2);
  }
  return e;
}

constexpr int kGraphIters = 4;
// Smallest half-batch for which the iterations run as two chains.
constexpr int kMinHalf = 16;

template <typename T>
fwi_status solve_batch(fwi_ctx* c, const cplx<T>* bvec, int conj_b, cplx<T>* X, bool warm,
                       int rhs0, int nb) {
  Batch<T> b = make_batch<T>(c, X, rhs0, nb);
  const double tol2 = c->tol * c->tol;
  const int wb = blocks_for((long long)nb * 32, 256, 1 << 30);
  // With a large enough batch the iterations run as two independent halves
  // on two streams of one graph, so that each chain's passes can start on
  // SMs the other chain's passes leave idle.  The halves share no
  // data, so every right-hand side follows exactly the same arithmetic as
  // in one chain.  Profiling mode times each launch and keeps one chain.
  const bool two = c->overlap && !c->profiling && c->stream2 != nullptr && nb >= 2 * kMinHalf;
  const int h0 = two ? nb / 2 : nb;
  const int nchains = two ? 2 : 1;
  Batch<T> hb[2] = {b, b};
  if (two) {
    hb[0] = make_batch<T>(c, X, rhs0, h0, 0, 0);
    hb[1] = make_batch<T>(c, X + (long long)h0 * c->N, rhs0 + h0, nb - h0, h0, 1);
  }
  // ---- initial residual and first search direction (whole batch) ----
  if (!warm) {
    FWI_CUDA(c, row_fwd(b, RF_INIT, false, nb, bvec, conj_b));
    Prof p(c, KC_KRYLOV_SCALAR);
    s0_kernel<<<wb, 256, 0, c->stream>>>(c->scal, c->partial, c->rows, nb, 0, tol2);
  } else {
    FWI_CUDA(c, row_fwd(b, RF_PLAIN, false, nb, X, 0));
    FWI_CUDA(c, columns(b, false, nb));
    FWI_CUDA(c, row_inv(b, RI_R0, false, nb, nullptr, nullptr, bvec, conj_b));
    Prof p(c, KC_KRYLOV_SCALAR);
    s0_kernel<<<wb, 256, 0, c->stream>>>(c->scal, c->partial, c->rows, nb, 1, tol2);
  }
  FWI_CUDA(c, cudaGetLastError());
  {
    Prof p(c, KC_KRYLOV_SCALAR, 0.0, 0.0, nchains);
    for (int k = 0; k < nchains; ++k)
      compact_kernel<<<1, 1024, 0, c->stream>>>(hb[k].scal, hb[k].nb, hb[k].active,
                                                hb[k].n_active);
  }
  FWI_CUDA(c, cudaGetLastError());
  if (warm) {
    for (int k = 0; k < nchains; ++k) {
      const double u = c->profiling ? (double)read_active(c, hb[k].n_active) : hb[k].nb;
      FWI_CUDA(c, row_fwd(hb[k], RF_START, true, u));
    }
  }
  const int max_replays = (c->max_it + kGraphIters - 1) / kGraphIters + 1;
  if (c->profiling) {
    // eager iterations, every pass bracketed by events
    for (int it = 0; it < c->max_it + 1; ++it) {
      const int na = read_active(c);
      if (na == 0) break;
      if (c->cancel.load()) return fail(c, FWI_ERR_CANCELLED, "solve cancelled");
      FWI_CUDA(c, iteration(b, (double)na));
      prof_flush(c);
    }
  } else {
    // ---- iterations: graph of kGraphIters bodies (per chain), replayed ----
    auto key = std::make_tuple((const void*)X, rhs0, nb, nchains);
    fwi_ctx::GraphRec rec{nullptr, 0};
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) {
      rec = it->second;
    } else {
      cudaGraph_t g = nullptr;
      FWI_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      c->capturing = true;
      c->capture_nodes = 0;
      cudaError_t e = cudaSuccess;
      if (two) {
        // both chains launch full persistent grids: a pass of one chain fills
        // the SMs that the other chain's pass leaves idle in its tail
        Batch<T> b0 = hb[0], b1 = hb[1];
        b1.st = c->stream2;
        // chain B starts when chain A's first column pass is done, so that
        // the chains run one pass apart and their passes interleave
        e = cudaEventRecord(c->ev_fork, c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream2, c->ev_fork, 0);
        for (int k = 0; k < kGraphIters && e == cudaSuccess; ++k) {
          e = iteration(b0, b0.nb);
          if (e == cudaSuccess) e = iteration(b1, b1.nb);
        }
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->stream2);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
      } else {
        for (int k = 0; k < kGraphIters && e == cudaSuccess; ++k) e = iteration(b, nb);
      }
      c->capturing = false;
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e, "capturing the Krylov iteration");
      }
      FWI_CUDA(c, e2);
      e = cudaGraphInstantiate(&rec.exec, g, 0);
      cudaGraphDestroy(g);
      FWI_CUDA(c, e);
      rec.nodes = c->capture_nodes;
      c->graphs[key] = rec;
    }
    for (int rep = 0; rep < max_replays; ++rep) {
      FWI_CUDA(c, cudaMemcpyAsync(c->h_n_active, c->n_active, sizeof(int) * nchains,
                                  cudaMemcpyDeviceToHost, c->stream));
      FWI_CUDA(c, cudaStreamSynchronize(c->stream));
      int act = 0;
      for (int k = 0; k < nchains; ++k) act += c->h_n_active[k];
      if (act == 0) break;
      if (c->cancel.load()) return fail(c, FWI_ERR_CANCELLED, "solve cancelled");
      FWI_CUDA(c, cudaGraphLaunch(rec.exec, c->stream));
      c->launches += rec.nodes;
    }
  }
  // ---- pending updates ----
  {
    Prof p(c, KC_FINALIZE);
    finalize_kernel<T><<<blocks_for(c->N * nb, 256, c->n_sm * 16), 256, 0, c->stream>>>(
        X, (const cplx<T>*)c->kv[2], (const cplx<T>*)c->kv[0], c->scal, nb, c->N);
  }
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

void fill_info(fwi_ctx* c, fwi_solve_info* info, int rhs0, int nb, bool first) {
  if (!info) return;
  if (first) {
    info->max_iters = 0;
    info->max_rel_resid = 0.0;
    info->n_not_converged = 0;
  }
  for (int i = 0; i < nb; ++i) {
    const Scal& s = c->h_scal[i];
    const double rr = s.bnorm2 > 0 ? std::sqrt(s.rnorm2 / s.bnorm2) : 0.0;
    const int g = rhs0 + i;
    if (g < info->n_rhs) {
      if (info->iters) info->iters[g] = s.iters;
      if (info->rel_resid) info->rel_resid[g] = rr;
      if (info->status) info->status[g] = s.status;
    }
    if (s.iters > info->max_iters) info->max_iters = s.iters;
    if (rr > info->max_rel_resid) info->max_rel_resid = rr;
    if (s.status != FWI_OK) info->n_not_converged += 1;
  }
}

template <typename T>
fwi_status solve_all(fwi_ctx* c, const cplx<T>* bvec, int conj_b, cplx<T>* X, bool warm,
                     fwi_solve_info* info) {
  FWI_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  fwi_status worst = FWI_OK;
  for (int rhs0 = 0; rhs0 < c->n_rhs; rhs0 += c->batch) {
    const int nb = (c->n_rhs - rhs0 < c->batch) ? c->n_rhs - rhs0 : c->batch;
    fwi_status st = solve_batch<T>(c, bvec + (long long)rhs0 * c->N, conj_b,
                                   X + (long long)rhs0 * c->N, warm, rhs0, nb);
    if (st != FWI_OK) return st;
    FWI_CUDA(c, cudaMemcpyAsync(c->h_scal, c->scal, sizeof(Scal) * nb,
                                cudaMemcpyDeviceToHost, c->stream));
    FWI_CUDA(c, cudaStreamSynchronize(c->stream));
    fill_info(c, info, rhs0, nb, rhs0 == 0);
    for (int i = 0; i < nb; ++i) {
      const int s = c->h_scal[i].status;
      if (s != FWI_OK && (worst == FWI_OK || s == FWI_ERR_NONFINITE)) worst = (fwi_status)s;
    }
  }
  FWI_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  FWI_CUDA(c, cudaEventSynchronize(c->ev1));
  prof_flush(c);
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->device_ms = ms;
  }
  if (worst != FWI_OK) {
    const char* what = worst == FWI_ERR_NOT_CONVERGED ? "some right-hand sides hit krylov_max_it"
                       : worst == FWI_ERR_BREAKDOWN   ? "BiCGSTAB breakdown"
                                                      : "non-finite value in a Krylov reduction";
    return fail(c, worst, what);
  }
  return FWI_OK;
}

template <typename T>
fwi_status apply_op_t(fwi_ctx* c, int kind, const void* m, int freq, int n_rhs,
                      const void* in, void* out) {
  if (m) {
    fwi_status st = set_contrast(c, m);
    if (st != FWI_OK) return st;
  }
  Batch<T> b = make_batch<T>(c, (cplx<T>*)c->kv[0], 0, n_rhs);
  b.cz.freq_fixed = freq;  // every vector of the call is at frequency `freq`
  const cplx<T>* src = (const cplx<T>*)in;
  if (kind == 0) {  // K
    FWI_CUDA(c, row_fwd(b, RF_PLAIN, false, n_rhs, src, 0, 0));
    FWI_CUDA(c, columns(b, false, n_rhs));
    FWI_CUDA(c, row_inv(b, RI_K, false, n_rhs, nullptr, (cplx<T>*)out));
  } else if (kind == 1) {  // A
    FWI_CUDA(c, row_fwd(b, RF_PLAIN, false, n_rhs, src, 0, 1));
    FWI_CUDA(c, columns(b, false, n_rhs));
    FWI_CUDA(c, row_inv(b, RI_A, false, n_rhs, src, (cplx<T>*)out));
  } else {  // A^H
    FWI_CUDA(c, row_fwd(b, RF_PLAIN, false, n_rhs, src, 1, 0));
    FWI_CUDA(c, columns(b, false, n_rhs));
    FWI_CUDA(c, row_inv(b, RI_AH, false, n_rhs, src, (cplx<T>*)out));
  }
  return FWI_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times every tile-shape variant of the operator passes on the
// context's full batch (scratch vectors) and keeps the fastest.  Variants
// differ only in how many lines / columns a CTA holds; every one gives
// bitwise-identical results.  Choices are cached in a text file keyed by
// (architecture, precision, length, batch, pass).
std::string tune_cache_path() {
  const char* p = std::getenv("LIBFWI_TUNE_CACHE");
  if (p && *p) return p;
  const char* h = std::getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/libfwi/autotune.txt";
}

std::map<std::string, int> read_tune_cache() {
  std::map<std::string, int> m;
  FILE* f = std::fopen(tune_cache_path().c_str(), "r");
  if (!f) return m;
  char key[256];
  int v = 0;
  while (std::fscanf(f, "%255s %d", key, &v) == 2) m[key] = v;
  std::fclose(f);
  return m;
}

void append_tune_cache(const std::vector<std::pair<std::string, int>>& rows) {
  const std::string path = tune_cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    std::string dir = path.substr(0, slash);
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);  // parents, no shell
  }
  FILE* f = std::fopen(path.c_str(), "a");
  if (!f) return;
  for (auto& r : rows) std::fprintf(f, "%s %d\n", r.first.c_str(), r.second);
  std::fclose(f);
}

template <typename T>
fwi_status autotune_t(fwi_ctx* c) {
  const char* env = std::getenv("LIBFWI_AUTOTUNE");
  if (env && env[0] == '0') return FWI_OK;
  const int nvr = Lsop<T>::variants(c->lx, 0);
  const int nvc = Lsop<T>::variants(c->lz, 2);
  const int nvy = c->dim == 3 ? Lsop<T>::variants(c->ly, 2) : 1;
  if (nvr <= 1 && nvc <= 1 && nvy <= 1) return FWI_OK;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
  char base[160];
  std::snprintf(base, sizeof(base), "sm%d%d|%s|d%d|%dx%dx%d|b%d|", major, minor,
                sizeof(T) == 4 ? "c64" : "c128", c->dim, c->lx, c->ly, c->lz, c->batch);
  const std::string kb(base);
  const char* kinds[4] = {"row_fwd", "row_inv", "col_z", "col_y"};
  std::map<std::string, int> cache = read_tune_cache();
  int* vars[4] = {&c->var_rf, &c->var_ri, &c->var_cz, &c->var_cy};
  const int nv[4] = {nvr, Lsop<T>::variants(c->lx, 1), nvc, nvy};
  bool all_cached = true;
  for (int k = 0; k < 4; ++k) {
    auto it = cache.find(kb + kinds[k]);
    if (nv[k] > 1 && it == cache.end()) all_cached = false;
  }
  if (all_cached) {
    for (int k = 0; k < 4; ++k) {
      auto it = cache.find(kb + kinds[k]);
      if (it != cache.end() && it->second >= 0 && it->second < nv[k]) *vars[k] = it->second;
    }
    return FWI_OK;
  }
  // scratch: zero input vectors in kv[0], output into kv[1]
  const long long nvec = c->N * (long long)c->batch;
  FWI_CUDA(c, cudaMemsetAsync(c->kv[0], 0, sizeof(cplx<T>) * nvec, c->stream));
  const bool saved_prof = c->profiling;
  c->profiling = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FWI_CUDA(c, cudaEventCreate(&e0));
  FWI_CUDA(c, cudaEventCreate(&e1));
  auto time_it = [&](auto launch) -> float {
    cudaError_t e = launch();  // warm-up (also sets up the launch grid)
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch();
    if (e != cudaSuccess) return -1.f;
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch();
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return e == cudaSuccess ? ms / 3.f : -1.f;
  };
  std::vector<std::pair<std::string, int>> rows;
  Batch<T> b = make_batch<T>(c, (cplx<T>*)c->kv[2], 0, c->batch);
  b.cz.freq_fixed = 0;
  const cplx<T>* src = (const cplx<T>*)c->kv[0];
  cplx<T>* dst = (cplx<T>*)c->kv[1];
  for (int k = 0; k < 4; ++k) {
    if (nv[k] <= 1) continue;
    float best = 1e30f;
    int bestv = 0;
    for (int v = 0; v < nv[k]; ++v) {
      float ms = -1.f;
      if (k == 0) {
        RowFwdArgs<T> r = b.rf;
        r.mode = RF_PLAIN; r.in = src; r.use_m = 1; r.active = nullptr;
        const int lpc = Lsop<T>::row_lines_per_cta(c->lx, v);
        r.ntiles = (c->rows + lpc - 1) / lpc;
        ms = time_it([&] { return Lsop<T>::row_fwd(c->lx, r, c->stream, v); });
      } else if (k == 1) {
        RowInvArgs<T> q = b.ri;
        q.mode = RI_A; q.in = src; q.out = dst; q.active = nullptr;
        const int lpc = Lsop<T>::row_lines_per_cta(c->lx, v);
        q.ntiles = (c->rows + lpc - 1) / lpc;
        ms = time_it([&] { return Lsop<T>::row_inv(c->lx, q, c->stream, v); });
      } else if (k == 2) {
        ColArgs<T> z = b.cz;
        z.active = nullptr;
        ms = time_it([&] { return Lsop<T>::col(c->lz, z, c->stream, v); });
      } else {
        ColArgs<T> y = b.cy_fwd;
        y.active = nullptr;
        ms = time_it([&] { return Lsop<T>::col(c->ly, y, c->stream, v); });
      }
      c->tune_ms[k][v] = ms;
      if (ms > 0.f && ms < best) {
        best = ms;
        bestv = v;
      }
    }
    *vars[k] = bestv;
    rows.emplace_back(kb + kinds[k], bestv);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->profiling = saved_prof;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
  c->tuned = 1;
  append_tune_cache(rows);
  return FWI_OK;
}

}  // namespace

fwi_status autotune(fwi_ctx* c) {
  return c->fp64 ? autotune_t<double>(c) : autotune_t<float>(c);
}

fwi_status forward_solve(fwi_ctx* c, const void* m, bool warm, fwi_solve_info* info) {
  fwi_status st = set_contrast(c, m);
  if (st != FWI_OK) return st;
  st = c->fp64 ? solve_all<double>(c, (const double2*)c->p0, 0, (double2*)c->fields, warm, info)
               : solve_all<float>(c, (const float2*)c->p0, 0, (float2*)c->fields, warm, info);
  c->fields_valid = (st == FWI_OK || st == FWI_ERR_NOT_CONVERGED);
  return st;
}

// Solves A y = conj(src) (conj_src = 1) or A y = src (conj_src = 0) into
// c->lam.  The adjoint field is lambda = conj(y).
fwi_status adjoint_solve(fwi_ctx* c, const void* m, const void* src, bool conj_src,
                         fwi_solve_info* info) {
  fwi_status st = set_contrast(c, m);
  if (st != FWI_OK) return st;
  return c->fp64 ? solve_all<double>(c, (const double2*)src, conj_src, (double2*)c->lam, false, info)
                 : solve_all<float>(c, (const float2*)src, conj_src, (float2*)c->lam, false, info);
}

fwi_status apply_op(fwi_ctx* c, int kind, const void* m, int freq, int n_rhs,
                    const void* in, void* out) {
  return c->fp64 ? apply_op_t<double>(c, kind, m, freq, n_rhs, in, out)
                 : apply_op_t<float>(c, kind, m, freq, n_rhs, in, out);
}

fwi_status copy_field(fwi_ctx* c, void* dst, const void* src, long long n, int conj) {
  const int blocks = blocks_for(n, 256, c->n_sm * 16);
  Prof p(c, KC_MISC, 2.0 * n * c->csz);
  if (c->fp64)
    copy_conj_kernel<double><<<blocks, 256, 0, c->stream>>>((double2*)dst, (const double2*)src, n, conj);
  else
    copy_conj_kernel<float><<<blocks, 256, 0, c->stream>>>((float2*)dst, (const float2*)src, n, conj);
  FWI_CUDA(c, cudaGetLastError());
  return FWI_OK;
}

}  // namespace fwi
