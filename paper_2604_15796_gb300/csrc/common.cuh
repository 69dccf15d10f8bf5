// Shared declarations of libfwi's CUDA sources: complex helpers, the
// per-right-hand-side Krylov scalar record, and error plumbing.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "fft_core.cuh"

namespace fwi {

// Per-RHS BiCGSTAB state (FP64 scalars, Sec. IV-A solver; van der Vorst's
// BiCGSTAB with the residual norm updated from the s/t inner products).
struct Scal {
  double2 rho;     // <rhat, r>
  double2 alpha;   // rho / <rhat, v>
  double2 omega;   // <t, s> / <t, t>
  double2 beta;    // (rho_new / rho) (alpha / omega)
  double bnorm2;   // ||b||^2
  double rnorm2;   // ||r||^2 (recursive estimate)
  int iters;       // completed iterations
  int status;      // fwi_status code of this RHS
  int pending;     // 1: the last x/r update is still to be applied
  int active;      // 1 while the RHS iterates
};

// Number of complex partial-sum slots per row tile.
constexpr int NSLOT = 5;

enum RowFwdMode { RF_PLAIN = 0, RF_INIT = 1, RF_START = 2, RF_ITER = 3, RF_S = 4 };
enum RowInvMode { RI_K = 0, RI_A = 1, RI_AH = 2, RI_V = 3, RI_T = 4, RI_R0 = 5 };
enum ColMode { C_CONV = 0, C_FWD = 1, C_INV = 2 };

template <typename T> struct RowFwdArgs {
  int mode;
  int conj_in;     // PLAIN / INIT: use conj(in)
  int use_m;       // multiply the FFT input by m
  int full;        // input rows hold L samples (no zero padding), pitch L
  const cplx<T>* in;   // PLAIN / INIT source, [B][N] (or [B][rows][L] if full)
  const cplx<T>* m;    // [N] contrast (field precision)
  cplx<T>* X; cplx<T>* R; cplx<T>* RH; cplx<T>* P; cplx<T>* V; cplx<T>* Tt;
  cplx<T>* plane;      // out: [B][rows][L]
  const cplx<T>* tw;   // twiddles exp(-2 pi i j / L), j < L
  const int* active;   // active RHS list, or NULL for 0..nb-1
  const int* n_active;
  int nb;
  const Scal* scal;
  double2* partial;    // [B][NSLOT][rows] per-row partial sums
  int nx;              // samples per input row (L/2, or L if full)
  int rows;            // lines per RHS
  int ntiles;
  long long N;         // elements per RHS vector
  int l2pf;            // prefetch the next item's rows into L2
  int stage;           // FP32, zero-padded rows: stage the rows with bulk copies
  int* err;            // error word of bounded waits (or NULL)
};

template <typename T> struct RowInvArgs {
  int mode;
  int conj_b;
  const cplx<T>* plane;  // in: [B][rows][L]
  const cplx<T>* in;     // A / AH: the vector the operator acts on
  cplx<T>* out;          // K / A / AH result
  const cplx<T>* m;
  const cplx<T>* B;      // R0: right-hand side
  cplx<T>* X; cplx<T>* R; cplx<T>* RH; cplx<T>* P; cplx<T>* V; cplx<T>* Tt;
  const cplx<T>* tw;
  const int* active; const int* n_active; int nb;
  double2* partial;
  int nx, rows, ntiles;
  long long N;
  int l2pf;              // prefetch the next item's rows into L2
};

template <typename T> struct ColArgs {
  int mode;
  int full;                 // FWD: input holds all L samples of each line
  const cplx<T>* in; cplx<T>* out;
  long long in_rhs_stride, out_rhs_stride;
  long long in_plane_stride, out_plane_stride;
  long long line_stride;    // element distance between samples of a line
  int ncols, nplanes;
  const cplx<T>* ghat;      // CONV: [freq][L][ncols], scaled
  long long ghat_freq_stride;
  int n_freq;               // frequencies held in ghat
  const cplx<T>* tw;
  const int* active; const int* n_active; int nb;
  int rhs0, n_elem;         // global RHS index = rhs0 + slot; freq = idx / n_elem
  int freq_fixed;           // >= 0: every RHS uses this frequency
  int tma;                  // FP32, zero-padded input: stage tiles with TMA
  int gstage;               // with tma: also stage the kernel-spectrum tiles
  int pairs;                // with gstage: two columns per thread where the plan allows
  int* err;                 // error word of bounded waits (or NULL)
};

// Host-side launch interface, specialised per precision in the
// instantiation units.  L is the transform length along the pass axis.
// ``var`` selects a tile-shape variant (0 = default; see Lsop::variants).
template <typename T> struct Lsop {
  static bool supported(int L);
  static int variants(int L, int kind);  // kind 0 row_fwd, 1 row_inv, 2 col
  static cudaError_t row_fwd(int L, const RowFwdArgs<T>& a, cudaStream_t s, int var = 0);
  static cudaError_t row_inv(int L, const RowInvArgs<T>& a, cudaStream_t s, int var = 0);
  static cudaError_t col(int L, const ColArgs<T>& a, cudaStream_t s, int var = 0);
  static int row_lines_per_cta(int L, int var = 0);
};

}  // namespace fwi
