// Host-side context of libfwi: descriptor copy, device workspace and the
// cached CUDA graphs.  Shared by the library's translation units.
#pragma once

#include <atomic>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/libfwi.h"
#include "common.cuh"

struct fwi_ctx {
  // ---- problem ----
  int dim = 2;
  int nx = 0, ny = 1, nz = 0;       // grid
  int lx = 0, ly = 1, lz = 0;       // doubled lattice
  long long N = 0;                  // voxels
  int rows = 0;                     // x-lines per field (ny * nz)
  int n_elem = 0, n_freq = 0, n_rhs = 0, batch = 0;
  double h = 0, c0 = 0, tol = 1e-6;
  int max_it = 1000;
  bool fp64 = false;
  size_t csz = 8;                   // bytes of one field element
  std::vector<double> elem, freq, kwave;
  // plane-wave transmits (0: point transmits at every element); n_t = N_T
  int n_tx = 0, n_t = 0;
  std::vector<double> tx_angle;
  double elem_length = 0;           // 3D line elements along y (0: points)
  // attenuating background: complex k_l, and the complex scales k_l^2 dV
  // applied in data space (the contraction kernels then scale by 1)
  double alpha0 = 0;
  std::vector<double2> kc;
  double2* sdat = nullptr;          // [n_freq] k_l^2 dV (lossy only)
  double2* dlossy = nullptr;        // [n_freq][n_elem][n_elem] scratch (lossy only)
  // inversion mesh: cells of rf x ry x rf pixels (ry = 1 in 2D)
  int rf = 1, ry = 1, inx = 0, iny = 1, inz = 0;
  long long Ninv = 0;
  // ---- device ----
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;  // created when the caller passes NULL
  cudaStream_t stream2 = nullptr;     // second chain of the Krylov iteration graph
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool overlap = true;                // iterate large batches as two chains (2-D default)
  int device = 0, n_sm = 0;
  // workspace (field precision unless noted)
  void* ghat = nullptr;             // [n_freq][lz][ly][lx], scaled k^2/(lx ly lz)
  void* tw_x = nullptr;             // twiddle tables exp(-2 pi i j/L)
  void* tw_y = nullptr;
  void* tw_z = nullptr;
  void* p0 = nullptr;               // [n_rhs][N] incident fields
  void* fields = nullptr;           // [n_rhs][N] forward solution
  void* rfields = nullptr;          // [n_rhs][N] receiver-field snapshot (hybrid_born)
  bool rfields_frozen = false;      // J / J^H take ptilde from rfields
  void* lam = nullptr;              // [n_rhs][N] adjoint work / solution
  void* asrc = nullptr;             // [n_rhs][N] adjoint right-hand sides
  void* kv[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // R, RH, P, V, T
  void* plane1 = nullptr;           // [batch][rows][lx]
  void* plane2 = nullptr;           // 3D: [batch][nz][ly][lx]
  void* mF = nullptr;               // [N] contrast in field precision
  fwi::Scal* scal = nullptr;        // [batch]
  double2* partial = nullptr;       // [batch][NSLOT][ntiles]
  int ntiles = 0;
  int* active = nullptr;            // [batch]
  int* n_active = nullptr;          // [1]
  int* h_n_active = nullptr;        // pinned host mirror
  fwi::Scal* h_scal = nullptr;      // pinned host mirror [batch]
  // Jacobian / data / ADMM workspace
  double2* dres = nullptr;          // [n_freq][n_elem][n_elem] c128 scratch
  void* dF = nullptr;               // [n_freq][max(n_t, n_elem)][n_elem] field precision
  double2* W = nullptr;             // [n_freq][n_tx][n_elem] plane-wave weights
  double2* WhW = nullptr;           // [n_freq][n_elem][n_elem] W^H W
  double2* dpw = nullptr;           // [n_freq][n_tx][n_elem] plane-wave data / residual
  double2* dsyn = nullptr;          // [n_freq][n_elem][n_elem] synthesis scratch
  void* jsplit = nullptr;           // split-K partials of pixel contractions
  int jsplit_n = 0;
  void* zpart = nullptr;            // per-(freq, e-block) partials of J^H
  void* aF = nullptr;               // [N] field-precision vector
  double2* vN[8] = {};              // [N] c128 ADMM / CG vectors
  double2* vD[3] = {};              // [dim][N] c128 ADMM vectors
  double2* vfwd = nullptr;          // [N] c128 forward-mesh scratch (inversion mesh only)
  void* tc_bops = nullptr;          // tensor-core J^H: B operand stages (FP32 only)
  int* tc_err = nullptr;            // error word of the tensor-core kernels
  int* h_tc_err = nullptr;          // pinned host mirror
  bool use_tc = true;               // tensor-core pixel contractions (FP32 fields)
  int col_tma = 1;                  // column passes stage tiles with TMA (FP32)
  int col_gstage = 1;               // ... and the convolution's kernel-spectrum tiles
  int row_l2pf = 1;                 // row passes prefetch their next item into L2
  int jac_tma = 1;                  // tensor-core contractions take raw tiles by TMA
  int row_stage = 1;                // forward row pass stages its rows (FP32)
  int col_pairs = 1;                // convolution: two columns per thread (FP32)
  int tc_stall = 0;                 // next contraction withholds its first stage (test)
  double* red = nullptr;            // reduction scratch (doubles)
  double* h_red = nullptr;          // pinned host mirror
  int red_n = 0;
  bool fields_valid = false;
  // graphs keyed by (solution pointer, batch start, batch size, chains),
  // with the number of kernel nodes each replay launches
  struct GraphRec { cudaGraphExec_t exec; long long nodes; };
  std::map<std::tuple<const void*, int, int, int>, GraphRec> graphs;
  // tile-shape variants of the operator passes (autotuned at creation)
  int var_rf = 0, var_ri = 0, var_cz = 0, var_cy = 0;
  int tuned = 0;
  float tune_ms[4][4] = {};
  // instrumentation (launch counts always; event timing when profiling)
  long long launches = 0;
  bool capturing = false;
  long long capture_nodes = 0;
  bool profiling = false;
  struct KStat { double ms = 0, bytes = 0, flops = 0; long long launches = 0; };
  KStat kstats[32];
  struct Pending { int cls; cudaEvent_t a, b; double bytes, flops; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // caller-supplied sum over ranks (frequency sharding), or none
  fwi_reduce_fn reduce_fn = nullptr;
  void* reduce_user = nullptr;
  std::atomic<bool> cancel{false};
  std::string err;
  size_t bytes = 0;
};

// Implemented in the library's units.
namespace fwi {
fwi_status fail(fwi_ctx* c, fwi_status s, const std::string& msg);
fwi_status cuda_fail(fwi_ctx* c, cudaError_t e, const char* where);
size_t workspace_bytes(const fwi_problem_desc* d, std::string* why);
fwi_status setup_operator(fwi_ctx* c);
fwi_status autotune(fwi_ctx* c);
fwi_status forward_solve(fwi_ctx* c, const void* m, bool warm, fwi_solve_info* info);
fwi_status adjoint_solve(fwi_ctx* c, const void* m, const void* src, bool conj_src,
                         fwi_solve_info* info);
fwi_status set_contrast(fwi_ctx* c, const void* m);
fwi_status apply_op(fwi_ctx* c, int kind, const void* m, int freq, int n_rhs,
                    const void* in, void* out);
// data / Jacobian / ADMM
fwi_status project_data(fwi_ctx* c, const void* m, void* data_out);
fwi_status residual_misfit(fwi_ctx* c, const void* d_obs, double* misfit);
fwi_status adjoint_sources_conj(fwi_ctx* c, void* out);
fwi_status assemble_gradient(fwi_ctx* c, void* grad);
fwi_status jac_forward(fwi_ctx* c, const void* a_c128, double2* y);
fwi_status jac_adjoint(fwi_ctx* c, const double2* y, double2* z);
// Sum of `count` doubles at device address buf over the ranks of a
// frequency-sharded run (the caller's reducer; a no-op without one).
fwi_status reduce_sum(fwi_ctx* c, void* buf, size_t count);
// the fields the Jacobian's receiver side (ptilde) is taken from
inline const void* receiver_fields(const fwi_ctx* c) {
  return c->rfields_frozen ? c->rfields : c->fields;
}
// plane-wave synthesis out[l] = op(A[l]) in[l] (op: A, or A^H when herm),
// op(A[l]) of R x K, in[l] of K x n_elem; conj_out (field precision) or NULL
fwi_status synth(fwi_ctx* c, const double2* A, int herm, int R, int K, const double2* in,
                 double2* out, void* conj_out);
fwi_status admm_init(fwi_ctx* c, const void* m0, void* g, void* u);
fwi_status admm_step(fwi_ctx* c, void* m, void* g, void* u, const void* grad,
                     const fwi_admm_params* p, double* sos);
fwi_status contrast_from_sos(fwi_ctx* c, const double* sos, const double* alpha, void* m);
fwi_status sos_attenuation_from_contrast(fwi_ctx* c, const void* m, double* sos, double* alpha);
// tensor-core pixel contractions (jac_tc.cu)
bool tc_usable(const fwi_ctx* c);
size_t tc_bops_bytes(int n_elem, int n_freq);
int tc_contract_partials(fwi_ctx* c, const float2* X, const float2* a, const float2* Q,
                         float2* part);
int tc_jh_partials(fwi_ctx* c, const double2* y, const float2* Q, const float2* X,
                   float2* zpart);
int tc_adjoint_sources(fwi_ctx* c, const float2* B, const float2* Q, float2* out);
void tc_err_fetch(fwi_ctx* c);
fwi_status tc_err_check(fwi_ctx* c);
}  // namespace fwi

#define FWI_CUDA(c, call)                                          \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return fwi::cuda_fail((c), e_, #call);  \
  } while (0)
