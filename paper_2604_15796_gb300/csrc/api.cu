// C entry points of libfwi (include/libfwi.h): argument checks, context
// creation and workspace accounting, and the composition of the hot-path
// steps into the calls of the paper's problem statement (Sec. II-III).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "ctx.cuh"
#include "prof.cuh"

namespace fwi {

static thread_local std::string g_create_error;

fwi_status fail(fwi_ctx* c, fwi_status s, const std::string& msg) {
  if (c) c->err = msg; else g_create_error = msg;
  return s;
}

fwi_status cuda_fail(fwi_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
  return fail(c, FWI_ERR_CUDA, m);
}

fwi_status copy_field(fwi_ctx* c, void* dst, const void* src, long long n, int conj);

namespace {

bool fft_len_ok(int L) {
  switch (L) {
    case 16: case 32: case 64: case 128: case 192: case 256: case 320: case 384:
    case 512: case 640: case 768: case 1024: return true;
    default: return false;
  }
}

// Everything fwi_create derives from the descriptor.
struct Layout {
  int dim, nx, ny, nz, lx, ly, lz, rows, n_elem, n_freq, n_rhs, batch, ntiles, split;
  int n_tx, n_t;  // plane-wave transmits (0: point transmits); N_T
  int rf, ry;     // inversion-mesh cell (rf x ry x rf pixels)
  long long Ninv;
  long long N;
  size_t csz;
  size_t b_ghat, b_field, b_kv, b_plane1, b_plane2, b_small, b_jsplit, b_zpart, b_vec, b_tc;
  size_t b_rfield;  // receiver-field snapshot (hybrid_born), else 0
  size_t total;
};

bool make_layout(const fwi_problem_desc* d, Layout& L, std::string* why) {
  auto bad = [&](const char* m) { if (why) *why = m; return false; };
  if (!d) return bad("descriptor is NULL");
  if (d->dim != 2 && d->dim != 3) return bad("dim must be 2 or 3");
  L.dim = d->dim;
  L.nx = d->n[0];
  L.ny = (d->dim == 3) ? d->n[1] : 1;
  L.nz = d->n[2];
  if (L.nx <= 0 || L.ny <= 0 || L.nz <= 0) return bad("grid sizes must be positive");
  L.lx = 2 * L.nx; L.ly = (d->dim == 3) ? 2 * L.ny : 1; L.lz = 2 * L.nz;
  if (!fft_len_ok(L.lx) || !fft_len_ok(L.lz) || (d->dim == 3 && !fft_len_ok(L.ly)))
    return bad("2*n must be one of 16,32,64,128,192,256,320,384,512,640,768,1024");
  if (!(d->h > 0) || !(d->c0 > 0) || !std::isfinite(d->h) || !std::isfinite(d->c0))
    return bad("h and c0 must be finite and positive");
  if (d->n_elem <= 0 || !d->elem_pos) return bad("n_elem must be positive with elem_pos");
  if (d->n_freq <= 0 || !d->freq_hz) return bad("n_freq must be positive with freq_hz");
  for (int l = 0; l < d->n_freq; ++l)
    if (!(d->freq_hz[l] > 0) || !std::isfinite(d->freq_hz[l]))
      return bad("frequencies must be finite and positive");
  if (d->precision != FWI_MIXED && d->precision != FWI_FP64) return bad("unknown precision");
  if (d->n_tx < 0 || (d->n_tx > 0 && !d->tx_angle))
    return bad("n_tx must be >= 0, with tx_angle when positive");
  for (int i = 0; i < d->n_tx; ++i)
    if (!std::isfinite(d->tx_angle[i])) return bad("tx_angle must be finite");
  if (!(d->elem_length >= 0) || !std::isfinite(d->elem_length))
    return bad("elem_length must be finite and >= 0");
  if (!(d->alpha0 >= 0) || !std::isfinite(d->alpha0))
    return bad("alpha0 must be finite and >= 0");
  L.rf = d->inv_factor > 1 ? d->inv_factor : 1;
  L.ry = (d->dim == 3) ? L.rf : 1;
  L.n_elem = d->n_elem; L.n_freq = d->n_freq;
  L.n_tx = d->n_tx;
  L.n_t = d->n_tx > 0 ? d->n_tx : d->n_elem;
  L.n_rhs = d->n_elem * d->n_freq;
  L.batch = (d->max_batch > 0 && d->max_batch < L.n_rhs) ? d->max_batch : L.n_rhs;
  L.N = (long long)L.nx * L.ny * L.nz;
  {
    // the FFT passes index their work items (batch x lines or column tiles)
    // with 32-bit arithmetic
    const long long per = std::max({(long long)L.ny * L.nz, (long long)L.lx * L.ly,
                                    (long long)L.nz * L.lx});
    const long long cap = 0x7fffffffLL / per;
    if (cap < 1) return bad("grid too large");
    if (L.batch > cap) L.batch = (int)cap;
  }
  L.rows = L.ny * L.nz;
  if (L.nx % L.rf || L.nz % L.rf || L.ny % L.ry)
    return bad("every grid size must be a multiple of inv_factor");
  L.Ninv = L.N / ((long long)L.rf * L.rf * L.ry);
  L.csz = (d->precision == FWI_FP64) ? 16 : 8;
  const int lpc = (d->precision == FWI_FP64) ? Lsop<double>::row_lines_per_cta(L.lx)
                                             : Lsop<float>::row_lines_per_cta(L.lx);
  L.ntiles = (L.rows + lpc - 1) / lpc;  // default tile shape (informational)
  const long long P = (long long)L.lx * L.ly * L.lz;
  const long long NE2 = (long long)L.n_elem * L.n_elem;
  const int nbe = (L.n_elem + 63) / 64;
  // split-K partials of the pixel contractions: at most ~1024 CTAs' tiles
  const int tiles = nbe * nbe * L.n_freq;
  L.split = (1024 / tiles) > 1 ? 1024 / tiles : 1;
  L.b_ghat = (size_t)L.n_freq * P * L.csz;
  L.b_field = (size_t)L.n_rhs * L.N * L.csz;
  L.b_kv = (size_t)L.batch * L.N * L.csz;
  L.b_plane1 = (size_t)L.batch * L.rows * L.lx * L.csz;
  L.b_plane2 = (d->dim == 3) ? (size_t)L.batch * L.nz * L.ly * L.lx * L.csz : 0;
  // data-space buffers: dres and (plane waves) W, W^H W, dpw, dsyn; dF holds
  // max(N_T, n_elem) rows of field-precision data
  const long long NTE = (long long)L.n_t * L.n_elem;
  const long long NDF = std::max(NTE, NE2);
  const size_t b_pw = L.n_tx > 0 ? (size_t)L.n_freq * (2 * NTE + 2 * NE2) * 16 : 0;
  const size_t b_lossy = d->alpha0 > 0 ? (size_t)L.n_freq * (NE2 + 1) * 16 : 0;
  L.b_small = (size_t)L.batch * (sizeof(Scal) + NSLOT * (size_t)L.rows * sizeof(double2) +
                                 sizeof(int)) +
              64 + (size_t)L.n_freq * (NE2 * 16 + NDF * L.csz) + b_pw + b_lossy + 3 * 1024 * L.csz;
  size_t js1 = (size_t)L.split * L.n_freq * NE2 * L.csz;
  size_t js2 = (size_t)8 * L.N * sizeof(double2);
  L.b_jsplit = js1 > js2 ? js1 : js2;
  L.b_zpart = (size_t)L.n_freq * nbe * L.N * L.csz;
  L.b_vec = (size_t)L.N * L.csz * 2 + (size_t)8 * L.N * 16 + (size_t)3 * L.dim * L.N * 16 +
            (L.rf > 1 ? (size_t)L.N * 16 : 0) +
            sizeof(double) * (L.n_freq + 256 + 512 + 16);
  L.b_tc = (d->precision == FWI_FP64) ? 0 : tc_bops_bytes(L.n_elem, L.n_freq);
  if (d->hybrid_born != 0 && d->hybrid_born != 1) return bad("hybrid_born must be 0 or 1");
  L.b_rfield = d->hybrid_born ? L.b_field : 0;
  L.total = L.b_ghat + 4 * L.b_field + 5 * L.b_kv + L.b_plane1 + L.b_plane2 + L.b_small +
            L.b_jsplit + L.b_zpart + L.b_vec + L.b_tc + L.b_rfield + 256;
  return true;
}

}  // namespace

size_t workspace_bytes(const fwi_problem_desc* d, std::string* why) {
  Layout L;
  if (!make_layout(d, L, why)) return 0;
  return L.total;
}

fwi_status reduce_sum(fwi_ctx* c, void* buf, size_t count) {
  if (!c->reduce_fn) return FWI_OK;
  const int rc = c->reduce_fn(buf, count, (void*)c->stream, c->reduce_user);
  if (rc != 0)
    return fail(c, FWI_ERR_REDUCE, "reducer returned " + std::to_string(rc));
  return FWI_OK;
}

}  // namespace fwi

using namespace fwi;

static void release(fwi_ctx* c) {
  if (!c) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->device);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  prof_flush(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  void* bufs[] = {c->ghat, c->tw_x, c->tw_y, c->tw_z, c->p0, c->fields, c->rfields, c->lam,
                  c->asrc,
                  c->kv[0], c->kv[1], c->kv[2], c->kv[3], c->kv[4], c->plane1, c->plane2,
                  c->mF, c->scal, c->partial, c->active, c->n_active, c->dres, c->dF,
                  c->W, c->WhW, c->dpw, c->dsyn, c->vfwd, c->sdat, c->dlossy,
                  c->jsplit, c->zpart, c->aF, c->red, c->tc_bops, c->tc_err};
  // stream-ordered frees: no device-wide synchronisation, so a context can be
  // retired while other contexts' work runs
  for (void* p : bufs) if (p) cudaFreeAsync(p, c->stream);
  for (auto* p : c->vN) if (p) cudaFreeAsync(p, c->stream);
  for (auto* p : c->vD) if (p) cudaFreeAsync(p, c->stream);
  cudaStreamSynchronize(c->stream);
  if (c->h_n_active) cudaFreeHost(c->h_n_active);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_red) cudaFreeHost(c->h_red);
  if (c->h_tc_err) cudaFreeHost(c->h_tc_err);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->stream2) cudaStreamDestroy(c->stream2);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
  cudaSetDevice(cur);
}

// NVTX range over one library call (visible in nsys / ncu timelines; a no-op
// without a profiler attached).
struct CallRange {
  explicit CallRange(const char* name) { nvtxRangePushA(name); }
  ~CallRange() { nvtxRangePop(); }
};

extern "C" {

const char* fwi_version(void) { return "libfwi 0.1 (sm_103a)"; }

size_t fwi_workspace_bytes(const fwi_problem_desc* desc) {
  return workspace_bytes(desc, nullptr);
}

const char* fwi_last_error(const fwi_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

fwi_status fwi_cancel(fwi_ctx* ctx) {
  if (!ctx) return FWI_ERR_INVALID_ARG;
  ctx->cancel.store(true);
  return FWI_OK;
}

fwi_status fwi_create(const fwi_problem_desc* d, void* stream, fwi_ctx** out) {
  CallRange nvtx_range("fwi_create");
  if (!out) return fail(nullptr, FWI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  g_create_error.clear();
  Layout L;
  std::string why;
  if (!make_layout(d, L, &why)) return fail(nullptr, FWI_ERR_INVALID_ARG, why);
  for (size_t i = 0; i < (size_t)d->n_elem * d->dim; ++i)
    if (!std::isfinite(d->elem_pos[i]))
      return fail(nullptr, FWI_ERR_INVALID_ARG, "elem_pos must be finite");
  fwi_ctx* c = new fwi_ctx();
  c->dim = L.dim; c->nx = L.nx; c->ny = L.ny; c->nz = L.nz;
  // Two chains pay off on 2-D lattices (3-4 % on the 256^2 and 512^2
  // workloads); on 3-D lattices one chain is 6 % faster (160x160x128): a
  // half batch's pass already spans hundreds of waves, and the second
  // chain's streams evict the kernel-spectrum tiles the convolution keeps in
  // L2 across right-hand sides.
  c->overlap = L.dim != 3;
  c->lx = L.lx; c->ly = L.ly; c->lz = L.lz; c->N = L.N; c->rows = L.rows;
  c->n_elem = L.n_elem; c->n_freq = L.n_freq; c->n_rhs = L.n_rhs; c->batch = L.batch;
  c->h = d->h; c->c0 = d->c0;
  c->tol = d->krylov_tol > 0 ? d->krylov_tol : 1e-6;
  c->max_it = d->krylov_max_it > 0 ? d->krylov_max_it : 1000;
  c->fp64 = (d->precision == FWI_FP64);
  c->csz = L.csz;
  c->ntiles = L.ntiles;
  c->jsplit_n = L.split;
  c->elem.assign(d->elem_pos, d->elem_pos + (size_t)d->n_elem * d->dim);
  c->freq.assign(d->freq_hz, d->freq_hz + d->n_freq);
  for (double f : c->freq) c->kwave.push_back(2.0 * 3.141592653589793238462643383279502884 * f / c->c0);
  c->n_tx = L.n_tx;
  c->n_t = L.n_t;
  if (L.n_tx > 0) c->tx_angle.assign(d->tx_angle, d->tx_angle + L.n_tx);
  c->elem_length = (L.dim == 3) ? d->elem_length : 0.0;
  c->alpha0 = d->alpha0;
  for (double f : c->freq) {
    // k = omega sqrt(1/c0^2 + i alpha0 / (pi c0)), the root with Im k >= 0
    const double w = 2.0 * 3.141592653589793238462643383279502884 * f;
    const std::complex<double> kk =
        w * std::sqrt(std::complex<double>(1.0 / (c->c0 * c->c0),
                                           c->alpha0 / (3.141592653589793238462643383279502884 * c->c0)));
    c->kc.push_back(make_double2(kk.real(), kk.imag()));
  }
  c->rf = L.rf;
  c->ry = L.ry;
  c->inx = L.nx / L.rf;
  c->iny = L.ny / L.ry;
  c->inz = L.nz / L.rf;
  c->Ninv = L.Ninv;
  c->stream = (cudaStream_t)stream;
  c->bytes = L.total;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess && !stream) {
    // The legacy default stream cannot be graph-captured; a blocking stream
    // is implicitly ordered with it, so callers on the default stream see
    // the same ordering.
    e = cudaStreamCreate(&c->own_stream);
    c->stream = c->own_stream;
  }
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
  // stream-ordered allocations from the device's default memory pool
  auto alloc = [&](void** p, size_t bytes) {
    if (e != cudaSuccess || bytes == 0) return;
    e = cudaMallocAsync(p, bytes, c->stream);
  };
  alloc(&c->ghat, L.b_ghat);
  alloc(&c->p0, L.b_field);
  alloc(&c->fields, L.b_field);
  alloc(&c->rfields, L.b_rfield);
  alloc(&c->lam, L.b_field);
  alloc(&c->asrc, L.b_field);
  for (int i = 0; i < 5; ++i) alloc(&c->kv[i], L.b_kv);
  alloc(&c->plane1, L.b_plane1);
  if (L.b_plane2) alloc(&c->plane2, L.b_plane2);
  alloc(&c->mF, (size_t)L.N * L.csz);
  alloc((void**)&c->scal, sizeof(Scal) * L.batch);
  alloc((void**)&c->partial, sizeof(double2) * NSLOT * (size_t)L.rows * L.batch);
  alloc((void**)&c->active, sizeof(int) * L.batch);
  alloc((void**)&c->n_active, 64);
  const size_t NE2 = (size_t)L.n_elem * L.n_elem;
  const size_t NTE = (size_t)L.n_t * L.n_elem;
  alloc((void**)&c->dres, 16 * L.n_freq * NE2);
  alloc(&c->dF, L.csz * L.n_freq * std::max(NTE, NE2));
  if (d->alpha0 > 0) {
    alloc((void**)&c->sdat, 16 * L.n_freq);
    alloc((void**)&c->dlossy, 16 * L.n_freq * NE2);
  }
  if (L.n_tx > 0) {
    alloc((void**)&c->W, 16 * L.n_freq * NTE);
    alloc((void**)&c->WhW, 16 * L.n_freq * NE2);
    alloc((void**)&c->dpw, 16 * L.n_freq * NTE);
    alloc((void**)&c->dsyn, 16 * L.n_freq * NE2);
  }
  alloc(&c->jsplit, L.b_jsplit);
  alloc(&c->zpart, L.b_zpart);
  alloc(&c->aF, (size_t)L.N * L.csz);
  for (int i = 0; i < 6; ++i) alloc((void**)&c->vN[i], (size_t)L.N * 16);
  alloc((void**)&c->vD[0], (size_t)L.dim * L.N * 16);
  if (L.rf > 1) alloc((void**)&c->vfwd, (size_t)L.N * 16);
  c->red_n = L.n_freq + 256 + 512 + 16;
  alloc((void**)&c->red, sizeof(double) * c->red_n);
  alloc(&c->tc_bops, L.b_tc);
  alloc((void**)&c->tc_err, 256);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_n_active, 64);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_scal, sizeof(Scal) * L.batch);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_red, sizeof(double) * c->red_n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_tc_err, sizeof(int));
  if (e == cudaSuccess) *c->h_tc_err = 0;
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fwi_status st = (e == cudaErrorMemoryAllocation) ? FWI_ERR_NOMEM : FWI_ERR_CUDA;
    fail(nullptr, st, std::string("workspace allocation: ") + cudaGetErrorString(e));
    cudaGetLastError();
    release(c);
    return st;
  }
  // per-frequency scales k_l^2 dV for the Jacobian / data contractions
  // (lossy background: the contraction kernels scale by 1 and the complex
  // k_l^2 dV is applied in data space)
  std::vector<double> sc(L.n_freq);
  std::vector<double2> scc(L.n_freq);
  for (int l = 0; l < L.n_freq; ++l) {
    const double dv = std::pow(c->h, c->dim);
    sc[l] = c->alpha0 > 0 ? 1.0 : c->kwave[l] * c->kwave[l] * dv;
    const std::complex<double> kk(c->kc[l].x, c->kc[l].y);
    const std::complex<double> s = kk * kk * dv;
    scc[l] = make_double2(s.real(), s.imag());
  }
  e = cudaMemcpy(c->red, sc.data(), sizeof(double) * L.n_freq, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && c->alpha0 > 0) {
    e = cudaMemcpyAsync(c->sdat, scc.data(), sizeof(double2) * L.n_freq, cudaMemcpyHostToDevice,
                        c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e == cudaSuccess && L.n_tx > 0) {
    // plane-wave weights w_{l,i,e} = exp(i k_l x_e sin theta_i) and W^H W
    const int nt = L.n_tx, ne = L.n_elem;
    std::vector<double2> w((size_t)L.n_freq * nt * ne), whw((size_t)L.n_freq * ne * ne);
    for (int l = 0; l < L.n_freq; ++l) {
      for (int i = 0; i < nt; ++i)
        for (int q = 0; q < ne; ++q) {
          const double ph = c->kwave[l] * c->elem[(size_t)q * c->dim] * std::sin(c->tx_angle[i]);
          w[((size_t)l * nt + i) * ne + q] = make_double2(std::cos(ph), std::sin(ph));
        }
      for (int a = 0; a < ne; ++a)
        for (int b = 0; b < ne; ++b) {
          double sx = 0.0, sy = 0.0;
          for (int i = 0; i < nt; ++i) {
            const double2 u = w[((size_t)l * nt + i) * ne + a], v = w[((size_t)l * nt + i) * ne + b];
            sx += u.x * v.x + u.y * v.y;  // conj(u) v
            sy += u.x * v.y - u.y * v.x;
          }
          whw[((size_t)l * ne + a) * ne + b] = make_double2(sx, sy);
        }
    }
    // ordered after the stream-ordered allocations; the host vectors live
    // until the synchronisation
    e = cudaMemcpyAsync(c->W, w.data(), sizeof(double2) * w.size(), cudaMemcpyHostToDevice,
                        c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->WhW, whw.data(), sizeof(double2) * whw.size(),
                          cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) {
    fail(nullptr, FWI_ERR_CUDA, std::string("scale upload: ") + cudaGetErrorString(e));
    release(c);
    return FWI_ERR_CUDA;
  }
  fwi_status st = setup_operator(c);
  if (st == FWI_OK) st = autotune(c);
  if (st != FWI_OK) {
    g_create_error = c->err;
    release(c);
    return st;
  }
  *out = c;
  return FWI_OK;
}

fwi_status fwi_destroy(fwi_ctx* ctx) {
  if (!ctx) return FWI_ERR_INVALID_ARG;
  cudaStreamSynchronize(ctx->stream);
  release(ctx);
  return FWI_OK;
}

fwi_status fwi_contrast_from_sos(fwi_ctx* ctx, const double* sos, const double* alpha, void* m) {
  CallRange nvtx_range("fwi_contrast_from_sos");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!sos || !m) return fail(ctx, FWI_ERR_INVALID_ARG, "sos and m are required");
  ctx->err.clear();
  return contrast_from_sos(ctx, sos, alpha, m);
}

fwi_status fwi_sos_attenuation_from_contrast(fwi_ctx* ctx, const void* m, double* sos,
                                             double* alpha) {
  CallRange nvtx_range("fwi_sos_attenuation_from_contrast");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!m) return fail(ctx, FWI_ERR_INVALID_ARG, "m is required");
  ctx->err.clear();
  return sos_attenuation_from_contrast(ctx, m, sos, alpha);
}

fwi_status fwi_forward(fwi_ctx* ctx, const void* m, void* fields, int warm_start, void* data,
                       fwi_solve_info* info) {
  CallRange nvtx_range("fwi_forward");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!m) return fail(ctx, FWI_ERR_INVALID_ARG, "m is NULL");
  if (warm_start && !fields) return fail(ctx, FWI_ERR_INVALID_ARG, "warm start needs fields");
  ctx->err.clear();
  ctx->cancel.store(false);
  const long long nf = (long long)ctx->n_rhs * ctx->N;
  if (warm_start) {
    fwi_status st = copy_field(ctx, ctx->fields, fields, nf, 0);
    if (st != FWI_OK) return st;
  }
  fwi_status st = forward_solve(ctx, m, warm_start != 0, info);
  if (st != FWI_OK && st != FWI_ERR_NOT_CONVERGED) return st;
  fwi_status st2 = FWI_OK;
  if (fields) st2 = copy_field(ctx, fields, ctx->fields, nf, 0);
  if (st2 == FWI_OK) st2 = project_data(ctx, m, data);
  if (st2 == FWI_OK) {
    tc_err_fetch(ctx);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fwi_forward");
    st2 = tc_err_check(ctx);
  }
  return st2 != FWI_OK ? st2 : st;
}

fwi_status fwi_adjoint(fwi_ctx* ctx, const void* m, const void* src, void* lambda,
                       fwi_solve_info* info) {
  CallRange nvtx_range("fwi_adjoint");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!m || !src || !lambda) return fail(ctx, FWI_ERR_INVALID_ARG, "m, src, lambda are required");
  ctx->err.clear();
  ctx->cancel.store(false);
  fwi_status st = adjoint_solve(ctx, m, src, true, info);
  if (st != FWI_OK && st != FWI_ERR_NOT_CONVERGED) return st;
  fwi_status st2 = copy_field(ctx, lambda, ctx->lam, (long long)ctx->n_rhs * ctx->N, 1);
  if (st2 == FWI_OK) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fwi_adjoint");
  }
  return st2 != FWI_OK ? st2 : st;
}

fwi_status fwi_gradient(fwi_ctx* ctx, const void* m, const void* d_obs, void* grad,
                        double* misfit, void* data, fwi_solve_info* info_fwd,
                        fwi_solve_info* info_adj) {
  CallRange nvtx_range("fwi_gradient");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!m || !d_obs || !grad) return fail(ctx, FWI_ERR_INVALID_ARG, "m, d_obs, grad are required");
  ctx->err.clear();
  ctx->cancel.store(false);
  fwi_status st = forward_solve(ctx, m, false, info_fwd);
  if (st != FWI_OK && st != FWI_ERR_NOT_CONVERGED) return st;
  fwi_status worst = st;
  st = project_data(ctx, m, data);
  if (st != FWI_OK) return st;
  st = residual_misfit(ctx, d_obs, misfit);
  if (st != FWI_OK) return st;
  st = adjoint_sources_conj(ctx, ctx->asrc);
  if (st != FWI_OK) return st;
  st = adjoint_solve(ctx, m, ctx->asrc, false, info_adj);
  if (st != FWI_OK && st != FWI_ERR_NOT_CONVERGED) return st;
  if (st != FWI_OK) worst = st;
  st = assemble_gradient(ctx, grad);
  if (st != FWI_OK) return st;
  // frequency sharding: the gradient of all frequencies (Sec. IV-D)
  st = reduce_sum(ctx, grad, 2 * (size_t)ctx->Ninv);
  if (st != FWI_OK) return st;
  tc_err_fetch(ctx);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fwi_gradient");
  st = tc_err_check(ctx);
  return st != FWI_OK ? st : worst;
}

fwi_status fwi_admm_tv_step(fwi_ctx* ctx, void* m, void* g, void* u, const void* grad,
                            const fwi_admm_params* p, double* sos_out) {
  CallRange nvtx_range("fwi_admm_tv_step");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!m || !g || !u || !grad || !p) return fail(ctx, FWI_ERR_INVALID_ARG, "missing argument");
  if (!(p->rho > 0) || p->lambda < 0 || p->gamma < 0 || p->n_cg < 0)
    return fail(ctx, FWI_ERR_INVALID_ARG, "need rho > 0, lambda >= 0, gamma >= 0, n_cg >= 0");
  ctx->err.clear();
  fwi_status st = admm_step(ctx, m, g, u, grad, p, sos_out);
  if (st != FWI_OK) return st;
  tc_err_fetch(ctx);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fwi_admm_tv_step");
  return tc_err_check(ctx);
}

fwi_status fwi_admm_init(fwi_ctx* ctx, const void* m0, void* g, void* u) {
  CallRange nvtx_range("fwi_admm_init");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!m0 || !g || !u) return fail(ctx, FWI_ERR_INVALID_ARG, "missing pointer");
  ctx->err.clear();
  return admm_init(ctx, m0, g, u);
}

fwi_status fwi_set_reducer(fwi_ctx* ctx, fwi_reduce_fn fn, void* user) {
  if (!ctx) return FWI_ERR_INVALID_ARG;
  ctx->reduce_fn = fn;
  ctx->reduce_user = fn ? user : nullptr;
  return FWI_OK;
}

fwi_status fwi_freeze_receiver_fields(fwi_ctx* ctx, int freeze) {
  CallRange nvtx_range("fwi_freeze_receiver_fields");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!ctx->rfields)
    return fail(ctx, FWI_ERR_INVALID_ARG,
                "the context has no receiver-field snapshot (create it with hybrid_born = 1)");
  if (freeze != 0 && freeze != 1) return fail(ctx, FWI_ERR_INVALID_ARG, "freeze must be 0 or 1");
  ctx->err.clear();
  if (freeze) {
    if (!ctx->fields_valid)
      return fail(ctx, FWI_ERR_INVALID_ARG, "no forward fields: call fwi_forward or fwi_gradient first");
    FWI_CUDA(ctx, cudaMemcpyAsync(ctx->rfields, ctx->fields,
                                  (size_t)ctx->n_rhs * ctx->N * ctx->csz,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  }
  ctx->rfields_frozen = freeze == 1;
  return FWI_OK;
}

static fwi_status apply_common(fwi_ctx* ctx, int kind, const void* m, int freq, int n_rhs,
                               const void* in, void* out) {
  CallRange nvtx_range(kind == 0 ? "fwi_apply_K" : kind == 1 ? "fwi_apply_A" : "fwi_apply_AH");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!in || !out || (kind != 0 && !m)) return fail(ctx, FWI_ERR_INVALID_ARG, "missing pointer");
  if (in == out) return fail(ctx, FWI_ERR_INVALID_ARG, "in and out must not alias");
  if (freq < 0 || freq >= ctx->n_freq) return fail(ctx, FWI_ERR_INVALID_ARG, "freq out of range");
  if (n_rhs < 1 || n_rhs > ctx->batch) return fail(ctx, FWI_ERR_INVALID_ARG, "n_rhs out of range");
  ctx->err.clear();
  return apply_op(ctx, kind, m, freq, n_rhs, in, out);
}

fwi_status fwi_apply_K(fwi_ctx* ctx, int freq, int n_rhs, const void* in, void* out) {
  return apply_common(ctx, 0, nullptr, freq, n_rhs, in, out);
}
fwi_status fwi_apply_A(fwi_ctx* ctx, const void* m, int freq, int n_rhs, const void* in,
                       void* out) {
  return apply_common(ctx, 1, m, freq, n_rhs, in, out);
}
fwi_status fwi_apply_AH(fwi_ctx* ctx, const void* m, int freq, int n_rhs, const void* in,
                        void* out) {
  return apply_common(ctx, 2, m, freq, n_rhs, in, out);
}

fwi_status fwi_jac_forward(fwi_ctx* ctx, const void* a, void* y) {
  CallRange nvtx_range("fwi_jac_forward");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!a || !y) return fail(ctx, FWI_ERR_INVALID_ARG, "missing pointer");
  if (!ctx->fields_valid) return fail(ctx, FWI_ERR_INVALID_ARG, "no forward fields");
  ctx->err.clear();
  if (ctx->n_tx == 0) return jac_forward(ctx, a, (double2*)y);
  // J = W J_point
  fwi_status st = jac_forward(ctx, a, ctx->dres);
  if (st != FWI_OK) return st;
  return synth(ctx, ctx->W, 0, ctx->n_tx, ctx->n_elem, ctx->dres, (double2*)y, nullptr);
}

fwi_status fwi_jac_adjoint(fwi_ctx* ctx, const void* y, void* z) {
  CallRange nvtx_range("fwi_jac_adjoint");
  if (!ctx) return FWI_ERR_INVALID_ARG;
  if (!y || !z) return fail(ctx, FWI_ERR_INVALID_ARG, "missing pointer");
  if (!ctx->fields_valid) return fail(ctx, FWI_ERR_INVALID_ARG, "no forward fields");
  ctx->err.clear();
  fwi_status st;
  if (ctx->n_tx == 0) {
    st = jac_adjoint(ctx, (const double2*)y, (double2*)z);
  } else {
    // J^H = J_point^H W^H
    st = synth(ctx, ctx->W, 1, ctx->n_elem, ctx->n_tx, (const double2*)y, ctx->dsyn, nullptr);
    if (st == FWI_OK) st = jac_adjoint(ctx, ctx->dsyn, (double2*)z);
  }
  if (st != FWI_OK) return st;
  return reduce_sum(ctx, z, 2 * (size_t)ctx->Ninv);  // frequency sharding
}

fwi_status fwi_get_tuning(const fwi_ctx* ctx, fwi_tuning* out) {
  if (!ctx || !out) return FWI_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->row_fwd_variant = ctx->var_rf;
  out->row_inv_variant = ctx->var_ri;
  out->col_variant = ctx->var_cz;
  out->col_y_variant = ctx->var_cy;
  out->tuned = ctx->tuned;
  out->jac_tensor_cores = ctx->use_tc ? 1 : 0;
  out->overlap_halves = ctx->overlap ? 1 : 0;
  out->col_tma = ctx->col_tma;
  out->col_spectrum_stage = ctx->col_gstage;
  out->jac_tma = ctx->jac_tma;
  out->row_l2_prefetch = ctx->row_l2pf;
  out->row_stage = ctx->row_stage;
  out->col_pairs = ctx->col_pairs;
  for (int k = 0; k < 4; ++k)
    for (int v = 0; v < 4; ++v) out->ms[k][v] = ctx->tune_ms[k][v];
  return FWI_OK;
}

fwi_status fwi_set_tuning(fwi_ctx* ctx, const fwi_tuning* in) {
  if (!ctx || !in) return FWI_ERR_INVALID_ARG;
  const int lims[4] = {ctx->fp64 ? 1 : Lsop<float>::variants(ctx->lx, 0),
                       ctx->fp64 ? 1 : Lsop<float>::variants(ctx->lx, 1),
                       ctx->fp64 ? 1 : Lsop<float>::variants(ctx->lz, 2),
                       (ctx->fp64 || ctx->dim != 3) ? 1 : Lsop<float>::variants(ctx->ly, 2)};
  const int req[4] = {in->row_fwd_variant, in->row_inv_variant, in->col_variant,
                      in->col_y_variant};
  for (int k = 0; k < 4; ++k)
    if (req[k] < 0 || req[k] >= lims[k]) return fail(ctx, FWI_ERR_INVALID_ARG, "variant out of range");
  if (in->jac_tensor_cores != 0 && in->jac_tensor_cores != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "jac_tensor_cores must be 0 or 1");
  if (in->overlap_halves != 0 && in->overlap_halves != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "overlap_halves must be 0 or 1");
  if (in->debug_stall_once != 0 && in->debug_stall_once != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "debug_stall_once must be 0 or 1");
  if (in->col_tma != 0 && in->col_tma != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "col_tma must be 0 or 1");
  if (in->row_l2_prefetch != 0 && in->row_l2_prefetch != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "row_l2_prefetch must be 0 or 1");
  if (in->col_spectrum_stage != 0 && in->col_spectrum_stage != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "col_spectrum_stage must be 0 or 1");
  if (in->jac_tma != 0 && in->jac_tma != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "jac_tma must be 0 or 1");
  if (in->row_stage != 0 && in->row_stage != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "row_stage must be 0 or 1");
  if (in->col_pairs != 0 && in->col_pairs != 1)
    return fail(ctx, FWI_ERR_INVALID_ARG, "col_pairs must be 0 or 1");
  ctx->col_tma = in->col_tma;
  ctx->col_gstage = in->col_spectrum_stage;
  ctx->jac_tma = in->jac_tma;
  ctx->row_l2pf = in->row_l2_prefetch;
  ctx->row_stage = in->row_stage;
  ctx->col_pairs = in->col_pairs;
  ctx->tc_stall = in->debug_stall_once;
  ctx->use_tc = in->jac_tensor_cores == 1;
  ctx->overlap = in->overlap_halves == 1;
  ctx->var_rf = req[0];
  ctx->var_ri = req[1];
  ctx->var_cz = req[2];
  ctx->var_cy = req[3];
  ctx->tuned = 0;
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
  ctx->graphs.clear();  // captured launches carry the old variants
  return FWI_OK;
}

fwi_status fwi_set_profiling(fwi_ctx* ctx, int on) {
  if (!ctx) return FWI_ERR_INVALID_ARG;
  ctx->profiling = (on != 0);
  return FWI_OK;
}

fwi_status fwi_get_stats(const fwi_ctx* ctx, fwi_stats* out) {
  if (!ctx || !out) return FWI_ERR_INVALID_ARG;
  prof_flush(const_cast<fwi_ctx*>(ctx));
  std::memset(out, 0, sizeof(*out));
  out->kernel_launches = ctx->launches;
  int n = 0;
  for (int k = 0; k < KC_COUNT && n < FWI_MAX_KERNEL_STATS; ++k) {
    const auto& s = ctx->kstats[k];
    if (s.launches == 0) continue;
    fwi_kernel_stat& o = out->kernels[n++];
    std::strncpy(o.name, kclass_name(k), sizeof(o.name) - 1);
    o.ms = s.ms;
    o.launches = s.launches;
    o.bytes = s.bytes;
    o.flops = s.flops;
  }
  out->n_kernel_stats = n;
  return FWI_OK;
}

fwi_status fwi_reset_stats(fwi_ctx* ctx) {
  if (!ctx) return FWI_ERR_INVALID_ARG;
  prof_flush(ctx);
  ctx->launches = 0;
  for (auto& s : ctx->kstats) s = fwi_ctx::KStat{};
  return FWI_OK;
}

}  // extern "C"
