// Serving runtime: continuous batching of whole reconstructions
// (Algorithm 1) over several contexts and CUDA streams, with FIFO first-fit
// admission by device-memory footprint.  Host code only; every step of a
// reconstruction runs through the library's own entry points.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ctx.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  long long id = 0;
  fwi_problem_desc desc{};
  std::vector<double> elem, freq, tx, sos0, sos_out;
  std::vector<char> d_obs;
  fwi_admm_params admm{};
  int n_iter = 1;
  int refresh_every = 1;
  long long n = 0;       // voxels
  size_t csz = 8;        // field element bytes
  size_t bytes = 0;      // admitted footprint
  Clock::time_point t_submit, t_admit, t_done;
  fwi_request_result res{};
  bool done = false;
  bool waited = false;
  std::atomic<bool> cancelled{false};
  fwi_ctx* ctx = nullptr;  // while running (guarded by the server's mutex)
};

// Footprint of a request: context workspace plus the request's vectors.
size_t request_bytes(const fwi_problem_desc& d, long long n, size_t csz, size_t& ws) {
  ws = fwi_workspace_bytes(&d);
  if (ws == 0) return 0;
  const size_t ne = (size_t)d.n_elem;
  const size_t nt = d.n_tx > 0 ? (size_t)d.n_tx : ne;  // transmits N_T
  const size_t vec = (size_t)n * (16 /*m*/ + 16 /*grad*/ + 8 /*sos*/ + 8 /*sos0*/ +
                                  2 * (size_t)d.dim * 16 /*g, u*/);
  return ws + vec + (size_t)d.n_freq * nt * ne * csz + (1 << 20);
}

}  // namespace

struct fwi_server {
  size_t budget = 0, in_use = 0;
  int max_active = 1, active = 0, device = 0;
  bool stopping = false;
  long long next_id = 1;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<long long, std::shared_ptr<Request>> all;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::thread> workers;
};

namespace {

// One reconstruction on its own context and stream.
void run_request(fwi_server* srv, Request& r) {
  fwi_request_result& res = r.res;
  cudaSetDevice(srv->device);
  cudaStream_t st = nullptr;
  fwi_ctx* ctx = nullptr;
  void *m = nullptr, *g = nullptr, *u = nullptr, *grad = nullptr, *sos = nullptr,
       *sos0 = nullptr, *dobs = nullptr;
  fwi_status status = FWI_OK;
  auto fail_cuda = [&](cudaError_t e) {
    if (e != cudaSuccess && status == FWI_OK) status = FWI_ERR_CUDA;
    return e != cudaSuccess;
  };
  do {
    if (fail_cuda(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) break;
    r.desc.elem_pos = r.elem.data();
    r.desc.freq_hz = r.freq.data();
    r.desc.tx_angle = r.tx.empty() ? nullptr : r.tx.data();
    if (r.cancelled.load()) { status = FWI_ERR_CANCELLED; break; }
    status = fwi_create(&r.desc, st, &ctx);
    if (status != FWI_OK) break;
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      r.ctx = ctx;  // fwi_server_cancel can now interrupt its solves
    }
    const size_t nd = r.d_obs.size();
    const size_t gsz = (size_t)r.desc.dim * r.n * 16;
    bool bad = false;
    for (auto pr : {std::make_pair(&m, (size_t)r.n * 16), std::make_pair(&g, gsz),
                    std::make_pair(&u, gsz), std::make_pair(&grad, (size_t)r.n * 16),
                    std::make_pair(&sos, (size_t)r.n * 8), std::make_pair(&sos0, (size_t)r.n * 8),
                    std::make_pair(&dobs, nd)})
      if (!bad) bad = fail_cuda(cudaMallocAsync(pr.first, pr.second, st));
    if (bad) break;
    if (fail_cuda(cudaMemcpyAsync(sos0, r.sos0.data(), (size_t)r.n * 8, cudaMemcpyHostToDevice, st)))
      break;
    if (fail_cuda(cudaMemcpyAsync(dobs, r.d_obs.data(), nd, cudaMemcpyHostToDevice, st))) break;
    if ((status = fwi_contrast_from_sos(ctx, (const double*)sos0, nullptr, m)) != FWI_OK) break;
    if ((status = fwi_admm_init(ctx, m, g, u)) != FWI_OK) break;
    double iters_sum = 0.0;
    int iters_n = 0;
    for (int k = 0; k < r.n_iter; ++k) {
      // a cancel between calls (a call's own start clears the context's flag)
      if (r.cancelled.load()) { status = FWI_ERR_CANCELLED; break; }
      double mis = 0.0;
      fwi_solve_info inf[2];
      std::memset(inf, 0, sizeof(inf));
      inf[0].n_rhs = inf[1].n_rhs = r.desc.n_elem * r.desc.n_freq;
      fwi_status s1 = fwi_gradient(ctx, m, dobs, grad, &mis, nullptr, &inf[0], &inf[1]);
      if (s1 != FWI_OK && s1 != FWI_ERR_NOT_CONVERGED) { status = s1; break; }
      for (const fwi_solve_info& f : inf) {
        if (f.max_iters > res.krylov_iters_max) res.krylov_iters_max = f.max_iters;
        iters_sum += f.max_iters;
        iters_n += 1;
        res.not_converged += f.n_not_converged;
      }
      res.krylov_iters_mean = iters_n ? iters_sum / iters_n : 0.0;
      if (k == 0) res.misfit_first = mis;
      res.misfit_last = mis;
      // hybrid Born schedule (Sec. IV-B): receiver fields of this
      // iteration's forward solve on iterations 0, K, 2K, ..., frozen between
      if (r.refresh_every > 1 && k % r.refresh_every == 0) {
        const fwi_status s3 = fwi_freeze_receiver_fields(ctx, 1);
        if (s3 != FWI_OK) { status = s3; break; }
      }
      fwi_status s2 = fwi_admm_tv_step(ctx, m, g, u, grad, &r.admm,
                                       k == r.n_iter - 1 ? (double*)sos : nullptr);
      if (s2 != FWI_OK) { status = s2; break; }
      res.rhs_solves += 2LL * r.desc.n_elem * r.desc.n_freq;
    }
    if (status != FWI_OK) break;
    r.sos_out.resize(r.n);
    if (fail_cuda(cudaMemcpyAsync(r.sos_out.data(), sos, (size_t)r.n * 8,
                                  cudaMemcpyDeviceToHost, st)))
      break;
    fail_cuda(cudaStreamSynchronize(st));
  } while (0);
  for (void* p : {m, g, u, grad, sos, sos0, dobs})
    if (p) cudaFreeAsync(p, st);
  if (ctx) {
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      r.ctx = nullptr;
    }
    fwi_destroy(ctx);
  }
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  res.status = status;
}

// First admissible request in FIFO order, or the end of the queue.
std::deque<std::shared_ptr<Request>>::iterator next_fit(fwi_server* s) {
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
    if (s->in_use + (*it)->bytes <= s->budget) return it;
  return s->queue.end();
}

void worker_loop(fwi_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        return (s->stopping && s->queue.empty()) ||
               (!s->queue.empty() && next_fit(s) != s->queue.end());
      });
      if (s->queue.empty()) return;
      auto it = next_fit(s);
      r = *it;
      s->queue.erase(it);
      s->in_use += r->bytes;
      s->active += 1;
      r->t_admit = Clock::now();
    }
    run_request(s, *r);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->t_done = Clock::now();
      r->res.queue_ms = ms_between(r->t_submit, r->t_admit);
      r->res.run_ms = ms_between(r->t_admit, r->t_done);
      r->res.latency_ms = ms_between(r->t_submit, r->t_done);
      r->res.bytes = r->bytes;
      r->done = true;
      s->in_use -= r->bytes;
      s->active -= 1;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

using fwi::fail;

extern "C" {

fwi_status fwi_server_create(size_t hbm_budget, int max_active, fwi_server** out) {
  if (!out || max_active < 1) return fail(nullptr, FWI_ERR_INVALID_ARG, "bad server arguments");
  *out = nullptr;
  auto* s = new fwi_server();
  cudaGetDevice(&s->device);
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return fail(nullptr, FWI_ERR_CUDA, "cudaMemGetInfo failed");
    }
    hbm_budget = (size_t)(0.9 * (double)fr);
  }
  s->budget = hbm_budget;
  s->max_active = max_active;
  for (int i = 0; i < max_active; ++i) s->workers.emplace_back(worker_loop, s);
  *out = s;
  return FWI_OK;
}

fwi_status fwi_server_submit(fwi_server* s, const fwi_request* r, long long* id) {
  if (!s || !r || !id || !r->sos0 || !r->d_obs || r->n_iter < 1 || r->admm.m_ref)
    return fail(nullptr, FWI_ERR_INVALID_ARG, "bad request");
  const fwi_problem_desc& d = r->problem;
  if (!d.elem_pos || !d.freq_hz || d.n_elem <= 0 || d.n_freq <= 0 || (d.dim != 2 && d.dim != 3) ||
      d.n_tx < 0 || (d.n_tx > 0 && !d.tx_angle))
    return fail(nullptr, FWI_ERR_INVALID_ARG, "bad request problem descriptor");
  auto q = std::make_shared<Request>();
  q->desc = d;
  q->elem.assign(d.elem_pos, d.elem_pos + (size_t)d.n_elem * d.dim);
  q->freq.assign(d.freq_hz, d.freq_hz + d.n_freq);
  if (d.n_tx > 0) q->tx.assign(d.tx_angle, d.tx_angle + d.n_tx);
  // the request's model vectors (m, g, u, grad, sos) live on the inversion mesh
  const long long rfac = d.inv_factor > 1 ? d.inv_factor : 1;
  q->n = (long long)d.n[0] * (d.dim == 3 ? d.n[1] : 1) * d.n[2] /
         (rfac * rfac * (d.dim == 3 ? rfac : 1));
  q->csz = (d.precision == FWI_FP64) ? 16 : 8;
  q->sos0.assign(r->sos0, r->sos0 + q->n);
  const size_t nt = d.n_tx > 0 ? (size_t)d.n_tx : (size_t)d.n_elem;
  const size_t nd = (size_t)d.n_freq * nt * d.n_elem * q->csz;
  q->d_obs.assign((const char*)r->d_obs, (const char*)r->d_obs + nd);
  q->admm = r->admm;
  q->n_iter = r->n_iter;
  q->refresh_every = r->refresh_every > 1 ? r->refresh_every : 1;
  // the hybrid Born schedule needs the context's receiver-field snapshot
  q->desc.hybrid_born = q->refresh_every > 1 ? 1 : 0;
  size_t ws = 0;
  q->bytes = request_bytes(q->desc, q->n, q->csz, ws);
  if (q->bytes == 0) return fail(nullptr, FWI_ERR_INVALID_ARG, "unsupported request problem");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (q->bytes > s->budget)
      return fail(nullptr, FWI_ERR_NOMEM, "request footprint exceeds the server budget");
    q->id = s->next_id++;
    q->t_submit = Clock::now();
    s->queue.push_back(q);
    s->all[q->id] = q;
    *id = q->id;
  }
  s->cv_work.notify_all();
  return FWI_OK;
}

fwi_status fwi_server_wait(fwi_server* s, long long id, double* sos_out, fwi_request_result* res) {
  if (!s) return FWI_ERR_INVALID_ARG;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end() || it->second->waited)
      return fail(nullptr, FWI_ERR_INVALID_ARG, "unknown request id");
    r = it->second;
    s->cv_done.wait(lk, [&] { return r->done; });
    r->waited = true;
    s->all.erase(it);
  }
  if (res) *res = r->res;
  if (sos_out && !r->sos_out.empty())
    std::memcpy(sos_out, r->sos_out.data(), sizeof(double) * r->sos_out.size());
  return (fwi_status)r->res.status;
}

fwi_status fwi_server_cancel(fwi_server* s, long long id) {
  if (!s) return FWI_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end() || it->second->waited)
      return fail(nullptr, FWI_ERR_INVALID_ARG, "unknown request id");
    const std::shared_ptr<Request>& r = it->second;
    if (r->done) return FWI_OK;  // finished already: its result stands
    r->cancelled.store(true);
    auto q = std::find(s->queue.begin(), s->queue.end(), r);
    if (q != s->queue.end()) {
      // still queued: leaves the queue, completed as cancelled
      s->queue.erase(q);
      r->t_admit = r->t_done = Clock::now();
      r->res.queue_ms = ms_between(r->t_submit, r->t_done);
      r->res.run_ms = 0.0;
      r->res.latency_ms = r->res.queue_ms;
      r->res.status = FWI_ERR_CANCELLED;
      r->done = true;
    } else if (r->ctx) {
      fwi_cancel(r->ctx);  // running: its solve stops at the next host check
    }
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  return FWI_OK;
}

fwi_status fwi_server_stats(fwi_server* s, int* active, int* queued, size_t* bytes) {
  if (!s) return FWI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (active) *active = s->active;
  if (queued) *queued = (int)s->queue.size();
  if (bytes) *bytes = s->in_use;
  return FWI_OK;
}

fwi_status fwi_server_destroy(fwi_server* s) {
  if (!s) return FWI_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return FWI_OK;
}

}  // extern "C"
