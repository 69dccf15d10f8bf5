// Launch counting and optional per-launch CUDA-event timing of libfwi's
// kernels (profiling mode), accumulated per kernel class.
#pragma once

#include "ctx.cuh"

namespace fwi {

enum KClass {
  KC_ROW_FWD_INIT, KC_ROW_FWD_ITER, KC_ROW_FWD_S, KC_ROW_FWD_PLAIN, KC_COL_CONV,
  KC_COL_FWD, KC_COL_INV, KC_ROW_INV_V, KC_ROW_INV_T, KC_ROW_INV_OTHER, KC_KRYLOV_SCALAR,
  KC_FINALIZE, KC_CONTRACT, KC_MIX_SOURCES, KC_MIX_JH, KC_GRADIENT, KC_ADMM, KC_SETUP,
  KC_MISC, KC_COUNT
};

inline const char* kclass_name(int k) {
  static const char* names[KC_COUNT] = {
      "row_fwd_init", "row_fwd_iter", "row_fwd_s", "row_fwd_plain", "col_conv",
      "col_fwd", "col_inv", "row_inv_v", "row_inv_t", "row_inv_other", "krylov_scalar",
      "krylov_finalize", "contract_pixels", "mix_adjoint_sources", "mix_jac_adjoint",
      "gradient_assembly", "admm_vector", "setup", "misc"};
  return (k >= 0 && k < KC_COUNT) ? names[k] : "?";
}

inline cudaEvent_t prof_event(fwi_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Scope around one kernel launch: counts it and, in profiling mode outside
// graph capture, brackets it with events.
struct Prof {
  fwi_ctx* c;
  int cls;
  double bytes, flops;
  cudaEvent_t a = nullptr;
  Prof(fwi_ctx* ctx, int k, double by = 0.0, double fl = 0.0, int n = 1)
      : c(ctx), cls(k), bytes(by), flops(fl) {
    if (c->capturing) {
      c->capture_nodes += n;
    } else {
      c->launches += n;
      if (c->profiling) {
        a = prof_event(c);
        cudaEventRecord(a, c->stream);
      }
    }
  }
  ~Prof() {
    if (a) {
      cudaEvent_t b = prof_event(c);
      cudaEventRecord(b, c->stream);
      c->pending.push_back({cls, a, b, bytes, flops});
    }
  }
};

// Resolve the pending timings (synchronises the last recorded event).
inline void prof_flush(fwi_ctx* c) {
  if (c->pending.empty()) return;
  cudaEventSynchronize(c->pending.back().b);
  for (auto& p : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto& k = c->kstats[p.cls];
    k.ms += ms;
    k.launches += 1;
    k.bytes += p.bytes;
    k.flops += p.flops;
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
}

}  // namespace fwi
