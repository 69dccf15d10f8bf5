/*
 * libfwi -- C ABI of the data-parallel hot path of TV-regularised
 * frequency-domain full-waveform inversion for single-sided linear arrays
 * (Guo, Auerbach, Eldar, "TV-Regularized Frequency-Domain Full-Waveform
 * Inversion for Single-Sided Linear Ultrasound Array Data").
 *
 * One process, one GPU (sm_103a).  Every computational step runs in the
 * library's own CUDA kernels; there is no CPU fallback.
 *
 * Conventions used by every call
 * ------------------------------
 *  - Time dependence e^{-i omega t} (the paper writes e^{+j omega t}; all
 *    complex quantities here are the complex conjugates of the paper's).
 *  - Grid n[0] x n[1] x n[2] = Nx x Ny x Nz (Ny = 1 in 2D), pixel edge h.
 *    Arrays over the grid are depth-major, x fastest: index
 *    (iz * Ny + iy) * Nx + ix.  Pixel centres x = (ix + 1/2 - Nx/2) h,
 *    y = (iy + 1/2 - Ny/2) h, z = iz h.  N = Nx * Ny * Nz.
 *  - Complex numbers are interleaved (re, im): "c128" = 2 doubles,
 *    "c64" = 2 floats.  "cF" denotes the field type of the context:
 *    c64 for FWI_MIXED, c128 for FWI_FP64.
 *  - Transmitters and receivers are the same n_elem elements; data are
 *    stored [n_freq][n_elem (transmit)][n_elem (receive)].
 *  - Fields are stored [n_freq][n_elem][N].
 *  - "dev" pointers are device memory of the context's device, owned by the
 *    caller, and must not alias one another unless a call says so.  "host"
 *    pointers are host memory owned by the caller.  The library owns only
 *    the context and its workspace (allocated in fwi_create, freed in
 *    fwi_destroy); no call allocates device memory after fwi_create.
 *  - All device work is enqueued on the context's stream.  Calls that fill
 *    a host result (fwi_solve_info, misfit) synchronise that stream before
 *    returning; the others only enqueue.
 *  - Errors: every call returns an fwi_status; on failure the context keeps
 *    a message readable with fwi_last_error.  No exception crosses the ABI.
 *    Device-side loops are bounded (krylov_max_it) and report a per-RHS
 *    status; no kernel traps.
 */
#ifndef LIBFWI_H
#define LIBFWI_H

#include <stddef.h>

#if defined(__GNUC__)
#define FWI_API __attribute__((visibility("default")))
#else
#define FWI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fwi_status {
  FWI_OK = 0,
  FWI_ERR_INVALID_ARG = 1,   /* bad descriptor, size, pointer or index */
  FWI_ERR_NOMEM = 2,         /* workspace allocation failed in fwi_create */
  FWI_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  FWI_ERR_NOT_CONVERGED = 4, /* some RHS hit krylov_max_it (results written) */
  FWI_ERR_BREAKDOWN = 5,     /* BiCGSTAB breakdown (rho or omega = 0) */
  FWI_ERR_NONFINITE = 6,     /* a non-finite value reached a reduction */
  FWI_ERR_CANCELLED = 7,     /* fwi_cancel was called during the solve */
  FWI_ERR_UNSUPPORTED = 8,   /* grid size without a compiled FFT plan */
  FWI_ERR_REDUCE = 9         /* the caller's reducer (fwi_set_reducer) failed */
} fwi_status;

typedef enum fwi_precision {
  FWI_MIXED = 0, /* c64 fields and operator, FP64 Krylov scalars/reductions */
  FWI_FP64 = 1   /* c128 fields and operator throughout */
} fwi_precision;

/* Problem statement (Sec. II): geometry, background, array, frequencies. */
typedef struct fwi_problem_desc {
  int dim;                 /* 2 or 3 */
  int n[3];                /* Nx, Ny, Nz (Ny = 1 when dim == 2).  Each of
                              2*Nx, 2*Ny (3D), 2*Nz must be a supported FFT
                              length: 16, 32, 64, 128, 192, 256, 320, 384,
                              512, 640, 768, 1024. */
  double h;                /* pixel / voxel edge [m], finite and > 0 */
  double c0;               /* background speed of sound [m/s], finite and
                              > 0 */
  int n_elem;              /* number of array elements (N_T = N_R) */
  const double* elem_pos;  /* host [n_elem][dim], (x, z) or (x, y, z) [m],
                              finite; read and copied in fwi_create */
  int n_freq;
  const double* freq_hz;   /* host [n_freq], finite and > 0; copied in
                              fwi_create */
  double krylov_tol;       /* BiCGSTAB relative residual (<= 0: 1e-6) */
  int krylov_max_it;       /* BiCGSTAB iteration cap (<= 0: 1000) */
  int precision;           /* fwi_precision */
  int max_batch;           /* right-hand sides per Krylov launch
                              (<= 0: all n_elem * n_freq in one launch) */
  /* Transmits (Sec. V-A).  n_tx = 0: every element transmits a unit point
     source in turn (N_T = n_elem).  n_tx > 0: N_T = n_tx plane waves
     synthesised with all elements, transmit i weighting element e by
     w_{l,i,e} = exp(i k_l x_e sin tx_angle[i]) (delay x_e sin(theta) / c0
     under e^{-i omega t}; x_e the element's lateral coordinate).  By
     superposition the library solves the n_elem point-source fields and
     synthesises: data, residuals and Jacobian rows of transmit i are the
     w-weighted sums over elements.  Every element receives.  Data arrays
     (data, d_obs, J a, J^H b input) are [n_freq][N_T][n_elem]. */
  int n_tx;
  const double* tx_angle;  /* host [n_tx] steering angles [rad] or NULL when
                              n_tx = 0; copied in fwi_create */
  double elem_length;      /* 3D: length of each element along y [m] (finite
                              elevation, Sec. V-B); 0 = point elements.  A
                              line element transmits and senses the mean of
                              the point Green's function over its length
                              (centred on elem_pos).  Ignored when dim == 2. */
  int inv_factor;          /* inversion mesh (Sec. IV): cells of inv_factor^dim
                              forward pixels (<= 1: the forward mesh).  Each
                              of Nx, Nz (and Ny in 3D) must be a multiple.
                              The contrast m, its gradient, J's input a and
                              J^H's output z, the TV variables g, u, m_ref
                              and sos are then [N_inv] = N / inv_factor^dim
                              on the inversion mesh (contrast constant over a
                              cell; gradients summed over its pixels). */
  double alpha0;           /* attenuation of the background [Np/m/Hz] (Eq. 1-2;
                              0: lossless).  Then k_l = omega_l sqrt(1/c0^2 +
                              i alpha0/(pi c0)) (Im k > 0), the Green's
                              functions are those of complex k, and the
                              contrast is m = kappa/kappa0 - 1 with both
                              compressibilities complex (a background pixel
                              has m = 0; fwi_contrast_from_sos without an
                              alpha map gives every pixel alpha0). */
  int hybrid_born;         /* 1: the context keeps one more field array, the
                              receiver-field snapshot of the hybrid Born /
                              distorted-Born Jacobian (Sec. IV-B; see
                              fwi_freeze_receiver_fields); 0: none (the
                              Jacobian always uses the current fields). */
} fwi_problem_desc;

/* Per-call Krylov report.  The caller sets n_rhs and the optional host
   arrays (each NULL or of length n_rhs >= n_elem * n_freq); the library
   fills them.  RHS index = freq * n_elem + elem. */
typedef struct fwi_solve_info {
  int n_rhs;
  int* iters;            /* host: BiCGSTAB iterations per RHS */
  double* rel_resid;     /* host: final ||b - A x|| / ||b|| (recursive) */
  int* status;           /* host: FWI_OK, FWI_ERR_NOT_CONVERGED, ... */
  int max_iters;         /* out */
  double max_rel_resid;  /* out */
  int n_not_converged;   /* out */
  float device_ms;       /* out: device time of the call (CUDA events) */
} fwi_solve_info;

/* ADMM-TV parameters (Eq. 7-8, Algorithm 1). */
typedef struct fwi_admm_params {
  double lambda;     /* TV weight */
  double rho;        /* ADMM penalty */
  double gamma;      /* reference-model weight */
  double dual_step;  /* factor of the u-update (<= 0: rho, as printed) */
  int n_cg;          /* CG iterations of the Gauss-Newton m-step */
  const void* m_ref; /* dev c128 [N] reference model, or NULL for 0 */
} fwi_admm_params;

typedef struct fwi_ctx fwi_ctx;

/* Device bytes fwi_create will allocate for this descriptor (admission
   control).  Returns 0 for an invalid or unsupported descriptor. */
FWI_API size_t fwi_workspace_bytes(const fwi_problem_desc* desc);

/* Create a context on the current CUDA device, bound to cuda_stream (a
   cudaStream_t).  NULL: the context creates its own blocking stream, which
   is implicitly ordered with the legacy default stream (the Krylov
   iterations are CUDA graphs, and the legacy stream cannot be captured).  Allocates the workspace and
   precomputes, per frequency, the FFT of the cell-integrated Green's
   function on the doubled lattice (Sec. IV-A) and the incident fields
   p0 = G(x, x_e) (Eq. 5).  On failure *out is NULL. */
FWI_API fwi_status fwi_create(const fwi_problem_desc* desc, void* cuda_stream,
                      fwi_ctx** out);
FWI_API fwi_status fwi_destroy(fwi_ctx* ctx);
/* Message of the last failure on ctx ("" if none); valid until the next
   call on ctx.  fwi_last_error(NULL) reports fwi_create failures. */
FWI_API const char* fwi_last_error(const fwi_ctx* ctx);
/* Request that a running or next solve stop at its next host check
   (thread-safe); the solve returns FWI_ERR_CANCELLED. */
FWI_API fwi_status fwi_cancel(fwi_ctx* ctx);

/* Contrast m = kappa/kappa0 - 1 (Eq. 1-3) from speed of sound and optional
   attenuation: m = c0^2/c^2 - 1 + i alpha c0^2/(pi c) for a lossless
   background; with alpha0 > 0, rho0 kappa = 1/c^2 + i alpha/(pi c) over
   rho0 kappa0 = 1/c0^2 + i alpha0/(pi c0), minus 1 (alpha NULL: every pixel
   has alpha0).  sos: dev double [N_inv] (m/s); alpha: dev double [N_inv]
   (Np/m/Hz) or NULL; m: dev c128 [N_inv] (out). */
FWI_API fwi_status fwi_contrast_from_sos(fwi_ctx* ctx, const double* sos,
                                 const double* alpha, void* m);

/* Speed of sound and attenuation from a contrast, the inverse of Eq. 1-3:
   with rho0 kappa = (1/c0^2 + i alpha0/(pi c0)) (1 + m), c = 1/sqrt(Re(rho0
   kappa)) and alpha = pi c Im(rho0 kappa) [Np/m/Hz] (attenuation
   inversion: the complex contrast that fwi_admm_tv_step updates carries
   both).  m: dev c128 [N_inv]; sos, alpha: dev double [N_inv] or NULL
   (out). */
FWI_API fwi_status fwi_sos_attenuation_from_contrast(fwi_ctx* ctx, const void* m, double* sos,
                                                     double* alpha);

/* Forward simulation F(m) (Eq. 4-5; Algorithm 1 "forward simulation"):
   solves A_l p = p0_{l,e}, A_l = I - K_l diag(m), for every transmit e and
   frequency l by batched BiCGSTAB, and projects the data
   P^s_{l,e,j} = k_l^2 dV sum_n G_l(x_j, x_n) m_n p_{l,e}(n).
   m: dev c128 [N].  fields: dev cF [n_freq][n_elem][N] or NULL (out; with
   warm_start != 0 also the initial guess, otherwise the guess is 0).
   data: dev cF [n_freq][N_T][n_elem] or NULL (out; with plane-wave
   transmits the w-weighted sums of the point-source data).  The fields
   (always the n_elem point-source fields) stay in the context for
   fwi_admm_tv_step.  info: host or NULL. */
FWI_API fwi_status fwi_forward(fwi_ctx* ctx, const void* m, void* fields,
                       int warm_start, void* data, fwi_solve_info* info);

/* Adjoint-state solves (Sec. IV-B): (I - diag(m) K_l)^H lambda = src for
   every (l, e).  Computed as lambda = conj(A_l^{-1} conj(src)) because K is
   complex-symmetric.  src, lambda: dev cF [n_freq][n_elem][N]. */
FWI_API fwi_status fwi_adjoint(fwi_ctx* ctx, const void* m, const void* src,
                       void* lambda, fwi_solve_info* info);

/* One gradient evaluation of phi = 1/2 ||F(m) - d_obs||^2 (Eq. 7, 17):
   forward solves, residual r = F(m) - d_obs, adjoint sources
   s_{l,e} = sum_j conj(R_{l,j}) r_{l,e,j}, adjoint solves, and
   grad_n = sum_{l,e} conj(p_{l,e}(n)) lambda_{l,e}(n) = (J^H r)_n.
   d_obs: dev cF [n_freq][N_T][n_elem]; grad: dev c128 [N] (out);
   misfit: host double (out) or NULL; data: dev cF (out, the predicted
   data F(m)) or NULL.  The forward fields stay in the context.  With
   plane-wave transmits r is the plane-wave residual and the adjoint
   sources of element e carry the residual W^H r (the gradient of the
   synthesised data map by the chain rule). */
FWI_API fwi_status fwi_gradient(fwi_ctx* ctx, const void* m, const void* d_obs,
                        void* grad, double* misfit, void* data,
                        fwi_solve_info* info_fwd, fwi_solve_info* info_adj);

/* One ADMM-TV iteration after the gradient (Algorithm 1 lines 4-7,
   Eq. 9-14): solves (J^H J + rho nabla^T nabla + gamma I) dm = b with
   b = -grad + rho nabla^T(g + u - nabla m) + gamma (m_ref - m) by n_cg CG
   iterations from 0 (J from the fields of the last fwi_forward /
   fwi_gradient), m += dm, g = shrink_{lambda/rho}(nabla m - u),
   u += dual_step (g - nabla m), and optionally c = c0 / sqrt(1 + Re m).
   nabla: forward differences in index units, zero on the last slice.
   With plane-wave transmits J^H J = J_point^H (W^H W) J_point: the exact
   distorted-Born Jacobian at the current model every iteration (the
   receiver fields are the point-source fields solved anyway).
   m: dev c128 [N] (in/out); g, u: dev c128 [dim][N] (in/out, component
   order x, [y], z); grad: dev c128 [N]; sos_out: dev double [N] or NULL. */
FWI_API fwi_status fwi_admm_tv_step(fwi_ctx* ctx, void* m, void* g, void* u,
                            const void* grad, const fwi_admm_params* p,
                            double* sos_out);

/* Receiver fields of the Jacobian (Sec. IV-B, hybrid Born / distorted-Born
   approximation).  The Jacobian rows are dP_{l,e,j}/dm_n =
   ptilde_{l,j}(n) p_{l,e}(n) with the receiver fields ptilde_{l,j} =
   A_l^{-1} R_{l,j}; with receivers at the element positions ptilde_{l,j} =
   k_l^2 dV p_{l,j}, the element fields.  By default J and J^H (and so the
   m-step of fwi_admm_tv_step) take ptilde from the current forward fields
   (the strict distorted-Born Jacobian).  The paper refreshes the receiver
   fields only every few iterations and keeps them fixed in between:
     freeze = 1: copy the current forward fields (of the last fwi_forward or
                 fwi_gradient) into the context's snapshot; until the next
                 call, J and J^H take ptilde from the snapshot and p_{l,e}
                 from the current fields;
     freeze = 0: back to the current fields.
   Needs a context created with hybrid_born = 1 (FWI_ERR_INVALID_ARG
   otherwise) and, for freeze = 1, forward fields.  Enqueued on the context
   stream (a device-to-device copy of n_freq * n_elem * N field elements). */
FWI_API fwi_status fwi_freeze_receiver_fields(fwi_ctx* ctx, int freeze);

/* ---- Sharding over GPUs by frequency (Sec. IV-D) -------------------------
   The paper spreads its sources over workers and aggregates the partial
   Jacobian products.  Here the work is split by frequency: each rank (one
   process per GPU) creates its context with a subset of the frequencies and
   the matching rows of d_obs, so its solves, data and Jacobian rows are its
   own, and every sum the method takes over frequencies is completed by a
   reduction the caller supplies (NCCL on the context stream, or any other
   all-reduce).  With a reducer set the library calls it, on the host thread
   of the library call, on
     - fwi_gradient: the misfit's per-block partial sums (before the host
       adds them) and the assembled gradient (2 N_inv doubles), so that
       every rank returns the misfit and gradient of all frequencies;
     - fwi_admm_tv_step: each CG iteration's J^H J d (2 N_inv doubles), so
       that every rank runs the same CG iterates and returns the same m, g,
       u and SoS (given the same inputs on every rank);
     - fwi_jac_adjoint: its output z.
   fn must replace the `count` doubles at device address buf by their sum
   over all ranks.  Work the library enqueued on cuda_stream (the context's
   stream) before the call produces buf; work it enqueues after the call
   reads the result, so fn must order its writes before that work (a
   collective on cuda_stream, or a synchronise and a blocking copy back).
   Every rank must make the same sequence of library calls.  fn returns 0
   on success; anything else makes the library call return FWI_ERR_REDUCE.
   fn = NULL removes the reducer.  The library itself never communicates. */
typedef int (*fwi_reduce_fn)(void* buf, size_t count, void* cuda_stream, void* user);
FWI_API fwi_status fwi_set_reducer(fwi_ctx* ctx, fwi_reduce_fn fn, void* user);

/* ADMM initialisation (Algorithm 1): g = nabla m0, u = 0.
   m0: dev c128 [N]; g, u: dev c128 [dim][N] (out). */
FWI_API fwi_status fwi_admm_init(fwi_ctx* ctx, const void* m0, void* g, void* u);

/* Single operator applications (Sec. IV-A) on n_rhs vectors at frequency
   index freq: out = K in, A in = in - K(m in), or A^H in
   = in - conj(m) K^H in.  in, out: dev cF [n_rhs][N] (must not alias);
   m: dev c128 [N].  1 <= n_rhs <= the context's batch. */
FWI_API fwi_status fwi_apply_K(fwi_ctx* ctx, int freq, int n_rhs, const void* in,
                       void* out);
FWI_API fwi_status fwi_apply_A(fwi_ctx* ctx, const void* m, int freq, int n_rhs,
                       const void* in, void* out);
FWI_API fwi_status fwi_apply_AH(fwi_ctx* ctx, const void* m, int freq, int n_rhs,
                        const void* in, void* out);

/* Implicit Jacobian products at the fields of the last forward solve
   (Eq. 16-17, receiver fields ptilde_{l,j} = k_l^2 dV p_{l,j}):
   (J a)_{l,e,j} = sum_n p_{l,e}(n) ptilde_{l,j}(n) a_n and
   (J^H b)_n = sum_{l,e,j} conj(p_{l,e}(n) ptilde_{l,j}(n)) b_{l,e,j}.
   a: dev c128 [N]; y: dev c128 [n_freq][N_T][n_elem] (out of J, in of
   J^H; with plane-wave transmits J = W J_point, J^H = J_point^H W^H);
   z: dev c128 [N] (out). */
FWI_API fwi_status fwi_jac_forward(fwi_ctx* ctx, const void* a, void* y);
FWI_API fwi_status fwi_jac_adjoint(fwi_ctx* ctx, const void* y, void* z);

/* ---- Serving: continuous batching of reconstructions -------------------
   A server runs whole reconstructions (Algorithm 1: contrast from the
   starting SoS, g0 = nabla m0, u0 = 0, then n_iter x [fwi_gradient,
   (receiver-field refresh), fwi_admm_tv_step]) for requests of different grids, arrays and frequency
   sets.  Requests wait in FIFO order and are admitted, first fit, as soon as
   a worker slot is free and their device footprint (fwi_workspace_bytes of
   the request plus its vectors) fits in the remaining HBM budget.  Each
   admitted request owns a context and a non-blocking CUDA stream, so the
   work of concurrent requests overlaps on the device; its fields, Krylov
   state and ADMM state stay device-resident until it completes.  Results
   are independent of the mix: each request computes exactly what it would
   compute alone. */
typedef struct fwi_server fwi_server;
typedef struct fwi_request {
  fwi_problem_desc problem;  /* host arrays are copied at submit */
  const double* sos0;        /* host double [N]: starting speed of sound */
  const void* d_obs;         /* host cF [n_freq][N_T][n_elem]: observed data */
  fwi_admm_params admm;      /* m_ref must be NULL */
  int n_iter;                /* ADMM-TV iterations (>= 1) */
  int refresh_every;         /* hybrid Born schedule (Sec. IV-B): <= 1 uses
                                the current receiver fields in every m-step;
                                K > 1 refreshes them on iterations 0, K,
                                2K, ... (fwi_freeze_receiver_fields right
                                after that iteration's gradient) and keeps
                                them fixed in between */
} fwi_request;
typedef struct fwi_request_result {
  int status;                /* fwi_status of the reconstruction */
  double queue_ms;           /* submit -> admission */
  double run_ms;             /* admission -> completion */
  double latency_ms;         /* submit -> completion */
  double misfit_first;       /* 1/2 ||F(m0) - d||^2 */
  double misfit_last;        /* misfit at the last iterate's forward solve */
  long long rhs_solves;      /* forward + adjoint BiCGSTAB solves */
  size_t bytes;              /* admitted device footprint */
  int krylov_iters_max;      /* most BiCGSTAB iterations of any solve */
  double krylov_iters_mean;  /* mean over the request's forward / adjoint batches
                                of their largest iteration count */
  long long not_converged;   /* solves that stopped at krylov_max_it */
} fwi_request_result;
/* hbm_budget: bytes the server may hold for admitted requests (0: 90 % of
   the free device memory at creation); max_active: worker slots (>= 1).
   Uses the current CUDA device. */
FWI_API fwi_status fwi_server_create(size_t hbm_budget, int max_active, fwi_server** out);
/* Queue a request (inputs copied); *id identifies it.  A request whose
   footprint exceeds the whole budget is rejected (FWI_ERR_NOMEM). */
FWI_API fwi_status fwi_server_submit(fwi_server* s, const fwi_request* r, long long* id);
/* Block until request id completes; sos_out: host double [N] (final SoS) or
   NULL; res: host or NULL.  Each id can be waited for once. */
FWI_API fwi_status fwi_server_wait(fwi_server* s, long long id, double* sos_out,
                                   fwi_request_result* res);
/* Cancel request id: a queued request leaves the queue at once; a running
   one stops at its solve's next host check or before its next iteration.
   Either completes with status FWI_ERR_CANCELLED and no SoS (its wait
   returns that status); a finished request keeps its result.  Thread-safe.
   FWI_ERR_INVALID_ARG for an unknown or already waited id. */
FWI_API fwi_status fwi_server_cancel(fwi_server* s, long long id);
/* Current admitted count, queued count and admitted bytes (any may be NULL). */
FWI_API fwi_status fwi_server_stats(fwi_server* s, int* active, int* queued, size_t* bytes);
/* Finish every submitted request, then release the workers. */
FWI_API fwi_status fwi_server_destroy(fwi_server* s);

/* ---- Allocation-free contraction (no counterpart in the paper) ----------
   For callers that cannot allocate device memory: code that runs where
   cudaMalloc is forbidden or unavailable (inside another framework's memory
   pool, under a stream-ordered allocator policy, in a plugin that must not
   touch the allocator, or before a context could be sized), and so cannot
   call fwi_create.  It computes, without any allocation,
       Y[l][e][j] = scale[l] * sum_n X[l][e][n] a[n] Q[l][j][n]
   -- the pixel contraction behind the data projection and J a (with
   X = Q = fields and scale = k_l^2 dV) -- for complex FP32 inputs.
   X, Q: dev c64 [n_freq][n_elem][N]; a: dev c64 [N] or NULL (a = 1);
   scale: host double [n_freq]; Y: dev c128 [n_freq][n_elem][n_elem] (out);
   cuda_stream: cudaStream_t (NULL = legacy default stream).
   Limits: n_freq <= FWI_NOALLOC_MAX_FREQ and n_freq * n_elem^2 <= 524288
   (the split partial sums live in one 4 MiB file-scope device array, which
   every GPU that loads the library holds until exit); larger sizes return
   FWI_ERR_INVALID_ARG with a message (fwi_last_error(NULL)).
   cuda_stream and X, a, Q, Y must belong to the current device (a stream
   of another device is rejected with FWI_ERR_INVALID_ARG).
   The first call on a device looks up the array's device address
   (cudaGetSymbolAddress) and caches it for the current CUDA context; a
   later context on that device (after cudaDeviceReset, say) looks it up
   again on its first call.  Make each such first call outside any stream
   capture.  Every call shares the array, which keeps the last
   call's contents (no part of it needs to start at zero: each call writes
   every partial it reads).  Calls whose work overlaps on the GPU (other
   streams, other host threads) race on the array; serialise them.
   Enqueues on cuda_stream and returns without synchronising. */
#define FWI_NOALLOC_MAX_FREQ 32
FWI_API fwi_status fwi_contract_pixels_noalloc(const void* X, const void* a, const void* Q,
                                               int n_freq, int n_elem, long long N,
                                               const double* scale, void* Y,
                                               void* cuda_stream);

/* ---- Instrumentation (no counterpart in the paper) ----------------------
   Kernel launch counting is always on.  With profiling on, the Krylov
   iterations run without CUDA graphs and every kernel launch of the
   library is bracketed by CUDA events on the context stream; durations,
   launch counts and algorithmic bytes (operator passes) or flops
   (contractions) are accumulated per kernel class. */
#define FWI_MAX_KERNEL_STATS 24
typedef struct fwi_kernel_stat {
  char name[40];       /* kernel class, e.g. "col_conv" */
  double ms;           /* summed device time (profiling mode) */
  long long launches;  /* launches timed */
  double bytes;        /* algorithmic HBM bytes of those launches */
  double flops;        /* algorithmic flops of those launches */
} fwi_kernel_stat;
typedef struct fwi_stats {
  long long kernel_launches;  /* kernels launched so far (graph nodes counted) */
  int n_kernel_stats;
  fwi_kernel_stat kernels[FWI_MAX_KERNEL_STATS];
} fwi_stats;
FWI_API fwi_status fwi_set_profiling(fwi_ctx* ctx, int on);
FWI_API fwi_status fwi_get_stats(const fwi_ctx* ctx, fwi_stats* out);
FWI_API fwi_status fwi_reset_stats(fwi_ctx* ctx);

/* Tile-shape tuning of the operator passes.  fwi_create times every
   variant on the context's batch (unless the environment variable
   LIBFWI_AUTOTUNE=0) and keeps the fastest; choices are cached in
   $LIBFWI_TUNE_CACHE (default ~/.cache/libfwi/autotune.txt).  Variants change
   only how many lines / columns a thread block holds: results are
   bitwise identical for every variant.  fwi_set_tuning forces variants. */
typedef struct fwi_tuning {
  int row_fwd_variant;  /* 0: 128 threads per CTA, 1: 64, 2: 256 */
  int row_inv_variant;
  int col_variant;      /* 0: default column tile, 1: half width */
  int col_y_variant;    /* 3-D y passes */
  int tuned;            /* 1 if chosen by timing */
  float ms[4][4];       /* measured ms per pass kind and variant (0: not timed) */
  int jac_tensor_cores; /* 1 (default): FP32 pixel contractions of the data
                           projection, J a and J^H b on the tensor cores
                           (tcgen05, 3xTF32 products, FP32 accumulation);
                           0: CUDA-core FP32 kernels.  FP64 contexts and odd
                           pixel counts always use the CUDA-core kernels. */
  int overlap_halves;   /* 1 (default on 2-D lattices): batches of >= 32
                           right-hand sides iterate as two independent
                           halves on two streams of one CUDA graph, so that
                           the passes of one half fill the SMs the other
                           half's passes leave idle; 0 (default on 3-D
                           lattices, whose passes already fill the GPU):
                           one chain.  Results are bitwise the same. */
  int debug_stall_once; /* test of the failure path: 1 makes the next
                           tensor-core contraction withhold its first
                           pipeline stage, so that its bounded waits give up
                           after about 1 s and the call returns FWI_ERR_CUDA
                           ("pipeline wait timed out"); the context stays
                           usable.  Applies once; reads back as 0. */
  int col_tma;          /* 1 (default): the FP32 column passes stage their
                           input tiles (and, for the 3-D and smaller 2-D
                           convolutions, their kernel-spectrum tiles) in
                           shared memory with TMA tensor copies, the next
                           tile's copy overlapping the current tile's
                           transforms, and read their twiddles from shared
                           memory; 0: plain loads from global memory.  The
                           same arithmetic on the same values: results agree
                           to FP32 rounding. */
  int col_spectrum_stage; /* 1 (default): with col_tma, the convolution also
                           stages its kernel-spectrum tiles with TMA where
                           they fit (half the column's rows, the spectrum
                           being even; at most 256 rows); 0: the spectrum
                           is read from global memory.  Results agree to
                           FP32 rounding. */
  int jac_tma;          /* 1 (default): the tensor-core pixel contractions
                           receive their raw FP32 operand tiles by TMA
                           tensor copies issued by one producer thread;
                           0: every producer copies its rows with cp.async.
                           Results are bitwise the same. */
  int row_l2_prefetch;  /* 1 (default): the row passes prefetch the HBM rows
                           of their next work item into L2 while the
                           current item transforms; 0: no prefetch.
                           Results are bitwise the same. */
  int row_stage;        /* 1 (default): the FP32 forward row pass copies the
                           rows of its next work item (every array it
                           reads) into shared memory with bulk copies while
                           the current item transforms, and reads its
                           samples there; 0: loads from global memory (with
                           row_l2_prefetch).  Results agree to FP32
                           rounding. */
  int col_pairs;        /* 1 (default): the FP32 convolution pass, where its
                           transform length is 16, 64 or 256 and its kernel
                           spectrum is staged, computes two columns per
                           thread with packed f32x2 arithmetic on column
                           pairs; 0: one column per thread.  Results agree
                           to FP32 rounding. */
} fwi_tuning;
FWI_API fwi_status fwi_get_tuning(const fwi_ctx* ctx, fwi_tuning* out);
FWI_API fwi_status fwi_set_tuning(fwi_ctx* ctx, const fwi_tuning* in);

/* Library version string. */
FWI_API const char* fwi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBFWI_H */
