/*
 * tctf2r.h -- C ABI of the GB300 TCTF2R traffic-tensor completion library.
 *
 * The library runs the per-iteration hot path of the TCTF2R Algorithm
 * (arXiv 2005.09838, Sec. 4.1) on one CUDA device: the generalized-inverse
 * X/Y updates of every frequency slice (Eq. (updataXYW1)), the product
 * Z~_k = X~_k Y~_k and its inverse mode-3 DFT (Eq. (barAAk)), the W-update
 * (Eq. (subquKKT) / Eq. (Wkiom)) and the forward mode-3 DFT of the new W
 * (Eq. (bar BA-k)).  Only floor(n3/2)+1 slices are solved; the others are
 * their complex conjugates (remark after the TCTF2R Algorithm).
 *
 * Conventions shared by every entry point
 *  - Every function returns a tc_status; none aborts or exits.  On failure
 *    tc_last_error() returns a message (thread-local, valid until the next
 *    call from the same thread).
 *  - Tensors are dense, column-major with the first index fastest: element
 *    (i1, i2, i3) of an n1 x n2 x n3 tensor is at i1 + n1*(i2 + n2*i3).  This
 *    is the element order of the paper's unfold (Sec. 2.1).
 *  - Real element type follows tc_params.precision: double for TC_FP64,
 *    float for TC_FP32, TC_TF32 and TC_BF16.
 *  - The caller owns every pointer it passes; the library copies what it
 *    needs and never keeps a caller pointer past the call.
 *  - A context is bound to the CUDA device that was current at tc_init and to
 *    the stream given there; all work is stream-ordered on that stream.  A
 *    context must not be used from two host threads at once.
 *  - After TC_ERR_CUDA or TC_ERR_TIMEOUT a context is poisoned: every later
 *    call on it returns TC_ERR_STATE except tc_free.
 */
#ifndef TCTF2R_H
#define TCTF2R_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TC_OK = 0,
  TC_ERR_ARG = 1,         /* invalid argument (sizes, NULL pointers, ranges) */
  TC_ERR_NOMEM = 2,       /* device or host allocation failed */
  TC_ERR_CUDA = 3,        /* a CUDA runtime call or kernel failed */
  TC_ERR_NUMERIC = 4,     /* non-finite objective or state */
  TC_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  TC_ERR_STATE = 6,       /* context poisoned by an earlier error */
  TC_ERR_UNSUPPORTED = 7  /* option not implemented by this build */
} tc_status;

/* Arithmetic of the iteration.
 *  TC_FP64, TC_FP32: every step in that type (the r x r pseudo-inverses too).
 *  TC_TF32, TC_BF16 (the precision form; data and state in float): for
 *    r > 16 the slice contractions Q = R~Y~^H run on the tensor cores with
 *    operands rounded to TF32 (BF16) and FP32 accumulation, each operand
 *    split into a rounded part and a rounded remainder (three products per
 *    step) unless TC_FLAG_SINGLE_PASS is set; for every r the two r x r
 *    Gram pseudo-inverses of each slice are taken in FP64.  Everything else
 *    runs in FP32. */
typedef enum { TC_FP64 = 0, TC_FP32 = 1, TC_TF32 = 2, TC_BF16 = 3 } tc_precision;

/* tc_params.flags bits. */
enum {
  /* TC_TF32 / TC_BF16 only: operands rounded once (one product per step);
   * faster, with the rounding error of the format (2^-11 TF32, 2^-8 BF16)
   * in every contraction. */
  TC_FLAG_SINGLE_PASS = 1
};

/* Step rule of Eq. (updataXYW1).  TC_STEP_EXACT takes alpha_kl = L_k1 and
 * beta_kl = L_k2 (unit steps along d_X, d_Y: exact minimisation of the
 * quadratic h_k in each block).  TC_STEP_SCALED uses the fixed alpha, beta
 * below divided by L_k1 = ||H_rho1||_2 ||Y~Y~^*||_2 and L_k2 = ||X~^* H_rho1 X~||_2
 * (no line search); the Gram matrices then go through the eigendecomposition,
 * which gives the 2-norms. */
typedef enum { TC_STEP_EXACT = 0, TC_STEP_SCALED = 1 } tc_step;

/* Problem statement of the TCTF2R Algorithm (Sec. 4.1, "Input").  H and K are
 * the fixed first-difference matrices of Eq. (Toeplitz) acting on modes 1 and
 * 2, so they are implied by n1 and n2.  Layout: 96 bytes, no implicit padding. */
typedef struct {
  int64_t n1, n2, n3;  /* tensor sizes (paper m1, m2, m3), each >= 1 */
  int32_t r;           /* tubal rank, 1 <= r <= min(n1, n2, 32) */
  int32_t precision;   /* tc_precision */
  double mu;           /* weight of ||W||^2, >= 0 (Eq. (TETP-optim)) */
  double rho1;         /* weight of the temporal-stability term on mode 1, >= 0 */
  double rho2;         /* weight of the periodicity term on mode 2, >= 0 */
  int32_t step;        /* tc_step */
  int32_t flags;       /* TC_FLAG_* bits; 0 for TC_FP64 and TC_FP32 */
  double alpha, beta;  /* step sizes, used only with TC_STEP_SCALED, > 0 */
  double eps;          /* stopping tolerance of step 6; 0 = run exactly n iterations */
  double pinv_rtol;    /* Gram eigenvalues <= pinv_rtol * lambda_max are cut by the
                          pseudo-inverse; <= 0 selects r times the machine epsilon
                          of the solve precision: 2^-52 for TC_FP64, for the
                          precision form and for TC_FP32 with r > 16 (whose r x r
                          solves are carried in FP64 storage with double-FP32
                          arithmetic), 2^-23 for TC_FP32 with r <= 16 */
} tc_params;

typedef struct tc_ctx tc_ctx;

/* Create a context and set the initial point of the TCTF2R Algorithm
 * ("Initialize"): W0 = P_Omega(G) (Sec. 3.1, missing entries filled with 0),
 * Y~0 and X~0 the mode-3 DFTs (Eq. (bar BA-k)) of Y0 and X0.
 *   out    : receives the new context (set to NULL on failure)
 *   p      : parameters, copied
 *   G      : n1*n2*n3 reals, observed tensor; entries off the mask are ignored
 *   mask   : n1*n2*n3 bytes, nonzero = observed (the set Omega)
 *   Y0     : r*n2*n3 reals, initial factor Y in the spatial domain (required)
 *   X0     : n1*r*n3 reals, initial factor X, or NULL for zero
 *   inputs_on_device : 1 if G, mask, Y0, X0 are device pointers on the current
 *            device, 0 if they are host pointers
 *   cuda_stream : cudaStream_t to order all work on (NULL = legacy default)
 * Device memory of the context is allocated here (cudaMalloc) and released by
 * tc_free; the CUDA graph of one iteration is captured and uploaded here too,
 * so tc_iterate only launches it.  Synchronises the stream before returning.
 * Errors: TC_ERR_ARG for invalid sizes/parameters/NULL inputs, TC_ERR_NOMEM,
 * TC_ERR_CUDA, TC_ERR_UNSUPPORTED for precisions or options not built. */
tc_status tc_init(tc_ctx** out, const tc_params* p, const void* G, const uint8_t* mask,
                  const void* Y0, const void* X0, int32_t inputs_on_device, void* cuda_stream);

/* Run n_iters iterations of the TCTF2R Algorithm (steps 1-4 and 7 of Sec. 4.1;
 * step 5 keeps r fixed).  Asynchronous: work is enqueued on the context's
 * stream and the call returns without waiting.  With p->eps > 0 the stopping
 * test of step 6 (||X~' - X~||_inf <= eps, ||Y~' - Y~||_inf <= eps and
 * ||W' - W||_F <= eps, ||.||_inf the largest modulus of an entry) is evaluated
 * on the device after every iteration; once it holds, the remaining launched
 * iterations do no work and the state stays at the iterate that passed it.
 *   done : receives the number of iterations run in this call (may be NULL;
 *          when given and p->eps > 0 the call synchronises the stream)
 * Errors: TC_ERR_ARG (n_iters < 0), TC_ERR_CUDA, TC_ERR_STATE. */
tc_status tc_iterate(tc_ctx* c, int32_t n_iters, int32_t* done);

/* Objective f0 of Eq. (TETP-optim) at the current iterate (X, Y, W), reduced in
 * FP64, and optionally ||P_Omega(X*Y - G)||_F.  Synchronises the stream.
 *   f0        : receives f0 (required)
 *   resid_obs : receives the observed-entry residual norm (may be NULL)
 * Errors: TC_ERR_ARG, TC_ERR_CUDA, TC_ERR_NUMERIC (non-finite f0), TC_ERR_STATE. */
tc_status tc_objective(tc_ctx* c, double* f0, double* resid_obs);

/* Copy the current iterate out (TCTF2R Algorithm, "Output"): W (n1*n2*n3 reals),
 * and optionally the spatial factors X (n1*r*n3) and Y (r*n2*n3), in the
 * column-major layout above.  dst_on_device selects device or host buffers.
 * Synchronises the stream.  Errors: TC_ERR_ARG, TC_ERR_CUDA, TC_ERR_STATE. */
tc_status tc_result(tc_ctx* c, void* W, void* X, void* Y, int32_t dst_on_device);

/* Profiling aid: run n_iters real iterations (they advance the state exactly
 * like tc_iterate) but launch the four per-iteration kernels one by one, with
 * CUDA events recorded around each on the context's stream, then synchronise.
 *   ms : receives 4 values, the mean device time per launch in milliseconds of
 *        the four kernels of one iteration, in launch order: the X-step
 *        contraction R~Y~^H, the X-step (with the r x r Y-step preparation),
 *        the Y-step, and the slab kernel (synthesis / inverse DFT / W-step /
 *        forward DFT).  The pseudo-inverse A^+ of the next X-step, which the
 *        captured iteration forms on a graph branch beside the slab kernel, runs
 *        after the slab kernel here and is not timed.
 * Errors: TC_ERR_ARG (n_iters < 1 or ms NULL), TC_ERR_CUDA, TC_ERR_STATE. */
tc_status tc_profile(tc_ctx* c, int32_t n_iters, double* ms);

/* State of the stopping test of step 6 (contexts created with p->eps > 0).
 * Synchronises the stream.
 *   changes   : receives 3 values of the last iteration run: ||X~' - X~||_inf,
 *               ||Y~' - Y~||_inf (largest modulus over the half spectrum, equal
 *               to that over all slices) and ||W' - W||_F (spatial)
 *   stopped   : receives 1 once the test has held, else 0 (may be NULL)
 *   iters_run : receives the iterations run since tc_init (may be NULL)
 * Errors: TC_ERR_ARG (changes NULL), TC_ERR_STATE (eps = 0 or poisoned),
 * TC_ERR_CUDA. */
tc_status tc_convergence(tc_ctx* c, double* changes, int32_t* stopped, int64_t* iters_run);

/* Step 5 of the TCTF2R Algorithm (Sec. 4.1): "adjust the rank vector and the
 * sizes of X~_k and Y~_k".  The paper leaves the rule open; this library reads
 * it as a rank decrease.  After the W-update of each iteration every solved
 * slice k takes the eigendecomposition of its Y-step Gram
 * G_k = X~_k^* H_rho1 X~_k; while at least one eigenvalue of its active
 * directions is <= tol * lambda_max(G_k) a per-slice count grows (else it
 * restarts), and when the count reaches patience the slice keeps only the
 * directions above that level (X~_k <- X~_k V_keep, Y~_k <- V_keep^* Y~_k) and
 * its rank r_k shrinks.  W~ is not changed by the step.  Slices past
 * floor(n3/2) follow by conjugate symmetry, so r_k = r_{n3-k+2} (1-based).
 * The initial rank vector is r for every slice; ranks never grow.
 * tc_rank_rule: tol in [0, 1) (0 turns the rule off for the following
 *   iterations; the ranks reached so far stay), patience >= 1.  Recaptures the
 *   iteration graph and synchronises the stream; set it before adding the
 *   context to a batch (a batch holds the graph captured at tc_batch_create).
 *   Errors: TC_ERR_ARG, TC_ERR_NOMEM, TC_ERR_CUDA, TC_ERR_STATE.
 * tc_ranks: ranks receives n3 values, the rank of every frontal slice of the
 *   DFT (r for all while the rule has never been on).  Synchronises the stream.
 *   Errors: TC_ERR_ARG, TC_ERR_CUDA, TC_ERR_STATE. */
tc_status tc_rank_rule(tc_ctx* c, double tol, int32_t patience);
tc_status tc_ranks(tc_ctx* c, int32_t* ranks);

/* Batched form: many independent completions (contexts of any sizes and either
 * precision, on the current device) advanced together, one CUDA graph launch
 * per iteration.  The graph holds each instance's captured iteration in K
 * independent chains, instance i in chain i mod K, so small instances that
 * leave most of the GPU idle fill it
 * together; the slices and tubes of every instance are independent
 * (Eq. (BDFT): the t-product separates by slice), so no instance waits on
 * another.  The first iterations of tc_batch_iterate time each candidate K
 * in {1, 4, 16, count} (every trial is a real iteration of all instances,
 * with identical results for every K) and keep the fastest.
 *
 * tc_batch_create: ctxs holds count distinct contexts (the caller keeps
 *   ownership; they must outlive the batch); cuda_stream is the stream the
 *   batch launches on.
 * tc_batch_iterate: n_iters iterations of every instance.  Ordered after the
 *   work queued on each context's stream and before its later calls; with a
 *   context whose p->eps > 0 the stopping test applies to that instance.
 *   Synchronises only while the tuning trials run.
 * tc_batch_branches: receives the chosen K (0 while tuning).
 * tc_batch_free: NULL-safe; the contexts stay valid.
 * Errors: TC_ERR_ARG, TC_ERR_STATE (poisoned context), TC_ERR_CUDA. */
typedef struct tc_batch tc_batch;
tc_status tc_batch_create(tc_batch** out, tc_ctx* const* ctxs, int32_t count, void* cuda_stream);
tc_status tc_batch_iterate(tc_batch* b, int32_t n_iters);
tc_status tc_batch_branches(tc_batch* b, int32_t* branches);
/* Once the tuning trials have chosen K, tc_batch_iterate runs all of its
 * remaining iterations in ONE graph launch: a CUDA while-node whose body is the
 * batched iteration followed by a one-thread kernel that counts the iterations
 * down on the device (the count only decreases, so the loop ends after n
 * passes).  Where conditional graph nodes are unavailable it falls back to one
 * launch per iteration.
 * tc_batch_launches: launches receives the graph launches made by
 *   tc_batch_iterate so far; device_loop (may be NULL) receives 1 once the
 *   device-side loop is in use.  Errors: TC_ERR_ARG. */
tc_status tc_batch_launches(tc_batch* b, int64_t* launches, int32_t* device_loop);
tc_status tc_batch_free(tc_batch* b);

/* Differentiation form: the factor terms of f0 (Eq. (TETP-optim)) with W held
 * at G on the mask, as a loss of spatial factors X (n1 x r x n3) and Y
 * (r x n2 x n3),
 *   L(X, Y) = 1/2 ||P_Omega(X*Y - G)||_F^2 + rho1/2 ||H unfold(X*Y, 1)||_F^2,
 * and its gradient, by the adjoint of the t-product (conjugate transpose of
 * Sec. 2): with E = P_Omega(Z - G) + rho1 (H^T H) x_1 Z, Z = X*Y,
 *   dL/dX = E * Y^*,  dL/dY = X^* * E,
 * evaluated per slice of the half spectrum (Eq. (bar BA-k), Eq. (barAAk)).
 * The gradients are those of Eq. (hkXYDer) gathered over the slices.
 *
 * tc_grad_init: p gives n1, n2, n3, r, rho1 and precision (TC_FP64 or TC_FP32;
 *   mu, rho2, step, eps are not used); G and mask as for tc_init (copied).
 * tc_grad_eval: X, Y in the precision's type, column-major (i1 fastest) like
 *   X0, Y0 of tc_init; loss receives L in FP64 (required); dX, dY receive the
 *   gradients in the layouts of X, Y (each may be NULL: then it is not
 *   formed).  on_device selects device or host buffers for X, Y, dX, dY.
 *   Synchronises the stream.  Errors: TC_ERR_ARG, TC_ERR_CUDA,
 *   TC_ERR_NUMERIC (non-finite loss).
 * tc_grad_free: NULL-safe. */
typedef struct tc_grad tc_grad;
tc_status tc_grad_init(tc_grad** out, const tc_params* p, const void* G, const uint8_t* mask,
                       int32_t inputs_on_device, void* cuda_stream);
tc_status tc_grad_eval(tc_grad* g, const void* X, const void* Y, double* loss, void* dX, void* dY,
                       int32_t on_device);
tc_status tc_grad_free(tc_grad* g);

/* Allocation-free completion of a small tensor (this entry point has no
 * counterpart in the paper; it is a deployment aid).  Some callers cannot call
 * cudaMalloc: code hosted in a framework whose allocator owns the device
 * memory, and latency-critical loops in which cudaMalloc/cudaFree could
 * synchronise the device and stall other streams.  tc_complete_static runs the
 * same computation as tc_init + tc_iterate(n_iters) + tc_result(W) (+
 * tc_objective) without allocating anything: every intermediate array lives in
 * one file-scope device array of 16 MiB, which every GPU that loads the library
 * holds until the process exits.
 *   p       : parameters (exact steps, eps = 0)
 *   G, mask, Y0, X0 : DEVICE pointers on the current device, layouts as for
 *             tc_init (X0 may be NULL); W : DEVICE output, n1*n2*n3 reals
 *   f0      : host pointer receiving f0 of the final iterate, or NULL
 *   cuda_stream : stream to run on; the call synchronises it before returning
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress).  The call reads its results back into host
 * variables and synchronises the stream, so it must not be made on a stream
 * that is being captured into a CUDA graph: it then returns TC_ERR_STATE.
 * All calls share the array and it keeps the last call's contents; the call
 * clears what must start at zero.  Calls that overlap on the GPU (other host
 * threads or streams) race on the array and must be serialised by the caller.
 * Errors: TC_ERR_ARG for bad arguments, for a buffer that is not device
 * memory of the current device (checked with cudaPointerGetAttributes; the
 * sizes of the buffers cannot be checked and must match the layouts above),
 * or for a problem whose arrays exceed the 16 MiB scratch (the message gives
 * the bytes needed), TC_ERR_STATE, TC_ERR_UNSUPPORTED, TC_ERR_CUDA,
 * TC_ERR_NUMERIC. */
tc_status tc_complete_static(const tc_params* p, const void* G, const uint8_t* mask, const void* Y0,
                             const void* X0, int32_t n_iters, void* W, double* f0, void* cuda_stream);

/* Tile of the mode-3 transform chosen for this context (the library's own
 * tuning, no counterpart in the paper).  Tube lengths other than the ones with
 * dedicated kernels (7, 112, 168 in FP32; 7 in FP64) use a transform written as
 * a product with the DFT matrix of Eq. (bar BA-k) / Eq. (barAAk), each work
 * item covering one tube and slab_tile rows (inverse) or slices (forward);
 * tc_init times slab_tile = 2, 4 and 8 on the initial pass (every choice gives
 * the same sums in the same order) and keeps the fastest.
 *   slab_tile : receives the chosen tile, 0 for a dedicated-kernel length.
 * Errors: TC_ERR_ARG. */
tc_status tc_tile(tc_ctx* c, int32_t* slab_tile);

/* Release a context and its device memory.  NULL-safe.  Synchronises the
 * context's stream first. */
tc_status tc_free(tc_ctx* c);

/* Message of the last failing call on this thread ("" if none). */
const char* tc_last_error(void);

/* Library version string. */
const char* tc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TCTF2R_H */
