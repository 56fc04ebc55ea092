/*
 * edaa.h -- C ABI of the GB300 (sm_103a) implementation of Entropic Descent
 * Archetypal Analysis (EDAA; Zouaoui et al., arXiv 2209.11002).
 *
 * The library solves, for each of M runs on each of one or more hyperspectral
 * cubes,   min_{A,B} 1/2 ||X - X B A||_F^2   with the columns of A (p x N) on
 * the simplex Delta_p and the columns of B (N x p) on Delta_N (Sec. III-A,
 * eq. AA), by the alternating entropic descent of Algorithm 1, and then
 * applies the model-selection rule of Algorithm 2.
 *
 * Conventions shared by every entry point
 *   - X is given PIXEL-MAJOR: an N x L row-major float32 array in which pixel
 *     i's L band values are contiguous (the paper's L x N matrix stored column
 *     by column).  X may live in host or device memory; host data is copied
 *     with cudaMemcpyAsync on the context's stream.
 *   - Outputs use the paper's shapes in row-major order: E is L x p, A is
 *     p x N, B is N x p.  Output pointers may be host or device memory; they
 *     are always caller-owned and never freed by the library.
 *   - Every call is asynchronous on the stream given to edaa_init unless it
 *     says it synchronises.  The library owns only what edaa_init allocated.
 *   - Errors: every call returns an edaa_status; no exception crosses the
 *     ABI.  edaa_last_error() returns a thread-local message for the last
 *     failure on the calling thread.  A device-side status word records
 *     barrier time-outs and non-finite merges; synchronising calls report it,
 *     after which the context only accepts edaa_destroy (EDAA_ERR_STATE).
 *   - There is no CPU fallback: without a CUDA device every compute call
 *     fails with EDAA_ERR_CUDA.
 */
#ifndef EDAA_H
#define EDAA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EDAA_OK = 0,
  EDAA_ERR_ARG = 1,         /* invalid argument (shape, pointer, index)        */
  EDAA_ERR_CUDA = 2,        /* a CUDA runtime call failed (no device, launch)  */
  EDAA_ERR_OOM = 3,         /* device allocation failed                        */
  EDAA_ERR_STATE = 4,       /* context unusable after an earlier device error  */
  EDAA_ERR_NONFINITE = 5,   /* a merge met a non-finite or empty softmax sum   */
  EDAA_ERR_TIMEOUT = 6,     /* a bounded grid barrier gave up waiting          */
  EDAA_ERR_UNSUPPORTED = 7  /* shape outside the compiled kernels' range       */
} edaa_status;

/* Contraction types of the X-streaming passes.  EDAA_FP32: CUDA cores.
 * EDAA_TF32, EDAA_BF16: tensor cores with TF32 or BF16 operands and FP32
 * accumulation.  EDAA_TF32X3: tensor cores at FP32 accuracy; every operand is
 * split into two TF32 parts (x = hi + lo, lo = tf32(x - hi)) and each product
 * is formed as hi*hi + hi*lo + lo*hi (the dropped lo*lo term is about 2^-22
 * relative), with the element-wise steps in full FP32.  The tensor-core modes
 * apply to cubes whose ensembles make the contractions dense (M p >= 64);
 * other cubes use the CUDA-core FP32 pass. */
typedef enum { EDAA_FP32 = 0, EDAA_TF32 = 1, EDAA_BF16 = 2, EDAA_TF32X3 = 3 } edaa_precision;

typedef struct {
  int T;              /* outer iterations (Algorithm 1; paper: 100)                 */
  int K1;             /* A-steps per outer iteration (paper: 5)                     */
  int K2;             /* B-steps per outer iteration (paper: 5)                     */
  int normalize;      /* 1: l2-normalise every pixel first (eq. normalization)      */
  int precision;      /* edaa_precision of the X-streaming contractions             */
  int fit_norm;       /* Algorithm 2 fit: 0 entrywise sum |X-EA|, 1 max column sum  */
  int coherence;      /* eq. coherence: 0 cosine of columns of E, 1 raw inner product */
  double fit_ratio;   /* Algorithm 2 threshold factor (paper: 1.05)                 */
  int persistent;     /* 1: one persistent launch per solve with bounded grid
                         barriers; 0: one launch per pass, replayed from a graph    */
  int autotune;       /* 1: time candidate tile shapes at init and keep the best    */
  double barrier_timeout_ms; /* give-up time of a grid barrier wait (default 2000)  */
  int center;         /* 1 (default): iterate on X minus its mean pixel.  EDAA's
                         iterates are unchanged by a common translation of all
                         pixels (each gradient changes by a constant along its
                         softmax axis), and centring avoids the cancellation in
                         E A A^T - X A^T; outputs and reported gradients are in
                         the paper's uncentred terms either way.                   */
  int trace;          /* 1: record when each phase of a launch sequence starts and
                         ends (GPU global timer; read with edaa_trace_read).  0
                         (default): no recording.                                   */
  int tile[4];        /* explicit launch shape of the CUDA-core passes, applied to
                         every CUDA-core cube: {runs per CTA group, pixel warps of
                         phase 1, pixels per lane of phase 1 (1, 2, or 4 for
                         p >= 3), pixel warps of phase 2}; the pixel tile is
                         32 x tile[1] x tile[2] (32..128).  All zero (default):
                         the built-in shape, or the autotuner's with autotune = 1.
                         A shape outside the compiled register tiles or the shared
                         memory of one CTA fails edaa_init with EDAA_ERR_ARG.
                         On tensor-core cubes tile[0] alone applies (1..M, the
                         other entries unchecked): the runs per CTA group, capped
                         by what tensor memory holds.                             */
  int record_loss;    /* 1: every outer iteration ends with the fit pass (one more
                         stream of X per outer iteration) and logs each run's
                         loss ||X - X B A||_F^2 (read with edaa_loss_history);
                         0 (default): no log.                                       */
} edaa_config;

typedef struct {
  const float* X;          /* N x L pixel-major float32, host or device             */
  int L, N, p, M;          /* bands, pixels, endmembers, ensemble runs              */
  const uint64_t* seeds;   /* host, length M: run seeds s_m (Algorithm 2)           */
  const double* gammas;    /* host, length M: step factors gamma_m in eq. (eta0A)   */
} edaa_cube;

typedef struct edaa_ctx edaa_ctx;

/* Fills the paper's defaults: T=100, K1=K2=5, normalize=1 (Sec. III-C),
 * FP32, entrywise l1 fit, cosine coherence, fit_ratio=1.05 (Algorithm 2),
 * persistent=1, autotune=0, barrier_timeout_ms=2000, center=1. */
void edaa_config_default(edaa_config* cfg);

/* Creates a context for n_cubes cubes (1..16), each with its own L, N, p, M,
 * all sharing T, K1, K2 (Algorithm 1).  Copies and normalises X (eq.
 * normalization), draws B^0 = softmax(0.1 u) per run from SplitMix64 seeded
 * with s_m (eq. initB0; entry (i,j) uses generator output i*p+j+1, top 24
 * bits), sets A^0 = 1/p (eq. initA0), and the step sizes eta1 =
 * gamma_m / sigma_max^2(X B^0), eta2 = sqrt(p/N) eta1 (eqs. eta0A, eta0B).
 * Limits: 1 <= p <= 8, p <= N, 1 <= L <= 319, M >= 1.  `stream` is a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns all
 * device memory it allocated; free it with edaa_destroy. */
edaa_status edaa_init(edaa_ctx** out, const edaa_cube* cubes, int n_cubes,
                      const edaa_config* cfg, void* stream);

/* Re-runs the initialisation of edaa_init on the existing buffers (no
 * allocation).  If X is not NULL it replaces cube `cube`'s data (same shape,
 * host or device, pixel-major); cube = -1 with X = NULL resets every cube. */
edaa_status edaa_reset(edaa_ctx* ctx, int cube, const float* X);

/* Runs n_outer outer iterations of Algorithm 1 (each: K1 A-steps, eq.
 * update_A, then K2 B-steps, eq. update_B) on every run of every cube. */
edaa_status edaa_step(edaa_ctx* ctx, int n_outer);

/* Runs the remaining outer iterations up to T, then computes per run the
 * fit ||X - E A||_1, the loss ||X - X B A||_F^2 and the coherence of E
 * (Algorithm 2, eq. coherence).  Replays a captured CUDA graph when the
 * context is at iteration 0. */
edaa_status edaa_solve(edaa_ctx* ctx);

/* Synchronises; applies Algorithm 2 to cube `cube`: I = {m : fit_m <=
 * fit_ratio * min fit}, best = argmin_{m in I} mu_m, ties to the lowest m,
 * non-finite fits excluded.  Writes *best and, when not NULL, fit[M] and
 * mu[M] (host arrays).  Needs a preceding edaa_solve. */
edaa_status edaa_select(edaa_ctx* ctx, int cube, int* best, double* fit, double* mu);

/* Algorithm 2's rule alone, on host arrays (no device work).  Returns the
 * selected index, or -1 when no fit is finite or M < 1. */
int edaa_select_rule(const double* fit, const double* mu, int M, double fit_ratio);

/* Copies run `run` of cube `cube`: E = X B (L x p), A (p x N), B (N x p),
 * row-major, to caller buffers (host or device; NULL skips). */
edaa_status edaa_get(edaa_ctx* ctx, int cube, int run, float* E, float* A, float* B);

/* Gradients of ||X - X B A||_F^2 at the current state of one run:
 * gA = 2 (E^T E A - E^T X) (p x N row-major) and gB = 2 X^T (E A A^T - X A^T)
 * (N x p row-major) -- twice the terms inside eqs. (update_A), (update_B).
 * Caller buffers, host or device; NULL skips. */
edaa_status edaa_grad(edaa_ctx* ctx, int cube, int run, float* gA, float* gB);

/* Synchronises; writes loss[m] = ||X - X B A||_F^2 (FP64 accumulation) for
 * every run of cube `cube` at the current state (host array, length M). */
edaa_status edaa_loss(edaa_ctx* ctx, int cube, double* loss);

/* The loss log (needs config.record_loss = 1): row t (0-based) holds every
 * run's loss ||X - X B A||_F^2 (FP64 accumulation) after outer iteration
 * t + 1 of Algorithm 1 since the last init/reset, for t < T.  Writes up to
 * `cap` rows of M doubles to the host array `hist` (NULL skips) and the
 * number of rows recorded to *n.  Synchronises; EDAA_ERR_STATE when the log
 * is off. */
edaa_status edaa_loss_history(edaa_ctx* ctx, int cube, int cap, double* hist, int* n);

/* Checkpoint and resume (the paper has none).  edaa_checkpoint synchronises
 * and copies the iteration state of every run of every cube -- A and B (for
 * tensor-core cubes: the running sums S, R and Lambda that regenerate B),
 * E, the merges' sums, the step sizes, fits, coherences and the loss log --
 * and the count of outer iterations done into the host buffer `buf`
 * (capacity `cap` bytes); *bytes receives the size needed (buf = NULL only
 * queries it).  edaa_restore loads such a buffer into a context created with
 * cubes of the same shapes, runs and precision and the same loss-log
 * setting, holding the same data X (checked through its FP64 band sums);
 * anything else returns EDAA_ERR_ARG before any state changes.  Later
 * edaa_step / edaa_solve calls continue from the restored iteration and give
 * the results the checkpointed context would have given. */
edaa_status edaa_checkpoint(edaa_ctx* ctx, void* buf, size_t cap, size_t* bytes);
edaa_status edaa_restore(edaa_ctx* ctx, const void* buf, size_t bytes);

/* Step sizes in use for cube `cube` (host arrays of length M; NULL skips). */
edaa_status edaa_step_sizes(edaa_ctx* ctx, int cube, double* eta1, double* eta2);

/* Phase trace (needs config.trace = 1).  For the last launch sequence of
 * kind `which` (0: the outer iterations of the last edaa_step / edaa_solve,
 * 1: initialisation, 2: the fit and coherence phases of edaa_solve), writes up
 * to `cap` entries: phase[i] (0 A-pass, 1 A-merge, 2 B-pass, 3 B-merge,
 * 4 initial B-pass, 5 initial A-pass, 6 step sizes, 7 fit pass, 8 fit merge,
 * 9 first B-merge), start_us[i] (when the first block began it, relative to
 * the sequence's first phase) and dur_us[i] (until the last block finished
 * it), from the GPU's global timer; *n receives the number of phases
 * recorded (at most 4096 per sequence).  Host arrays; synchronises the
 * context's stream.  A persistent launch includes the grid-barrier wait in
 * each phase's time.  EDAA_ERR_STATE when tracing is off. */
edaa_status edaa_trace_read(edaa_ctx* ctx, int which, int cap, int* n, int* phase, double* start_us,
                            double* dur_us);

/* Synchronises the context's stream and reports the device status word. */
edaa_status edaa_sync(edaa_ctx* ctx);

/* Outer iterations completed since the last init/reset. */
int edaa_outer_done(const edaa_ctx* ctx);

/* Describes the launch shape picked for cube `cube` (for logs and tests):
 * runs per CTA group, pixel tile, CTAs per run group, persistent grid size,
 * the number of kernel launches the last edaa_solve enqueued, and the graph
 * state: 1 when the last edaa_solve replayed its captured CUDA graph, -1 when
 * capturing failed and solves launch their kernels directly (the capture
 * error was left in edaa_last_error by that edaa_solve, which still
 * succeeded), 0 before the first edaa_solve.  NULL outputs are skipped. */
edaa_status edaa_describe(const edaa_ctx* ctx, int cube, int* runs_per_group, int* pixel_tile,
                          int* ctas_per_group, int* grid, int* launches_per_solve, int* graph_state);

/* The CUDA-core launch shape of cube `cube` in the form of edaa_config.tile
 * ({runs per CTA group, phase-1 pixel warps, pixels per lane, phase-2 pixel
 * warps}), e.g. the one the autotuner kept, so that a later context can pin
 * it.  Tensor-core cubes report the shape of their fit pass. */
edaa_status edaa_describe_tile(const edaa_ctx* ctx, int cube, int tile[4]);

void edaa_destroy(edaa_ctx* ctx);

/* Thread-local text of the last error on this thread ("" if none). */
const char* edaa_last_error(void);

/* Failure injection for tests of the out-of-memory path (the paper has no
 * counterpart): with k >= 0 the k-th device allocation the library makes from
 * now on (0: the next one) fails with EDAA_ERR_OOM, without asking the
 * driver; k < 0 switches it off.  Process-wide.  edaa_init then releases
 * whatever it had allocated and returns EDAA_ERR_OOM. */
void edaa_debug_fail_alloc(int k);

/* Failure-detection self-test: launches the persistent kernel's grid barrier
 * on `grid` CTAs while waiting for grid + extra arrivals, with the given
 * time-out.  With extra > 0 the barrier cannot complete, so every CTA must
 * give up after timeout_ms and the call must return EDAA_ERR_TIMEOUT with the
 * device still usable (no trap, no hang).  extra = 0 must return EDAA_OK. */
edaa_status edaa_selftest_barrier(int grid, int extra, double timeout_ms, void* stream);

/* Measures the FP32 FMA throughput of the current device (TFLOP/s, best of
 * five timed launches of a register-resident loop of independent FMA chains,
 * about 0.1 s in total) on `stream`; synchronises.  It is the roofline
 * denominator of the CUDA-core passes, whose work is FP32 FMAs (Algorithm 1's
 * contractions and element-wise steps); the paper has no counterpart. */
edaa_status edaa_measure_fma_peak(double* tflops, void* stream);

/* ---- Differentiable unrolled solve (one run) ------------------------------
 * Algorithm 1 unrolled for T outer iterations with one step size per block:
 * eta_A[t] for the K1 A-steps (eq. update_A) and eta_B[t] for the K2 B-steps
 * (eq. update_B) of outer iteration t; A^0 = 1/p (eq. initA0), B^0 =
 * softmax(0.1 u) with u from SplitMix64(seed) exactly as in edaa_init (eq.
 * initB0).  X is used as given (no normalisation inside).  The forward keeps
 * one checkpoint (log A, log B) per outer iteration and the iteration's
 * grid-level reductions (E = X B, W = A A^T, and per B-step R and the column
 * normaliser: O(T K2 L p) floats); the backward recomputes each outer
 * iteration from its checkpoint and those reductions and runs hand-written
 * adjoint kernels, returning d loss / d X and d loss / d eta from
 * d loss / d E_hat and d loss / d A_hat, where E_hat = X B_hat and A_hat are
 * the outputs.  Results are deterministic (fixed-order reductions).
 * Limits: 1 <= p <= 8, p <= N, L <= 320, K1 <= 5.  All device buffers are
 * allocated by edaa_unrolled_create: about 8 N L + 8 N p T (K2 + 3) + 150 N p
 * bytes (111 MB at L=285, N=13542, p=4, T=20, K2=5); `stream` is a
 * cudaStream_t. */
typedef struct edaa_unrolled edaa_unrolled;

edaa_status edaa_unrolled_create(edaa_unrolled** out, int L, int N, int p, int T, int K1, int K2, void* stream);

/* X: N x L pixel-major float32 (host or device); eta_A, eta_B: host arrays of
 * length T; outputs E_out (L x p) and A_out (p x N), row-major, host or
 * device, NULL skips.  Synchronous with respect to the host only for host
 * outputs. */
edaa_status edaa_unrolled_forward(edaa_unrolled* u, const float* X, uint64_t seed, const double* eta_A,
                                  const double* eta_B, float* E_out, float* A_out);

/* dE: L x p, dA: p x N (host or device, NULL = zero); outputs dX (N x L,
 * host or device, NULL skips) and d_eta_A, d_eta_B (host, length T, NULL
 * skips).  Needs a preceding forward; synchronises. */
edaa_status edaa_unrolled_backward(edaa_unrolled* u, const float* dE, const float* dA, float* dX, double* d_eta_A,
                                   double* d_eta_B);

void edaa_unrolled_destroy(edaa_unrolled* u);

/* Allocation-free evaluation of the fit and loss of given solutions.  The
 * paper has no counterpart: this entry point serves callers that cannot call
 * cudaMalloc -- a process whose device memory belongs to another allocator
 * (for example a framework's caching pool that reserved the whole GPU), or a
 * latency-bound loop that must not block in the driver's allocator.  It does
 * the work of the fit pass behind edaa_solve / edaa_loss for M runs given
 * explicitly, and keeps its per-block partial sums in a fixed 384 KiB static
 * device array that is part of the library (every GPU that loads the
 * library holds it until exit); it calls no allocating routine.
 *   X: N x L pixel-major float32 (the data the solutions were computed on,
 *      already normalised the way they saw it); E: M x L x p float32 (run m's
 *      E, row-major); A: M x p x N float32.  All inputs and the outputs
 *      fit[M] = sum |X - E A|, fitmax[M] = max_i sum_l |X - E A|,
 *      loss[M] = ||X - E A||_F^2 (FP64, NULL skips) must be device memory.
 * Limits: 1 <= p <= 8 and 1 <= M <= 64 (the size of the static array);
 * larger sizes return EDAA_ERR_UNSUPPORTED with a message, nothing runs.
 * Inputs and outputs must be memory of the current device (or managed);
 * anything else returns EDAA_ERR_ARG.  Asynchronous on `stream` (a
 * cudaStream_t).  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Under CUDA's default lazy module loading
 * the library's device image -- its code and this array -- is loaded onto a
 * device by the first library call that needs it there, which is this
 * lookup when no other library call came first on that device; the load
 * takes device memory from the driver.  A caller whose allocator will
 * reserve the whole GPU makes one library call on each device before that;
 * a load that finds no memory returns EDAA_ERR_OOM.  Calls on one device
 * share the array, so calls whose GPU work overlaps race: the caller
 * serialises them (one stream, or an event between streams). */
edaa_status edaa_fit_eval_static(const float* X, int L, int N, int p, int M, const float* E, const float* A,
                                 double* fit, double* fitmax, double* loss, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* EDAA_H */
