// Internal declarations shared by the CUDA translation units of libedaa.
// Layouts (all device memory, row-major):
//   X     N x Ls float32, pixel i's L bands contiguous, CENTRED: the mean
//         pixel xbar (of the l2-normalised pixels) is subtracted.  EDAA's
//         iterates do not change under a common translation of the pixels
//         (the gradients change by a constant per softmax column, which the
//         softmax removes), and centring removes the large cancelling terms
//         of R = E (A A^T) - X A^T.  E is kept centred too; xbar is added
//         back wherever the paper's uncentred E is needed (step sizes,
//         coherence, outputs, reported gradients).  Column L holds 1.0
//         (a "ones band": contracting it with the softmax weights yields the
//         softmax denominators for free), columns L+1..Ls-1 are zero.
//         Ls = smallest multiple of 4 >= L+1 with Ls/4 odd, so 16-byte rows
//         and conflict-free 128-bit shared-memory reads across pixels.
//   logA  Mp x Nst z = log a - max_j log a per pixel and run (A = softmax_j z);
//                  row m*p+j is abundance j of run m over the pixels, rows
//                  padded to Nst = N rounded up to 32 (a warp's 32 pixels of
//                  one column are one 128-byte line)
//   logB  Mp x Nst logits u of B in the frame log(N b): B = exp(u - lse - log N)
//                  with lse stored as (log-sum-exp - log N); both stay near 0
//                  while B is near uniform, where float32 spacing is finest
//   Ef/Ed L x Mp   E = X B (float32 panel and float64 master copy)
//   Rf    L x Mp   R = E (A A^T) - X A^T, the factor of the B-gradient X^T R
//   XAt   L x Mp   X A^T (float64), AAt M x p x p (float64)
//   part  Pg x Mp x (L+1)  per-CTA partial sums of X W, one column of W after
//                  another (band L: sum of W), so that lanes holding
//                  consecutive bands write consecutive addresses
// Tensor-core cubes keep no B logits: eq. (update_B)'s gradient row of pixel
// i is x_i^T R, linear in the pixel, so after s B-steps the logits are
//     u_i = 0.1 r_i - Lambda - x_i^T S,   S = sum over the steps of eta2 R
// (r: the SplitMix64 uniforms of eq. initB0, Lambda: the per-column sum of
// the log-normalisers).  The B-pass regenerates them from r, S and Lambda:
//   Sd    L x Mp   S after the last completed B-step (float64)
//   Rd    L x Mp   R in float64 (the B-merge commits Sd += eta2 Rd of the
//                  step just taken)
//   lamd  Mp       Lambda after the last completed B-step (float64)
//   panelS Mp x kp the next B-pass's S + eta2 R, K-major, as a high and a
//                  low part in the compute type (two MMAs per product)
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace edaa {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCubes = 16;
constexpr int kMaxP = 8;
constexpr int kMaxL = 319;

// device status bits
constexpr int kStatTimeout = 1;

// kernel programs (sequences of phases)
enum Mode { MODE_OUTER = 0, MODE_INIT = 1, MODE_FIT = 2 };
constexpr int kTraceCap = 4096;  // traced phases per launch sequence
enum Phase {
  PH_A = 0,      // A-pass: K1 fused A-steps per pixel, partials of X A^T, A A^T
  PH_AM = 1,     // merge A partials; R = E AAt - XAt
  PH_B = 2,      // B-pass: one B-step, online-softmax partials of X B
  PH_BM = 3,     // merge B partials: E, lse, R
  PH_INITB = 4,  // B^0 logits from SplitMix64, partials of X B^0
  PH_INITA = 5,  // A^0 = 1/p, partials of X A^T, A A^T
  PH_ETA = 6,    // sigma_max^2(X B^0) by Jacobi, eta1, eta2
  PH_FIT = 7,    // residual pass: sum |r|, max column sum, sum r^2 per run
  PH_FITM = 8,   // merge fit partials, coherence
  PH_BM0 = 9     // merge of the B^0 partials (reference logit 0.05 instead of -log N)
};

// Shifted accumulation: the passes accumulate X (W - w_ref) instead of X W,
// with w_ref = 1/p for A and, for B, the weight of logit 0 in the frame
// log(N b) (the weight of a uniform column) in the power-of-two softmax frame;
// the merge adds w_ref * sum_i x_i back in FP64.  While A or B are close to
// uniform (the first iterations) this keeps the FP32 rounding of the partial
// sums proportional to the small deviation from uniform instead of to the
// full weights.

struct CubeDev {
  int L, Ls, Lr, N, p, M, Mp, LT;
  int Nst;                     // row length of the state arrays logA / logB (N rounded up to 32)
  double logN;                 // log N (the B logits live in the frame log(N b))
  int Rm, RG, Pg, Nt, WP1, SPT, WP2, ntiles;
  int cta0;                    // first pass work item of this cube
  int lchunk, nlchunk, unit0;  // merge work items: M * nlchunk from unit0
  int run0;                    // first run index of this cube in the batch
  float* X;
  double* xbar;    // L: mean pixel that was subtracted (zero when centring is off)
  double* sx;      // L+1: FP64 sum over pixels of the centred X as stored; sx[L] = N
  float* logA;
  float* logB;
  float* Ef;
  double* Ed;
  float* Rf;
  double* XAt;
  double* AAt;
  float* lse;
  float* eta1;
  float* eta2;
  double* eta1d;
  double* eta2d;
  double* sig2;
  float* part;
  float* pmax;
  float* paa;
  double* pfit;
  double* fit;
  double* fitmax;
  double* loss2;
  double* mu;
  double* loss_hist;  // hist_cap x M: loss after each outer iteration (with record_loss)
  double* rho;     // nlchunk x Mp: per band chunk, sum_l E[l][c] R[l][c] (FP64) for the next B-pass
  int* bref;       // Mp: reference exponent k of the B-pass just run (weights shifted by 2^k)
  double* gpart;   // nlchunk x M x p x p: per band chunk, E^T E of each run (FP64)
  const uint64_t* seeds;
  const double* gammas;
  // tensor-core path (precision TF32 or BF16): 0 = CUDA-core FP32 passes
  int tc;       // 0 off, 1 TF32, 2 BF16
  int tc_rgp;   // run-group columns padded to a multiple of 16 (MMA N)
  int tc_nkc;   // 128-byte K chunks over the bands (contraction 1)
  int tc_nbt;   // 128-band tiles (contraction 2)
  int tc_kp;    // row length (elements) of the K-major X copy and panels
  const CUtensorMap* tmaps;  // TM_COUNT maps in TcMap order
  const void* Xk;            // N x tc_kp compute-type copy of the centred X (split: then its low part)
  void* panelE;              // Mp x tc_kp, compute type (K-major E^T)
  void* panelS;              // 2 x Mp x tc_kp, compute type: high, then low part of (S + eta2 R)^T
  double* Sd;                // L x Mp: S of the last completed B-step (tensor-core cubes)
  double* Rd;                // L x Mp: R in float64 (tensor-core cubes)
  double* lamd;              // Mp: Lambda of the last completed B-step (tensor-core cubes)
  uint16_t* r16;             // Mp x Nst: the B^0 uniforms of tensor-core cubes in 16-bit fixed point
};

// The TF32 and BF16 tensor-core passes read the uniforms of eq. (initB0)
// from a table filled once per initialisation: entry (column c = m p + j,
// pixel i) is the top 16 bits q of SplitMix64 output i p + j + 1 of run m's
// seed, and the uniform is (q + 1/2) 2^-16, within 2^-17 of the 24-bit draw
// the CUDA-core passes use (the logits 0.1 u differ by at most 7.6e-7, far
// below those modes' operand rounding).  The split-operand mode, held to the
// FP32 path's accuracy, draws the 24-bit uniforms in the pass instead: near
// uniform B the B-gradient factor cancels to the deviation of B^0 from
// uniform (about 3 %), which magnifies the table's error about 30-fold.
constexpr float kR16Scale = 0.1f / 65536.f;

// Tensor maps of a tensor-core cube, in this order.
enum TcMap {
  TM_X = 0,      // X pixel-major (contraction 1's A operand)
  TM_XT = 1,     // X band-major (contraction 2's A operand)
  TM_E = 2,      // panel E (A-pass contraction 1)
  TM_S = 3,      // panel S + eta2 R, high part (B-pass contraction 1)
  TM_XLO = 4,    // split operands: low parts of X, X band-major, E
  TM_XTLO = 5,
  TM_ELO = 6,
  TM_SLO = 7,    // panel S + eta2 R, low part
  TM_STATE = 8,  // the log-abundance state (Mp x Nst float32), boxes of 128 pixels x one run group
  TM_R16 = 9,    // the B^0 uniforms (Mp x Nst uint16), same boxes
  TM_COUNT = 10
};

struct Batch {
  int n_cubes;
  int pass_items;     // total pass work items (one per (cube, run group, pixel group))
  int merge_units;    // total merge work items
  int total_runs;
  int K1, K2;
  int coh_mode;
  long long timeout_ns;
  unsigned int smem_bytes;  // dynamic shared memory of every launch of the program kernel
  int record_loss;          // 1: every outer iteration ends with the fit pass and logs its loss
  int hist_cap;             // rows of each cube's loss log
  int* status;
  unsigned int* bar;  // [0] arrivals, [1] generation
  // phase trace (null when off): [mode][phase] first-start / last-end global-timer ns
  unsigned long long* trace_start;
  unsigned long long* trace_end;
  CubeDev c[kMaxCubes];
};

// Shared-memory carve-up of a pass work item (in floats).
struct PassSmem {
  int RgS4, RgSo, RgW;
  int off_ps, off_gs, off_bar, off_xs, off_ss, off_ws, off_col, off_run, total;
};

__host__ __device__ inline PassSmem pass_smem(int L, int Ls, int Lr, int p, int Rm, int Nt) {
  PassSmem s;
  const int P4 = (p + 3) & ~3;
  s.RgS4 = Rm * P4;
  s.RgSo = (Rm * p) | 1;
  int rw = s.RgS4;
  if (((rw >> 2) & 1) == 0) rw += 4;
  s.RgW = rw;
  int o = 0;
  s.off_ps = o; o += Lr * s.RgS4;
  s.off_gs = o; o += Rm * p * P4;  // G of each run, rows padded to P4
  s.off_bar = o; o += 4;             // the X tile's mbarrier (below the end-of-pass buffer)
  s.off_xs = o; o += Nt * Ls;
  s.off_ss = o; o += (Nt * s.RgSo + 3) & ~3;
  s.off_ws = o; o += Nt * s.RgW;
  s.off_col = o; o += 7 * s.RgS4;  // B: lse, frame, tile key, reference k, 2^-Mn, frame of the tile, 2^(k-Mn)
  s.off_run = o; o += (2 * Rm + 3) & ~3;
  // end-of-pass reduction buffer ((L+1) x RgS4) reuses the region from off_xs
  const int need = s.off_xs + (L + 1) * s.RgS4 + kWarps * Rm * 36;
  if (need > o) o = need;
  s.total = o;
  return s;
}

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Shared memory of a merge work item (one run, one chunk of lchunk bands), in doubles.
struct MergeSmem {
  int saat, sw, ssx, sxa, sE, sraw, sprod, sscale, sEf, sSd, sRd, total;
};
__host__ __device__ inline MergeSmem merge_smem(int lchunk, int p, int Pg) {
  MergeSmem s;
  int o = 0;
  s.saat = o; o += 64;                // A A^T of the run
  s.sw = o; o += 2 * kMaxP;           // B: frame, then reference weight and denominator per column
  s.ssx = o; o += lchunk;             // centred band sums of the chunk
  s.sxa = o; o += lchunk * p;         // X A^T of the chunk
  s.sE = o; o += lchunk * p;          // E of the chunk
  s.sraw = o; o += (lchunk + 1) * p;  // B: scaled partial sums (last row: the ones band)
  s.sprod = o; o += lchunk * p;       // E R products
  s.sscale = o; o += Pg * p;          // B: per-CTA scale factors
  s.sEf = o; o += (lchunk * p + 1) / 2;  // B: E of the chunk (floats)
  s.sSd = o; o += lchunk * p;         // tensor-core cubes: S and R of the chunk, loaded up front
  s.sRd = o; o += lchunk * p;
  s.total = o;
  return s;
}

inline int padded_ld(int L) {
  int ls = round_up(L + 1, 4);
  if (((ls >> 2) & 1) == 0) ls += 4;
  return ls;
}

// Launch helpers implemented in edaa_kernels.cu.
// outer0: outer iterations completed before this launch sequence (the loss
// log's row of its first outer iteration)
cudaError_t launch_program(const Batch* d_batch, int mode, int outer0, int ph_lo, int ph_hi, int grid,
                           size_t smem, bool cooperative, cudaStream_t stream);
cudaError_t launch_normalize(const float* Xin, float* X, double* scale, double* bsum, double* xbar, double* sx,
                             int L, int Ls, int N, int normalize, int center, cudaStream_t s);
int normalize_blocks(int N);
cudaError_t launch_grad(const CubeDev* d_cube, const CubeDev& hc, int run, float* gA, float* gB, cudaStream_t s);
cudaError_t launch_gather(const CubeDev& hc, int run, float* E, float* A, float* B, cudaStream_t s);
cudaError_t launch_barrier_test(unsigned int* bar, int* status, int grid, int expected, long long timeout_ns,
                                cudaStream_t s);
cudaError_t set_program_smem(size_t smem);
cudaError_t program_occupancy(int* blocks_per_sm, size_t smem);
int program_phase_count(int mode, int n_outer, int K2, int record);
int program_phase_id(int mode, int s, int K2, int record);
cudaError_t launch_tc_prepare(const CubeDev& hc, void* Xk, void* XT, int Npad, cudaStream_t s);
cudaError_t launch_fill_r16(const CubeDev& hc, cudaStream_t s);
cudaError_t launch_fma_peak(float* out, int blocks, int iters, cudaStream_t s);
double fma_peak_flops_per_launch(int blocks, int iters);

}  // namespace edaa
