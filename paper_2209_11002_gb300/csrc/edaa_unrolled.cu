// Differentiable unrolled EDAA for one run: the forward pass of Algorithm 1
// with per-block step sizes (eta_A[t] for the K1 A-steps and eta_B[t] for the
// K2 B-steps of outer iteration t), a checkpoint of (log A, log B) at the
// start of every outer iteration, and hand-written adjoint kernels giving
// d(loss)/dX and d(loss)/d(eta) from d(loss)/dE_hat and d(loss)/dA_hat.
//
// State (pixel-major, N x p): z = log A (normalised per pixel), l = log B
// (normalised per column), both float-float (hi + lo).  One A-step (eq.
// update_A in softmax form):
//   z' = log_softmax_j(z - eta (G a - c)),  a = exp z, G = E^T E, c = E^T x_i
// One B-step (eq. update_B):
//   l' = log_softmax_i(l - eta g),  g_i = x_i^T R,  R = X (B W - A^T), W = A A^T
// (R is formed from the per-pixel deviations W b_i - a_i, i.e. directly as
// the paper's X^T (X - X B A) A^T factor, without the cancelling E W - X A^T).
//
// Adjoints (per step; bars are adjoints, s = column sums of l'-bar):
//   B-step:  zeta = lbar' - B' diag(s);  P = X zeta;  Dbar = -eta X^T P;
//            lbar = zeta + B o (Dbar W);  Abar += -Dbar^T + (Wbar + Wbar^T) A
//            with Wbar = B^T Dbar;  Xbar += -eta (R zeta^T + P D^T),
//            D = B W - A^T;  d eta += -<zeta, g>.
//   A-step:  zeta = zbar' - a' (1^T zbar');  d eta += -<zeta, g>;
//            Cbar += eta zeta;  Gbar += -eta zeta a^T;
//            zbar = zeta - eta a o (G zeta).
//   A-phase inputs: Ebar = E (Gbar + Gbar^T) + X Cbar^T;
//            Xbar += E Cbar + Ebar B^T;  lbar += B o (X^T Ebar).
// Every reduction over pixels is per-CTA partials in float32 followed by a
// fixed-order float-float merge: results are deterministic.
//
// Each sweep (the forward, the backward) is one cooperative launch of a
// persistent kernel: CTA g owns the contiguous pixels [N g / G, N (g+1) / G)
// and every per-pixel quantity of them, so that only reductions over pixels
// need the whole grid.  Those are the grid barriers: a contraction over
// pixels (E = X B, R = X D, P = X zeta, X Cbar) writes per-CTA partials,
// one barrier, a distributed merge (each CTA a few of the L x p entries),
// a second barrier; a small reduction (W, log-sum-exp, column sums, Gbar)
// is merged by every CTA for itself after one barrier.  That is 18 barriers
// per outer iteration forward and 18 backward: the forward keeps the
// iteration's grid-level reductions (E_t, W, every R_k and column
// normaliser; O(T K2 L p) floats), so that the backward's recompute of an
// iteration from its checkpoint needs none.  d(loss)/dX is a sum of
// rank-p terms: the backward records them and forms each CTA's rows once at
// the end.
//
// Precision: d(loss)/dX holds the residual X - E_hat A_hat, small where the
// model fits, so rounding that moves the trajectory shows up there
// amplified.  Hence the float-float logs (a float's rounding of a log was the
// largest error), and G a - c and W b - a (which cancel near a fit) formed
// from G and W exact for the float E and A and evaluated in float-float.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/edaa.h"
#include "edaa_pass.cuh"

namespace edaa {
void set_last_error(const char* msg);
}

namespace eu {

constexpr int kT = 256;      // threads per CTA
constexpr int kW = kT / 32;  // warps per CTA
constexpr int kMaxP = 8;
constexpr int kLT = 10;      // L <= 320: bands per lane in the X contractions
constexpr int kLPMax = 320 * kMaxP;
constexpr int kMaxG = 256;   // CTAs of a sweep at most
constexpr int kSmall = 80;   // per-CTA slots of a small reduction (>= p^2 + 1, >= 2p)

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Float-float accumulation (Knuth's TwoSum: s + e == hi + x exactly).  This
// GPU's FP64 rate is a small fraction of its FP32 rate; two-float sums keep
// about 44 bits at FP32 speed.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}
// butterfly over the warp in a fixed order (every lane ends with the total)
__device__ __forceinline__ double ff_warp_total(float hi, float lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, h2);
    lo += l2;
  }
  return (double)hi + (double)lo;
}

// Everything a sweep touches.  Per-pixel arrays are pixel-major N x p.
struct UArgs {
  int L, N, P, T, K1, K2, LP;  // LP = L p
  uint64_t seed;
  const float* X;              // N x L
  const double* eta;           // 2T: eta_A[t], then eta_B[t]
  float2 *z, *l;               // log A, log B as float-float (x + y): a float's rounding of a log
                               // is the sweep's largest error
  float *b, *a, *C, *g, *d, *lbar, *zbar, *Abar, *zeta, *Dbar, *bp, *tmp;
  float2 *zck, *lck;           // (T + 1) x N x p: log A, log B at the start of every outer iteration
  float2* ls;                  // backward recompute: (K2 + 1) logits (N x p)
  float* gs;                   // K2 B-gradients (N x p) of the iteration being reversed
  float* Rs;                   // T x K2 x L x p: R of every B-step (kept by the forward)
  float* Ws;                   // T x 2p^2: W = A A^T of every outer iteration (high, low parts)
  float2* lses;                // T x K2 x p: the column normalisers of every B-step
  float* Xbar;                 // N x L
  float* U;                    // N x RK: per-pixel coefficients of the rank-p terms of Xbar
  float* V;                    // RK x Lv: their panel columns (Lv >= L, zero padded)
  int RK, Lv;
  const float *dE, *dA;        // backward inputs: L x p, p x N
  float *Eout, *Aout;          // forward outputs: E_hat (L x p), A_hat (p x N)
  float* part;                 // G x LP per-CTA partials of an X contraction
  float* part2;                // G x kSmall per-CTA partials of a small reduction
  double* part2d;              // G x kSmall per-CTA FP64 partials (W = A A^T)
  float* peta;                 // G x 2T per-CTA partials of d eta
  float *E32, *P32;            // merged L x p (float)
  float* Es;                   // T x L x p: E_t = X B_t of every outer iteration (float) ...
  double* Eds;                 // ... and FP64, kept by the forward for the reverse sweep
  double *Ed, *XCd;            // merged L x p (FP64)
  double* deta;                // 2T
  unsigned* bar;               // arrivals at the grid barriers of this launch (zeroed before it)
  int* status;
  long long timeout_ns;
  int maxpx;                   // the most pixels a CTA owns
  int res_state, res_x;        // the per-pixel arrays / the CTA's X rows live in shared memory
  int Ls;                      // row stride of X as the sweeps read it (L, or padded in shared memory)
  int Qx;                      // quad stride of xw_part's chunk sums in shared memory (>= ceil(L/4))
};
constexpr int kPixD = 2;   // per-pixel float-float arrays: z, l
constexpr int kPixF = 12;  // per-pixel float arrays: b, a, C, g, d, lbar, zbar, Abar, zeta, Dbar, bp, tmp

// Float-float logs v = v.x + v.y (|v.y| <= ulp(v.x)).
// exp to float accuracy: expf of the high part times 1 + the low part (the
// first-order term of exp of the low part)
__device__ __forceinline__ float ff_exp(float2 v) {
  const float e = expf(v.x);
  return fmaf(e, v.y, e);
}
// h + l -= x (Knuth's TwoSum of h and -x, then renormalised)
__device__ __forceinline__ void ff_sub(float& h, float& l, float x) {
  const float s = h - x;
  const float bp = s - h;
  const float e = (h - (s - bp)) - (x + bp);
  l += e;
  h = s + l;
  l -= h - s;
}
// v - w for float-float w
__device__ __forceinline__ float2 ff_minus(float2 v, float2 w) {
  ff_sub(v.x, v.y, w.x);
  ff_sub(v.x, v.y, w.y);
  return v;
}
// a double as float-float
__device__ __forceinline__ float2 ff_split(double d) {
  const float h = (float)d;
  return make_float2(h, (float)(d - (double)h));
}

// shared memory of a CTA
struct Sm {
  alignas(16) float p0[kLPMax];  // L x p panels
  alignas(16) float p1[kLPMax];
  float xs[4 * kMaxP * kT];      // the pixel-chunk sums of an X contraction
  float red[kW * kSmall];                     // per-warp partials of a small reduction
  float W[64], G[64], Wb[64], Wacc[64], tmp[kSmall];
  double Gb[64], lse[kMaxP], sd[kMaxP];
  float2 lse2[kMaxP], sd2[kMaxP];  // lse and sd as float-float
  float Gl[64], Wl[64];          // low parts: G + Gl = E^T E, W + Wl = A A^T, exact for the float E, A
};

__device__ __forceinline__ void prange(int N, int& lo, int& hi) {
  lo = (int)((long long)N * blockIdx.x / gridDim.x);
  hi = (int)((long long)N * (blockIdx.x + 1) / gridDim.x);
}
// Grid barrier on a monotonic arrival counter: the k-th barrier of a launch
// completes when the counter reaches k G.  Thread 0 of each CTA arrives
// (release) and polls (acquire); a wait beyond timeout_ns, or another CTA's
// time-out, sets the status bit and returns false.  `nb` counts this CTA's
// barriers.
__device__ __forceinline__ bool gbar_wait(const UArgs& a, unsigned& nb) {
  __shared__ int s_ok;
  __syncthreads();
  ++nb;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = nb * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.bar) : "memory");
    const unsigned long long t0 = edaa::global_ns();
    for (unsigned spin = 0;; ++spin) {
      if ((int)(edaa::ld_acquire_u32(a.bar) - target) >= 0) break;
      if ((spin & 255u) == 255u) {
        if (edaa::ld_volatile_i32(a.status) & edaa::kStatTimeout) { ok = 0; break; }
        if ((long long)(edaa::global_ns() - t0) > a.timeout_ns) {
          atomicOr(a.status, edaa::kStatTimeout);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}
#define gbar(a) gbar_wait(a, nbar)

// Dot product of n terms x[k sx] y[k sy] in blocks of 64: four interleaved
// FMA chains of 16 terms, each block's sum added into a float-float total
// (the error stays that of a 16-term chain however long the dot product).
__device__ __forceinline__ float dot_blocked(const float* x, size_t sx, const float* y, size_t sy, int n) {
  float hi = 0.f, lo = 0.f;
  for (int k0 = 0; k0 < n; k0 += 64) {
    const int k1 = min(n, k0 + 64);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int k = k0;
#pragma unroll 4
    for (; k + 3 < k1; k += 4) {
      s0 = fmaf(x[k * sx], y[k * sy], s0);
      s1 = fmaf(x[(k + 1) * sx], y[(k + 1) * sy], s1);
      s2 = fmaf(x[(k + 2) * sx], y[(k + 2) * sy], s2);
      s3 = fmaf(x[(k + 3) * sx], y[(k + 3) * sy], s3);
    }
    for (; k < k1; ++k) s0 = fmaf(x[k * sx], y[k * sy], s0);
    ff_add(hi, lo, (s0 + s1) + (s2 + s3));
  }
  return hi + lo;
}

// row j of an L x p panel in shared memory (16-byte aligned) into registers
template <int P>
__device__ __forceinline__ void ld_row(const float* r, float (&v)[P]) {
  if constexpr (P % 4 == 0) {
#pragma unroll
    for (int j = 0; j < P; j += 4) {
      const float4 t = *reinterpret_cast<const float4*>(r + j);
      v[j] = t.x; v[j + 1] = t.y; v[j + 2] = t.z; v[j + 3] = t.w;
    }
  } else if constexpr (P % 2 == 0) {
#pragma unroll
    for (int j = 0; j < P; j += 2) {
      const float2 t = *reinterpret_cast<const float2*>(r + j);
      v[j] = t.x; v[j + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < P; ++j) v[j] = r[j];
  }
}

// ---- a.part[g] = sum over this CTA's pixels of x_i w_i^T (L x p).
// X rows in shared memory (row stride Ls: a multiple of 4, zero padded): a
// thread per (4 bands, pixel chunk); per pixel one 16-byte load of x and p
// broadcast loads of w feed 4p FMAs; chains of 16 pixels go into float-float
// sums; the C chunk sums of an entry are then added in chunk order.
// X in global memory: a thread per entry (l, j), pixels in order.
template <int P>
__device__ void xw_part(const UArgs& a, const float* __restrict__ w, Sm& S) {
  const int L = a.L, LP = a.LP, tid = threadIdx.x;
  int lo, hi;
  prange(a.N, lo, hi);
  float* dst = a.part + (size_t)blockIdx.x * LP;
  if (!a.res_x) {
    for (int e = tid; e < LP; e += kT) {
      const int l = e / P, j = e - l * P;
      const float* xp = a.X + (size_t)lo * L + l;
      const float* wp = w + (size_t)lo * P + j;
      dst[e] = dot_blocked(xp, (size_t)L, wp, (size_t)P, hi - lo);
    }
    return;
  }
  const int Ls = a.Ls, Q = (L + 3) >> 2, C = min(8, max(1, kT / Q)), npx = hi - lo, Qs = a.Qx;
  if (tid < Q * C) {
    const int c = tid / Q, q = tid - c * Q;
    const int k0 = lo + npx * c / C, k1 = lo + npx * (c + 1) / C;
    float sh[4][P], sl[4][P], s[4][P];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < P; ++j) sh[r][j] = sl[r][j] = s[r][j] = 0.f;
    const float* xp = a.X + (size_t)k0 * Ls + 4 * q;
    const float* wp = w + (size_t)k0 * P;
    for (int kb = k0; kb < k1; kb += 16) {
      const int ke = min(k1, kb + 16);
#pragma unroll 4
      for (int k = kb; k < ke; ++k) {
        const float4 x4 = *reinterpret_cast<const float4*>(xp);
        float wv[P];
#pragma unroll
        for (int j = 0; j < P; ++j) wv[j] = wp[j];
#pragma unroll
        for (int j = 0; j < P; ++j) {
          s[0][j] = fmaf(x4.x, wv[j], s[0][j]);
          s[1][j] = fmaf(x4.y, wv[j], s[1][j]);
          s[2][j] = fmaf(x4.z, wv[j], s[2][j]);
          s[3][j] = fmaf(x4.w, wv[j], s[3][j]);
        }
        xp += Ls;
        wp += P;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < P; ++j) {
          ff_add(sh[r][j], sl[r][j], s[r][j]);
          s[r][j] = 0.f;
        }
    }
    float* xs = S.xs + (size_t)c * 4 * P * Qs;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < P; ++j) xs[(r * P + j) * Qs + q] = sh[r][j] + sl[r][j];
  }
  __syncthreads();
  for (int e = tid; e < LP; e += kT) {
    const int l = e / P, j = e - l * P, q = l >> 2, r = l & 3;
    float h = 0.f, lw = 0.f;
    for (int c = 0; c < C; ++c) ff_add(h, lw, S.xs[((size_t)c * 4 * P + r * P + j) * Qs + q]);
    dst[e] = h + lw;
  }
}

// ---- after a barrier: entry e of the merged L x p contraction (sum of the
// CTAs' partials in a fixed order, float-float), a few entries per CTA
__device__ void merge_dist(const UArgs& a, double* outd, float* outf, float* outf2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
  for (int e = blockIdx.x * kW + warp; e < a.LP; e += G * kW) {
    float hi = 0.f, lo = 0.f;
    for (int b = lane; b < G; b += 32) ff_add(hi, lo, a.part[(size_t)b * a.LP + e]);
    const double s = ff_warp_total(hi, lo);
    if (lane == 0) {
      if (outd) outd[e] = s;
      if (outf) outf[e] = (float)s;
      if (outf2) outf2[e] = (float)s;
    }
  }
}

// ---- after a barrier: every CTA merges the CTAs' n small partials for itself
__device__ void merge_small(const UArgs& a, int n, float* outf, double* outd) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
  for (int e = warp; e < n; e += kW) {
    float hi = 0.f, lo = 0.f;
    for (int b = lane; b < G; b += 32) ff_add(hi, lo, a.part2[(size_t)b * kSmall + e]);
    const double s = ff_warp_total(hi, lo);
    if (lane == 0) {
      if (outf) outf[e] = (float)s;
      if (outd) outd[e] = s;
    }
  }
  __syncthreads();
}

// ---- W = A A^T: this CTA's share, exact for the float A to about 2^-44
// (each product split into its rounded value and fma remainder, float-float
// sums; a warp per entry, lanes over the pixels, a fixed butterfly) into
// a.part2d[g]; after a barrier every CTA sums the CTAs' partials in order into
// outf + out_lo (float-float)
template <int P>
__device__ void aat_part(const UArgs& a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lo, hi;
  prange(a.N, lo, hi);
  for (int e = warp; e < P * P; e += kW) {
    const int j = e / P, k = e - j * P;
    float sh = 0.f, sl = 0.f;
    for (int i = lo + lane; i < hi; i += 32) {
      const float x = a.a[(size_t)i * P + j], y = a.a[(size_t)i * P + k];
      const float pr = __fmul_rn(x, y);
      ff_add(sh, sl, pr);
      sl += fmaf(x, y, -pr);
    }
    const double s = ff_warp_total(sh, sl);
    if (lane == 0) a.part2d[(size_t)blockIdx.x * kSmall + e] = s;
  }
}
__device__ void merge_small_d(const UArgs& a, int n, float* out_lo, float* outf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
  for (int e = warp; e < n; e += kW) {
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += a.part2d[(size_t)b * kSmall + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      outf[e] = (float)s;
      out_lo[e] = (float)(s - (double)outf[e]);
    }
  }
  __syncthreads();
}

// ---- NV per-thread values summed over the CTA (warps in a fixed order) into
// a.part2[g][0..NV)
template <int NV>
__device__ void block_part(const UArgs& a, const float (&v)[NV], Sm& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < NV; ++e) {
    const float s = wsum(v[e]);
    if (lane == 0) S.red[warp * kSmall + e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NV; e += kT) {
    float s = 0.f;
    for (int w = 0; w < kW; ++w) s += S.red[w * kSmall + e];
    a.part2[(size_t)blockIdx.x * kSmall + e] = s;
  }
  __syncthreads();
}
// the same into S.tmp (this CTA's total only)
template <int NV>
__device__ void block_total(const float (&v)[NV], Sm& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < NV; ++e) {
    const float s = wsum(v[e]);
    if (lane == 0) S.red[warp * kSmall + e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NV; e += kT) {
    float s = 0.f;
    for (int w = 0; w < kW; ++w) s += S.red[w * kSmall + e];
    S.tmp[e] = s;
  }
  __syncthreads();
}

// ---- out_i = scale x_i^T panel (panel: L x p in shared memory, 16-byte aligned).
// X rows in shared memory: a warp takes 16 pixels; lane (h, q) takes pixels
// q and q + 8 over quarter h of the bands.  Per 4 bands two 16-byte loads of
// x and four panel rows feed 8p FMAs; chains of 16 bands go into float-float
// sums, and the quarters meet by shuffles.  X in global memory: a thread per
// (pixel, j), bands in order.
template <int P>
__device__ void xdot(const UArgs& a, const float* panel, float scale, float* __restrict__ out) {
  const int L = a.L;
  int lo, hi;
  prange(a.N, lo, hi);
  if (!a.res_x) {
    for (int e = threadIdx.x; e < (hi - lo) * P; e += kT) {
      const int il = e / P, j = e - il * P;
      const float* xp = a.X + (size_t)(lo + il) * L;
      out[(size_t)lo * P + e] = scale * dot_blocked(xp, 1, panel + j, (size_t)P, L);
    }
    __syncthreads();
    return;
  }
  const int Ls = a.Ls, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, h = lane >> 3, pp = lane & 7;
  const int Qf = L >> 2;
  const int qa = Qf * h / 4, qz = Qf * (h + 1) / 4;
  for (int ib = lo + warp * 16; ib < hi; ib += kW * 16) {
    const int i0 = ib + pp, i1 = ib + 8 + pp;
    const bool live0 = i0 < hi, live1 = i1 < hi;
    const float* x0 = a.X + (size_t)(live0 ? i0 : ib) * Ls;
    const float* x1 = a.X + (size_t)(live1 ? i1 : ib) * Ls;
    float sh0[P], sl0[P], s0[P], sh1[P], sl1[P], s1[P];
#pragma unroll
    for (int j = 0; j < P; ++j) sh0[j] = sl0[j] = s0[j] = sh1[j] = sl1[j] = s1[j] = 0.f;
    for (int q0 = qa; q0 < qz; q0 += 4) {
      const int qe = min(qz, q0 + 4);
      for (int q = q0; q < qe; ++q) {
        const float4 a4 = *reinterpret_cast<const float4*>(x0 + 4 * q);
        const float4 b4 = *reinterpret_cast<const float4*>(x1 + 4 * q);
        const float* pr = panel + (size_t)q * 4 * P;
        float v0[P], v1[P], v2[P], v3[P];
        ld_row<P>(pr, v0);
        ld_row<P>(pr + P, v1);
        ld_row<P>(pr + 2 * P, v2);
        ld_row<P>(pr + 3 * P, v3);
#pragma unroll
        for (int j = 0; j < P; ++j) {
          s0[j] = fmaf(a4.x, v0[j], s0[j]);
          s1[j] = fmaf(b4.x, v0[j], s1[j]);
          s0[j] = fmaf(a4.y, v1[j], s0[j]);
          s1[j] = fmaf(b4.y, v1[j], s1[j]);
          s0[j] = fmaf(a4.z, v2[j], s0[j]);
          s1[j] = fmaf(b4.z, v2[j], s1[j]);
          s0[j] = fmaf(a4.w, v3[j], s0[j]);
          s1[j] = fmaf(b4.w, v3[j], s1[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < P; ++j) {
        ff_add(sh0[j], sl0[j], s0[j]);
        ff_add(sh1[j], sl1[j], s1[j]);
        s0[j] = s1[j] = 0.f;
      }
    }
    if (h == 3) {
      for (int l = 4 * Qf; l < L; ++l)
#pragma unroll
        for (int j = 0; j < P; ++j) {
          s0[j] = fmaf(x0[l], panel[l * P + j], s0[j]);
          s1[j] = fmaf(x1[l], panel[l * P + j], s1[j]);
        }
#pragma unroll
      for (int j = 0; j < P; ++j) {
        ff_add(sh0[j], sl0[j], s0[j]);
        ff_add(sh1[j], sl1[j], s1[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
      float H0 = sh0[j], L0 = sl0[j], H1 = sh1[j], L1 = sl1[j];
#pragma unroll
      for (int o = 8; o <= 16; o <<= 1) {
        const float a_ = __shfl_xor_sync(0xffffffffu, H0, o), b_ = __shfl_xor_sync(0xffffffffu, L0, o);
        const float c_ = __shfl_xor_sync(0xffffffffu, H1, o), d_ = __shfl_xor_sync(0xffffffffu, L1, o);
        ff_add(H0, L0, a_);
        L0 += b_;
        ff_add(H1, L1, c_);
        L1 += d_;
      }
      if (h == 0) {
        if (live0) out[(size_t)i0 * P + j] = scale * (H0 + L0);
        if (live1) out[(size_t)i1 * P + j] = scale * (H1 + L1);
      }
    }
  }
  __syncthreads();
}

// ---- Xbar = sum of rank-p terms s L R^T (L: an L x p panel in shared memory;
// R: per-pixel coefficients).  A term is recorded: s R into this CTA's rows of
// U (columns ru..ru+p), the panel's columns into rows ru.. of V (shared out
// among the CTAs: the panels are the same in every CTA).  dx_contract forms
// the sum once, after the last grid barrier.
template <int P>
__device__ void rank_record(const UArgs& a, int& ru, const float* L1, const float* R1, float s1, const float* L2,
                            const float* R2, float s2) {
  int lo, hi;
  prange(a.N, lo, hi);
  const int nt = L2 ? 2 : 1;
  for (int e = lo * P + (int)threadIdx.x; e < hi * P; e += kT) {
    const int i = e / P, j = e - i * P;
    float* u = a.U + (size_t)i * a.RK + ru;
    u[j] = s1 * R1[e];
    if (L2) u[P + j] = s2 * R2[e];
  }
  // the panels' columns: spread over the CTAs (each holds the same panels),
  // bands fastest so that consecutive threads write consecutive floats of V
  for (int e = blockIdx.x * kT + threadIdx.x; e < nt * a.LP; e += gridDim.x * kT) {
    const int r = e / a.L, l = e - r * a.L, t = r / P, j = r - t * P;
    a.V[(size_t)(ru + r) * a.Lv + l] = (t ? L2 : L1)[l * P + j];
  }
  ru += nt * P;
  __syncthreads();
}

// ---- Xbar_i = U_i V over this CTA's pixels (the nr recorded terms, FP32 FMAs
// in the order they were recorded).  Blocks of kDxBlk pixels; a thread per
// tile of kDxPx pixels x kDxB bands; kKC terms at a time staged in shared
// memory, the next kKC terms' loads in flight meanwhile.
constexpr int kDxPx = 8, kDxB = 14, kDxBlk = 96, kKC = 8, kLvMax = 322;
constexpr int kUL = (kKC * kDxBlk + kT - 1) / kT, kVL = (kKC * kLvMax + kT - 1) / kT;
__device__ __forceinline__ void dx_contract(const UArgs& a, int nr, Sm& S) {
  int lo, hi;
  prange(a.N, lo, hi);
  const int Lv = a.Lv, tid = threadIdx.x, nbg = Lv / kDxB;
  float* Us = S.xs;                 // [kKC][kDxBlk]
  float* Vs = S.xs + kKC * kDxBlk;  // [kKC][Lv]
  const int nc = (nr + kKC - 1) / kKC;
  for (int p0 = lo; p0 < hi; p0 += kDxBlk) {
    const int np = min(kDxBlk, hi - p0);
    const int ntile = ((np + kDxPx - 1) / kDxPx) * nbg;
    for (int tb = 0; tb < ntile; tb += kT) {
      const int tau = tb + tid;
      const bool mine = tau < ntile;
      const int pg = mine ? tau / nbg : 0, bg = mine ? tau - pg * nbg : 0;
      float acc[kDxPx][kDxB];
#pragma unroll
      for (int q = 0; q < kDxPx; ++q)
#pragma unroll
        for (int b = 0; b < kDxB; ++b) acc[q][b] = 0.f;
      float ur[kUL], vr[kVL];
      auto fetch = [&](int c) {
        const int r0 = c * kKC;
#pragma unroll
        for (int u = 0; u < kUL; ++u) {
          const int e = tid + u * kT, px = e / kKC, r = e - px * kKC;
          ur[u] = (px < np && r0 + r < nr) ? a.U[(size_t)(p0 + px) * a.RK + r0 + r] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kVL; ++u) {
          const int e = tid + u * kT, r = e / Lv, l = e - r * Lv;
          vr[u] = (r < kKC && r0 + r < nr) ? a.V[(size_t)(r0 + r) * Lv + l] : 0.f;
        }
      };
      fetch(0);
      for (int c = 0; c < nc; ++c) {
#pragma unroll
        for (int u = 0; u < kUL; ++u) {
          const int e = tid + u * kT, px = e / kKC, r = e - px * kKC;
          if (px < kDxBlk) Us[r * kDxBlk + px] = ur[u];
        }
#pragma unroll
        for (int u = 0; u < kVL; ++u) {
          const int e = tid + u * kT, r = e / Lv, l = e - r * Lv;
          if (r < kKC) Vs[r * Lv + l] = vr[u];
        }
        __syncthreads();
        if (c + 1 < nc) fetch(c + 1);
        if (mine) {
#pragma unroll
          for (int r = 0; r < kKC; ++r) {
            const float4 u0 = *reinterpret_cast<const float4*>(Us + r * kDxBlk + pg * kDxPx);
            const float4 u1 = *reinterpret_cast<const float4*>(Us + r * kDxBlk + pg * kDxPx + 4);
            const float uv[kDxPx] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
            float vv[kDxB];
#pragma unroll
            for (int m = 0; m < kDxB / 2; ++m) {
              const float2 t2 = *reinterpret_cast<const float2*>(Vs + r * Lv + bg * kDxB + 2 * m);
              vv[2 * m] = t2.x;
              vv[2 * m + 1] = t2.y;
            }
#pragma unroll
            for (int q = 0; q < kDxPx; ++q)
#pragma unroll
              for (int b = 0; b < kDxB; ++b) acc[q][b] = fmaf(uv[q], vv[b], acc[q][b]);
          }
        }
        __syncthreads();
      }
      if (mine)
#pragma unroll
        for (int q = 0; q < kDxPx; ++q) {
          const int i = pg * kDxPx + q;
          if (i < np)
#pragma unroll
            for (int b = 0; b < kDxB; ++b) {
              const int l = bg * kDxB + b;
              if (l < a.L) a.Xbar[(size_t)(p0 + i) * a.L + l] = acc[q][b];
            }
        }
    }
  }
}

// ---- G = E^T E from E in shared memory: warp per entry, lanes over the bands
// (each product split exactly into its rounded value and error, both summed,
// so that G + Gl is E^T E of the float E to about 2^-44)
__device__ void gram(const UArgs& a, const float* E, float* G, float* Gl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, P = a.P, L = a.L;
  for (int e = warp; e < P * P; e += kW) {
    const int j = e / P, k = e % P;
    float hi = 0.f, lo = 0.f;
    for (int l = lane; l < L; l += 32) {
      const float x = E[l * P + j], y = E[l * P + k];
      const float pr = __fmul_rn(x, y);
      ff_add(hi, lo, pr);
      lo += fmaf(x, y, -pr);
    }
    const double s = ff_warp_total(hi, lo);
    if (lane == 0) {
      G[e] = (float)s;
      Gl[e] = (float)(s - (double)G[e]);
    }
  }
  __syncthreads();
}

// ---- per-column log-sum-exp of the logits v over all pixels: this CTA's
// (max m, sum of exp(v - m)) pairs into part2 (two passes: the column maxima
// over the CTA, then the sums), then (after a barrier) every CTA merges
template <int P>
__device__ void lse_part(const UArgs& a, const float2* __restrict__ v, Sm& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lo, hi;
  prange(a.N, lo, hi);
  float m[P], s[P];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    m[j] = -INFINITY;
    s[j] = 0.f;
  }
  for (int i = lo + (int)threadIdx.x; i < hi; i += kT)
#pragma unroll
    for (int j = 0; j < P; ++j) m[j] = fmaxf(m[j], v[(size_t)i * P + j].x);
#pragma unroll
  for (int j = 0; j < P; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m[j] = fmaxf(m[j], __shfl_xor_sync(0xffffffffu, m[j], o));
    if (lane == 0) S.red[warp * kSmall + j] = m[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < P; ++j) {
    float mm = S.red[j];
    for (int w = 1; w < kW; ++w) mm = fmaxf(mm, S.red[w * kSmall + j]);
    m[j] = mm;  // the CTA's column maximum (-inf for a CTA without pixels: the merge skips it)
  }
  for (int i = lo + (int)threadIdx.x; i < hi; i += kT)
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const float2 x = v[(size_t)i * P + j];
      s[j] += expf((x.x - m[j]) + x.y);
    }
#pragma unroll
  for (int j = 0; j < P; ++j) {
    s[j] = wsum(s[j]);
    if (lane == 0) S.red[warp * kSmall + P + j] = s[j];
  }
  __syncthreads();
  if (threadIdx.x < P) {
    const int j = threadIdx.x;
    float ss = 0.f;
    for (int w = 0; w < kW; ++w) ss += S.red[w * kSmall + P + j];
    a.part2[(size_t)blockIdx.x * kSmall + 2 * j] = m[j];
    a.part2[(size_t)blockIdx.x * kSmall + 2 * j + 1] = ss;
  }
  __syncthreads();
}
// every CTA: lse_j = M + log sum_g s_g exp(m_g - M), M the largest m_g (the
// CTAs' pairs loaded once, a warp per column)
__device__ void lse_merge(const UArgs& a, double* lse, float2* lse2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
  constexpr int kB = kMaxG / 32;
  if (warp < a.P) {
    const int j = warp;
    float mb[kB], sb[kB], m = -INFINITY;
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int b = lane + 32 * u;
      mb[u] = b < G ? a.part2[(size_t)b * kSmall + 2 * j] : -INFINITY;
      sb[u] = b < G ? a.part2[(size_t)b * kSmall + 2 * j + 1] : 0.f;
      m = fmaxf(m, mb[u]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int u = 0; u < kB; ++u)
      if (mb[u] != -INFINITY) ff_add(hi, lo, sb[u] * expf(mb[u] - m));
    const double sum = ff_warp_total(hi, lo);
    // log sum = k ln 2 + log f, sum = f 2^k, f in [1/2, 1): logf of f's float
    // part plus the first-order term of its remainder (about 2^-24 absolute;
    // FP64's log is a long chain of FP64 operations)
    if (lane == 0) {
      int k2;
      const double f = frexp(sum, &k2);
      const float fh = (float)f;
      lse[j] = (double)m + (double)k2 * 0.6931471805599453 + (double)logf(fh) + (double)((float)(f - (double)fh) / fh);
      lse2[j] = ff_split(lse[j]);
    }
  }
  __syncthreads();
}

// one pixel's A-phase: K1 mirror steps; keeps the iterates when `zs` is given
// z = zh + zl (float-float) through the steps and in memory; the
// normaliser lz is a float: its rounding is common to the pixel's p entries,
// which the next normalisation takes out again
// sum_q (h_q + l_q) v_q - c for float-float weights (h, l) and float v, c:
// every product split exactly (its rounded value and the fma remainder), the
// sum carried as float-float; good to about 2^-44 of the largest term
template <int P>
__device__ __forceinline__ float ff_dot_sub(const float* h, const float* l, const float* v, float c) {
  float s = -c, e = 0.f;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const float pr = __fmul_rn(h[q], v[q]);
    const float pe = fmaf(h[q], v[q], -pr);
    const float t = s + pr;
    const float bp = t - s;
    e += ((s - (t - bp)) + (pr - bp)) + fmaf(l[q], v[q], pe);
    s = t;
  }
  return s + e;
}

// The gradient g = G a - c cancels near a fit: it is evaluated from G + Gl =
// E^T E, exact for the float E, and the float a and c (ff_dot_sub).
template <int P>
__device__ __forceinline__ void a_steps(float2* z, const float* c, const float* G, const float* Gl, double eta,
                                        int K1, float (*zs)[kMaxP]) {
  float zh[P], zl[P];
#pragma unroll
  for (int j = 0; j < P; ++j) {
    zh[j] = z[j].x;
    zl[j] = z[j].y;
  }
  const float et = (float)eta;
  for (int k = 0; k < K1; ++k) {
    if (zs)
#pragma unroll
      for (int j = 0; j < P; ++j) zs[k][j] = zh[j];
    float av[P], mx = -INFINITY;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const float e = expf(zh[j]);
      av[j] = fmaf(e, zl[j], e);
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const float g = ff_dot_sub<P>(G + j * P, Gl + j * P, av, c[j]);
      ff_sub(zh[j], zl[j], __fmul_rn(et, g));  // (a rounded product: not contracted into the sum)
      mx = fmaxf(mx, zh[j]);
    }
    float se = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) se += expf((zh[j] - mx) + zl[j]);
    const float lz = mx + logf(se);
#pragma unroll
    for (int j = 0; j < P; ++j) ff_sub(zh[j], zl[j], lz);
  }
  if (zs)
#pragma unroll
    for (int j = 0; j < P; ++j) zs[K1][j] = zh[j];
#pragma unroll
  for (int j = 0; j < P; ++j) z[j] = make_float2(zh[j], zl[j]);
}

// l <- l - lse (per column), b = exp(l); optionally a copy of l
template <int P>
__device__ void shift_exp(const UArgs& a, const float2* lse, float2* copy) {
  int lo, hi;
  prange(a.N, lo, hi);
  for (int e = lo * P + (int)threadIdx.x; e < hi * P; e += kT) {
    const float2 v = ff_minus(a.l[e], lse[e % P]);
    a.l[e] = v;
    a.b[e] = ff_exp(v);
    if (copy) copy[e] = v;
  }
  __syncthreads();
}
// dst = src (logs) over this CTA's pixels (p values each); b = exp(src) when b is given
template <int P>
__device__ void copy_px(const UArgs& a, const float2* __restrict__ src, float2* __restrict__ dst, float* __restrict__ eb) {
  int lo, hi;
  prange(a.N, lo, hi);
  for (int e = lo * P + (int)threadIdx.x; e < hi * P; e += kT) {
    const float2 v = src[e];
    if (dst) dst[e] = v;
    if (eb) eb[e] = ff_exp(v);
  }
  __syncthreads();
}

// ---- one outer iteration forward from (z, l normalised, b = exp l): the
// A-phase, then K2 B-steps.  The forward (rec false) forms the grid-level
// reductions of the iteration and keeps them: E_t (Es, Eds), W (Ws), every
// R_k (Rs) and every column normaliser (lses).  The reverse sweep's
// recompute (rec true) reads them back, so it needs no grid barrier and
// reproduces the forward's per-pixel values bit for bit; it keeps the
// logits ls[k] and B-gradients gs[k] for the reverse B-steps.  Ends with
// z = z_{t+1}, a = exp z, W in S.W + S.Wl.
template <int P>
__device__ bool fwd_outer(const UArgs& a, Sm& S, int t, bool rec, unsigned& nbar) {
  const int tid = threadIdx.x, LP = a.LP;
  int lo, hi;
  prange(a.N, lo, hi);
  // E = X B (FP64 and float; kept by the forward, read back by the
  // recompute), G = E^T E
  float* Et = a.Es + (size_t)t * LP;
  if (!rec) {
    xw_part<P>(a, a.b, S);
    if (!gbar(a)) return false;
    merge_dist(a, a.Eds + (size_t)t * LP, Et, nullptr);
    if (!gbar(a)) return false;
  }
  for (int e = tid; e < LP; e += kT) S.p0[e] = Et[e];
  __syncthreads();
  gram(a, S.p0, S.G, S.Gl);
  // c = E^T x_i, the K1 A-steps, a = exp z, and this CTA's share of W = A A^T
  xdot<P>(a, S.p0, 1.f, a.C);
  const double etaA = a.eta[t];
  for (int i = lo + tid; i < hi; i += kT) {
    float2 z[kMaxP];
    float c[kMaxP];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      z[j] = a.z[(size_t)i * P + j];
      c[j] = a.C[(size_t)i * P + j];
    }
    a_steps<P>(z, c, S.G, S.Gl, etaA, a.K1, nullptr);
#pragma unroll
    for (int j = 0; j < P; ++j) {
      a.z[(size_t)i * P + j] = z[j];
      a.a[(size_t)i * P + j] = ff_exp(z[j]);
    }
  }
  __syncthreads();
  float* Wt = a.Ws + (size_t)t * 2 * P * P;
  if (!rec) {
    aat_part<P>(a);
    if (!gbar(a)) return false;
    merge_small_d(a, P * P, S.Wl, S.W);
    if (blockIdx.x == 0)
      for (int e = tid; e < P * P; e += kT) {
        Wt[e] = S.W[e];
        Wt[P * P + e] = S.Wl[e];
      }
  } else {
    copy_px<P>(a, a.l, a.ls, nullptr);
    for (int e = tid; e < P * P; e += kT) {
      S.W[e] = Wt[e];
      S.Wl[e] = Wt[P * P + e];
    }
    __syncthreads();
  }
  const float etaB = (float)a.eta[a.T + t];
  for (int k = 0; k < a.K2; ++k) {
    float* Rk = a.Rs + ((size_t)t * a.K2 + k) * LP;
    float2* lk = a.lses + ((size_t)t * a.K2 + k) * P;
    if (!rec) {
      // d_i = W b_i - a_i (cancels near a fit: from the exact W + Wl by
      // ff_dot_sub); R = X D, kept
      for (int i = lo + tid; i < hi; i += kT) {
        float bv[P];
#pragma unroll
        for (int q = 0; q < P; ++q) bv[q] = a.b[(size_t)i * P + q];
#pragma unroll
        for (int j = 0; j < P; ++j)
          a.d[(size_t)i * P + j] = ff_dot_sub<P>(S.W + j * P, S.Wl + j * P, bv, a.a[(size_t)i * P + j]);
      }
      __syncthreads();
      xw_part<P>(a, a.d, S);
      if (!gbar(a)) return false;
      merge_dist(a, nullptr, Rk, nullptr);
      if (!gbar(a)) return false;
    }
    for (int e = tid; e < LP; e += kT) S.p0[e] = Rk[e];
    __syncthreads();
    // g_i = x_i^T R; l' = l - eta g, normalised per column
    xdot<P>(a, S.p0, 1.f, a.g);
    for (int e = lo * P + tid; e < hi * P; e += kT) {
      const float gv = a.g[e];
      float2 v = a.l[e];
      ff_sub(v.x, v.y, __fmul_rn(etaB, gv));  // (a rounded product: not contracted into the sum)
      a.l[e] = v;
      if (rec) a.gs[(size_t)k * a.N * P + e] = gv;
    }
    __syncthreads();
    if (!rec) {
      lse_part<P>(a, a.l, S);
      if (!gbar(a)) return false;
      lse_merge(a, S.lse, S.lse2);
      if (blockIdx.x == 0 && tid < P) lk[tid] = S.lse2[tid];
    } else {
      if (tid < P) S.lse2[tid] = lk[tid];
      __syncthreads();
    }
    shift_exp<P>(a, S.lse2, rec ? a.ls + (size_t)(k + 1) * a.N * P : nullptr);
  }
  return true;
}

// ---- the forward sweep: A^0, B^0, T outer iterations with their
// checkpoints, then E_hat = X B_T and A_hat (p x N)
// This CTA's view of the arrays: with residency, its per-pixel arrays and its
// X rows live in shared memory (addressed with the global pixel index, like
// the arrays in global memory).
__device__ UArgs local_view(const UArgs& g, float* dyn) {
  UArgs a = g;
  int lo, hi;
  prange(g.N, lo, hi);
  const int P = g.P, L = g.L;
  float* q = dyn;
  if (g.res_x) {  // rows padded with zeros to the stride Ls (a multiple of 4)
    const int Ls = g.Ls;
    const float* src = g.X + (size_t)lo * L;
    for (int e = threadIdx.x; e < (hi - lo) * Ls; e += kT) {
      const int r = e / Ls, l = e - r * Ls;
      q[e] = l < L ? src[(size_t)r * L + l] : 0.f;
    }
    a.X = q - (size_t)lo * Ls;
    q += (size_t)g.maxpx * Ls;
  }
  if (g.res_state) {  // the kPixD float-float arrays first (q is 16-byte aligned here), then the kPixF float ones
    auto nextd = [&]() {
      float2* r = reinterpret_cast<float2*>(q) - (size_t)lo * P;
      q += (size_t)g.maxpx * P * 2;
      return r;
    };
    auto nextf = [&]() {
      float* r = q - (size_t)lo * P;
      q += (size_t)g.maxpx * P;
      return r;
    };
    a.z = nextd(); a.l = nextd();
    a.b = nextf(); a.a = nextf(); a.C = nextf(); a.g = nextf(); a.d = nextf(); a.lbar = nextf();
    a.zbar = nextf(); a.Abar = nextf(); a.zeta = nextf(); a.Dbar = nextf(); a.bp = nextf(); a.tmp = nextf();
  }
  __syncthreads();
  return a;
}

template <int P>
__global__ void __launch_bounds__(kT, 1) k_unrolled_fwd(UArgs ag) {
  __shared__ Sm S;
  extern __shared__ __align__(16) float dyn[];
  const UArgs a = local_view(ag, dyn);
  unsigned nbar = 0;
  const int tid = threadIdx.x;
  const size_t n = (size_t)a.N * P;
  int lo, hi;
  prange(a.N, lo, hi);
  // A^0 = 1/p (eq. initA0); B^0 = softmax(0.1 u), u from SplitMix64 (eq. initB0)
  const float2 z0 = ff_split(-log((double)P));
  for (int e = lo * P + tid; e < hi * P; e += kT) {
    a.z[e] = z0;
    a.l[e] = ff_split(0.1 * ((double)(sm64(a.seed, (uint64_t)e + 1) >> 40) * (1.0 / 16777216.0)));
  }
  __syncthreads();
  lse_part<P>(a, a.l, S);
  if (!gbar(a)) return;
  lse_merge(a, S.lse, S.lse2);
  shift_exp<P>(a, S.lse2, nullptr);
  for (int t = 0; t < a.T; ++t) {
    copy_px<P>(a, a.z, a.zck + (size_t)t * n, nullptr);
    copy_px<P>(a, a.l, a.lck + (size_t)t * n, nullptr);
    if (!fwd_outer<P>(a, S, t, false, nbar)) return;
  }
  copy_px<P>(a, a.z, a.zck + (size_t)a.T * n, nullptr);
  copy_px<P>(a, a.l, a.lck + (size_t)a.T * n, nullptr);
  xw_part<P>(a, a.b, S);
  if (!gbar(a)) return;
  merge_dist(a, a.Ed, a.E32, a.Eout);
  for (int i = lo + tid; i < hi; i += kT)
#pragma unroll
    for (int j = 0; j < P; ++j) a.Aout[(size_t)j * a.N + i] = ff_exp(a.z[(size_t)i * P + j]);
}

// ---- the reverse sweep: from d(loss)/dE_hat (dE) and d(loss)/dA_hat (dA),
// d(loss)/dX (Xbar) and d(loss)/d eta (deta)
template <int P>
__global__ void __launch_bounds__(kT, 1) k_unrolled_bwd(UArgs ag) {
  __shared__ Sm S;
  extern __shared__ __align__(16) float dyn[];
  const UArgs a = local_view(ag, dyn);
  unsigned nbar = 0;
  const int tid = threadIdx.x, LP = a.LP, T = a.T;
  const size_t n = (size_t)a.N * P;
  int lo, hi;
  prange(a.N, lo, hi);
  float* peta = a.peta + (size_t)blockIdx.x * 2 * T;  // this CTA's d eta partials
  for (int e = tid; e < 2 * T; e += kT) peta[e] = 0.f;
  int ru = 0;  // rank-p terms of Xbar recorded so far
  for (int e = lo * P + tid; e < hi * P; e += kT) {
    a.zbar[e] = 0.f;
    const int i = e / P, j = e - i * P;
    a.Abar[e] = a.dA[(size_t)j * a.N + i];  // A_hat = exp(z_T): its adjoint starts at dA
  }
  // E_hat = X B_T: Xbar += dE B^T; lbar = B o (X^T dE)
  copy_px<P>(a, a.lck + (size_t)T * n, a.l, a.b);
  for (int e = tid; e < LP; e += kT) S.p0[e] = a.dE[e];
  __syncthreads();
  rank_record<P>(a, ru, S.p0, a.b, 1.f, nullptr, nullptr, 0.f);
  xdot<P>(a, S.p0, 1.f, a.tmp);
  for (int e = lo * P + tid; e < hi * P; e += kT) a.lbar[e] = a.b[e] * a.tmp[e];
  __syncthreads();
  for (int t = T - 1; t >= 0; --t) {
    // ---- recompute outer iteration t from its checkpoint
    copy_px<P>(a, a.zck + (size_t)t * n, a.z, nullptr);
    copy_px<P>(a, a.lck + (size_t)t * n, a.l, a.b);
    if (!fwd_outer<P>(a, S, t, true, nbar)) return;
    // now z = z_{t+1}, a = exp z_{t+1}, S.W = A A^T; ls[k], gs[k], Rs[k]
    const float etaB = (float)a.eta[T + t], etaA = (float)a.eta[t];
    for (int e = tid; e < P * P; e += kT) S.Wacc[e] = 0.f;
    // ---- reverse the B-steps
    for (int k = a.K2 - 1; k >= 0; --k) {
      copy_px<P>(a, a.ls + (size_t)(k + 1) * n, nullptr, a.bp);
      copy_px<P>(a, a.ls + (size_t)k * n, nullptr, a.b);
      // s = column sums of lbar; zeta = lbar - B' diag(s)
      {
        float cs[P];
#pragma unroll
        for (int j = 0; j < P; ++j) cs[j] = 0.f;
        for (int i = lo + tid; i < hi; i += kT)
#pragma unroll
          for (int j = 0; j < P; ++j) cs[j] += a.lbar[(size_t)i * P + j];
        block_part<P>(a, cs, S);
      }
      if (!gbar(a)) return;
      merge_small(a, P, nullptr, S.sd);
      if (tid < P) S.sd2[tid] = ff_split(S.sd[tid]);
      __syncthreads();
      // zeta; d eta_B += -<zeta, g_k>
      {
        float de[1] = {0.f};
        const float* gk = a.gs + (size_t)k * n;
        for (int e = lo * P + tid; e < hi * P; e += kT) {
          // lbar - bp sd with sd float-float: the product split exactly
          const float2 sd = S.sd2[e % P];
          const float bpv = a.bp[e], pr = __fmul_rn(bpv, sd.x);
          const float pe = fmaf(bpv, sd.x, -pr) + bpv * sd.y;
          const float zt = (a.lbar[e] - pr) - pe;
          a.zeta[e] = zt;
          de[0] = fmaf(-zt, gk[e], de[0]);
        }
        block_total<1>(de, S);
        if (tid == 0) peta[T + t] += S.tmp[0];
      }
      // P = X zeta; Dbar = -eta X^T P
      xw_part<P>(a, a.zeta, S);
      if (!gbar(a)) return;
      merge_dist(a, nullptr, a.P32, nullptr);
      if (!gbar(a)) return;
      for (int e = tid; e < LP; e += kT) {
        S.p0[e] = a.P32[e];
        S.p1[e] = a.Rs[((size_t)t * a.K2 + k) * LP + e];
      }
      __syncthreads();
      xdot<P>(a, S.p0, -etaB, a.Dbar);
      // D = B W - A^T (per pixel); Xbar += -eta (R zeta^T + P D^T); Wbar += B^T Dbar;
      // lbar = zeta + B o (Dbar W); Abar -= Dbar
      float wb[P * P];
#pragma unroll
      for (int e = 0; e < P * P; ++e) wb[e] = 0.f;
      for (int i = lo + tid; i < hi; i += kT) {
        float bv[P], av[P], db[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
          bv[j] = a.b[(size_t)i * P + j];
          av[j] = a.a[(size_t)i * P + j];
          db[j] = a.Dbar[(size_t)i * P + j];
        }
#pragma unroll
        for (int j = 0; j < P; ++j) {
          float s = -av[j], sw = 0.f;
#pragma unroll
          for (int q = 0; q < P; ++q) {
            s = fmaf(S.W[j * P + q], bv[q], s);
            sw = fmaf(db[q], S.W[q * P + j], sw);
            wb[j * P + q] = fmaf(bv[j], db[q], wb[j * P + q]);
          }
          a.d[(size_t)i * P + j] = s;
          a.lbar[(size_t)i * P + j] = fmaf(bv[j], sw, a.zeta[(size_t)i * P + j]);
          a.Abar[(size_t)i * P + j] -= db[j];
        }
      }
      __syncthreads();
      rank_record<P>(a, ru, S.p1, a.zeta, -etaB, S.p0, a.d, -etaB);
      block_total<P * P>(wb, S);
      for (int e = tid; e < P * P; e += kT) S.Wacc[e] += S.tmp[e];
      __syncthreads();
    }
    // ---- Wbar over all pixels; zbar(z_{t+1}) += a o (Abar + (Wbar + Wbar^T) a); Abar = 0
    for (int e = tid; e < P * P; e += kT) a.part2[(size_t)blockIdx.x * kSmall + e] = S.Wacc[e];
    __syncthreads();
    if (!gbar(a)) return;
    merge_small(a, P * P, S.Wb, nullptr);
    for (int i = lo + tid; i < hi; i += kT) {
      float av[P];
#pragma unroll
      for (int j = 0; j < P; ++j) av[j] = a.a[(size_t)i * P + j];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        float s = a.Abar[(size_t)i * P + j];
#pragma unroll
        for (int q = 0; q < P; ++q) s = fmaf(S.Wb[j * P + q] + S.Wb[q * P + j], av[q], s);
        a.zbar[(size_t)i * P + j] = fmaf(av[j], s, a.zbar[(size_t)i * P + j]);
        a.Abar[(size_t)i * P + j] = 0.f;
      }
    }
    __syncthreads();
    // ---- reverse the A-steps from z_t with E_t = X B_t, its Gram, and c = E_t^T x
    // (G and c are still those the recompute of iteration t formed)
    copy_px<P>(a, a.lck + (size_t)t * n, a.l, a.b);
    const double* Edt = a.Eds + (size_t)t * LP;
    for (int e = tid; e < LP; e += kT) S.p0[e] = a.Es[(size_t)t * LP + e];
    __syncthreads();
    {
      float gacc[P * P + 1];
#pragma unroll
      for (int e = 0; e <= P * P; ++e) gacc[e] = 0.f;
      for (int i = lo + tid; i < hi; i += kT) {
        float2 z[kMaxP];
        float c[kMaxP], zb[P], cb[P];
        float zs[6][kMaxP];  // K1 <= 5 recorded iterates + the result
#pragma unroll
        for (int j = 0; j < P; ++j) {
          z[j] = a.zck[(size_t)t * n + (size_t)i * P + j];
          c[j] = a.C[(size_t)i * P + j];
          zb[j] = a.zbar[(size_t)i * P + j];
          cb[j] = 0.f;
        }
        a_steps<P>(z, c, S.G, S.Gl, a.eta[t], a.K1, zs);
        for (int k = a.K1 - 1; k >= 0; --k) {
          float ak[P], ap[P], zeta[P], sz = 0.f;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            ak[j] = expf(zs[k][j]);
            ap[j] = expf(zs[k + 1][j]);
            sz += zb[j];
          }
#pragma unroll
          for (int j = 0; j < P; ++j) zeta[j] = fmaf(-ap[j], sz, zb[j]);
#pragma unroll
          for (int j = 0; j < P; ++j) {
            float g = -c[j], gz = 0.f;
#pragma unroll
            for (int q = 0; q < P; ++q) {
              g = fmaf(S.G[j * P + q], ak[q], g);
              gz = fmaf(S.G[j * P + q], zeta[q], gz);
            }
            gacc[P * P] = fmaf(-zeta[j], g, gacc[P * P]);  // d eta_A
            cb[j] = fmaf(etaA, zeta[j], cb[j]);
#pragma unroll
            for (int q = 0; q < P; ++q) gacc[j * P + q] = fmaf(-etaA * zeta[j], ak[q], gacc[j * P + q]);
            zb[j] = fmaf(-etaA * ak[j], gz, zeta[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < P; ++j) {
          a.zbar[(size_t)i * P + j] = zb[j];
          a.tmp[(size_t)i * P + j] = cb[j];  // Cbar
        }
      }
      block_part<P * P + 1>(a, gacc, S);
      if (tid == 0) peta[t] += a.part2[(size_t)blockIdx.x * kSmall + P * P];
    }
    // Ebar = E (Gbar + Gbar^T) + X Cbar^T ; Xbar += E Cbar + Ebar B^T ; lbar += B o (X^T Ebar)
    // (the Gbar partials and the X Cbar^T partials share one barrier)
    xw_part<P>(a, a.tmp, S);
    if (!gbar(a)) return;
    merge_small(a, P * P, nullptr, S.Gb);
    merge_dist(a, a.XCd, nullptr, nullptr);
    if (!gbar(a)) return;
    for (int e = tid; e < LP; e += kT) {
      const int l = e / P, j = e - l * P;
      double s = a.XCd[e];
#pragma unroll
      for (int k = 0; k < P; ++k) s += Edt[l * P + k] * (S.Gb[k * P + j] + S.Gb[j * P + k]);
      S.p1[e] = (float)s;
    }
    __syncthreads();
    rank_record<P>(a, ru, S.p0, a.tmp, 1.f, S.p1, a.b, 1.f);
    xdot<P>(a, S.p1, 1.f, a.d);
    for (int e = lo * P + tid; e < hi * P; e += kT) a.lbar[e] = fmaf(a.b[e], a.d[e], a.lbar[e]);
    __syncthreads();
  }
  // d eta: the CTAs' partials in a fixed order; Xbar from the recorded terms
  if (!gbar(a)) return;
  if (blockIdx.x == 0) {
    const int lane = tid & 31, warp = tid >> 5, G = gridDim.x;
    for (int e = warp; e < 2 * T; e += kW) {
      float hi2 = 0.f, lo2 = 0.f;
      for (int b = lane; b < G; b += 32) ff_add(hi2, lo2, a.peta[(size_t)b * 2 * T + e]);
      const double s = ff_warp_total(hi2, lo2);
      if (lane == 0) a.deta[e] = s;
    }
  }
  dx_contract(a, ru, S);
}

template <class F>
cudaError_t by_p(int P, F&& f) {
  switch (P) {
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 3: return f(std::integral_constant<int, 3>());
    case 4: return f(std::integral_constant<int, 4>());
    case 5: return f(std::integral_constant<int, 5>());
    case 6: return f(std::integral_constant<int, 6>());
    case 7: return f(std::integral_constant<int, 7>());
    default: return f(std::integral_constant<int, 8>());
  }
}

// ---------------------------------------------------------------------------
// host engine
// ---------------------------------------------------------------------------
struct Buf {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&p, n * sizeof(T) + 16);
    ptrs.push_back(p);
    return (T*)p;
  }
  ~Buf() {
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
};

}  // namespace eu

struct edaa_unrolled {
  int L, N, P, T, K1, K2, G = 0;
  size_t dyn = 0;  // dynamic shared memory of the sweeps
  cudaStream_t caller = nullptr;  // the stream the caller orders our work on
  cudaStream_t s = nullptr;       // our own stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  eu::Buf buf;
  eu::UArgs a{};
  double* eta_d = nullptr;
  float *dE_d = nullptr, *dA_d = nullptr;
  bool have_forward = false;
};

namespace eu {

// one cooperative launch of the sweep kernel over every SM
template <int P>
cudaError_t launch_sweep(edaa_unrolled* u, bool forward) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)u->G);
  lc.blockDim = dim3(kT);
  lc.dynamicSmemBytes = u->dyn;
  lc.stream = u->s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaError_t e = cudaMemsetAsync(u->a.bar, 0, sizeof(unsigned), u->s);  // the barrier counter starts at 0
  if (e != cudaSuccess) return e;
  return forward ? cudaLaunchKernelEx(&lc, k_unrolled_fwd<P>, u->a) : cudaLaunchKernelEx(&lc, k_unrolled_bwd<P>, u->a);
}
// the sweeps' dynamic shared memory (the per-pixel arrays, then also the X
// rows, where they fit next to the static part)
template <int P>
cudaError_t set_dyn(size_t dyn) {
  cudaError_t e = cudaFuncSetAttribute(k_unrolled_fwd<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_unrolled_bwd<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  return e;
}
cudaError_t sweep(edaa_unrolled* u, bool forward) {
  return by_p(u->P, [&](auto pc) { return launch_sweep<decltype(pc)::value>(u, forward); });
}
// xw_part's chunk sums sit in shared memory at [c][r][j][q] with quad stride
// Qx: the smallest Qx >= ceil(L/4) (up to 32 more) whose reads in the
// combine loop (thread e takes entry (l, j) = (e / p, e % p)) fall in the
// fewest banks at once; writes (consecutive q) are conflict-free for any Qx
int xs_stride(int L, int P) {
  const int Q = (L + 3) >> 2, C = std::min(8, std::max(1, kT / Q)), LP = L * P;
  int best = Q, bestw = 1 << 30;
  for (int Qp = Q; Qp <= Q + 32 && C * 4 * P * Qp <= 4 * kMaxP * kT; ++Qp) {
    int w = 1;
    for (int c = 0; c < C; ++c)
      for (int e0 = 0; e0 < LP; e0 += 32) {
        int cnt[32] = {0};
        for (int lane = 0; lane < 32 && e0 + lane < LP; ++lane) {
          const int e = e0 + lane, l = e / P, j = e - l * P, q = l >> 2, r = l & 3;
          w = std::max(w, ++cnt[(((c * 4 + r) * P + j) * Qp + q) & 31]);
        }
      }
    if (w < bestw) {
      bestw = w;
      best = Qp;
    }
    if (bestw == 1) break;
  }
  return best;
}
// the largest grid a cooperative launch of the sweeps can take: every SM, one CTA each
cudaError_t grid_size(int P, size_t dyn, int* G) {
  int dev = 0, sms = 0, bps = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = by_p(P, [&](auto pc) {
    constexpr int PP = decltype(pc)::value;
    int b1 = 0, b2 = 0;
    cudaError_t r = set_dyn<PP>(dyn);
    if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_unrolled_fwd<PP>, kT, dyn);
    if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_unrolled_bwd<PP>, kT, dyn);
    bps = std::min(b1, b2);
    return r;
  });
  if (e != cudaSuccess) return e;
  *G = bps >= 1 ? std::min(sms, kMaxG) : 0;
  return cudaSuccess;
}

}  // namespace eu

using namespace eu;

static edaa_status ufail(edaa_status st, const char* m) {
  edaa::set_last_error(m);
  return st;
}

#define UCK(x, m)                                              \
  do {                                                         \
    cudaError_t e__ = (x);                                     \
    if (e__ != cudaSuccess) {                                  \
      edaa::set_last_error((std::string(m) + ": " + cudaGetErrorString(e__)).c_str()); \
      return EDAA_ERR_CUDA;                                    \
    }                                                          \
  } while (0)

extern "C" {

edaa_status edaa_unrolled_create(edaa_unrolled** out, int L, int N, int p, int T, int K1, int K2, void* stream) {
  if (!out) return ufail(EDAA_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (L < 1 || N < p || p < 1 || T < 1 || K1 < 0 || K2 < 0) return ufail(EDAA_ERR_ARG, "bad shape");
  if (L > 32 * kLT || p > kMaxP || K1 > 5) return ufail(EDAA_ERR_UNSUPPORTED, "L <= 320, p <= 8, K1 <= 5");
  edaa_unrolled* u = new edaa_unrolled();
  u->L = L; u->N = N; u->P = p; u->T = T; u->K1 = K1; u->K2 = K2;
  u->caller = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&u->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&u->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&u->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    edaa_unrolled_destroy(u);
    return ufail(EDAA_ERR_CUDA, "stream or event creation failed in edaa_unrolled_create");
  }
  {
    // one CTA per SM; the per-pixel arrays and then the X rows of a CTA go to
    // shared memory where they fit beside the static part (227 KB per CTA)
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      edaa_unrolled_destroy(u);
      return ufail(EDAA_ERR_CUDA, "edaa_unrolled_create: no device");
    }
    const size_t maxpx = (size_t)(N + sms - 1) / sms + 1;
    const size_t room = 232448 - sizeof(Sm) - 1024;
    // resident X rows: stride a multiple of 4 floats (16-byte loads) and an
    // odd multiple of 4 (eight rows' 16-byte words fall in distinct banks)
    int Ls = (L + 3) & ~3;
    if (Ls % 8 == 0) Ls += 4;
    const size_t st = maxpx * p * (kPixF * 4 + kPixD * 8), xs = maxpx * (size_t)Ls * 4;
    u->a.maxpx = (int)maxpx;
    u->a.res_state = st <= room;
    u->a.res_x = u->a.res_state && st + xs <= room;
    u->a.Ls = u->a.res_x ? Ls : L;
    u->a.Qx = xs_stride(L, p);
    u->dyn = (u->a.res_state ? st : 0) + (u->a.res_x ? xs : 0);
    if (grid_size(p, u->dyn, &u->G) != cudaSuccess || u->G < 1) {
      edaa_unrolled_destroy(u);
      return ufail(EDAA_ERR_CUDA, "edaa_unrolled_create: the sweep kernels do not fit on an SM");
    }
  }
  const size_t n = (size_t)N * p, lp = (size_t)L * p, G = (size_t)u->G;
  Buf& B = u->buf;
  UArgs& a = u->a;
  a.L = L; a.N = N; a.P = p; a.T = T; a.K1 = K1; a.K2 = K2; a.LP = (int)lp;  // (maxpx, res_* set above)
  a.timeout_ns = 2000000000ll;
  a.X = B.get<float>((size_t)N * L);
  u->eta_d = B.get<double>((size_t)2 * T);
  a.eta = u->eta_d;
  a.z = B.get<float2>(n); a.l = B.get<float2>(n); a.b = B.get<float>(n); a.a = B.get<float>(n);
  a.C = B.get<float>(n); a.g = B.get<float>(n); a.d = B.get<float>(n);
  a.lbar = B.get<float>(n); a.zbar = B.get<float>(n); a.Abar = B.get<float>(n); a.zeta = B.get<float>(n);
  a.Dbar = B.get<float>(n); a.bp = B.get<float>(n); a.tmp = B.get<float>(n);
  a.zck = B.get<float2>((T + 1) * n); a.lck = B.get<float2>((T + 1) * n);
  a.ls = B.get<float2>((size_t)(K2 + 1) * n); a.gs = B.get<float>((size_t)std::max(K2, 1) * n);
  a.Rs = B.get<float>((size_t)T * std::max(K2, 1) * lp);
  a.Ws = B.get<float>((size_t)T * 2 * p * p);
  a.lses = B.get<float2>((size_t)T * std::max(K2, 1) * p);
  a.Xbar = B.get<float>((size_t)N * L);
  a.RK = (p * (1 + 2 * T * (K2 + 1)) + 7) & ~7;  // the rank-p terms of Xbar: dE B^T, 2 per B-step, 2 per A-phase
  a.Lv = (L + kDxB - 1) / kDxB * kDxB;
  a.U = B.get<float>((size_t)N * a.RK);
  a.V = B.get<float>((size_t)a.RK * a.Lv);
  u->dE_d = B.get<float>(lp); u->dA_d = B.get<float>(n);
  a.dE = u->dE_d; a.dA = u->dA_d;
  a.Eout = B.get<float>(lp); a.Aout = B.get<float>(n);
  a.part = B.get<float>(G * lp); a.part2 = B.get<float>(G * kSmall); a.peta = B.get<float>(G * 2 * T);
  a.part2d = B.get<double>(G * kSmall);
  a.E32 = B.get<float>(lp); a.P32 = B.get<float>(lp);
  a.Es = B.get<float>((size_t)T * lp); a.Eds = B.get<double>((size_t)T * lp);
  a.Ed = B.get<double>(lp); a.XCd = B.get<double>(lp); a.deta = B.get<double>((size_t)2 * T);
  a.bar = B.get<unsigned>(2); a.status = B.get<int>(1);
  if (B.err != cudaSuccess) {
    edaa_unrolled_destroy(u);
    return ufail(EDAA_ERR_OOM, "cudaMalloc failed in edaa_unrolled_create");
  }
  if (cudaMemset(a.bar, 0, 2 * sizeof(unsigned)) != cudaSuccess || cudaMemset(a.status, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(a.V, 0, (size_t)a.RK * a.Lv * 4) != cudaSuccess) {
    edaa_unrolled_destroy(u);
    return ufail(EDAA_ERR_CUDA, "edaa_unrolled_create: memset failed");
  }
  *out = u;
  return EDAA_OK;
}

void edaa_unrolled_destroy(edaa_unrolled* u) {
  if (!u) return;
  if (u->s) cudaStreamSynchronize(u->s);
  if (u->ev_in) cudaEventDestroy(u->ev_in);
  if (u->ev_out) cudaEventDestroy(u->ev_out);
  if (u->s) cudaStreamDestroy(u->s);
  delete u;
}

edaa_status edaa_unrolled_forward(edaa_unrolled* u, const float* X, uint64_t seed, const double* eta_A,
                                  const double* eta_B, float* E_out, float* A_out) {
  if (!u || !X || !eta_A || !eta_B) return ufail(EDAA_ERR_ARG, "edaa_unrolled_forward: NULL argument");
  const int N = u->N, P = u->P, L = u->L, n = N * P;
  std::vector<double> eta(2 * u->T);
  for (int t = 0; t < u->T; ++t) {
    eta[t] = eta_A[t];
    eta[u->T + t] = eta_B[t];
  }
  u->a.seed = seed;
  // our stream follows the caller's
  UCK(cudaEventRecord(u->ev_in, u->caller), "order after the caller's stream");
  UCK(cudaStreamWaitEvent(u->s, u->ev_in, 0), "order after the caller's stream");
  UCK(cudaMemcpyAsync(u->eta_d, eta.data(), eta.size() * sizeof(double), cudaMemcpyHostToDevice, u->s), "copy eta");
  UCK(cudaMemcpyAsync((void*)u->a.X, X, (size_t)N * L * 4, cudaMemcpyDefault, u->s), "copy X");
  UCK(sweep(u, true), "forward sweep");
  if (E_out) UCK(cudaMemcpyAsync(E_out, u->a.Eout, (size_t)L * P * 4, cudaMemcpyDefault, u->s), "copy E");
  if (A_out) UCK(cudaMemcpyAsync(A_out, u->a.Aout, (size_t)n * 4, cudaMemcpyDefault, u->s), "copy A");
  UCK(cudaEventRecord(u->ev_out, u->s), "order the caller's stream after ours");
  UCK(cudaStreamWaitEvent(u->caller, u->ev_out, 0), "order the caller's stream after ours");
  UCK(cudaGetLastError(), "forward");
  u->have_forward = true;
  return EDAA_OK;
}

edaa_status edaa_unrolled_backward(edaa_unrolled* u, const float* dE, const float* dA, float* dX, double* d_eta_A,
                                   double* d_eta_B) {
  if (!u || !u->have_forward) return ufail(EDAA_ERR_STATE, "edaa_unrolled_backward needs a forward first");
  const int N = u->N, P = u->P, L = u->L, n = N * P, lp = L * P;
  std::vector<double> deta(2 * u->T, 0.0);
  int status = 0;
  UCK(cudaEventRecord(u->ev_in, u->caller), "order after the caller's stream");
  UCK(cudaStreamWaitEvent(u->s, u->ev_in, 0), "order after the caller's stream");
  // the adjoints of the outputs (zeros when absent) go into the engine's buffers
  if (dE) UCK(cudaMemcpyAsync(u->dE_d, dE, (size_t)lp * 4, cudaMemcpyDefault, u->s), "copy dE");
  else UCK(cudaMemsetAsync(u->dE_d, 0, (size_t)lp * 4, u->s), "zero");
  if (dA) UCK(cudaMemcpyAsync(u->dA_d, dA, (size_t)n * 4, cudaMemcpyDefault, u->s), "copy dA");
  else UCK(cudaMemsetAsync(u->dA_d, 0, (size_t)n * 4, u->s), "zero");
  UCK(sweep(u, false), "backward sweep");
  if (dX) UCK(cudaMemcpyAsync(dX, u->a.Xbar, (size_t)N * L * 4, cudaMemcpyDefault, u->s), "copy dX");
  UCK(cudaMemcpyAsync(deta.data(), u->a.deta, 2 * u->T * sizeof(double), cudaMemcpyDeviceToHost, u->s), "copy");
  UCK(cudaMemcpyAsync(&status, u->a.status, sizeof(int), cudaMemcpyDeviceToHost, u->s), "copy status");
  UCK(cudaStreamSynchronize(u->s), "sync");
  UCK(cudaEventRecord(u->ev_out, u->s), "order the caller's stream after ours");
  UCK(cudaStreamWaitEvent(u->caller, u->ev_out, 0), "order the caller's stream after ours");
  if (status & edaa::kStatTimeout) {
    cudaMemsetAsync(u->a.status, 0, sizeof(int), u->s);
    cudaMemsetAsync(u->a.bar, 0, 2 * sizeof(unsigned), u->s);
    return ufail(EDAA_ERR_TIMEOUT, "a grid barrier of the unrolled sweeps timed out");
  }
  if (d_eta_A) for (int t = 0; t < u->T; ++t) d_eta_A[t] = deta[t];
  if (d_eta_B) for (int t = 0; t < u->T; ++t) d_eta_B[t] = deta[u->T + t];
  return EDAA_OK;
}

}  // extern "C"
