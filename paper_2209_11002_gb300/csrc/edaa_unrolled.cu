// Differentiable unrolled EDAA for one run: the forward pass of Algorithm 1
// with per-block step sizes (eta_A[t] for the K1 A-steps and eta_B[t] for the
// K2 B-steps of outer iteration t), a checkpoint of (log A, log B) at the
// start of every outer iteration, and hand-written adjoint kernels giving
// d(loss)/dX and d(loss)/d(eta) from d(loss)/dE_hat and d(loss)/dA_hat.
//
// State (pixel-major, N x p): z = log A (normalised per pixel), l = log B
// (normalised per column).  One A-step (eq. update_A in softmax form):
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
// Every reduction over pixels is per-block partials in float32 followed by a
// fixed-order FP64 merge: results are deterministic.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/edaa.h"

namespace edaa {
void set_last_error(const char* msg);
}

namespace eu {

constexpr int kT = 256;     // threads per block
constexpr int kW = kT / 32;
constexpr int kMaxP = 8;
constexpr int kLT = 10;     // L <= 320
constexpr int kBlocks = 304;

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

// ---- part[blk][l*P + j] = sum_{pixels i of blk} x_i[l] * w_i[j]  (warp per pixel)
template <int P>
__global__ void __launch_bounds__(kT) k_xw(const float* __restrict__ X, int L, int N, const float* __restrict__ w,
                                         float* __restrict__ part) {
  extern __shared__ float sbuf[];  // L * P
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[kLT][P];
#pragma unroll
  for (int k = 0; k < kLT; ++k)
#pragma unroll
    for (int j = 0; j < P; ++j) acc[k][j] = 0.f;
  for (int i = blockIdx.x * kW + warp; i < N; i += gridDim.x * kW) {
    float wv[P];
#pragma unroll
    for (int j = 0; j < P; ++j) wv[j] = w[(size_t)i * P + j];
    const float* x = X + (size_t)i * L;
#pragma unroll
    for (int k = 0; k < kLT; ++k) {
      const int l = lane + 32 * k;
      const float xv = (l < L) ? x[l] : 0.f;
#pragma unroll
      for (int j = 0; j < P; ++j) acc[k][j] = fmaf(xv, wv[j], acc[k][j]);
    }
  }
  // fixed-order reduction over the block's warps
  for (int r = 0; r < kW; ++r) {
    if (warp == r) {
#pragma unroll
      for (int k = 0; k < kLT; ++k) {
        const int l = lane + 32 * k;
        if (l < L) {
#pragma unroll
          for (int j = 0; j < P; ++j) sbuf[l * P + j] = (r == 0) ? acc[k][j] : sbuf[l * P + j] + acc[k][j];
        }
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < L * P; e += kT) part[(size_t)blockIdx.x * L * P + e] = sbuf[e];
}

// ---- out[i*P + j] = scale * sum_l x_i[l] panel[l*P + j]  (warp per pixel)
template <int P>
__global__ void __launch_bounds__(kT) k_xdot(const float* __restrict__ X, int L, int N,
                                           const float* __restrict__ panel, float scale0,
                                           const float* __restrict__ smul, float* __restrict__ out) {
  // scale = scale0 times the step size at smul when given (read on the device, so that a
  // captured graph serves every call)
  const float scale = smul ? scale0 * *smul : scale0;
  extern __shared__ float sp[];  // L * P
  for (int e = threadIdx.x; e < L * P; e += kT) sp[e] = panel[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = blockIdx.x * kW + warp; i < N; i += gridDim.x * kW) {
    const float* x = X + (size_t)i * L;
    float c[P];
#pragma unroll
    for (int j = 0; j < P; ++j) c[j] = 0.f;
    for (int l = lane; l < L; l += 32) {
      const float xv = x[l];
#pragma unroll
      for (int j = 0; j < P; ++j) c[j] = fmaf(xv, sp[l * P + j], c[j]);
    }
#pragma unroll
    for (int j = 0; j < P; ++j) c[j] = wsum(c[j]);
    if (lane < P) {
      float v = c[0];
#pragma unroll
      for (int j = 1; j < P; ++j)
        if (lane == j) v = c[j];
      out[(size_t)i * P + lane] = scale * v;
    }
  }
}

// ---- Xbar_i[l] += s1 sum_j L1[l,j] R1[i,j] + s2 sum_j L2[l,j] R2[i,j]  (rank-p updates of dX)
template <int P>
__global__ void __launch_bounds__(kT) k_rank(float* __restrict__ Xbar, int L, int N, const float* __restrict__ L1,
                                           const float* __restrict__ R1, float s1m, const float* __restrict__ L2,
                                           const float* __restrict__ R2, float s2m, const float* __restrict__ smul) {
  const float s1 = smul ? s1m * *smul : s1m, s2 = smul ? s2m * *smul : s2m;
  extern __shared__ float sp[];  // 2 * L * P
  float* l1 = sp;
  float* l2 = sp + L * P;
  for (int e = threadIdx.x; e < L * P; e += kT) {
    l1[e] = L1[e];
    l2[e] = L2 ? L2[e] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = blockIdx.x * kW + warp; i < N; i += gridDim.x * kW) {
    float r1[P], r2[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      r1[j] = s1 * R1[(size_t)i * P + j];
      r2[j] = R2 ? s2 * R2[(size_t)i * P + j] : 0.f;
    }
    float* xb = Xbar + (size_t)i * L;
    for (int l = lane; l < L; l += 32) {
      float v = xb[l];
#pragma unroll
      for (int j = 0; j < P; ++j) v = fmaf(l1[l * P + j], r1[j], fmaf(l2[l * P + j], r2[j], v));
      xb[l] = v;
    }
  }
}

// ---- reductions of per-pixel p-vectors: mode 0: sum w1 w2^T (P x P);
// mode 1: column sums of w1 (P); mode 2: per-column sum of w1 o w2 (P)
__global__ void __launch_bounds__(kT) k_pred(const float* __restrict__ w1, const float* __restrict__ w2, int N, int P,
                                           int mode, float* __restrict__ part) {
  __shared__ float red[kT];
  const int n_out = (mode == 0) ? P * P : P;
  float acc[kMaxP * kMaxP];
  for (int e = 0; e < n_out; ++e) acc[e] = 0.f;
  for (int i = blockIdx.x * kT + threadIdx.x; i < N; i += gridDim.x * kT) {
    const float* a = w1 + (size_t)i * P;
    const float* b = w2 ? w2 + (size_t)i * P : nullptr;
    if (mode == 0) {
      for (int j = 0; j < P; ++j)
        for (int k = 0; k < P; ++k) acc[j * P + k] = fmaf(a[j], b[k], acc[j * P + k]);
    } else if (mode == 1) {
      for (int j = 0; j < P; ++j) acc[j] += a[j];
    } else {
      for (int j = 0; j < P; ++j) acc[j] = fmaf(a[j], b[j], acc[j]);
    }
  }
  for (int e = 0; e < n_out; ++e) {
    red[threadIdx.x] = acc[e];
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * n_out + e] = red[0];
    __syncthreads();
  }
}

// fixed-order merge of per-block partials (FP64), optional scale and float copy
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
// butterfly over the warp in a fixed order (lane 0 ends with the total)
__device__ __forceinline__ double ff_warp_total(float hi, float lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    ff_add(hi, lo, h2);
    lo += l2;
  }
  return (double)hi + (double)lo;
}

// out[e] = scale * sum_b part[b][e]: one warp per output, lanes over the
// partials (fixed order, float-float)
__global__ void k_merge(const float* __restrict__ part, int nb, int n, double scale, double* outd, float* outf) {
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= n) return;  // whole warps leave together
  float hi = 0.f, lo = 0.f;
  for (int b = lane; b < nb; b += 32) ff_add(hi, lo, part[(size_t)b * n + e]);
  const double s = ff_warp_total(hi, lo) * scale;
  if (lane == 0) {
    if (outd) outd[e] = s;
    if (outf) outf[e] = (float)s;
  }
}
inline int merge_blocks(int n) { return (n + 7) / 8; }  // 8 warps (outputs) per 256-thread block

// ---- column log-sum-exp over pixels (online per thread, fixed-order merges)
__global__ void __launch_bounds__(kT) k_lse_part(const float* __restrict__ u, int N, int P, float* __restrict__ part) {
  __shared__ float sm[kT], ss[kT];
  for (int j = 0; j < P; ++j) {
    float m = -INFINITY, s = 0.f;
    for (int i = blockIdx.x * kT + threadIdx.x; i < N; i += gridDim.x * kT) {
      const float v = u[(size_t)i * P + j];
      if (v > m) {
        s = s * expf(m - v) + 1.f;
        m = v;
      } else {
        s += expf(v - m);
      }
    }
    sm[threadIdx.x] = m;
    ss[threadIdx.x] = s;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) {
        const float m1 = sm[threadIdx.x], m2 = sm[threadIdx.x + h];
        const float mm = fmaxf(m1, m2);
        float s1 = ss[threadIdx.x], s2 = ss[threadIdx.x + h];
        s1 = (m1 == -INFINITY) ? 0.f : s1 * expf(m1 - mm);
        s2 = (m2 == -INFINITY) ? 0.f : s2 * expf(m2 - mm);
        sm[threadIdx.x] = mm;
        ss[threadIdx.x] = s1 + s2;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      part[((size_t)blockIdx.x * P + j) * 2 + 0] = sm[0];
      part[((size_t)blockIdx.x * P + j) * 2 + 1] = ss[0];
    }
    __syncthreads();
  }
}

__global__ void k_lse_merge(const float* __restrict__ part, int nb, int P, double* __restrict__ lse) {
  // one warp per column: m = max of the block maxima, then sum_b s_b e^(m_b - m)
  const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
  if (j >= P) return;
  float m = -INFINITY;
  for (int b = lane; b < nb; b += 32) m = fmaxf(m, part[((size_t)b * P + j) * 2]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  float hi = 0.f, lo = 0.f;
  for (int b = lane; b < nb; b += 32) {
    const float mb = part[((size_t)b * P + j) * 2];
    if (mb != -INFINITY) ff_add(hi, lo, part[((size_t)b * P + j) * 2 + 1] * expf(mb - m));
  }
  const double sum = ff_warp_total(hi, lo);
  if (lane == 0) lse[j] = (double)m + log(sum);
}

// l -= lse (per column); b = exp(l)
__global__ void k_shift_exp(float* __restrict__ l, const double* __restrict__ lse, int N, int P, float* __restrict__ b) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * P) return;
  const float v = (float)((double)l[e] - lse[e % P]);
  l[e] = v;
  if (b) b[e] = expf(v);
}

__global__ void k_exp(const float* __restrict__ z, int n, float* __restrict__ a) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) a[e] = expf(z[e]);
}

__global__ void k_init_logits(uint64_t seed, int N, int P, float* __restrict__ l) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * P) return;
  l[e] = 0.1f * ((float)(sm64(seed, (uint64_t)e + 1) >> 40) * (1.0f / 16777216.0f));
}

__global__ void k_fill(float* __restrict__ z, int n, float v) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) z[e] = v;
}

// G = E^T E (P x P) from the FP64 E, one block
__global__ void k_gram(const double* __restrict__ E, int L, int P, float* __restrict__ G) {
  // one warp per entry (j, k) of G = E^T E, lanes over the bands
  const int lane = threadIdx.x & 31, e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= P * P) return;
  const int j = e / P, k = e % P;
  double s = 0.0;
  for (int l = lane; l < L; l += 32) s += E[l * P + j] * E[l * P + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) G[e] = (float)s;
}

// one pixel's A-phase: K1 mirror steps; keeps the iterates when `rec` is set
__device__ __forceinline__ void a_steps(float* z, const float* c, const float* G, float eta, int K1, int P,
                                        float (*zs)[kMaxP]) {
  for (int k = 0; k < K1; ++k) {
    if (zs)
      for (int j = 0; j < P; ++j) zs[k][j] = z[j];
    float a[kMaxP], mx = -INFINITY;
    for (int j = 0; j < P; ++j) a[j] = expf(z[j]);
    for (int j = 0; j < P; ++j) {
      float g = -c[j];
      for (int q = 0; q < P; ++q) g = fmaf(G[j * P + q], a[q], g);
      z[j] = fmaf(-eta, g, z[j]);
      mx = fmaxf(mx, z[j]);
    }
    float se = 0.f;
    for (int j = 0; j < P; ++j) se += expf(z[j] - mx);
    const float lz = mx + logf(se);
    for (int j = 0; j < P; ++j) z[j] -= lz;
  }
  if (zs)
    for (int j = 0; j < P; ++j) zs[K1][j] = z[j];
}

__global__ void k_a_fwd(const float* __restrict__ C, const float* __restrict__ Gg, const float* __restrict__ etap,
                        int K1, int N, int P, const float* zin, float* zout) {  // zin may be zout (in place)
  const float eta = *etap;
  __shared__ float G[kMaxP * kMaxP];
  if (threadIdx.x < P * P) G[threadIdx.x] = Gg[threadIdx.x];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float z[kMaxP], c[kMaxP];
  for (int j = 0; j < P; ++j) {
    z[j] = zin[(size_t)i * P + j];
    c[j] = C[(size_t)i * P + j];
  }
  a_steps(z, c, G, eta, K1, P, nullptr);
  for (int j = 0; j < P; ++j) zout[(size_t)i * P + j] = z[j];
}

// d_i = W b_i - a_i
__global__ void k_dev(const float* __restrict__ b, const float* __restrict__ a, const float* __restrict__ W, int N,
                      int P, float* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int j = 0; j < P; ++j) {
    float s = -a[(size_t)i * P + j];
    for (int k = 0; k < P; ++k) s = fmaf(W[j * P + k], b[(size_t)i * P + k], s);
    d[(size_t)i * P + j] = s;
  }
}

// l' = l - eta g (unnormalised)
__global__ void k_axpy(const float* l, const float* __restrict__ g, const float* __restrict__ etap, int n,
                       float* o) {  // l may be o (in place)
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) o[e] = fmaf(-*etap, g[e], l[e]);
}

// zeta = lbar - bp o s
__global__ void k_zeta(const float* __restrict__ lbar, const float* __restrict__ bp, const double* __restrict__ s,
                       int N, int P, float* __restrict__ zeta) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * P) return;
  zeta[e] = (float)((double)lbar[e] - (double)bp[e] * s[e % P]);
}

// B-step adjoint, per pixel: lbar = zeta + b o (Dbar W); Abar -= Dbar
__global__ void k_bbwd(const float* __restrict__ zeta, const float* __restrict__ b, const float* __restrict__ Dbar,
                       const float* __restrict__ W, int N, int P, float* __restrict__ lbar, float* __restrict__ Abar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int j = 0; j < P; ++j) {
    float s = 0.f;
    for (int k = 0; k < P; ++k) s = fmaf(Dbar[(size_t)i * P + k], W[k * P + j], s);
    lbar[(size_t)i * P + j] = fmaf(b[(size_t)i * P + j], s, zeta[(size_t)i * P + j]);
    Abar[(size_t)i * P + j] -= Dbar[(size_t)i * P + j];
  }
}

// zbar += a o (Abar + (Wbar + Wbar^T) a)
__global__ void k_zbar(const float* __restrict__ a, const float* __restrict__ Abar, const float* __restrict__ Wb,
                       int N, int P, float* __restrict__ zbar) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int j = 0; j < P; ++j) {
    float s = Abar[(size_t)i * P + j];
    for (int k = 0; k < P; ++k) s = fmaf(Wb[j * P + k] + Wb[k * P + j], a[(size_t)i * P + k], s);
    zbar[(size_t)i * P + j] = fmaf(a[(size_t)i * P + j], s, zbar[(size_t)i * P + j]);
  }
}

// A-phase adjoint per pixel: recompute the K1 iterates from z_t, then reverse.
// Writes zbar (adjoint of z_t), Cbar; block partials of Gbar (P*P) and d eta (1).
__global__ void __launch_bounds__(kT) k_a_bwd(const float* __restrict__ C, const float* __restrict__ Gg,
                                            const float* __restrict__ etap, int K1, int N, int P,
                                            const float* __restrict__ zt, float* __restrict__ zbar,
                                            float* __restrict__ Cbar, float* __restrict__ part) {
  const float eta = *etap;
  __shared__ float G[kMaxP * kMaxP];
  __shared__ float red[kT];
  if (threadIdx.x < P * P) G[threadIdx.x] = Gg[threadIdx.x];
  __syncthreads();
  float gacc[kMaxP * kMaxP + 1];
  for (int e = 0; e <= P * P; ++e) gacc[e] = 0.f;
  for (int i = blockIdx.x * kT + threadIdx.x; i < N; i += gridDim.x * kT) {
    float z[kMaxP], c[kMaxP], zb[kMaxP], cb[kMaxP];
    float zs[6][kMaxP];  // K1 <= 5 recorded iterates + the result
    for (int j = 0; j < P; ++j) {
      z[j] = zt[(size_t)i * P + j];
      c[j] = C[(size_t)i * P + j];
      zb[j] = zbar[(size_t)i * P + j];
      cb[j] = 0.f;
    }
    a_steps(z, c, G, eta, K1, P, zs);
    for (int k = K1 - 1; k >= 0; --k) {
      float ak[kMaxP], ap[kMaxP], zeta[kMaxP], sz = 0.f;
      for (int j = 0; j < P; ++j) {
        ak[j] = expf(zs[k][j]);
        ap[j] = expf(zs[k + 1][j]);
        sz += zb[j];
      }
      for (int j = 0; j < P; ++j) zeta[j] = fmaf(-ap[j], sz, zb[j]);
      for (int j = 0; j < P; ++j) {
        float g = -c[j], gz = 0.f;
        for (int q = 0; q < P; ++q) {
          g = fmaf(G[j * P + q], ak[q], g);
          gz = fmaf(G[j * P + q], zeta[q], gz);
        }
        gacc[P * P] = fmaf(-zeta[j], g, gacc[P * P]);  // d eta
        cb[j] = fmaf(eta, zeta[j], cb[j]);
        for (int q = 0; q < P; ++q) gacc[j * P + q] = fmaf(-eta * zeta[j], ak[q], gacc[j * P + q]);
        zb[j] = fmaf(-eta * ak[j], gz, zeta[j]);
      }
    }
    for (int j = 0; j < P; ++j) {
      zbar[(size_t)i * P + j] = zb[j];
      Cbar[(size_t)i * P + j] = cb[j];
    }
  }
  for (int e = 0; e <= P * P; ++e) {
    red[threadIdx.x] = gacc[e];
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * (P * P + 1) + e] = red[0];
    __syncthreads();
  }
}

// Ebar = E (Gbar + Gbar^T) + XCbar^T  (L x P, FP64 inputs)
__global__ void k_ebar(const double* __restrict__ E, const double* __restrict__ Gb, const double* __restrict__ XC, int L,
                       int P, float* __restrict__ Ebar) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * P) return;
  const int l = e / P, j = e % P;
  double s = XC[e];
  for (int k = 0; k < P; ++k) s += E[l * P + k] * (Gb[k * P + j] + Gb[j * P + k]);
  Ebar[e] = (float)s;
}

// lbar += b o v (v = X^T Ebar per pixel)
__global__ void k_fma_inplace(float* __restrict__ lbar, const float* __restrict__ b, const float* __restrict__ v, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) lbar[e] = fmaf(b[e], v[e], lbar[e]);
}

// dst[0] += sign * sum(src[0..n)); dst and src FP64, one thread
__global__ void k_acc_sum(double* __restrict__ dst, const double* __restrict__ src, int n, double sign) {
  double v = 0.0;
  for (int e = 0; e < n; ++e) v += src[e];
  dst[0] += sign * v;
}
// dst += src (n doubles); also writes a float copy
__global__ void k_add_d(double* __restrict__ dst, const double* __restrict__ src, int n, float* __restrict__ f) {
  const int e = threadIdx.x;
  if (e >= n) return;
  dst[e] += src[e];
  if (f) f[e] = (float)dst[e];
}

__global__ void k_transpose_pn(const float* __restrict__ src, int N, int P, float* __restrict__ dst) {
  // src N x P (pixel-major) -> dst P x N
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * P) return;
  const int i = e / P, j = e % P;
  dst[(size_t)j * N + i] = src[e];
}
__global__ void k_transpose_np(const float* __restrict__ src, int N, int P, float* __restrict__ dst) {
  // src P x N -> dst N x P
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * P) return;
  const int i = e / P, j = e % P;
  dst[e] = src[(size_t)j * N + i];
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
  int L, N, P, T, K1, K2;
  cudaStream_t caller = nullptr;  // the stream the caller orders our work on
  cudaStream_t s = nullptr;       // our own stream (a captured graph needs one that is not the legacy default)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t g_fwd = nullptr, g_bwd = nullptr;
  eu::Buf buf;
  float *X, *zck, *lck, *z, *l, *b, *a, *C, *g, *d, *part, *G, *W, *E32, *R32;
  double *Ed, *Wd, *Rd, *lse, *scr;
  float *ls, *gs;              // recompute storage: (K2+1) x N x P logits, K2 x N x P B-gradients
  float *Rs;                   // K2 x L x P
  double* deta;                // 2T: d eta_A, d eta_B
  float* eta;                  // 2T on the device: eta_A[t], then eta_B[t]
  float* dAin;                 // p x N: d(loss)/dA_hat for the backward (zeros when absent)
  float *lbar, *zbar, *Abar, *Xbar, *zeta, *Dbar, *bp, *tmp, *P32, *Eb32, *Wb32, *Gb32;
  double *sd, *XCd, *Gbd, *Pd, *Wbd, *eta_scr;
  bool have_forward = false;
};

namespace eu {

inline int nb_pix(int N) { return std::min(kBlocks, (N + kW - 1) / kW); }
inline int nb_thr(int N) { return std::min(kBlocks, (N + kT - 1) / kT); }
inline int g1(int n) { return (n + 255) / 256; }

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

// out (FP64 and float) = X^T-contraction sum_i x_i w_i^T, L x P
cudaError_t xw(edaa_unrolled* u, const float* w, double* outd, float* outf, double scale = 1.0) {
  const int nb = nb_pix(u->N);
  cudaError_t e = by_p(u->P, [&](auto pc) {
    constexpr int PP = decltype(pc)::value;
    k_xw<PP><<<nb, kT, u->L * PP * sizeof(float), u->s>>>(u->X, u->L, u->N, w, u->part);
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  k_merge<<<merge_blocks(u->L * u->P), 256, 0, u->s>>>(u->part, nb, u->L * u->P, scale, outd, outf);
  return cudaGetLastError();
}

// out = scale * X panel, times the step size at smul when given
cudaError_t xdot(edaa_unrolled* u, const float* panel, float scale, float* out, const float* smul = nullptr) {
  const int nb = nb_pix(u->N);
  return by_p(u->P, [&](auto pc) {
    constexpr int PP = decltype(pc)::value;
    k_xdot<PP><<<nb, kT, u->L * PP * sizeof(float), u->s>>>(u->X, u->L, u->N, panel, scale, smul, out);
    return cudaGetLastError();
  });
}

cudaError_t rank(edaa_unrolled* u, const float* L1, const float* R1, float s1, const float* L2, const float* R2,
                 float s2, const float* smul = nullptr) {
  const int nb = nb_pix(u->N);
  return by_p(u->P, [&](auto pc) {
    constexpr int PP = decltype(pc)::value;
    k_rank<PP><<<nb, kT, 2 * u->L * PP * sizeof(float), u->s>>>(u->Xbar, u->L, u->N, L1, R1, s1, L2, R2, s2, smul);
    return cudaGetLastError();
  });
}

cudaError_t pred(edaa_unrolled* u, const float* w1, const float* w2, int mode, double* outd, float* outf,
                 double scale = 1.0) {
  const int nb = nb_thr(u->N);
  const int n_out = mode == 0 ? u->P * u->P : u->P;
  k_pred<<<nb, kT, 0, u->s>>>(w1, w2, u->N, u->P, mode, u->part);
  k_merge<<<merge_blocks(n_out), 256, 0, u->s>>>(u->part, nb, n_out, scale, outd, outf);
  return cudaGetLastError();
}

// l <- l - lse(l) per column; b = exp(l)
cudaError_t normalise_logits(edaa_unrolled* u, float* l, float* b) {
  const int nb = nb_thr(u->N);
  k_lse_part<<<nb, kT, 0, u->s>>>(l, u->N, u->P, u->part);
  k_lse_merge<<<1, 32 * u->P, 0, u->s>>>(u->part, nb, u->P, u->lse);
  k_shift_exp<<<g1(u->N * u->P), 256, 0, u->s>>>(l, u->lse, u->N, u->P, b);
  return cudaGetLastError();
}

// E (FP64 Ed, float E32) = X exp(l) (b must hold exp(l))
cudaError_t make_E(edaa_unrolled* u, const float* b) { return xw(u, b, u->Ed, u->E32); }

// W = A A^T (float W, FP64 Wd) from a = exp(z)
cudaError_t make_W(edaa_unrolled* u, const float* a) { return pred(u, a, a, 0, u->Wd, u->W); }

// R = X (B W - A^T), float R32 (FP64 Rd)
cudaError_t make_R(edaa_unrolled* u, const float* b, const float* a) {
  k_dev<<<g1(u->N), 256, 0, u->s>>>(b, a, u->W, u->N, u->P, u->d);
  return xw(u, u->d, u->Rd, u->R32);
}

// one outer iteration forward from (z, l normalised, b = exp l): A-phase then K2 B-steps.
// When rec is set, stores logits ls[k], B-gradients gs[k] and R_k.
cudaError_t outer_forward(edaa_unrolled* u, int t, bool rec) {
  cudaError_t e;
  const int n = u->N * u->P;
  if ((e = make_E(u, u->b)) != cudaSuccess) return e;
  k_gram<<<(u->P * u->P + 7) / 8, 256, 0, u->s>>>(u->Ed, u->L, u->P, u->G);
  if ((e = xdot(u, u->E32, 1.f, u->C)) != cudaSuccess) return e;
  k_a_fwd<<<g1(u->N), 256, 0, u->s>>>(u->C, u->G, u->eta + t, u->K1, u->N, u->P, u->z, u->z);
  k_exp<<<g1(n), 256, 0, u->s>>>(u->z, n, u->a);
  if ((e = make_W(u, u->a)) != cudaSuccess) return e;
  if (rec) cudaMemcpyAsync(u->ls, u->l, n * 4, cudaMemcpyDeviceToDevice, u->s);
  for (int k = 0; k < u->K2; ++k) {
    if ((e = make_R(u, u->b, u->a)) != cudaSuccess) return e;
    if ((e = xdot(u, u->R32, 1.f, u->g)) != cudaSuccess) return e;
    if (rec) {
      cudaMemcpyAsync(u->Rs + (size_t)k * u->L * u->P, u->R32, u->L * u->P * 4, cudaMemcpyDeviceToDevice, u->s);
      cudaMemcpyAsync(u->gs + (size_t)k * n, u->g, n * 4, cudaMemcpyDeviceToDevice, u->s);
    }
    k_axpy<<<g1(n), 256, 0, u->s>>>(u->l, u->g, u->eta + u->T + t, n, u->l);
    if ((e = normalise_logits(u, u->l, u->b)) != cudaSuccess) return e;
    if (rec) cudaMemcpyAsync(u->ls + (size_t)(k + 1) * n, u->l, n * 4, cudaMemcpyDeviceToDevice, u->s);
  }
  return cudaGetLastError();
}

// The T outer iterations with their checkpoints, then E_hat (E32) and A_hat
// (tmp, p x N).  Every input lives in the engine's buffers, so the sequence
// is captured once and replayed.
cudaError_t forward_body(edaa_unrolled* u) {
  const int N = u->N, P = u->P, n = N * P;
  cudaError_t e;
  for (int t = 0; t < u->T; ++t) {
    cudaMemcpyAsync(u->zck + (size_t)t * n, u->z, n * 4, cudaMemcpyDeviceToDevice, u->s);
    cudaMemcpyAsync(u->lck + (size_t)t * n, u->l, n * 4, cudaMemcpyDeviceToDevice, u->s);
    if ((e = outer_forward(u, t, false)) != cudaSuccess) return e;
  }
  cudaMemcpyAsync(u->zck + (size_t)u->T * n, u->z, n * 4, cudaMemcpyDeviceToDevice, u->s);
  cudaMemcpyAsync(u->lck + (size_t)u->T * n, u->l, n * 4, cudaMemcpyDeviceToDevice, u->s);
  if ((e = make_E(u, u->b)) != cudaSuccess) return e;
  k_exp<<<g1(n), 256, 0, u->s>>>(u->z, n, u->a);
  k_transpose_pn<<<g1(n), 256, 0, u->s>>>(u->a, N, P, u->tmp);
  return cudaGetLastError();
}

// The reverse sweep: from d(loss)/dE_hat (Eb32) and d(loss)/dA_hat (dAin),
// accumulates Xbar (dX) and deta (d eta_A, d eta_B).
cudaError_t backward_body(edaa_unrolled* u) {
  const int N = u->N, P = u->P, L = u->L, n = N * P, lp = L * P;
  cudaError_t e;
  cudaMemsetAsync(u->Xbar, 0, (size_t)N * L * 4, u->s);
  cudaMemsetAsync(u->zbar, 0, n * 4, u->s);
  // final state: b_T, a_T
  cudaMemcpyAsync(u->l, u->lck + (size_t)u->T * n, n * 4, cudaMemcpyDeviceToDevice, u->s);
  k_exp<<<g1(n), 256, 0, u->s>>>(u->l, n, u->b);
  // E_hat = X B_T: Xbar += dE B^T; lbar = B o (X^T dE)
  if ((e = rank(u, u->Eb32, u->b, 1.f, nullptr, nullptr, 0.f)) != cudaSuccess) return e;
  if ((e = xdot(u, u->Eb32, 1.f, u->tmp)) != cudaSuccess) return e;
  cudaMemsetAsync(u->lbar, 0, n * 4, u->s);
  k_fma_inplace<<<g1(n), 256, 0, u->s>>>(u->lbar, u->b, u->tmp, n);
  // A_hat = exp(z_T): the A-adjoint accumulator (pixel-major) starts at dA (p x N)
  k_transpose_np<<<g1(n), 256, 0, u->s>>>(u->dAin, N, P, u->Abar);
  cudaMemsetAsync(u->deta, 0, 2 * u->T * sizeof(double), u->s);
  for (int t = u->T - 1; t >= 0; --t) {
    // ---- recompute outer iteration t from its checkpoint
    cudaMemcpyAsync(u->z, u->zck + (size_t)t * n, n * 4, cudaMemcpyDeviceToDevice, u->s);
    cudaMemcpyAsync(u->l, u->lck + (size_t)t * n, n * 4, cudaMemcpyDeviceToDevice, u->s);
    k_exp<<<g1(n), 256, 0, u->s>>>(u->l, n, u->b);
    if ((e = outer_forward(u, t, true)) != cudaSuccess) return e;
    // after it: z = z_{t+1}, a = exp(z_{t+1}), W = A A^T; ls[k], gs[k], Rs[k]
    const float* etaA = u->eta + t;
    const float* etaB = u->eta + u->T + t;
    cudaMemsetAsync(u->Wbd, 0, 64 * 8, u->s);
    cudaMemsetAsync(u->Wb32, 0, 64 * 4, u->s);
    // ---- reverse the B-steps
    for (int k = u->K2 - 1; k >= 0; --k) {
      const float* lk = u->ls + (size_t)k * n;
      const float* lk1 = u->ls + (size_t)(k + 1) * n;
      k_exp<<<g1(n), 256, 0, u->s>>>(lk1, n, u->bp);
      k_exp<<<g1(n), 256, 0, u->s>>>(lk, n, u->b);
      // s = column sums of lbar; zeta = lbar - B' diag(s)
      if ((e = pred(u, u->lbar, nullptr, 1, u->sd, nullptr)) != cudaSuccess) return e;
      k_zeta<<<g1(n), 256, 0, u->s>>>(u->lbar, u->bp, u->sd, N, P, u->zeta);
      // d eta_B += -<zeta, g>
      if ((e = pred(u, u->zeta, u->gs + (size_t)k * n, 2, u->eta_scr, nullptr)) != cudaSuccess) return e;
      k_acc_sum<<<1, 1, 0, u->s>>>(u->deta + u->T + t, u->eta_scr, P, -1.0);
      // P = X zeta; Dbar = -eta X^T P
      if ((e = xw(u, u->zeta, u->Pd, u->P32)) != cudaSuccess) return e;
      if ((e = xdot(u, u->P32, -1.f, u->Dbar, etaB)) != cudaSuccess) return e;
      // D = B W - A^T (per pixel), Xbar += -eta (R zeta^T + P D^T)
      k_dev<<<g1(N), 256, 0, u->s>>>(u->b, u->a, u->W, N, P, u->d);
      if ((e = rank(u, u->Rs + (size_t)k * lp, u->zeta, -1.f, u->P32, u->d, -1.f, etaB)) != cudaSuccess) return e;
      // Wbar += B^T Dbar
      if ((e = pred(u, u->b, u->Dbar, 0, u->scr, nullptr)) != cudaSuccess) return e;
      k_add_d<<<1, 64, 0, u->s>>>(u->Wbd, u->scr, P * P, u->Wb32);
      // lbar = zeta + B o (Dbar W); Abar -= Dbar
      k_bbwd<<<g1(N), 256, 0, u->s>>>(u->zeta, u->b, u->Dbar, u->W, N, P, u->lbar, u->Abar);
    }
    // ---- A-phase: zbar(z_{t+1}) += a o (Abar + (Wbar + Wbar^T) a)
    k_zbar<<<g1(N), 256, 0, u->s>>>(u->a, u->Abar, u->Wb32, N, P, u->zbar);
    cudaMemsetAsync(u->Abar, 0, n * 4, u->s);
    // ---- reverse the A-steps from z_t with E_t = X B_t, its Gram, and c = E_t^T x
    cudaMemcpyAsync(u->l, u->lck + (size_t)t * n, n * 4, cudaMemcpyDeviceToDevice, u->s);
    k_exp<<<g1(n), 256, 0, u->s>>>(u->l, n, u->b);  // B_t
    if ((e = make_E(u, u->b)) != cudaSuccess) return e;
    k_gram<<<(u->P * u->P + 7) / 8, 256, 0, u->s>>>(u->Ed, L, P, u->G);
    if ((e = xdot(u, u->E32, 1.f, u->C)) != cudaSuccess) return e;
    {
      const int nb = nb_thr(N);
      k_a_bwd<<<nb, kT, 0, u->s>>>(u->C, u->G, etaA, u->K1, N, P, u->zck + (size_t)t * n, u->zbar, u->tmp, u->part);
      k_merge<<<merge_blocks(P * P + 1), 256, 0, u->s>>>(u->part, nb, P * P + 1, 1.0, u->Gbd, nullptr);
      k_acc_sum<<<1, 1, 0, u->s>>>(u->deta + t, u->Gbd + P * P, 1, 1.0);
    }
    // Ebar = E (Gbar + Gbar^T) + X Cbar^T ; Xbar += E Cbar + Ebar B^T ; lbar += B o (X^T Ebar)
    if ((e = xw(u, u->tmp, u->XCd, nullptr)) != cudaSuccess) return e;
    k_ebar<<<g1(lp), 256, 0, u->s>>>(u->Ed, u->Gbd, u->XCd, L, P, u->Eb32);
    if ((e = rank(u, u->E32, u->tmp, 1.f, u->Eb32, u->b, 1.f)) != cudaSuccess) return e;
    if ((e = xdot(u, u->Eb32, 1.f, u->d)) != cudaSuccess) return e;
    k_fma_inplace<<<g1(n), 256, 0, u->s>>>(u->lbar, u->b, u->d, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Runs body on the engine's stream: captured into *g on the first call,
// replayed afterwards.
template <class F>
cudaError_t run_captured(edaa_unrolled* u, cudaGraphExec_t* g, F&& body) {
  if (!*g) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(u->s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t eb = body();
    e = cudaStreamEndCapture(u->s, &graph);
    if (eb != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return eb;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(g, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      *g = nullptr;
      return e;
    }
  }
  return cudaGraphLaunch(*g, u->s);
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
  const size_t n = (size_t)N * p, lp = (size_t)L * p;
  Buf& B = u->buf;
  u->X = B.get<float>((size_t)N * L);
  u->zck = B.get<float>((size_t)(T + 1) * n);
  u->lck = B.get<float>((size_t)(T + 1) * n);
  u->z = B.get<float>(n); u->l = B.get<float>(n); u->b = B.get<float>(n); u->a = B.get<float>(n);
  u->C = B.get<float>(n); u->g = B.get<float>(n); u->d = B.get<float>(n);
  u->part = B.get<float>((size_t)kBlocks * std::max<size_t>(lp, (size_t)2 * p * p + 2 * p + 1) + 64);
  u->G = B.get<float>(64); u->W = B.get<float>(64); u->E32 = B.get<float>(lp); u->R32 = B.get<float>(lp);
  u->Ed = B.get<double>(lp); u->Wd = B.get<double>(64); u->Rd = B.get<double>(lp); u->lse = B.get<double>(8);
  u->scr = B.get<double>(lp);
  u->ls = B.get<float>((size_t)(K2 + 1) * n); u->gs = B.get<float>((size_t)std::max(K2, 1) * n);
  u->Rs = B.get<float>((size_t)std::max(K2, 1) * lp); u->deta = B.get<double>((size_t)2 * T);
  u->eta = B.get<float>((size_t)2 * T); u->dAin = B.get<float>(n);
  u->lbar = B.get<float>(n); u->zbar = B.get<float>(n); u->Abar = B.get<float>(n);
  u->Xbar = B.get<float>((size_t)N * L); u->zeta = B.get<float>(n); u->Dbar = B.get<float>(n);
  u->bp = B.get<float>(n); u->tmp = B.get<float>(n); u->P32 = B.get<float>(lp); u->Eb32 = B.get<float>(lp);
  u->Wb32 = B.get<float>(64); u->Gb32 = B.get<float>(72);
  u->sd = B.get<double>(8); u->XCd = B.get<double>(lp); u->Gbd = B.get<double>(72); u->Pd = B.get<double>(lp);
  u->Wbd = B.get<double>(64); u->eta_scr = B.get<double>(8);
  if (B.err != cudaSuccess) {
    edaa_unrolled_destroy(u);
    return ufail(EDAA_ERR_OOM, "cudaMalloc failed in edaa_unrolled_create");
  }
  *out = u;
  return EDAA_OK;
}

void edaa_unrolled_destroy(edaa_unrolled* u) {
  if (!u) return;
  if (u->s) cudaStreamSynchronize(u->s);
  if (u->g_fwd) cudaGraphExecDestroy(u->g_fwd);
  if (u->g_bwd) cudaGraphExecDestroy(u->g_bwd);
  if (u->ev_in) cudaEventDestroy(u->ev_in);
  if (u->ev_out) cudaEventDestroy(u->ev_out);
  if (u->s) cudaStreamDestroy(u->s);
  delete u;
}

edaa_status edaa_unrolled_forward(edaa_unrolled* u, const float* X, uint64_t seed, const double* eta_A,
                                  const double* eta_B, float* E_out, float* A_out) {
  if (!u || !X || !eta_A || !eta_B) return ufail(EDAA_ERR_ARG, "edaa_unrolled_forward: NULL argument");
  const int N = u->N, P = u->P, L = u->L, n = N * P;
  std::vector<float> eta(2 * u->T);
  for (int t = 0; t < u->T; ++t) {
    eta[t] = (float)eta_A[t];
    eta[u->T + t] = (float)eta_B[t];
  }
  // our stream follows the caller's
  UCK(cudaEventRecord(u->ev_in, u->caller), "order after the caller's stream");
  UCK(cudaStreamWaitEvent(u->s, u->ev_in, 0), "order after the caller's stream");
  UCK(cudaMemcpyAsync(u->eta, eta.data(), eta.size() * sizeof(float), cudaMemcpyHostToDevice, u->s), "copy eta");
  UCK(cudaMemcpyAsync(u->X, X, (size_t)N * L * 4, cudaMemcpyDefault, u->s), "copy X");
  // A^0 = 1/p (eq. initA0): z = -log p; B^0 = softmax(0.1 u) (eq. initB0)
  k_fill<<<g1(n), 256, 0, u->s>>>(u->z, n, -logf((float)P));
  k_init_logits<<<g1(n), 256, 0, u->s>>>(seed, N, P, u->l);
  UCK(normalise_logits(u, u->l, u->b), "init logits");
  UCK(run_captured(u, &u->g_fwd, [&] { return forward_body(u); }), "forward");
  if (E_out) UCK(cudaMemcpyAsync(E_out, u->E32, (size_t)L * P * 4, cudaMemcpyDefault, u->s), "copy E");
  if (A_out) UCK(cudaMemcpyAsync(A_out, u->tmp, (size_t)n * 4, cudaMemcpyDefault, u->s), "copy A");
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
  std::vector<double> deA(u->T, 0.0), deB(u->T, 0.0);
  UCK(cudaEventRecord(u->ev_in, u->caller), "order after the caller's stream");
  UCK(cudaStreamWaitEvent(u->s, u->ev_in, 0), "order after the caller's stream");
  // the adjoints of the outputs (zeros when absent) go into the engine's buffers
  if (dE) UCK(cudaMemcpyAsync(u->Eb32, dE, (size_t)lp * 4, cudaMemcpyDefault, u->s), "copy dE");
  else UCK(cudaMemsetAsync(u->Eb32, 0, (size_t)lp * 4, u->s), "zero");
  if (dA) UCK(cudaMemcpyAsync(u->dAin, dA, (size_t)n * 4, cudaMemcpyDefault, u->s), "copy dA");
  else UCK(cudaMemsetAsync(u->dAin, 0, (size_t)n * 4, u->s), "zero");
  UCK(run_captured(u, &u->g_bwd, [&] { return backward_body(u); }), "backward");
  if (dX) UCK(cudaMemcpyAsync(dX, u->Xbar, (size_t)N * L * 4, cudaMemcpyDefault, u->s), "copy dX");
  UCK(cudaMemcpyAsync(deA.data(), u->deta, u->T * sizeof(double), cudaMemcpyDeviceToHost, u->s), "copy");
  UCK(cudaMemcpyAsync(deB.data(), u->deta + u->T, u->T * sizeof(double), cudaMemcpyDeviceToHost, u->s), "copy");
  UCK(cudaStreamSynchronize(u->s), "sync");
  UCK(cudaEventRecord(u->ev_out, u->s), "order the caller's stream after ours");
  UCK(cudaStreamWaitEvent(u->caller, u->ev_out, 0), "order the caller's stream after ours");
  if (d_eta_A) for (int t = 0; t < u->T; ++t) d_eta_A[t] = deA[t];
  if (d_eta_B) for (int t = 0; t < u->T; ++t) d_eta_B[t] = deB[t];
  return EDAA_OK;
}

}  // extern "C"
