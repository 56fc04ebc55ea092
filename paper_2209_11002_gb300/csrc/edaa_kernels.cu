// CUDA kernels of EDAA (arXiv 2209.11002) for sm_103a, CUDA-core FP32 path.
//
// One X pass per A-phase and one per B-step (Algorithm 1):
//   A-pass (eq. update_A): pixel i needs only x_i, E and E^T E, so the K1
//     A-steps of an outer iteration run in registers during one stream of X,
//     and the same pass accumulates X A^T and A A^T for the B-phase.
//   B-pass (eq. update_B): the B-gradient row of pixel i is x_i^T R with
//     R = E (A A^T) - X A^T, so one stream of X updates the logits u_i,
//     and the softmax over all N pixels of each column of B is merged across
//     CTAs online (running max + rescaled sums), giving E = X B for the next
//     step from the same pass.
// Every pass is followed by a deterministic FP64 merge of per-CTA partials
// (fixed order, no float atomics on results).  All phases live in one
// program kernel so that a whole solve can run as one persistent launch with
// bounded grid barriers, or one launch per phase replayed from a CUDA graph.
#include <math.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include <mutex>

#include "edaa_pass.cuh"

namespace edaa {

__device__ void pass_phase(const Batch* __restrict__ bt, int ph, float* smem) {
  for (int item = blockIdx.x; item < bt->pass_items; item += gridDim.x) {
    int ci = 0;
    while (ci + 1 < bt->n_cubes && item >= bt->c[ci + 1].cta0) ++ci;
    const CubeDev& cd = bt->c[ci];
    const int local = item - cd.cta0;
    const int rg = local / cd.Pg, pg = local - rg * cd.Pg;
    switch (cd.p) {
      case 1: pass_dispatch<1>(bt, cd, rg, pg, smem, ph); break;
      case 2: pass_dispatch<2>(bt, cd, rg, pg, smem, ph); break;
      case 3: pass_dispatch<3>(bt, cd, rg, pg, smem, ph); break;
      case 4: pass_dispatch<4>(bt, cd, rg, pg, smem, ph); break;
      case 5: pass_dispatch<5>(bt, cd, rg, pg, smem, ph); break;
      case 6: pass_dispatch<6>(bt, cd, rg, pg, smem, ph); break;
      case 7: pass_dispatch<7>(bt, cd, rg, pg, smem, ph); break;
      default: pass_dispatch<8>(bt, cd, rg, pg, smem, ph); break;
    }
  }
}

// ---------------------------------------------------------------------------
// Merges (one work item = one run m and a chunk of bands), FP64, fixed order.
// ---------------------------------------------------------------------------
// K-major copy of a panel for the tensor-core passes: row c (column of E or R),
// band l, in the compute type (TF32 rounded to nearest, or BF16)
__device__ __forceinline__ void store_panel(const CubeDev& cd, void* panel, int c, int l, double v) {
  const size_t o = (size_t)c * cd.tc_kp + l;
  if (cd.tc == 2) {
    reinterpret_cast<__nv_bfloat16*>(panel)[o] = __float2bfloat16_rn((float)v);
  } else {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)v));
    reinterpret_cast<float*>(panel)[o] = __uint_as_float(r);
  }
}

// rho[lc][c] = sum over the chunk's bands of E[l][c] R[l][c], in a fixed
// order (lanes strided over the bands, then a butterfly): the reference
// exponent of the next B-pass is derived from these sums.
__device__ void chunk_rho(const CubeDev& cd, int m, int lc, int nl, const double* sprod) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, P = cd.p;
  if (warp < P) {
    double s = 0.0;
    for (int li = lane; li < nl; li += 32) s += sprod[li * P + warp];
    s = warp_sum_d(s);
    if (lane == 0) cd.rho[(size_t)lc * cd.Mp + m * P + warp] = s;
  }
  __syncthreads();
}

// Sum over the Pg per-CTA partials of one element (stride apart), each
// scaled by scale[g * sstride] when scale is given.  Eight independent
// chains keep eight loads in flight; they are combined in a fixed tree, so
// the result does not depend on the launch mode.
__device__ __forceinline__ double sum_partials(const float* __restrict__ v, size_t stride, int Pg,
                                               const double* scale, int sstride) {
  double c[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int g = 0;
  for (; g + 8 <= Pg; g += 8) {
    float x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = v[(size_t)(g + q) * stride];
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] += (scale ? scale[(g + q) * sstride] : 1.0) * (double)x[q];
  }
  for (int q = 0; g < Pg; ++g, ++q) c[q] += (scale ? scale[g * sstride] : 1.0) * (double)v[(size_t)g * stride];
  return ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
}

__device__ void merge_a_unit(const CubeDev& cd, int m, int lc, float* smem) {
  const int tid = threadIdx.x;
  const int P = cd.p, L = cd.L, Mp = cd.Mp, Pg = cd.Pg;
  double* saat = reinterpret_cast<double*>(smem);  // P*P
  double* sx = saat + 64;                          // lchunk * P
  double* sprod = sx + cd.lchunk * P;              // lchunk * P: E R products
  for (int e = tid; e < P * P; e += kThreads) {
    double s = 0.0;
    s += sum_partials(cd.paa + (size_t)m * P * P + e, (size_t)cd.M * P * P, Pg, nullptr, 0);
    saat[e] = s;
    if (lc == 0) cd.AAt[(size_t)m * P * P + e] = s;
  }
  const int l0 = lc * cd.lchunk, nl = min(cd.lchunk, L - l0);
  const double aref = (double)(1.f / (float)P);
  for (int e = tid; e < nl * P; e += kThreads) {
    const int l = l0 + e / P, j = e - (e / P) * P;
    double s = aref * cd.sx[l];  // shifted accumulation: add back (1/p) sum_i x_i
    s += sum_partials(cd.part + (size_t)l * Mp + m * P + j, (size_t)(L + 1) * Mp, Pg, nullptr, 0);
    cd.XAt[(size_t)l * Mp + m * P + j] = s;
    sx[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < nl * P; e += kThreads) {
    const int l = l0 + e / P, j = e - (e / P) * P;
    double r = -sx[e];
    for (int k = 0; k < P; ++k) r += cd.Ed[(size_t)l * Mp + m * P + k] * saat[k * P + j];
    cd.Rf[(size_t)l * Mp + m * P + j] = (float)r;
    if (cd.tc) store_panel(cd, cd.panelR, m * P + j, l, r);
    sprod[e] = cd.Ed[(size_t)l * Mp + m * P + j] * r;
  }
  __syncthreads();
  chunk_rho(cd, m, lc, nl, sprod);
}

__device__ void merge_b_unit(const CubeDev& cd, int m, int lc, float* smem, bool init) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = cd.p, L = cd.L, Mp = cd.Mp, Pg = cd.Pg;
  double* sS = reinterpret_cast<double*>(smem);  // kMaxP: softmax denominators
  double* sW = sS + kMaxP;                        // kMaxP: w_ref / S
  double* sE = sW + kMaxP;                        // lchunk * P
  double* sprod = sE + cd.lchunk * P;             // lchunk * P: E R products
  double* sscale = sprod + cd.lchunk * P;         // Pg * P
  (void)init;
  const double logN = log((double)cd.N);
  if (warp < P) {
    // pmax holds each CTA's power-of-two exponent e_g: its weights are e^u 2^-e_g
    const int j = warp, c = m * P + j;
    float mx = -EDAA_INF;
    for (int g = lane; g < Pg; g += 32) mx = fmaxf(mx, cd.pmax[(size_t)g * Mp + c]);
    mx = warp_max(mx);
    double S = 0.0;
    for (int g = lane; g < Pg; g += 32) {
      const float eg = cd.pmax[(size_t)g * Mp + c];
      const double f = (eg == -EDAA_INF) ? 0.0 : ldexp(1.0, (int)(eg - mx));  // exact
      sscale[g * P + j] = f;
      S += f * (double)cd.part[((size_t)g * (L + 1) + L) * Mp + c];
    }
    S = warp_sum_d(S);
    if (lane == 0) {
      // shifted accumulation: every pixel contributed w - 2^(k-e_g), i.e.
      // 2^(k-mx) in the merged frame; add N * 2^(k-mx) back to the denominator
      const double wref = ldexp(1.0, cd.bref[c] - (int)mx);
      S += wref * (double)cd.N;
      sS[j] = S;
      sW[j] = wref / S;
      // stored logits live in the frame log(N b): keep lse - log N (small near uniform B)
      if (lc == 0) cd.lse[c] = (float)((double)mx * 0.69314718055994531 + log(S) - logN);
    }
  }
  __syncthreads();
  for (int e = tid; e < Pg * P; e += kThreads) sscale[e] /= sS[e % P];
  __syncthreads();
  const int l0 = lc * cd.lchunk, nl = min(cd.lchunk, L - l0);
  for (int e = tid; e < nl * P; e += kThreads) {
    const int l = l0 + e / P, j = e - (e / P) * P;
    double s = sW[j] * cd.sx[l];
    s += sum_partials(cd.part + (size_t)l * Mp + m * P + j, (size_t)(L + 1) * Mp, Pg, sscale + j, P);
    cd.Ed[(size_t)l * Mp + m * P + j] = s;
    cd.Ef[(size_t)l * Mp + m * P + j] = (float)s;
    if (cd.tc) store_panel(cd, cd.panelE, m * P + j, l, s);
    sE[e] = s;
  }
  __syncthreads();
  // G = E^T E of run m over this chunk's bands, bands in order (the tensor-core
  // A-pass sums the chunks; the CUDA-core A-pass forms G from its staged panel)
  for (int e = tid; e < P * P; e += kThreads) {
    const int j = e / P, k = e - j * P;
    double g = 0.0;
    for (int li = 0; li < nl; ++li) g += sE[li * P + j] * sE[li * P + k];
    cd.gpart[((size_t)lc * cd.M + m) * P * P + e] = g;
  }
  for (int e = tid; e < nl * P; e += kThreads) {
    const int li = e / P, l = l0 + li, j = e - li * P;
    double r = -cd.XAt[(size_t)l * Mp + m * P + j];
    for (int k = 0; k < P; ++k) r += sE[li * P + k] * cd.AAt[(size_t)m * P * P + k * P + j];
    cd.Rf[(size_t)l * Mp + m * P + j] = (float)r;
    if (cd.tc) store_panel(cd, cd.panelR, m * P + j, l, r);
    sprod[e] = sE[e] * r;
  }
  __syncthreads();
  chunk_rho(cd, m, lc, nl, sprod);
}

__device__ void merge_phase(const Batch* __restrict__ bt, int ph, float* smem) {
  for (int u = blockIdx.x; u < bt->merge_units; u += gridDim.x) {
    int ci = 0;
    while (ci + 1 < bt->n_cubes && u >= bt->c[ci + 1].unit0) ++ci;
    const CubeDev& cd = bt->c[ci];
    const int local = u - cd.unit0;
    const int m = local / cd.nlchunk, lc = local - m * cd.nlchunk;
    if (ph == PH_AM) merge_a_unit(cd, m, lc, smem);
    else merge_b_unit(cd, m, lc, smem, ph == PH_BM0);
  }
}

// ---------------------------------------------------------------------------
// Per-run scalar phases: step sizes (eqs. eta0A, eta0B) and fit/coherence.
// ---------------------------------------------------------------------------
// Largest eigenvalue of a symmetric p x p matrix by the cyclic Jacobi method
// (plane rotations that zero one off-diagonal entry at a time, Golub & Van
// Loan, "Matrix Computations", Sec. 8.5).
__device__ double jacobi_max_eig(double* a, int n) {
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += a[i * n + i] * a[i * n + i];
      for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
    }
    if (off <= 1e-30 * diag || off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (apq == 0.0) continue;
        const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
      }
    }
  }
  double mx = a[0];
  for (int i = 1; i < n; ++i) mx = fmax(mx, a[i * n + i]);
  return mx;
}

__device__ void eta_phase(const Batch* __restrict__ bt) {
  for (int g = blockIdx.x * kThreads + threadIdx.x; g < bt->total_runs; g += gridDim.x * kThreads) {
    int ci = 0;
    while (ci + 1 < bt->n_cubes && g >= bt->c[ci + 1].run0) ++ci;
    const CubeDev& cd = bt->c[ci];
    const int m = g - cd.run0, P = cd.p;
    double G[kMaxP * kMaxP];
    for (int e = 0; e < P * P; ++e) G[e] = 0.0;
    for (int l = 0; l < cd.L; ++l) {  // E^0 = X B^0 with the mean pixel added back
      const double* e = cd.Ed + (size_t)l * cd.Mp + m * P;
      const double xb = cd.xbar[l];
      for (int j = 0; j < P; ++j)
        for (int k = 0; k < P; ++k) G[j * P + k] += (e[j] + xb) * (e[k] + xb);
    }
    const double s2 = jacobi_max_eig(G, P);
    const double e1 = cd.gammas[m] / s2;
    const double e2 = sqrt((double)P / (double)cd.N) * e1;
    cd.sig2[m] = s2;
    cd.eta1d[m] = e1;
    cd.eta2d[m] = e2;
    cd.eta1[m] = (float)e1;
    cd.eta2[m] = (float)e2;
  }
}

__device__ void fitm_phase(const Batch* __restrict__ bt) {
  for (int g = blockIdx.x * kThreads + threadIdx.x; g < bt->total_runs; g += gridDim.x * kThreads) {
    int ci = 0;
    while (ci + 1 < bt->n_cubes && g >= bt->c[ci + 1].run0) ++ci;
    const CubeDev& cd = bt->c[ci];
    const int m = g - cd.run0, P = cd.p;
    double a1 = 0.0, am = 0.0, a2 = 0.0;
    for (int q = 0; q < cd.Pg; ++q) {
      const double* s = cd.pfit + ((size_t)q * cd.M + m) * 3;
      a1 += s[0];
      am = fmax(am, s[1]);
      a2 += s[2];
    }
    cd.fit[m] = a1;
    cd.fitmax[m] = am;
    cd.loss2[m] = a2;
    // coherence (eq. coherence) from the FP64 copy of E
    double G[kMaxP * kMaxP];
    for (int e = 0; e < P * P; ++e) G[e] = 0.0;
    for (int l = 0; l < cd.L; ++l) {  // uncentred E = E_c + xbar 1^T
      const double* e = cd.Ed + (size_t)l * cd.Mp + m * P;
      const double xb = cd.xbar[l];
      for (int j = 0; j < P; ++j)
        for (int k = j; k < P; ++k) G[j * P + k] += (e[j] + xb) * (e[k] + xb);
    }
    double mu = -INFINITY;
    for (int j = 0; j < P; ++j)
      for (int k = j + 1; k < P; ++k) {
        double v = G[j * P + k];
        if (bt->coh_mode == 0) {
          const double d = sqrt(G[j * P + j]) * sqrt(G[k * P + k]);
          v = d > 0.0 ? v / d : 0.0;
        }
        mu = fmax(mu, v);
      }
    cd.mu[m] = mu;
  }
}

// ---------------------------------------------------------------------------
// The program kernel.
// ---------------------------------------------------------------------------
__host__ __device__ inline int phase_of(int mode, int s, int K2) {
  if (mode == MODE_INIT) {
    const int seq[5] = {PH_INITB, PH_BM0, PH_ETA, PH_INITA, PH_AM};
    return seq[s];
  }
  if (mode == MODE_FIT) return s == 0 ? PH_FIT : PH_FITM;
  const int per = 2 + 2 * K2;
  const int k = s % per;
  if (k == 0) return PH_A;
  if (k == 1) return PH_AM;
  return (k & 1) ? PH_BM : PH_B;
}

int program_phase_count(int mode, int n_outer, int K2) {
  if (mode == MODE_INIT) return 5;
  if (mode == MODE_FIT) return 2;
  return n_outer * (2 + 2 * K2);
}

__global__ void __launch_bounds__(kThreads, 1)
k_edaa(const Batch* __restrict__ bt, int mode, int n_outer, int ph_lo, int ph_hi) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  (void)n_outer;
  for (int s = ph_lo; s < ph_hi; ++s) {
    if (s > ph_lo) {
      if (!grid_barrier(bt->bar, gridDim.x, bt->status, bt->timeout_ns)) return;
    }
    const int ph = phase_of(mode, s, bt->K2);
    switch (ph) {
      case PH_A:
      case PH_B:
      case PH_INITA:
      case PH_INITB:
      case PH_FIT: pass_phase(bt, ph, smem); break;
      case PH_AM:
      case PH_BM:
      case PH_BM0: merge_phase(bt, ph, smem); break;
      case PH_ETA: eta_phase(bt); break;
      case PH_FITM: fitm_phase(bt); break;
      default: break;
    }
  }
}

// The attribute is per kernel and process-wide: several contexts may coexist,
// so it only ever grows (a smaller request keeps the larger setting).
cudaError_t set_program_smem(size_t smem) {
  static std::mutex mu;
  static size_t current = 0;
  std::lock_guard<std::mutex> lock(mu);
  if (smem <= current) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_edaa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) current = smem;
  return e;
}

cudaError_t program_occupancy(int* blocks_per_sm, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_edaa, kThreads, smem);
}

cudaError_t launch_program(const Batch* d_batch, int mode, int n_outer, int ph_lo, int ph_hi, int grid,
                           size_t smem, bool cooperative, cudaStream_t stream) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)grid);
  lc.blockDim = dim3(kThreads);
  lc.dynamicSmemBytes = smem;
  lc.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = cooperative ? 1 : 0;
  return cudaLaunchKernelEx(&lc, k_edaa, d_batch, mode, n_outer, ph_lo, ph_hi);
}

// ---------------------------------------------------------------------------
// Auxiliary kernels: normalisation (eq. normalization), gradients, gathers,
// barrier self-test.
// ---------------------------------------------------------------------------
// eq. (normalization): x_i <- x_i / ||x_i||_2 (a zero pixel stays zero).
// Pass 1 (one warp per pixel): the FP64 norm of every pixel and per-block FP64
// band sums of the normalised pixels (for the mean pixel, in a fixed order).
// Pass 2 writes x_i/||x_i|| - xbar rounded to float32 once, so the stored
// centred pixel carries float32 rounding relative to itself, not to x_i.
constexpr int kNormWarps = 8, kNormPix = 16;  // pixels per warp

int normalize_blocks(int N) { return (N + kNormWarps * kNormPix - 1) / (kNormWarps * kNormPix); }

__global__ void __launch_bounds__(kNormWarps * 32) k_norms(const float* __restrict__ Xin, double* __restrict__ scale,
                                                         double* __restrict__ bsum, int L, int N, int normalize) {
  extern __shared__ double shn[];  // kNormWarps x L
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int KMAX = (kMaxL + 31) / 32;
  double acc[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) acc[k] = 0.0;
  for (int q = 0; q < kNormPix; ++q) {
    const int i = (blockIdx.x * kNormWarps + w) * kNormPix + q;
    if (i >= N) break;
    const float* x = Xin + (size_t)i * L;
    double ss = 0.0;
    for (int l = lane; l < L; l += 32) ss += (double)x[l] * (double)x[l];
    ss = warp_sum_d(ss);
    const double nrm = sqrt(ss);
    const double sc = (normalize && nrm > 0.0) ? 1.0 / nrm : 1.0;
    if (lane == 0) scale[i] = sc;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int l = lane + 32 * k;
      if (l < L) acc[k] += (double)x[l] * sc;
    }
  }
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int l = lane + 32 * k;
    if (l < L) shn[w * L + l] = acc[k];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < kNormWarps; ++q) s += shn[q * L + l];
    bsum[(size_t)blockIdx.x * L + l] = s;
  }
}

__global__ void k_mean(const double* __restrict__ bsum, int nb, int L, int N, int center, double* __restrict__ xbar) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += bsum[(size_t)b * L + l];
  xbar[l] = center ? s / (double)N : 0.0;
}

__global__ void k_write_x(const float* __restrict__ Xin, const double* __restrict__ scale,
                          const double* __restrict__ xbar, float* __restrict__ X, int L, int Ls, int N) {
  const size_t n = (size_t)N * Ls;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / Ls), l = (int)(e - (size_t)i * Ls);
    float v = 0.f;
    if (l < L) v = (float)((double)Xin[(size_t)i * L + l] * scale[i] - xbar[l]);
    else if (l == L) v = 1.f;  // the ones band
    X[e] = v;
  }
}

// Per-block band sums (FP64) of the stored X, for sum_i x_i after centring.
__global__ void __launch_bounds__(kNormWarps * 32) k_colsum(const float* __restrict__ X, double* __restrict__ bsum,
                                                          int L, int Ls, int N) {
  extern __shared__ double shn[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int KMAX = (kMaxL + 31) / 32;
  double acc[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) acc[k] = 0.0;
  for (int q = 0; q < kNormPix; ++q) {
    const int i = (blockIdx.x * kNormWarps + w) * kNormPix + q;
    if (i >= N) break;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int l = lane + 32 * k;
      if (l < L) acc[k] += (double)X[(size_t)i * Ls + l];
    }
  }
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int l = lane + 32 * k;
    if (l < L) shn[w * L + l] = acc[k];
  }
  __syncthreads();
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < kNormWarps; ++q) s += shn[q * L + l];
    bsum[(size_t)blockIdx.x * L + l] = s;
  }
}

__global__ void k_sum(const double* __restrict__ bsum, int nb, int L, int N, double* __restrict__ sx) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > L) return;
  if (l == L) {
    sx[L] = (double)N;  // the ones band
    return;
  }
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += bsum[(size_t)b * L + l];
  sx[l] = s;
}

cudaError_t launch_normalize(const float* Xin, float* X, double* scale, double* bsum, double* xbar, double* sx,
                             int L, int Ls, int N, int normalize, int center, cudaStream_t s) {
  const int nb = normalize_blocks(N);
  const size_t sh = kNormWarps * L * sizeof(double);
  k_norms<<<nb, kNormWarps * 32, sh, s>>>(Xin, scale, bsum, L, N, normalize);
  k_mean<<<(L + 127) / 128, 128, 0, s>>>(bsum, nb, L, N, center, xbar);
  k_write_x<<<1024, 256, 0, s>>>(Xin, scale, xbar, X, L, Ls, N);
  k_colsum<<<nb, kNormWarps * 32, sh, s>>>(X, bsum, L, Ls, N);
  k_sum<<<(L + 128) / 128, 128, 0, s>>>(bsum, nb, L, N, sx);
  return cudaGetLastError();
}

// Gradients of ||X - X B A||_F^2 at the current state, in the paper's
// uncentred terms: gA_i = 2 E^T (E a_i - x_i) with E = E_c + xbar 1^T (the
// residual E a_i - x_i equals E_c a_i - x_c,i because a_i sums to 1), and
// gB_i = 2 x_i^T R with x_i = x_c,i + xbar.  gA is p x N, gB is N x p.
__global__ void k_grad(const CubeDev* __restrict__ cdp, int m, float* gA, float* gB) {
  const CubeDev& cd = *cdp;
  const int P = cd.p, L = cd.L, Mp = cd.Mp;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cd.N) return;
  const float* x = cd.X + (size_t)i * cd.Ls;
  float a[kMaxP], ga[kMaxP], gb[kMaxP];
  float se = 0.f;
  for (int j = 0; j < P; ++j) {
    a[j] = expf(cd.logA[(size_t)(m * P + j) * cd.Nst + i]);
    se += a[j];
    ga[j] = 0.f;
    gb[j] = 0.f;
  }
  for (int j = 0; j < P; ++j) a[j] /= se;
  for (int l = 0; l < L; ++l) {
    const float* e = cd.Ef + (size_t)l * Mp + m * P;
    const float* r = cd.Rf + (size_t)l * Mp + m * P;
    const float xb = (float)cd.xbar[l];
    float res = -x[l];
    for (int k = 0; k < P; ++k) res = fmaf(e[k], a[k], res);
    for (int j = 0; j < P; ++j) {
      ga[j] = fmaf(e[j] + xb, res, ga[j]);
      gb[j] = fmaf(x[l] + xb, r[j], gb[j]);
    }
  }
  for (int j = 0; j < P; ++j) {
    if (gA) gA[(size_t)j * cd.N + i] = 2.f * ga[j];
    if (gB) gB[(size_t)i * P + j] = 2.f * gb[j];
  }
}

cudaError_t launch_grad(const CubeDev* d_cube, const CubeDev& hc, int run, float* gA, float* gB, cudaStream_t s) {
  k_grad<<<(hc.N + 255) / 256, 256, 0, s>>>(d_cube, run, gA, gB);
  return cudaGetLastError();
}

__global__ void k_gather_e(const double* Ed, const double* xbar, int L, int Mp, int p, int m, float* E) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= L * p) return;
  const int l = e / p, j = e % p;
  E[e] = (float)(Ed[(size_t)l * Mp + m * p + j] + xbar[l]);
}
__global__ void k_gather_ab(const float* logA, const float* logB, const float* lse, int N, int Nst, int p, int m,
                            float* A, float* B) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * p) return;
  const int i = e / p, j = e % p;
  const size_t src = (size_t)(m * p + j) * Nst + i;
  if (A) {  // softmax over the p max-normalised log abundances of pixel i
    double se = 0.0;
    for (int k = 0; k < p; ++k) se += exp((double)logA[(size_t)(m * p + k) * Nst + i]);
    A[(size_t)j * N + i] = (float)(exp((double)logA[src]) / se);
  }
  if (B) B[e] = (float)exp((double)logB[src] - (double)lse[m * p + j] - log((double)N));
}

cudaError_t launch_gather(const CubeDev& hc, int run, float* E, float* A, float* B, cudaStream_t s) {
  if (E) k_gather_e<<<(hc.L * hc.p + 255) / 256, 256, 0, s>>>(hc.Ed, hc.xbar, hc.L, hc.Mp, hc.p, run, E);
  if (A || B) k_gather_ab<<<(hc.N * hc.p + 255) / 256, 256, 0, s>>>(hc.logA, hc.logB, hc.lse, hc.N, hc.Nst, hc.p, run, A, B);
  return cudaGetLastError();
}

// Compute-type copies of the centred X for the tensor-core passes:
// Xk: N x kp pixel-major (bands >= L+1 zero), XT: (L+1) x Npad band-major
// (row L is the ones band), TF32 rounded to nearest or BF16.
__global__ void k_tc_prepare(const float* __restrict__ X, int L, int Ls, int N, int kp, int Npad, int bf16,
                             void* __restrict__ Xk, void* __restrict__ XT) {
  const size_t n = (size_t)N * kp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / kp), l = (int)(e - (size_t)i * kp);
    const float v = (l < Ls) ? X[(size_t)i * Ls + l] : 0.f;
    if (bf16) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      reinterpret_cast<__nv_bfloat16*>(Xk)[e] = h;
      if (l <= L) reinterpret_cast<__nv_bfloat16*>(XT)[(size_t)l * Npad + i] = h;
    } else {
      uint32_t r;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
      reinterpret_cast<float*>(Xk)[e] = __uint_as_float(r);
      if (l <= L) reinterpret_cast<float*>(XT)[(size_t)l * Npad + i] = __uint_as_float(r);
    }
  }
}

cudaError_t launch_tc_prepare(const CubeDev& hc, void* Xk, void* XT, int Npad, cudaStream_t s) {
  k_tc_prepare<<<1024, 256, 0, s>>>(hc.X, hc.L, hc.Ls, hc.N, hc.tc_kp, Npad, hc.tc == 2 ? 1 : 0, Xk, XT);
  return cudaGetLastError();
}

__global__ void k_barrier_test(unsigned* bar, int* status, unsigned expected, long long timeout_ns) {
  grid_barrier(bar, expected, status, timeout_ns);
}

cudaError_t launch_barrier_test(unsigned* bar, int* status, int grid, int expected, long long timeout_ns,
                                cudaStream_t s) {
  k_barrier_test<<<grid, 64, 0, s>>>(bar, status, (unsigned)expected, timeout_ns);
  return cudaGetLastError();
}

}  // namespace edaa
