// Device code of the streaming passes (A-pass, B-pass, fit pass), included by
// the per-p translation units edaa_pass_p.cu (compiled once per p = 1..8) and
// by edaa_kernels.cu for the shared helpers.
#pragma once
#include <math.h>
#include <stdint.h>

#include "edaa_internal.cuh"

namespace edaa {

#define EDAA_INF __int_as_float(0x7f800000)

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// order-preserving float <-> int map for atomicMax on floats of any sign
__device__ __forceinline__ int ord_key(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord_val(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// The B-pass keeps its online-softmax maximum as a power-of-two exponent e
// (weights e^u 2^-e), so every rescale between tiles and CTAs and the shifted
// reference weight 2^-e are exact powers of two: the merge can then add the
// reference term back without any rounding mismatch.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;
__device__ __forceinline__ float tile_exp(int key) {
  const float m = ord_val(key);
  return m == -EDAA_INF ? m : ceilf(m * kLog2e);
}

// Reference of the shifted B accumulation.  Column c subtracts the weight of
// the logit k ln 2 from every pixel and the merge adds N 2^k back.  Near
// uniform B (logits near 0) k = 0, so the summands are the small deviations
// from uniform.  Far from uniform, logit 0 can sit far above every logit of
// the column, and a reference of 2^0 would then dwarf the sum it is taken
// from; so k is capped by a lower bound of log mean_i e^{u_i} that is known
// before the pass.  With u_i = log(N b_i) - eta2 c_i, c = X^T R, Jensen's
// inequality under the weights b gives
//     log mean_i e^{u_i} = log sum_i b_i e^{-eta2 c_i} >= -eta2 sum_i b_i c_i
//                        = -eta2 E_c^T R_c,            E = X B, eq. (update_B),
// hence N 2^k <= sqrt(2) sum_i e^{u_i}: no overflow and no cancellation worse
// than a factor of about two.  The per-chunk sums are added in a fixed order,
// so every CTA and the merge compute the same k.
__device__ __forceinline__ int ref_exponent(const CubeDev& cd, int m, int c) {
  double s = 0.0;
  for (int lc0 = 0; lc0 < cd.nlchunk; lc0 += 8) {  // loads in batches, sum in chunk order
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = lc0 + u < cd.nlchunk ? cd.rho[(size_t)(lc0 + u) * cd.Mp + c] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (lc0 + u < cd.nlchunk) s += v[u];
  }
  const double t = -cd.eta2d[m] * s * 1.4426950408889634;
  if (!(fabs(t) < 16384.0)) return t < 0.0 ? -16384 : 0;  // also non-finite
  return (int)rint(t);
}

// The same with the column's powers of two precomputed: p2 = 2^-Mn and
// p2k = 2^(k-Mn) (a product with an exact power of two is the single rounding
// ldexpf makes, down to the subnormal range).
__device__ __forceinline__ float shifted_weight_p2(float u, float Mn, float p2, int k, float p2k) {
  if (k == 0) return (fabsf(u) < 1.f) ? expm1f(u) * p2 : exp2f(fmaf(u, kLog2e, -Mn)) - p2;
  const float s = fmaf(u, kLog2e, -(float)k);
  return (fabsf(s) < 1.5f) ? expm1f(s * kLn2) * p2k : exp2f(fmaf(u, kLog2e, -Mn)) - p2k;
}

// Shifted weight of logit u in the power-of-two frame Mn with reference 2^k:
// e^u 2^-Mn - 2^(k-Mn).  Near the reference the difference is formed by
// expm1 and is exact to rounding.
__device__ __forceinline__ float shifted_weight(float u, float Mn, int k) {
  if (k == 0)
    return (fabsf(u) < 1.f) ? ldexpf(expm1f(u), -(int)Mn) : exp2f(fmaf(u, kLog2e, -Mn)) - ldexpf(1.f, -(int)Mn);
  const float s = fmaf(u, kLog2e, -(float)k);  // log2 of e^u / 2^k
  return (fabsf(s) < 1.5f) ? ldexpf(expm1f(s * kLn2), k - (int)Mn)
                           : exp2f(fmaf(u, kLog2e, -Mn)) - ldexpf(1.f, k - (int)Mn);
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number n of the
// generator seeded with `seed` is the variant-13 finaliser of seed + n*gamma.
constexpr uint64_t kSplitMixGamma = 0x9E3779B97F4A7C15ull;
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t n) {
  return splitmix64_mix(seed + n * kSplitMixGamma);
}
// u ~ U[0,1) with 24 bits, exact in float32 (eq. initB0)
__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t n) {
  return (float)(splitmix64_out(seed, n) >> 40) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// mbarrier helpers (shared by the CUDA-core and tensor-core passes)
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, int c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* b) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// bounded wait for phase `par` of the barrier; false on time-out.  The clock
// is read only once the barrier is found incomplete (completed barriers are
// the common case on the critical path).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t par, long long timeout_ns) {
  {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(par)
        : "memory");
    if (ok) return true;
  }
  const unsigned long long t0 = global_ns();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(par)
        : "memory");
    if (ok) return true;
    if ((long long)(global_ns() - t0) > timeout_ns) return false;
  }
}
// non-blocking probe of phase `par` of the barrier: true if it has completed
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t par) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(par)
      : "memory");
  return ok != 0;
}
// One bulk (TMA) copy of `bytes` contiguous bytes global -> shared, completing
// on barrier b; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(b))
               : "memory");
}

// Bounded grid barrier: generation counter + arrival counter.  A CTA that
// waits longer than timeout_ns, or sees another CTA's time-out, sets the
// status bit and returns false so that the kernel can exit; it never traps.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned expected, int* status, long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();
    const unsigned prev = atomicAdd(bar, 1u);
    if (prev + 1u == expected) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u32(bar + 1) == gen) {
        if (ld_volatile_i32(status) & kStatTimeout) { ok = 0; break; }
        if ((long long)(global_ns() - t0) > timeout_ns) {
          atomicOr(status, kStatTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// Pass work item: one CTA, one run group (Rm runs), pixel tiles pg, pg+Pg, ...
// Template: P endmembers, LT = ceil((L+1)/32) l-values per lane in phase 2.
// ---------------------------------------------------------------------------
// Slot shapes of phase 1 and the element-wise step: SW = 0 is the default
// (up to SPTM pixels x RQ1M runs per thread); SW = 4 is four pixels x one
// run.  Phase 1 reloads every operand word it multiplies through the
// shared-memory pipe, whose register write-back (one word per lane per
// cycle per SM) is the limit: a thread tile of a pixels x b columns does a*b
// FMAs per a+b words, so 4 x P4 beats 2 x 2P4 (and 1 x P4 for p > 4).
template <int P, int SW = 0>
struct PassTraits {
  static constexpr int P4 = (P + 3) & ~3;
  static constexpr int PP = P * (P + 1) / 2;
  static constexpr int RQ1M = SW == 4 ? 1 : ((P <= 2) ? 4 : (P <= 4 ? 2 : 1));  // runs per warp, phase 1
  static constexpr int SPTM = SW == 4 ? 4 : ((P <= 4) ? 2 : 1);                 // pixels per lane, phase 1
  static constexpr int RQ2M = (P <= 2) ? 4 : (P <= 4 ? 2 : 1);  // runs per warp, phase 2
};

template <int P>
__device__ __forceinline__ void load_p4(const float* src, float (&v)[PassTraits<P>::P4]) {
#pragma unroll
  for (int h = 0; h < PassTraits<P>::P4 / 4; ++h) {
    const float4 t = *reinterpret_cast<const float4*>(src + 4 * h);
    v[4 * h + 0] = t.x;
    v[4 * h + 1] = t.y;
    v[4 * h + 2] = t.z;
    v[4 * h + 3] = t.w;
  }
}

// Asynchronous global -> shared copies (cp.async): the loads of a staging loop
// are all in flight together instead of one L2 round trip per iteration.
// With valid == false nothing is read and the destination is zero-filled.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                   static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// N floats (a multiple of 4) from 16-byte-aligned shared memory; volatile so
// that the compiler re-issues the load where it is written rather than
// keeping the values live in registers across a loop.
template <int N>
__device__ __forceinline__ void lds_row(const float* src, float (&v)[N]) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(src));
#pragma unroll
  for (int h = 0; h < N / 4; ++h)
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[4 * h]), "=f"(v[4 * h + 1]), "=f"(v[4 * h + 2]), "=f"(v[4 * h + 3])
                 : "r"(a + 16 * h));
}

__device__ __forceinline__ float f4c(const float4& v, int d) {
  return d == 0 ? v.x : (d == 1 ? v.y : (d == 2 ? v.z : v.w));
}

// kind: 0 = A-pass (K1 steps; init => A^0), 1 = B-pass (init => B^0 logits)
template <int P, int LT, bool IS_A, int SW>
__device__ __noinline__ void pass_item(const Batch* __restrict__ bt, const CubeDev& cd, int rg, int pg,
                                       float* smem, int K1, bool init) {
  using TR = PassTraits<P, SW>;
  constexpr int P4 = TR::P4;
  constexpr int PP = TR::PP;
  constexpr int RQ1M = TR::RQ1M;
  constexpr int SPTM = TR::SPTM;
  constexpr int RQ2M = TR::RQ2M;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int L = cd.L, Ls = cd.Ls, Lr = cd.Lr, N = cd.N, Mp = cd.Mp, Rm = cd.Rm;
  const int m0 = rg * Rm;
  const int nr = min(Rm, cd.M - m0);
  const int c0 = m0 * P, nc = nr * P;
  const int Nt = cd.Nt;
  const int WP1 = cd.WP1, WR1 = kWarps / WP1, SPT = cd.SPT;
  const int WP2 = cd.WP2, WR2 = kWarps / WP2;
  const int RQ1 = (Rm + WR1 - 1) / WR1, RQ2 = (Rm + WR2 - 1) / WR2;
  const PassSmem sm = pass_smem(L, Ls, Lr, P, Rm, Nt);
  float* Ps = smem + sm.off_ps;
  float* Gs = smem + sm.off_gs;
  float* Xs = smem + sm.off_xs;
  float* Ss = smem + sm.off_ss;
  float* Ws = smem + sm.off_ws;
  float* colLse = smem + sm.off_col;
  float* colM = colLse + sm.RgS4;
  int* colKey = reinterpret_cast<int*>(colM + sm.RgS4);
  int* colRef = colKey + sm.RgS4;  // B: reference exponent k of the shifted weights
  float* colP2 = reinterpret_cast<float*>(colRef + sm.RgS4);  // B: 2^-Mn of the current tile's frame
  float* colMn = colP2 + sm.RgS4;                              // B: the current tile's frame Mn
  float* colP2k = colMn + sm.RgS4;                             // B: 2^(k-Mn)
  float* runEta = smem + sm.off_run;
  const int RgS4 = sm.RgS4, RgSo = sm.RgSo, RgW = sm.RgW;

  // ---- stage the panel (E for A, R for B), per-run step sizes, column stats
  // Panel layout: band quads, then runs, then the quad's 4 bands x P4 columns,
  // so that phase 1 reads a run's 4 x P4 block at fixed offsets from one pointer.
  const bool need_panel = !init;
  if (need_panel) {
    const float* panel = IS_A ? cd.Ef : cd.Rf;
    for (int e = tid; e < Lr * RgS4; e += kThreads) {
      const int l = e / RgS4, cc = e - l * RgS4, r = cc / P4, j = cc - r * P4;
      const bool v = l < L && r < nr && j < P;
      cp_async4(Ps + (l >> 2) * 4 * RgS4 + r * 4 * P4 + (l & 3) * P4 + j,
                v ? panel + (size_t)l * Mp + c0 + r * P + j : panel, v);
    }
    // completed together with the first tile's copies
  }
  if (tid < Rm) runEta[tid] = (tid < nr) ? (IS_A ? cd.eta1[m0 + tid] : cd.eta2[m0 + tid]) : 0.f;
  if (!IS_A) {
    for (int c = tid; c < RgS4; c += kThreads) {
      const int r = c / P4, j = c - r * P4;
      const bool live = r < nr && j < P;
      colLse[c] = (!init && live) ? cd.lse[c0 + r * P + j] : 0.f;
      colM[c] = -EDAA_INF;
      colKey[c] = ord_key(-EDAA_INF);
      const int k = (!init && live) ? ref_exponent(cd, m0 + r, c0 + r * P + j) : 0;
      colRef[c] = k;
      if (pg == 0 && live) cd.bref[c0 + r * P + j] = k;
    }
  }
  bool g_pending = IS_A && need_panel && K1 > 0;  // G = P^T P, formed once the panel has landed
  // the X tile arrives by one bulk copy per tile, completing on xbar
  uint64_t* xbar = reinterpret_cast<uint64_t*>(smem + sm.off_bar);
  uint32_t xpar = 0;
  if (tid == 0) {
    mbar_init(xbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int wp = warp % WP1, wr = warp / WP1;
  const int wp2 = warp % WP2, wr2 = warp / WP2;

  float acc[LT][RQ2M][P];
#pragma unroll
  for (int k = 0; k < LT; ++k)
#pragma unroll
    for (int q = 0; q < RQ2M; ++q)
#pragma unroll
      for (int j = 0; j < P; ++j) acc[k][q][j] = 0.f;
  float aa[RQ1M][PP];
#pragma unroll
  for (int q = 0; q < RQ1M; ++q)
#pragma unroll
    for (int e = 0; e < PP; ++e) aa[q][e] = 0.f;

  float* St = IS_A ? cd.logA : cd.logB;
  const float4* Xs4 = reinterpret_cast<const float4*>(Xs);
  const float aref = 1.f / (float)P;  // A reference weight

  for (int tile = pg; tile < cd.ntiles; tile += cd.Pg) {
    const int i0 = tile * Nt;
    const int ni = min(Nt, N - i0);
    {  // X tile: ni contiguous rows of Ls floats (16-byte multiples) by one bulk copy; rows >= ni zero
      float4* xs4 = reinterpret_cast<float4*>(Xs);
      const int n4 = ni * (Ls >> 2), nt4 = Nt * (Ls >> 2);
      if (tid == 0) {
        mbar_expect(xbar, (uint32_t)n4 * 16u);
        bulk_copy(xs4, cd.X + (size_t)i0 * Ls, (uint32_t)n4 * 16u, xbar);
      }
      for (int e = n4 + tid; e < nt4; e += kThreads) xs4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!init) {  // a warp per state column, lanes along the pixels
      for (int cc = warp; cc < nc; cc += kWarps) {
        const float* src = St + (size_t)(c0 + cc) * cd.Nst + i0;
        for (int i = lane; i < ni; i += 32) cp_async4(Ss + i * RgSo + cc, src + i, true);
      }
    }
    cp_async_wait_all();
    const int x_late = mbar_wait(xbar, xpar, bt->timeout_ns) ? 0 : 1;
    xpar ^= 1u;
    if (__syncthreads_or(x_late)) {
      // The X tile's bulk copy did not arrive in time: report it, give the
      // copy a bounded time to land, and end the work item without touching
      // the tile or re-arming the barrier (the host reports EDAA_ERR_TIMEOUT
      // at its next synchronising call; this pass's partials are not written).
      if (tid == 0) {
        atomicOr(bt->status, kStatTimeout);
        const unsigned long long t0 = global_ns();
        while ((long long)(global_ns() - t0) < 50000000ll) __nanosleep(1000);
        mbar_inval(xbar);
      }
      __syncthreads();
      return;
    }
    if (g_pending) {
      for (int e = tid; e < nr * P * P; e += kThreads) {
        const int r = e / (P * P), jk = e - r * P * P, j = jk / P, k = jk - j * P;
        // four interleaved partial sums (the panel rows from L to Lr are zero)
        const float* pj = Ps + r * 4 * P4 + j;
        const float* pk = Ps + r * 4 * P4 + k;
        float s4[4] = {0.f, 0.f, 0.f, 0.f};
        for (int l = 0; l < Lr; l += 4) {
#pragma unroll
          for (int u = 0; u < 4; ++u) s4[u] = fmaf(pj[l * RgS4 + u * P4], pk[l * RgS4 + u * P4], s4[u]);
        }
        Gs[(r * P + j) * P4 + k] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
      }
      __syncthreads();
      g_pending = false;
    }

    // ---- phase 1: c = P^T x_i per (pixel, run), then the element-wise update
    float cr[SPTM][RQ1M][P];
#pragma unroll
    for (int s = 0; s < SPTM; ++s)
#pragma unroll
      for (int q = 0; q < RQ1M; ++q)
#pragma unroll
        for (int j = 0; j < P; ++j) cr[s][q][j] = 0.f;
    if (need_panel && (!IS_A || K1 > 0)) {
      // Branch-free inner loop: a slot beyond SPT re-reads slot 0's pixel and
      // a run beyond the group re-reads run 0's panel columns; their sums are
      // never stored, and every load stays inside the tile and the panel.
      const float4* xrow[SPTM];
      const float* prow[RQ1M];
#pragma unroll
      for (int s = 0; s < SPTM; ++s) xrow[s] = Xs4 + (((lane + 32 * (wp + (s < SPT ? WP1 * s : 0))) * Ls) >> 2);
#pragma unroll
      for (int q = 0; q < RQ1M; ++q) {
        const int r = wr + WR1 * q;
        prow[q] = Ps + ((q < RQ1 && r < nr) ? r : 0) * 4 * P4;
      }
#pragma unroll 4
      for (int l = 0; l < Lr; l += 4) {
        float4 xv[SPTM];
#pragma unroll
        for (int s = 0; s < SPTM; ++s) xv[s] = xrow[s][l >> 2];
#pragma unroll
        for (int q = 0; q < RQ1M; ++q) {
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            float pv[P4];
            load_p4<P>(prow[q] + l * RgS4 + d * P4, pv);
#pragma unroll
            for (int s = 0; s < SPTM; ++s) {
              const float x = f4c(xv[s], d);
#pragma unroll
              for (int j = 0; j < P; ++j) cr[s][q][j] = fmaf(x, pv[j], cr[s][q][j]);
            }
          }
        }
      }
    }

    if (IS_A) {
      // eq. (update_A) in softmax form, a+ = softmax(log a - eta (G a - c)),
      // for every (pixel, run) slot of this thread.  The K1 loop is outermost
      // so that the slots' independent chains interleave.  Inactive slots
      // (beyond SPT, RQ1 or the group's runs) compute on zeros with clamped
      // indices and store nothing.
      float z[SPTM][RQ1M][P], ea[SPTM][RQ1M][P], se[SPTM][RQ1M];
#pragma unroll
      for (int s = 0; s < SPTM; ++s) {
        const int il = lane + 32 * (wp + WP1 * s);
        const bool valid = s < SPT && il < ni;
#pragma unroll
        for (int q = 0; q < RQ1M; ++q) {
          const int r = wr + WR1 * q;
          const bool act = valid && q < RQ1 && r < nr;
          // z = log a - max_j log a (max-normalised log abundances; 0 for uniform a)
          se[s][q] = 0.f;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            z[s][q][j] = (init || !act) ? 0.f : Ss[il * RgSo + r * P + j];
            ea[s][q][j] = expf(z[s][q][j]);
            se[s][q] += ea[s][q][j];
          }
        }
      }
      for (int kk = 0; kk < K1; ++kk) {
#pragma unroll
        for (int s = 0; s < SPTM; ++s)
#pragma unroll
          for (int q = 0; q < RQ1M; ++q) {
            const int r = wr + WR1 * q;
            const int rr = (q < RQ1 && r < nr) ? r : 0;
            const float* G = Gs + rr * P * P4;
            const float eta = runEta[rr];
            const float inv = 1.f / se[s][q];
            float a[P], mx = -EDAA_INF;
#pragma unroll
            for (int j = 0; j < P; ++j) a[j] = ea[s][q][j] * inv;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              // G's row j is re-read from shared memory at every step (a
              // broadcast load) instead of being held in registers
              float grow[P4];
              lds_row<P4>(G + j * P4, grow);
              float g = -cr[s][q][j];
#pragma unroll
              for (int k = 0; k < P; ++k) g = fmaf(grow[k], a[k], g);
              z[s][q][j] = fmaf(-eta, g, z[s][q][j]);
              mx = fmaxf(mx, z[s][q][j]);
            }
            se[s][q] = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              z[s][q][j] -= mx;
              ea[s][q][j] = expf(z[s][q][j]);
              se[s][q] += ea[s][q][j];
            }
          }
      }
#pragma unroll
      for (int s = 0; s < SPTM; ++s) {
        if (s >= SPT) continue;
        const int il = lane + 32 * (wp + WP1 * s);
        const bool valid = il < ni;
#pragma unroll
        for (int q = 0; q < RQ1M; ++q) {
          const int r = wr + WR1 * q;
          if (!(q < RQ1 && r < nr)) continue;
          // a_j = e^{z_j} / sum_k e^{z_k}.  The accumulated deviation a_j - 1/p is
          // formed from d = expm1(z), exact to float rounding near uniform a
          // (where a_j - 1/p itself is small): a_j - 1/p = (p d_j - sd) / (p (p + sd)).
          float d[P];
          float sd = 0.f;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            d[j] = expm1f(z[s][q][j]);
            sd += d[j];
          }
          const float den = 1.f / ((float)P + sd);
          float a[P4], wa[P4];
#pragma unroll
          for (int j = 0; j < P4; ++j) {
            const int jj = j < P ? j : 0;
            a[j] = (j < P && valid) ? (1.f + d[jj]) * den : 0.f;
            wa[j] = (j < P && valid) ? ((float)P * d[jj] - sd) * den * aref : 0.f;  // a - 1/p
          }
          if (valid) {
#pragma unroll
            for (int j = 0; j < P; ++j) Ss[il * RgSo + r * P + j] = z[s][q][j];
          }
#pragma unroll
          for (int h = 0; h < P4 / 4; ++h)
            *reinterpret_cast<float4*>(Ws + il * RgW + r * P4 + 4 * h) =
                make_float4(wa[4 * h], wa[4 * h + 1], wa[4 * h + 2], wa[4 * h + 3]);
          int e = 0;
#pragma unroll
          for (int j = 0; j < P; ++j)
#pragma unroll
            for (int k = j; k < P; ++k) aa[q][e++] += a[j] * a[k];
        }
      }
      __syncthreads();
    } else {
      float ur[SPTM][RQ1M][P];
#pragma unroll
      for (int s = 0; s < SPTM; ++s) {
        const int il = lane + 32 * (wp + WP1 * s);
        const bool valid = (s < SPT) && il < ni;
#pragma unroll
        for (int q = 0; q < RQ1M; ++q) {
          const int r = wr + WR1 * q;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            float u = -EDAA_INF;
            if (valid && q < RQ1 && r < nr) {
              if (init) {
                u = 0.1f * uniform24(cd.seeds[m0 + r], (uint64_t)(i0 + il) * P + j + 1);
              } else {
                u = Ss[il * RgSo + r * P + j] - colLse[r * P4 + j] - runEta[r] * cr[s][q][j];
              }
            }
            ur[s][q][j] = u;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RQ1M; ++q) {
        const int r = wr + WR1 * q;
        if (!(q < RQ1 && r < nr)) continue;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          float m = ur[0][q][j];
#pragma unroll
          for (int s = 1; s < SPTM; ++s) m = fmaxf(m, ur[s][q][j]);
          m = warp_max(m);
          if (lane == 0) atomicMax(&colKey[r * P4 + j], ord_key(m));
        }
      }
      __syncthreads();
      for (int c = tid; c < RgS4; c += kThreads) {  // the tile's power-of-two frame of each column
        const float Mn = fmaxf(colM[c], tile_exp(colKey[c]));
        colMn[c] = Mn;
        colP2[c] = Mn == -EDAA_INF ? 0.f : ldexpf(1.f, -(int)Mn);
        colP2k[c] = Mn == -EDAA_INF ? 0.f : ldexpf(1.f, colRef[c] - (int)Mn);
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < SPTM; ++s) {
        if (s >= SPT) continue;
        const int il = lane + 32 * (wp + WP1 * s);
        const bool valid = il < ni;
#pragma unroll
        for (int q = 0; q < RQ1M; ++q) {
          const int r = wr + WR1 * q;
          if (!(q < RQ1 && r < nr)) continue;
          float w[P4];
#pragma unroll
          for (int j = 0; j < P4; ++j) {
            w[j] = 0.f;
            if (j < P && valid) {
              const int c = r * P4 + j;
              // w = e^u 2^-Mn minus the reference weight 2^(k-Mn) (k = 0: uniform b)
              w[j] = shifted_weight_p2(ur[s][q][j], colMn[c], colP2[c], colRef[c], colP2k[c]);
            }
          }
          if (valid) {
#pragma unroll
            for (int j = 0; j < P; ++j) Ss[il * RgSo + r * P + j] = ur[s][q][j];
          }
#pragma unroll
          for (int h = 0; h < P4 / 4; ++h)
            *reinterpret_cast<float4*>(Ws + il * RgW + r * P4 + 4 * h) =
                make_float4(w[4 * h], w[4 * h + 1], w[4 * h + 2], w[4 * h + 3]);
        }
      }
      __syncthreads();
    }

    // ---- write the new state back (coalesced along pixels)
    for (int cc = warp; cc < nc; cc += kWarps) {
      float* dst = St + (size_t)(c0 + cc) * cd.Nst + i0;
      for (int i = lane; i < ni; i += 32) dst[i] = Ss[i * RgSo + cc];
    }

    // ---- phase 2: acc[l][c] += sum_i X[i][l] W[i][c]  (l = 0..L, row L = ones band)
    if (!IS_A) {
#pragma unroll
      for (int q = 0; q < RQ2M; ++q) {
        const int r = wr2 + WR2 * q;
        if (!(q < RQ2 && r < nr)) continue;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          const int c = r * P4 + j;
          const float Mo = colM[c];
          const float Mn = fmaxf(Mo, tile_exp(colKey[c]));
          // exact rescale by a power of two (0 while nothing was accumulated)
          const float sc = (Mo == Mn) ? 1.f : (Mo == -EDAA_INF ? 0.f : ldexpf(1.f, (int)(Mo - Mn)));
#pragma unroll
          for (int k = 0; k < LT; ++k) acc[k][q][j] *= sc;
        }
      }
    }
    // Branch-free like phase 1: a run slot beyond the group accumulates run
    // 0's weights and is never written out.
    const float* wcol[RQ2M];
#pragma unroll
    for (int q = 0; q < RQ2M; ++q) {
      const int r = wr2 + WR2 * q;
      wcol[q] = Ws + ((q < RQ2 && r < nr) ? r : 0) * P4;
    }
    const bool last_in = lane + 32 * (LT - 1) <= L;  // bands of the earlier groups are all <= L
#pragma unroll 4
    for (int i = wp2; i < ni; i += WP2) {
      const float* xr = Xs + i * Ls + lane;
      float xv[LT];
#pragma unroll
      for (int k = 0; k < LT - 1; ++k) xv[k] = xr[32 * k];
      xv[LT - 1] = last_in ? xr[32 * (LT - 1)] : 0.f;
#pragma unroll
      for (int q = 0; q < RQ2M; ++q) {
        float w[P4];
        load_p4<P>(wcol[q] + i * RgW, w);
#pragma unroll
        for (int k = 0; k < LT; ++k)
#pragma unroll
          for (int j = 0; j < P; ++j) acc[k][q][j] = fmaf(xv[k], w[j], acc[k][q][j]);
      }
    }
    __syncthreads();
    if (!IS_A) {
      for (int c = tid; c < RgS4; c += kThreads) {
        colM[c] = fmaxf(colM[c], tile_exp(colKey[c]));
        colKey[c] = ord_key(-EDAA_INF);
      }
    }
  }  // tiles
  cp_async_wait_all();  // a work item without tiles still owns its panel copies
  if (tid == 0) mbar_inval(xbar);  // every wait on it has returned (the tile loop ends in a block barrier)

  // ---- end of pass: reduce phase-2 accumulators over pixel groups, write partials
  float* buf = Xs;  // column-major (L+1) x RgS4: a warp's lanes touch consecutive words
  for (int g = WP2 - 1; g >= 1; --g) {
    __syncthreads();
    if (wp2 == g) {
#pragma unroll
      for (int q = 0; q < RQ2M; ++q) {
        const int r = wr2 + WR2 * q;
        if (!(q < RQ2 && r < nr)) continue;
#pragma unroll
        for (int k = 0; k < LT; ++k) {
          const int l = lane + 32 * k;
          if (l <= L) {
#pragma unroll
            for (int j = 0; j < P; ++j) buf[(r * P4 + j) * (L + 1) + l] = acc[k][q][j];
          }
        }
      }
    }
    __syncthreads();
    if (wp2 == 0) {
#pragma unroll
      for (int q = 0; q < RQ2M; ++q) {
        const int r = wr2 + WR2 * q;
        if (!(q < RQ2 && r < nr)) continue;
#pragma unroll
        for (int k = 0; k < LT; ++k) {
          const int l = lane + 32 * k;
          if (l <= L) {
#pragma unroll
            for (int j = 0; j < P; ++j) acc[k][q][j] += buf[(r * P4 + j) * (L + 1) + l];
          }
        }
      }
    }
  }
  __syncthreads();
  if (wp2 == 0) {
    float* part = cd.part + (size_t)pg * (L + 1) * Mp;
#pragma unroll
    for (int q = 0; q < RQ2M; ++q) {
      const int r = wr2 + WR2 * q;
      if (!(q < RQ2 && r < nr)) continue;
#pragma unroll
      for (int k = 0; k < LT; ++k) {
        const int l = lane + 32 * k;
        if (l <= L) {
#pragma unroll
          for (int j = 0; j < P; ++j) part[(size_t)(c0 + r * P + j) * (L + 1) + l] = acc[k][q][j];
        }
      }
    }
  }
  if (IS_A) {
    // A A^T: sum over lanes (fixed butterfly), then over the WP1 warps of a run set
    float* abuf = buf + (L + 1) * RgS4;  // kWarps x Rm x 36 floats
#pragma unroll
    for (int q = 0; q < RQ1M; ++q) {
      const int r = wr + WR1 * q;
      const bool act = q < RQ1 && r < nr;
#pragma unroll
      for (int e = 0; e < PP; ++e) {
        const float v = warp_sum(aa[q][e]);
        if (act && lane == 0) abuf[(wp * Rm + r) * 36 + e] = v;
      }
    }
    __syncthreads();
    for (int e = tid; e < nr * PP; e += kThreads) {
      const int r = e / PP, pe = e - r * PP;
      float v = 0.f;
      for (int w = 0; w < WP1; ++w) v += abuf[(w * Rm + r) * 36 + pe];
      int j = 0, rem = pe;
      while (rem >= P - j) { rem -= P - j; ++j; }
      const int k = j + rem;
      float* dst = cd.paa + ((size_t)pg * cd.M + m0 + r) * P * P;
      dst[j * P + k] = v;
      dst[k * P + j] = v;
    }
  } else {
    for (int c = tid; c < nc; c += kThreads) {
      const int r = c / P, j = c - r * P;
      cd.pmax[(size_t)pg * Mp + c0 + c] = colM[r * P4 + j];
    }
  }
  __syncthreads();
}

// Fit pass: per (pixel, run) the residual r = x_i - E a_i over the L bands;
// accumulates sum |r| (entrywise l1), the largest per-pixel sum |r| (induced
// l1, max column sum) and sum r^2, FP32 within a pixel, FP64 across pixels.
template <int P>
__device__ __noinline__ void fit_item(const CubeDev& cd, int rg, int pg, float* smem) {
  using TR = PassTraits<P>;
  constexpr int P4 = TR::P4;
  constexpr int RQ1M = TR::RQ1M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int L = cd.L, Ls = cd.Ls, Lr = cd.Lr, N = cd.N, Mp = cd.Mp, Rm = cd.Rm;
  const int m0 = rg * Rm, nr_all = min(Rm, cd.M - m0);
  const int Nt = cd.Nt, WP1 = cd.WP1, WR1 = kWarps / WP1, SPT = cd.SPT;
  // runs are processed in blocks of RB = WR1 * RQ1M (the register tile of one pass over X)
  const int RB = min(Rm, WR1 * RQ1M);
  const PassSmem sm = pass_smem(L, Ls, Lr, P, RB, Nt);
  float* Ps = smem + sm.off_ps;
  float* Xs = smem + sm.off_xs;
  float* Ss = smem + sm.off_ss;
  const int RgS4 = sm.RgS4, RgSo = sm.RgSo;
  const int wp = warp % WP1, wr = warp / WP1;
  const float4* Xs4 = reinterpret_cast<const float4*>(Xs);
  double* dbuf = reinterpret_cast<double*>(Xs);  // kWarps x RB x 3, after the tiles
  for (int rb0 = 0; rb0 < nr_all; rb0 += RB) {
    const int nr = min(RB, nr_all - rb0);
    const int c0 = (m0 + rb0) * P, nc = nr * P;
    const int RQ1 = (nr + WR1 - 1) / WR1;
    __syncthreads();
    for (int e = tid; e < Lr * RgS4; e += kThreads) {
      const int l = e / RgS4, cc = e - l * RgS4, r = cc / P4, j = cc - r * P4;
      float v = 0.f;
      if (l < L && r < nr && j < P) v = cd.Ef[(size_t)l * Mp + c0 + r * P + j];
      Ps[e] = v;
    }
    __syncthreads();
    double s1[RQ1M], s2[RQ1M], smx[RQ1M];
#pragma unroll
    for (int q = 0; q < RQ1M; ++q) { s1[q] = 0.0; s2[q] = 0.0; smx[q] = 0.0; }
    for (int tile = pg; tile < cd.ntiles; tile += cd.Pg) {
      const int i0 = tile * Nt, ni = min(Nt, N - i0);
      {
        const float4* Xg = reinterpret_cast<const float4*>(cd.X + (size_t)i0 * Ls);
        float4* xs4 = reinterpret_cast<float4*>(Xs);
        const int n4 = ni * (Ls >> 2), nt4 = Nt * (Ls >> 2);
        for (int e = tid; e < nt4; e += kThreads) xs4[e] = (e < n4) ? __ldg(Xg + e) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int e = tid; e < ni * nc; e += kThreads) {
        const int cc = e / ni, i = e - cc * ni;
        Ss[i * RgSo + cc] = cd.logA[(size_t)(c0 + cc) * cd.Nst + i0 + i];
      }
      __syncthreads();
      for (int s = 0; s < SPT; ++s) {  // once per solve: a plain loop over the tile's pixel slots
        const int il = lane + 32 * (wp + WP1 * s);
        const bool valid = il < ni;
#pragma unroll
        for (int q = 0; q < RQ1M; ++q) {
          const int r = wr + WR1 * q;
          if (!(q < RQ1 && r < nr)) continue;
          float a[P], se = 0.f;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            a[j] = valid ? expf(Ss[il * RgSo + r * P + j]) : 0.f;
            se += a[j];
          }
          const float inv = valid ? 1.f / se : 0.f;
#pragma unroll
          for (int j = 0; j < P; ++j) a[j] *= inv;
          float t1 = 0.f, t2 = 0.f;
          for (int l = 0; l < Lr; l += 4) {
            const float4 xv = Xs4[(il * Ls + l) >> 2];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              if (l + d < L) {
                float pv[P4];
                load_p4<P>(Ps + (l + d) * RgS4 + r * P4, pv);
                float rr = f4c(xv, d);
#pragma unroll
                for (int j = 0; j < P; ++j) rr = fmaf(-pv[j], a[j], rr);
                t1 += fabsf(rr);
                t2 = fmaf(rr, rr, t2);
              }
            }
          }
          if (valid) {
            s1[q] += (double)t1;
            s2[q] += (double)t2;
            smx[q] = fmax(smx[q], (double)t1);
          }
        }
      }
      __syncthreads();
    }
    // reduce over lanes, then over the WP1 warps sharing a run set
#pragma unroll
    for (int q = 0; q < RQ1M; ++q) {
      const int r = wr + WR1 * q;
      const double a1 = warp_sum_d(s1[q]);
      const double a2 = warp_sum_d(s2[q]);
      const double am = warp_max_d(smx[q]);
      if (q < RQ1 && r < nr && lane == 0) {
        dbuf[(wp * RB + r) * 3 + 0] = a1;
        dbuf[(wp * RB + r) * 3 + 1] = am;
        dbuf[(wp * RB + r) * 3 + 2] = a2;
      }
    }
    __syncthreads();
    for (int r = tid; r < nr; r += kThreads) {
      double a1 = 0.0, a2 = 0.0, am = 0.0;
      for (int w = 0; w < WP1; ++w) {
        a1 += dbuf[(w * RB + r) * 3 + 0];
        am = fmax(am, dbuf[(w * RB + r) * 3 + 1]);
        a2 += dbuf[(w * RB + r) * 3 + 2];
      }
      double* dst = cd.pfit + ((size_t)pg * cd.M + m0 + rb0 + r) * 3;
      dst[0] = a1;
      dst[1] = am;
      dst[2] = a2;
    }
  }
  __syncthreads();
}

template <int P, bool IS_A, int PREC>
__device__ __noinline__ void tc_pass_item(const Batch* __restrict__ bt, const CubeDev& cd, int rg, int pg,
                                          unsigned char* smem_raw, int K1, bool init);

template <int P, int SW>
__device__ __forceinline__ void pass_lt(const Batch* bt, const CubeDev& cd, int rg, int pg, float* smem, int k1,
                                        bool init, bool is_a) {
  if (cd.LT <= 5) {
    if (is_a) pass_item<P, 5, true, SW>(bt, cd, rg, pg, smem, k1, init);
    else pass_item<P, 5, false, SW>(bt, cd, rg, pg, smem, k1, init);
  } else if (cd.LT <= 7) {
    if (is_a) pass_item<P, 7, true, SW>(bt, cd, rg, pg, smem, k1, init);
    else pass_item<P, 7, false, SW>(bt, cd, rg, pg, smem, k1, init);
  } else {
    if (is_a) pass_item<P, 10, true, SW>(bt, cd, rg, pg, smem, k1, init);
    else pass_item<P, 10, false, SW>(bt, cd, rg, pg, smem, k1, init);
  }
}

template <int P>
__device__ __forceinline__ void pass_dispatch_impl(const Batch* bt, const CubeDev& cd, int rg, int pg, float* smem,
                                                 int ph) {
  const int K1 = bt->K1;
  if (ph == PH_FIT) {
    fit_item<P>(cd, rg, pg, smem);
    return;
  }
  const bool is_a = (ph == PH_A || ph == PH_INITA);
  const bool init = (ph == PH_INITA || ph == PH_INITB);
  const int k1 = (ph == PH_INITA) ? 0 : K1;
  if (cd.tc) {
    unsigned char* sb = reinterpret_cast<unsigned char*>(smem);
    if (cd.tc == 2) {
      if (is_a) tc_pass_item<P, true, 1>(bt, cd, rg, pg, sb, k1, init);
      else tc_pass_item<P, false, 1>(bt, cd, rg, pg, sb, k1, init);
    } else if (cd.tc == 3) {
      if (is_a) tc_pass_item<P, true, 2>(bt, cd, rg, pg, sb, k1, init);
      else tc_pass_item<P, false, 2>(bt, cd, rg, pg, sb, k1, init);
    } else {
      if (is_a) tc_pass_item<P, true, 0>(bt, cd, rg, pg, sb, k1, init);
      else tc_pass_item<P, false, 0>(bt, cd, rg, pg, sb, k1, init);
    }
    return;
  }
  if (P >= 3 && cd.SPT == 4)
    pass_lt<P, 4>(bt, cd, rg, pg, smem, k1, init, is_a);
  else
    pass_lt<P, 0>(bt, cd, rg, pg, smem, k1, init, is_a);
}


// Defined (explicitly instantiated) in edaa_pass_p.cu, one object per p.
template <int P>
__device__ void pass_dispatch(const Batch* bt, const CubeDev& cd, int rg, int pg, float* smem, int ph);

}  // namespace edaa
