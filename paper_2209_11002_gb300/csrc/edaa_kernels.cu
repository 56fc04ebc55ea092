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
// (split operands: the high part here and the low part tf32(v - high) one
// panel further on)
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void store_panel(const CubeDev& cd, void* panel, int c, int l, double v) {
  const size_t o = (size_t)c * cd.tc_kp + l;
  if (cd.tc == 2) {
    reinterpret_cast<__nv_bfloat16*>(panel)[o] = __float2bfloat16_rn((float)v);
  } else {
    const float f = (float)v, hi = tf32_rna(f);
    reinterpret_cast<float*>(panel)[o] = hi;
    if (cd.tc == 3) reinterpret_cast<float*>(panel)[(size_t)cd.Mp * cd.tc_kp + o] = tf32_rna(f - hi);
  }
}

// The B-pass panel of a tensor-core cube: v = S + eta2 R (column c, band l)
// as a high part and a low part in the compute type, v ~ hi + lo to about
// 2^-17 (BF16) or 2^-22 (TF32) relative; contraction 1 adds both products.
__device__ __forceinline__ void store_panel_s(const CubeDev& cd, int c, int l, double v) {
  const size_t o = (size_t)c * cd.tc_kp + l, lo = (size_t)cd.Mp * cd.tc_kp;
  if (cd.tc == 2) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
    __nv_bfloat16* ps = reinterpret_cast<__nv_bfloat16*>(cd.panelS);
    ps[o] = h;
    ps[lo + o] = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
  } else {
    const float h = tf32_rna((float)v);
    float* ps = reinterpret_cast<float*>(cd.panelS);
    ps[o] = h;
    ps[lo + o] = tf32_rna((float)(v - (double)h));
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

// Asynchronous copies global -> shared of 8 or 4 bytes (both addresses
// aligned to the size): a merge issues the loads of its inputs this way, so
// that they are all in flight together and land while it forms the partial
// sums; cp_async_wait<n>() waits until at most n committed groups are pending.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Where element e's Pg per-CTA partials live: v[g * stride], each scaled by
// sc[g * sstride] when sc is given (exact powers of two <= 1).
struct PartialRow {
  const float* v;
  size_t stride;
  const float* sc;
  int sstride;
};

// Sums of the per-CTA partials of ne elements, in rounds of up to kThreads
// elements.  In a round a team of lanes (a power of two, as many as the
// block allows for the elements left) shares one element: lane `sub` takes
// g = sub, sub + team, ..., 16 float-float chains per lane with their loads
// in flight together, then a fixed tree over the chains and a fixed
// butterfly over the team.  The rounds, team sizes and every order depend
// only on ne and Pg, so the launch mode does not change the result.  Callers
// number the elements so that consecutive lanes read consecutive addresses.
// store(e, sum) receives each element's total once.
template <bool SCALED, typename Row, typename Store>
__device__ void team_sums(int ne, int Pg, Row row, Store store) {
  constexpr int W = 16;
  for (int e0 = 0; e0 < ne;) {
    int team = 32;
    while (team > 1 && (ne - e0) * team > kThreads) team >>= 1;
    const int per = kThreads / team, sub = (int)threadIdx.x & (team - 1);
    const int e = e0 + (int)threadIdx.x / team;
    float hi[W], lo[W];
#pragma unroll
    for (int q = 0; q < W; ++q) hi[q] = lo[q] = 0.f;
    if (e < ne) {
      const PartialRow r = row(e);
      for (int g0 = sub; g0 < Pg; g0 += W * team) {
        // all loads of the batch first (out-of-range partials read as 0 with scale 0)
        float x[W], sc[W];
#pragma unroll
        for (int q = 0; q < W; ++q) {
          const int g = min(g0 + q * team, Pg - 1);
          x[q] = r.v[(size_t)g * r.stride];
          sc[q] = SCALED ? r.sc[g * r.sstride] : 1.f;
        }
#pragma unroll
        for (int q = 0; q < W; ++q) {
          const float keep = (g0 + q * team < Pg) ? 1.f : 0.f;
          ff_add(hi[q], lo[q], (SCALED ? sc[q] * x[q] : x[q]) * keep);
        }
      }
    }
#pragma unroll
    for (int w = W / 2; w >= 1; w >>= 1)
#pragma unroll
      for (int q = 0; q < w; ++q) {
        ff_add(hi[q], lo[q], hi[q + w]);
        lo[q] += lo[q + w];
      }
    for (int o = team / 2; o >= 1; o >>= 1) {  // every lane of the warp takes part
      const float h2 = __shfl_xor_sync(0xffffffffu, hi[0], o);
      const float l2 = __shfl_xor_sync(0xffffffffu, lo[0], o);
      ff_add(hi[0], lo[0], h2);
      lo[0] += l2;
    }
    if (e < ne && sub == 0) store(e, (double)hi[0] + (double)lo[0]);
    e0 += per;
  }
}

// A-merge of run m over band chunk lc: X A^T = sum of the partials + (1/p) sum_i x_i
// (shifted accumulation), A A^T, and R = E A A^T - X A^T for the next B-pass.
// The loads of E, S and the band sums are in flight during the partial sums.
__device__ void merge_a_unit(const CubeDev& cd, int m, int lc, float* smem) {
  const int tid = threadIdx.x;
  const int P = cd.p, L = cd.L, Mp = cd.Mp, Pg = cd.Pg, c0 = m * P;
  const MergeSmem ms = merge_smem(cd.lchunk, P, Pg);
  double* sd = reinterpret_cast<double*>(smem);
  double *saat = sd + ms.saat, *ssx = sd + ms.ssx, *sxa = sd + ms.sxa, *sE = sd + ms.sE, *sprod = sd + ms.sprod;
  double* sSd = sd + ms.sSd;
  const int l0 = lc * cd.lchunk, nl = min(cd.lchunk, L - l0);
  for (int e = tid; e < nl * P; e += kThreads) {
    const size_t o = (size_t)(l0 + e / P) * Mp + c0 + e % P;
    cp_async8(sE + e, cd.Ed + o);
    if (cd.tc) cp_async8(sSd + e, cd.Sd + o);
  }
  for (int e = tid; e < nl; e += kThreads) cp_async8(ssx + e, cd.sx + l0 + e);
  cp_async_commit();
  team_sums<false>(
      P * P + nl * P, Pg,
      [&](int e) {
        if (e < P * P) return PartialRow{cd.paa + (size_t)m * P * P + e, (size_t)cd.M * P * P, nullptr, 0};
        const int f = e - P * P, j = f / nl, li = f - j * nl;  // bands fastest: coalesced
        return PartialRow{cd.part + (size_t)(c0 + j) * (L + 1) + l0 + li, (size_t)(L + 1) * Mp, nullptr, 0};
      },
      [&](int e, double v) {
        if (e < P * P) {
          saat[e] = v;
        } else {
          const int f = e - P * P, j = f / nl, li = f - j * nl;
          sxa[li * P + j] = v;
        }
      });
  cp_async_wait<0>();
  __syncthreads();
  if (lc == 0)
    for (int e = tid; e < P * P; e += kThreads) cd.AAt[(size_t)m * P * P + e] = saat[e];
  const double aref = (double)(1.f / (float)P);
  for (int e = tid; e < nl * P; e += kThreads) {
    const int li = e / P, l = l0 + li, j = e - li * P;
    const double xat = sxa[e] + aref * ssx[li];  // shifted accumulation: add back (1/p) sum_i x_i
    cd.XAt[(size_t)l * Mp + c0 + j] = xat;
    double r = -xat;
    for (int k = 0; k < P; ++k) r += sE[li * P + k] * saat[k * P + j];
    const size_t o = (size_t)l * Mp + c0 + j;
    cd.Rf[o] = (float)r;
    if (cd.tc) {  // the next B-pass contracts X with S + eta2 R
      cd.Rd[o] = r;
      store_panel_s(cd, c0 + j, l, sSd[e] + cd.eta2d[m] * r);
    }
    sprod[e] = sE[e] * r;
  }
  __syncthreads();
  chunk_rho(cd, m, lc, nl, sprod);
}

// B-merge of run m over band chunk lc: the online softmax over all pixels of
// each column of B, merged across CTAs.  CTA g kept its weights as
// e^u 2^-e_g; in the common frame mx = max_g e_g they scale by 2^(e_g - mx)
// (exact).  The ones band (row L) gives the denominator S, so
// E = X B = (sum_g 2^(e_g-mx) part_g + 2^(k-mx) sum_i x_i) / S, and the
// stored lse is mx ln 2 + log S - log N (logits live in the frame log(N b)).
// Then G = E^T E (chunk sums) and R = E A A^T - X A^T for the next pass.
// Tensor-core cubes keep no B logits (they are u = 0.1 r - Lambda - x^T S):
// a B-merge after a B-step (commit) first adds that step's eta2 R to S, and
// its lc == 0 unit adds the step's log-normaliser to Lambda (the first
// B-merge, after the initial pass, sets Lambda); the new R then gives the
// next B-pass's panel S + eta2 R.
__device__ void merge_b_unit(const CubeDev& cd, int m, int lc, float* smem, bool commit) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int P = cd.p, L = cd.L, Mp = cd.Mp, Pg = cd.Pg, c0 = m * P;
  const MergeSmem ms = merge_smem(cd.lchunk, P, Pg);
  double* sd = reinterpret_cast<double*>(smem);
  double *saat = sd + ms.saat, *sw = sd + ms.sw, *ssx = sd + ms.ssx, *sxa = sd + ms.sxa, *sE = sd + ms.sE;
  double *sraw = sd + ms.sraw, *sprod = sd + ms.sprod;
  float* sscale = reinterpret_cast<float*>(sd + ms.sscale);  // Pg x P
  float* sEf = reinterpret_cast<float*>(sd + ms.sEf);        // E of the chunk in float (the Gram sums)
  double *sSd = sd + ms.sSd, *sRd = sd + ms.sRd;
  const int l0 = lc * cd.lchunk, nl = min(cd.lchunk, L - l0);
  // every load that does not depend on the partial sums, in flight together:
  // first the per-CTA frames, then (landing during the sums) X A^T, S, R, the
  // band sums and A A^T
  for (int e = tid; e < Pg * P; e += kThreads) cp_async4(sscale + e, cd.pmax + (size_t)(e / P) * Mp + c0 + e % P);
  cp_async_commit();
  for (int e = tid; e < nl * P; e += kThreads) {
    const size_t o = (size_t)(l0 + e / P) * Mp + c0 + e % P;
    cp_async8(sxa + e, cd.XAt + o);
    if (cd.tc) {
      cp_async8(sSd + e, cd.Sd + o);
      cp_async8(sRd + e, cd.Rd + o);
    }
  }
  for (int e = tid; e < nl; e += kThreads) cp_async8(ssx + e, cd.sx + l0 + e);
  for (int e = tid; e < P * P; e += kThreads) cp_async8(saat + e, cd.AAt + (size_t)m * P * P + e);
  cp_async_commit();
  cp_async_wait<1>();
  __syncthreads();
  if (warp < P) {  // the common frame of column j and the per-CTA scale factors
    const int j = warp;
    float mx = -EDAA_INF;
    for (int g = lane; g < Pg; g += 32) mx = fmaxf(mx, sscale[g * P + j]);
    mx = warp_max(mx);
    for (int g = lane; g < Pg; g += 32) {
      const float eg = sscale[g * P + j];
      sscale[g * P + j] = (eg == -EDAA_INF) ? 0.f : ldexpf(1.f, (int)(eg - mx));  // exact (0 below 2^-149)
    }
    if (lane == 0) sw[j] = (double)mx;
  }
  __syncthreads();
  // second step: scaled sums of the partials of the chunk's bands and of the ones band
  team_sums<true>(
      (nl + 1) * P, Pg,
      [&](int e) {
        const int j = e / (nl + 1), li = e - j * (nl + 1);  // bands fastest: coalesced
        const int l = li < nl ? l0 + li : L;
        return PartialRow{cd.part + (size_t)(c0 + j) * (L + 1) + l, (size_t)(L + 1) * Mp, sscale + j, P};
      },
      [&](int e, double v) {
        const int j = e / (nl + 1), li = e - j * (nl + 1);
        sraw[li * P + j] = v;
      });
  cp_async_wait<0>();
  __syncthreads();
  if (tid < P) {
    const int j = tid, c = c0 + j;
    const double mx = sw[j];
    // shifted accumulation: every pixel contributed w - 2^(k-e_g), i.e.
    // 2^(k-mx) in the merged frame; add N 2^(k-mx) back to the denominator
    const double wref = ldexp(1.0, cd.bref[c] - (int)mx);
    const double S = sraw[nl * P + j] + wref * (double)cd.N;
    if (lc == 0) {
      // log S = e ln 2 + log f (S = f 2^e, f in [1/2, 1)): f rounded to float
      // and a float logarithm err by about 1e-7 absolute, below the float lse's
      // own rounding; this GPU's FP64 pipe makes a double log cost microseconds.
      int ex = 0;
      const double f = frexp(S, &ex);
      const double lse = (mx + (double)ex) * 0.69314718055994531 + (double)logf((float)f) - cd.logN;
      cd.lse[c] = (float)lse;
      if (cd.tc) cd.lamd[c] = (commit ? cd.lamd[c] : 0.0) + lse;
    }
    sw[j] = wref;
    sw[kMaxP + j] = 1.0 / S;
  }
  __syncthreads();
  for (int e = tid; e < nl * P; e += kThreads) {
    const int li = e / P, l = l0 + li, j = e - li * P;
    const double s = (sraw[e] + sw[j] * ssx[li]) * sw[kMaxP + j];
    cd.Ed[(size_t)l * Mp + c0 + j] = s;
    cd.Ef[(size_t)l * Mp + c0 + j] = (float)s;
    if (cd.tc) store_panel(cd, cd.panelE, c0 + j, l, s);
    sE[e] = s;
    sEf[e] = (float)s;
  }
  __syncthreads();
  // G = E^T E of run m over this chunk's bands, bands in order (the tensor-core
  // A-pass sums the chunks; the CUDA-core A-pass forms G from its staged panel)
  if (cd.tc)  // one warp per entry, lanes over the bands, fixed butterfly; FP32 like the A-pass's use of G
    for (int e = warp; e < P * P; e += kWarps) {
      const int j = e / P, k = e - j * P;
      float g = 0.f;
      for (int li = lane; li < nl; li += 32) g = fmaf(sEf[li * P + j], sEf[li * P + k], g);
      g = warp_sum(g);
      if (lane == 0) cd.gpart[((size_t)lc * cd.M + m) * P * P + e] = g;
    }
  const double eta2 = cd.tc ? cd.eta2d[m] : 0.0;
  for (int e = tid; e < nl * P; e += kThreads) {
    const int li = e / P, l = l0 + li, j = e - li * P;
    double r = -sxa[e];
    for (int k = 0; k < P; ++k) r += sE[li * P + k] * saat[k * P + j];
    const size_t o = (size_t)l * Mp + c0 + j;
    cd.Rf[o] = (float)r;
    if (cd.tc) {
      double sv = sSd[e];
      if (commit) {  // the step just taken used R from the previous merge
        sv += eta2 * sRd[e];
        cd.Sd[o] = sv;
      }
      cd.Rd[o] = r;
      store_panel_s(cd, c0 + j, l, sv + eta2 * r);
    }
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
    else merge_b_unit(cd, m, lc, smem, ph == PH_BM);
  }
}

// ---------------------------------------------------------------------------
// Per-run scalar phases: step sizes (eqs. eta0A, eta0B) and fit/coherence.
// ---------------------------------------------------------------------------
// Largest eigenvalue of a symmetric p x p matrix by the cyclic Jacobi method
// (plane rotations that zero one off-diagonal entry at a time, Golub & Van
// Loan, "Matrix Computations", Sec. 8.5).
template <typename F>
__device__ F jacobi_max_eig(F* a, int n) {
  const F tol = sizeof(F) == 4 ? (F)1e-14 : (F)1e-30;  // squared relative size of the off-diagonal part
  for (int sweep = 0; sweep < 60; ++sweep) {
    F off = 0, diag = 0;
    for (int i = 0; i < n; ++i) {
      diag += a[i * n + i] * a[i * n + i];
      for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
    }
    if (off <= tol * diag || off == (F)0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const F apq = a[p * n + q];
        if (apq == (F)0) continue;
        const F theta = (a[q * n + q] - a[p * n + p]) / ((F)2 * apq);
        const F t = (theta >= (F)0 ? (F)1 : (F)-1) / (fabs(theta) + sqrt(theta * theta + (F)1));
        const F c = (F)1 / sqrt(t * t + (F)1), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const F akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const F apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
      }
    }
  }
  F mx = a[0];
  for (int i = 1; i < n; ++i) mx = fmax(mx, a[i * n + i]);
  return mx;
}

// G = E^T E of run m with the mean pixel added back (E = E_c + xbar 1^T), by
// one warp: lanes stride over the bands, each entry is reduced in a fixed
// butterfly and lands in Gw (P x P, shared memory).
__device__ void warp_gram(const CubeDev& cd, int m, double* Gw, int lane) {
  const int P = cd.p;
  for (int e = 0; e < P * P; ++e) {
    const int j = e / P, k = e - j * P;
    double s = 0.0;
    if (k >= j)
      for (int l = lane; l < cd.L; l += 32) {
        const double* r = cd.Ed + (size_t)l * cd.Mp + m * P;
        const double xb = cd.xbar[l];
        s += (r[j] + xb) * (r[k] + xb);
      }
    s = warp_sum_d(s);
    if (lane == 0 && k >= j) Gw[j * P + k] = Gw[k * P + j] = s;
  }
  __syncwarp();
}

// Step sizes (eqs. eta0A, eta0B), one warp per run: sigma_max^2(X B^0) by
// Jacobi on G = E^0T E^0, eta1 = gamma / sigma_max^2, eta2 = sqrt(p / N) eta1.
__device__ void eta_phase(const Batch* __restrict__ bt, float* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* Gw = reinterpret_cast<double*>(smem) + warp * kMaxP * kMaxP;
  float* Gf = reinterpret_cast<float*>(reinterpret_cast<double*>(smem) + kWarps * kMaxP * kMaxP) + warp * kMaxP * kMaxP;
  for (int g = blockIdx.x * kWarps + warp; g < bt->total_runs; g += gridDim.x * kWarps) {
    int ci = 0;
    while (ci + 1 < bt->n_cubes && g >= bt->c[ci + 1].run0) ++ci;
    const CubeDev& cd = bt->c[ci];
    const int m = g - cd.run0, P = cd.p;
    warp_gram(cd, m, Gw, lane);
    if (lane == 0) {
      // FP64 Gram matrix, FP32 rotations: the largest eigenvalue to ~1e-7 relative
      for (int e = 0; e < P * P; ++e) Gf[e] = (float)Gw[e];
      const double s2 = (double)jacobi_max_eig(Gf, P);
      const double e1 = cd.gammas[m] / s2;
      const double e2 = sqrt((double)P / (double)cd.N) * e1;
      cd.sig2[m] = s2;
      cd.eta1d[m] = e1;
      cd.eta2d[m] = e2;
      cd.eta1[m] = (float)e1;
      cd.eta2[m] = (float)e2;
    }
    __syncwarp();
  }
}

// Fit merge and coherence (Algorithm 2, eq. coherence), one warp per run.
__device__ void fitm_phase(const Batch* __restrict__ bt, float* smem, int hist_t) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* Gw = reinterpret_cast<double*>(smem) + warp * kMaxP * kMaxP;
  for (int g = blockIdx.x * kWarps + warp; g < bt->total_runs; g += gridDim.x * kWarps) {
    int ci = 0;
    while (ci + 1 < bt->n_cubes && g >= bt->c[ci + 1].run0) ++ci;
    const CubeDev& cd = bt->c[ci];
    const int m = g - cd.run0, P = cd.p;
    double a1 = 0.0, am = 0.0, a2 = 0.0;
    for (int q = lane; q < cd.Pg; q += 32) {
      const double* s = cd.pfit + ((size_t)q * cd.M + m) * 3;
      a1 += s[0];
      am = fmax(am, s[1]);
      a2 += s[2];
    }
    a1 = warp_sum_d(a1);
    am = warp_max_d(am);
    a2 = warp_sum_d(a2);
    warp_gram(cd, m, Gw, lane);  // coherence from the FP64 copy of E, uncentred
    if (lane == 0) {
      cd.fit[m] = a1;
      cd.fitmax[m] = am;
      cd.loss2[m] = a2;
      // the loss log: row hist_t (the outer iteration just completed, 0-based)
      if (hist_t >= 0 && hist_t < bt->hist_cap) cd.loss_hist[(size_t)hist_t * cd.M + m] = a2;
      double mu = -INFINITY;
      for (int j = 0; j < P; ++j)
        for (int k = j + 1; k < P; ++k) {
          double v = Gw[j * P + k];
          if (bt->coh_mode == 0) {
            const double d = sqrt(Gw[j * P + j]) * sqrt(Gw[k * P + k]);
            v = d > 0.0 ? v / d : 0.0;
          }
          mu = fmax(mu, v);
        }
      cd.mu[m] = mu;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// The program kernel.
// ---------------------------------------------------------------------------
// Phases of an outer iteration: A-pass, A-merge, K2 x (B-pass, B-merge), and
// with the loss log the fit pass and fit merge.
__host__ __device__ inline int phases_per_outer(int K2, int record) { return 2 + 2 * K2 + (record ? 2 : 0); }

__host__ __device__ inline int phase_of(int mode, int s, int K2, int record) {
  if (mode == MODE_INIT) {
    const int seq[5] = {PH_INITB, PH_BM0, PH_ETA, PH_INITA, PH_AM};
    return seq[s];
  }
  if (mode == MODE_FIT) return s == 0 ? PH_FIT : PH_FITM;
  const int per = phases_per_outer(K2, record);
  const int k = s % per;
  if (k == 0) return PH_A;
  if (k == 1) return PH_AM;
  if (k >= 2 + 2 * K2) return k == 2 + 2 * K2 ? PH_FIT : PH_FITM;
  return (k & 1) ? PH_BM : PH_B;
}

int program_phase_id(int mode, int s, int K2, int record) { return phase_of(mode, s, K2, record); }

int program_phase_count(int mode, int n_outer, int K2, int record) {
  if (mode == MODE_INIT) return 5;
  if (mode == MODE_FIT) return 2;
  return n_outer * phases_per_outer(K2, record);
}

__global__ void __launch_bounds__(kThreads, 1)
k_edaa(const Batch* __restrict__ bt, int mode, int outer0, int ph_lo, int ph_hi) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int per = phases_per_outer(bt->K2, bt->record_loss);
  const bool tr = bt->trace_start != nullptr;
  for (int s = ph_lo; s < ph_hi; ++s) {
    if (s > ph_lo) {
      if (!grid_barrier(bt->bar, gridDim.x, bt->status, bt->timeout_ns)) return;
    }
    const size_t ti = (size_t)mode * kTraceCap + s;
    if (tr && threadIdx.x == 0 && s < kTraceCap) atomicMin(bt->trace_start + ti, (unsigned long long)global_ns());
    const int ph = phase_of(mode, s, bt->K2, bt->record_loss);
    switch (ph) {
      case PH_A:
      case PH_B:
      case PH_INITA:
      case PH_INITB:
      case PH_FIT: pass_phase(bt, ph, smem); break;
      case PH_AM:
      case PH_BM:
      case PH_BM0: merge_phase(bt, ph, smem); break;
      case PH_ETA: eta_phase(bt, smem); break;
      case PH_FITM: fitm_phase(bt, smem, mode == MODE_OUTER ? outer0 + s / per : -1); break;
      default: break;
    }
    if (tr) {
      __syncthreads();
      if (threadIdx.x == 0 && s < kTraceCap) atomicMax(bt->trace_end + ti, (unsigned long long)global_ns());
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

cudaError_t launch_program(const Batch* d_batch, int mode, int outer0, int ph_lo, int ph_hi, int grid,
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
  return cudaLaunchKernelEx(&lc, k_edaa, d_batch, mode, outer0, ph_lo, ph_hi);
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

// B of a tensor-core cube, regenerated: b_i = exp(0.1 r_i - Lambda - x_i^T S - log N),
// one thread per entry, FP64.  x is the centred pixel as contraction 1 saw it
// (the compute-type copy Xk: BF16, TF32, or the sum of its two TF32 parts),
// so that b is the B the solve's logits and normalisers describe.
__global__ void k_gather_b_regen(const void* __restrict__ Xk, int kp, int tc, const double* __restrict__ Sd,
                                 const double* __restrict__ lamd, const uint16_t* __restrict__ r16,
                                 const uint64_t* __restrict__ seeds, int Nst, int L, int N, int Mp, int p, int m,
                                 double logN, float* __restrict__ B) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * p) return;
  const int i = e / p, j = e % p, c = m * p + j;
  double dot = 0.0;
  for (int l = 0; l < L; ++l) {
    const size_t o = (size_t)i * kp + l;
    double x;
    if (tc == 2) {
      x = (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(Xk)[o]);
    } else {
      const float* xf = reinterpret_cast<const float*>(Xk);
      x = (double)xf[o] + (tc == 3 ? (double)xf[(size_t)N * kp + o] : 0.0);
    }
    dot += x * Sd[(size_t)l * Mp + c];
  }
  // as the tensor-core passes read it: the 16-bit table, or (split operands) the 24-bit draw
  const float u0 = tc == 3 ? 0.1f * uniform24(seeds[m], (uint64_t)i * p + j + 1)
                           : ((float)r16[(size_t)c * Nst + i] + 0.5f) * kR16Scale;
  B[e] = (float)exp((double)u0 - lamd[c] - dot - logN);
}

cudaError_t launch_gather(const CubeDev& hc, int run, float* E, float* A, float* B, cudaStream_t s) {
  if (E) k_gather_e<<<(hc.L * hc.p + 255) / 256, 256, 0, s>>>(hc.Ed, hc.xbar, hc.L, hc.Mp, hc.p, run, E);
  if (hc.tc) {
    if (A) k_gather_ab<<<(hc.N * hc.p + 255) / 256, 256, 0, s>>>(hc.logA, nullptr, nullptr, hc.N, hc.Nst, hc.p, run, A,
                                                                 nullptr);
    if (B)
      k_gather_b_regen<<<(hc.N * hc.p + 255) / 256, 256, 0, s>>>(hc.Xk, hc.tc_kp, hc.tc, hc.Sd, hc.lamd, hc.r16,
                                                                 hc.seeds, hc.Nst, hc.L, hc.N, hc.Mp, hc.p, run,
                                                                 hc.logN, B);
  } else if (A || B) {
    k_gather_ab<<<(hc.N * hc.p + 255) / 256, 256, 0, s>>>(hc.logA, hc.logB, hc.lse, hc.N, hc.Nst, hc.p, run, A, B);
  }
  return cudaGetLastError();
}

// Compute-type copies of the centred X for the tensor-core passes:
// Xk: N x kp pixel-major (band L is the ones band, bands > L zero), XT
// (TF32 only; null for BF16): (L+1) x Npad band-major, TF32 rounded to
// nearest or BF16.
// mode 1: TF32, 2: BF16, 3: split TF32 (high part, then the low part
// tf32(x - high) in a second copy of each array right after the first)
__global__ void k_tc_prepare(const float* __restrict__ X, int L, int Ls, int N, int kp, int Npad, int mode,
                             void* __restrict__ Xk, void* __restrict__ XT) {
  const size_t n = (size_t)N * kp, nT = (size_t)(L + 1) * Npad;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / kp), l = (int)(e - (size_t)i * kp);
    const float v = (l < Ls) ? X[(size_t)i * Ls + l] : 0.f;
    const size_t t = (size_t)l * Npad + i;
    if (mode == 2) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      reinterpret_cast<__nv_bfloat16*>(Xk)[e] = h;
      if (XT != nullptr && l <= L) reinterpret_cast<__nv_bfloat16*>(XT)[t] = h;
    } else {
      const float hi = tf32_rna(v);
      reinterpret_cast<float*>(Xk)[e] = hi;
      if (l <= L) reinterpret_cast<float*>(XT)[t] = hi;
      if (mode == 3) {
        const float lo = tf32_rna(v - hi);
        reinterpret_cast<float*>(Xk)[n + e] = lo;
        if (l <= L) reinterpret_cast<float*>(XT)[nT + t] = lo;
      }
    }
  }
}

// The uniforms of eq. (initB0) for the tensor-core passes: r16[c][i] = top 16
// bits of SplitMix64 output i p + j + 1 of run m's seed (c = m p + j); the
// padding pixels [N, Nst) hold 0.
__global__ void k_fill_r16(const uint64_t* __restrict__ seeds, int N, int Nst, int p, int Mp,
                           uint16_t* __restrict__ r16) {
  const size_t n = (size_t)Mp * Nst;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / Nst), i = (int)(e - (size_t)c * Nst);
    const int m = c / p, j = c - m * p;
    r16[e] = i < N ? (uint16_t)(splitmix64_out(seeds[m], (uint64_t)i * p + j + 1) >> 48) : (uint16_t)0;
  }
}

cudaError_t launch_fill_r16(const CubeDev& hc, cudaStream_t s) {
  k_fill_r16<<<1024, 256, 0, s>>>(hc.seeds, hc.N, hc.Nst, hc.p, hc.Mp, hc.r16);
  return cudaGetLastError();
}

cudaError_t launch_tc_prepare(const CubeDev& hc, void* Xk, void* XT, int Npad, cudaStream_t s) {
  k_tc_prepare<<<1024, 256, 0, s>>>(hc.X, hc.L, hc.Ls, hc.N, hc.tc_kp, Npad, hc.tc, Xk, XT);
  return cudaGetLastError();
}

// FP32 FMA throughput probe (the roofline denominator of the CUDA-core
// passes).  kFmaChains independent dependency chains per thread, unrolled so
// that loop control is a small fraction of the issued instructions; the
// chains are folded into one store per thread so that none is dead code.
constexpr int kFmaChains = 16;
__global__ void __launch_bounds__(256) k_fma_peak(float* __restrict__ out, int iters, float b, float c) {
  float a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = (float)threadIdx.x * 1e-3f + (float)k;
#pragma unroll 8
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = fmaf(a[k], b, c);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fma_peak(float* out, int blocks, int iters, cudaStream_t s) {
  k_fma_peak<<<blocks, 256, 0, s>>>(out, iters, 0.9999999f, 1e-7f);
  return cudaGetLastError();
}

double fma_peak_flops_per_launch(int blocks, int iters) { return 2.0 * kFmaChains * (double)iters * blocks * 256.0; }

__global__ void k_barrier_test(unsigned* bar, int* status, unsigned expected, long long timeout_ns) {
  grid_barrier(bar, expected, status, timeout_ns);
}

cudaError_t launch_barrier_test(unsigned* bar, int* status, int grid, int expected, long long timeout_ns,
                                cudaStream_t s) {
  k_barrier_test<<<grid, 64, 0, s>>>(bar, status, (unsigned)expected, timeout_ns);
  return cudaGetLastError();
}

}  // namespace edaa
