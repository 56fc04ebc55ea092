// The tcgen05 pass work item (see edaa_tc.cuh for the scheme).  Included by
// edaa_pass_p.cu, instantiated per p.
#pragma once
#include "edaa_tc.cuh"

namespace edaa {

// PREC: 0 TF32, 1 BF16, 2 split TF32 (x = hi + lo; products hi*hi + hi*lo + lo*hi,
// and the element-wise steps in full FP32 as in the CUDA-core pass).
template <int P, bool IS_A, int PREC>
__device__ __noinline__ void tc_pass_item(const Batch* __restrict__ bt, const CubeDev& cd, int rg, int pg,
                                          unsigned char* smem_raw, int K1, bool init) {
  constexpr bool BF = PREC == 1, SPLIT = PREC == 2;
  constexpr int SUB = SPLIT ? 2 : 1;  // stream chunks per 128-byte K chunk (split: high part, then low part)
  constexpr int PP = P * (P + 1) / 2;
  constexpr int ESZ = BF ? 2 : 4;
  constexpr int KCH = 128 / ESZ;   // elements per 128-byte row (32 tf32, 64 bf16)
  constexpr int NPC = 128 / KCH;   // pixel chunks per 128-pixel tile
  constexpr uint32_t FMT = BF ? 1u : 2u;
  constexpr int kRB = 4;           // runs whose state is loaded together in the B epilogue
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quarter = warp & 3, half = warp >> 2;
  const int L = cd.L, N = cd.N, Mp = cd.Mp, Rm = cd.Rm;
  const int m0 = rg * Rm, nr = min(Rm, cd.M - m0), c0 = m0 * P, nc = nr * P;
  const int Rgp = cd.tc_rgp, nkc = cd.tc_nkc, nbt = cd.tc_nbt;
  const long long tmo = bt->timeout_ns;
  const CUtensorMap* tmX = cd.tmaps + 0;
  const CUtensorMap* tmXT = cd.tmaps + 1;
  const CUtensorMap* tmPan = cd.tmaps + (IS_A ? 2 : 3);
  const CUtensorMap* tmXlo = cd.tmaps + 4;  // split operands: the low parts
  const CUtensorMap* tmXTlo = cd.tmaps + 5;
  const CUtensorMap* tmPanLo = cd.tmaps + (IS_A ? 6 : 7);
  const TcSmem S = tc_smem(Rgp, ESZ, SPLIT, P);
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Wsm = sm + (S.w_off - 1024u);
  const uint32_t wchunk = ((uint32_t)Rgp * 128u + 1023u) & ~1023u;
  const uint32_t pnl = wchunk;  // a panel chunk (Rgp rows of 128 B), 1024-byte aligned in its stage
  unsigned char* misc = sm + (S.misc_off - 1024u);
  uint64_t* full = reinterpret_cast<uint64_t*>(misc);      // kTcStages
  uint64_t* empty = full + kTcStages;                      // kTcStages
  uint64_t* bar_c1 = empty + kTcStages;
  uint64_t* bar_c2 = bar_c1 + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_c2 + 1);
  int* flags = reinterpret_cast<int*>(tmem_slot + 4);      // [0] bail, [1] rescale needed
  float* colM = reinterpret_cast<float*>(flags + 4);       // Rgp: running power-of-two exponent (B)
  int* colKey = reinterpret_cast<int*>(colM + 256);        // Rgp: tile maximum logit (B)
  float* colScale = reinterpret_cast<float*>(colKey + 256);  // Rgp
  float* colLse = colScale + 256;                          // Rgp
  float* runEta = colLse + 256;                            // Rm (<= 128)
  int* colRef = reinterpret_cast<int*>(runEta + 128);      // Rgp: reference exponent k (B)
  float* colRefW = reinterpret_cast<float*>(colRef + 256);  // Rgp: 2^(k - Mn), the reference weight (B)
  float* Gs = colRefW + 256;                               // Rm x P x P (A), <= 2048
  float* aaq = Gs + 2048;                                  // 4 x Rm x PP (A)

  // ---- set-up: barriers, TMEM (512 columns: one CTA per SM), per-run constants
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(512)
                 : "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(bar_c1, 1);
    mbar_init(bar_c2, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    flags[0] = 0;
    flags[1] = 0;
  }
  for (int c = tid; c < 256; c += kThreads) {
    colM[c] = -EDAA_INF;
    colKey[c] = ord_key(-EDAA_INF);
    colScale[c] = 1.f;
    colLse[c] = 0.f;
    colRefW[c] = 0.f;
  }
  if (!IS_A)
    for (int c = tid; c < 256; c += kThreads) {
      const int k = (!init && c < nc) ? ref_exponent(cd, m0 + c / P, c0 + c) : 0;
      colRef[c] = k;
      if (c < nc) {
        if (!init) colLse[c] = cd.lse[c0 + c];
        if (pg == 0) cd.bref[c0 + c] = k;
      }
    }
  for (int r = tid; r < Rm; r += kThreads) runEta[r] = r < nr ? (IS_A ? cd.eta1[m0 + r] : cd.eta2[m0 + r]) : 0.f;
  if (IS_A) {
    for (int e = tid; e < 4 * Rm * PP; e += kThreads) aaq[e] = 0.f;
    if (!init && K1 > 0) {
      for (int e = tid; e < nr * P * P; e += kThreads) {  // G = E^T E per run from the merge's band-chunk sums
        const int r = e / (P * P), jk = e - r * P * P;
        double s = 0.0;
        for (int lc = 0; lc < cd.nlchunk; ++lc) s += cd.gpart[((size_t)lc * cd.M + m0 + r) * P * P + jk];
        Gs[e] = (float)s;
      }
    }
  }
  // W: zero once (padding rows and invalid pixels must stay 0)
  for (uint32_t e = tid; e < (uint32_t)SUB * NPC * wchunk / 4; e += kThreads) reinterpret_cast<float*>(Wsm)[e] = 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tmem_slot;
  const uint32_t id = tc_idesc(128, Rgp, FMT);
  const bool do_c1 = !init;

  // ---- the chunk stream (thread 0).  Per tile: contraction 1 (nkc chunks of X
  // and the panel; not in the initial passes), then contraction 2 (nbt * NPC
  // chunks of the band-major X).  Chunk k uses ring stage k % kTcStages.  Loads
  // run up to kTcStages chunks ahead of the MMAs, so contraction 2's X streams
  // in during the epilogue and the next tile's contraction 1 during
  // contraction 2.
  const int nc1 = do_c1 ? nkc * SUB : 0;
  const int nc2 = nbt * NPC * SUB;
  const int per_tile = nc1 + nc2;
  const int ntl = pg < cd.ntiles ? (cd.ntiles - pg + cd.Pg - 1) / cd.Pg : 0;
  const uint32_t total = (uint32_t)(ntl * per_tile);
  uint32_t loaded = 0, issued = 0;
  auto load_chunk = [&](uint32_t k) -> bool {
    const uint32_t s = k % kTcStages;
    if (k >= kTcStages && !mbar_wait(empty + s, ((k / kTcStages) + 1) & 1, tmo)) return false;
    const int q = (int)(k / (uint32_t)per_tile), j = (int)(k - (uint32_t)(q * per_tile));
    const int ti0 = (pg + q * cd.Pg) * kTcTile;
    unsigned char* dst = sm + s * S.stage_bytes;
    if (j < nc1) {  // X chunk + panel chunk (split: [X hi | P hi | P lo], then [X lo | P hi])
      const int kc = j / SUB, part = j - kc * SUB;
      const bool two = SPLIT && part == 0;
      mbar_expect(full + s, 128u * 128u + (two ? 2u : 1u) * (uint32_t)Rgp * 128u);
      tma2d(dst, part ? tmXlo : tmX, kc * KCH, ti0, full + s);
      tma2d(dst + 128 * 128, tmPan, kc * KCH, c0, full + s);
      if (two) tma2d(dst + 128 * 128 + pnl, tmPanLo, kc * KCH, c0, full + s);
    } else {  // band-major X chunk (split: high part, then low part)
      const int jj = j - nc1, kc = jj / SUB, part = jj - kc * SUB, bti = kc / NPC, pc = kc - bti * NPC;
      mbar_expect(full + s, 128u * 128u);
      tma2d(dst, part ? tmXTlo : tmXT, ti0 + pc * KCH, bti * 128, full + s);
    }
    return true;
  };
  auto fill = [&]() -> bool {
    while (loaded < total && loaded < issued + kTcStages) {
      if (!load_chunk(loaded)) return false;
      ++loaded;
    }
    return true;
  };
  // MMAs of the next chunk; its stage is released by the MMAs' commit
  auto consume = [&](auto&& mma) -> bool {
    const uint32_t k = issued, s = k % kTcStages;
    if (!mbar_wait(full + s, (k / kTcStages) & 1, tmo)) return false;
    tc_fence_after();
    mma(sm + s * S.stage_bytes);
    tc_commit(empty + s);
    ++issued;
    return fill();
  };
  if (tid == 0 && !fill()) flags[0] = 1;

  // Split operands: contraction 2 of each tile restarts a tile accumulator T
  // (TMEM columns Rgp (1 + b)), and the threads add it into the running sums
  // S (columns Rgp (1 + nbt + b)) in FP32, S = S * scale + T, with the B-pass
  // frame change as the exact power-of-two scale.  The tensor core's FP32
  // accumulation then never runs over more than one tile: over long chains
  // (many tiles per CTA) it drifts by more than the FP32 path allows.
  const uint32_t tl0 = (uint32_t)((warp & 3) * 32) << 16;
  auto fold_tile = [&](bool first) {
    for (int b = 0; b < nbt; ++b)
      for (int cc = (warp >> 2) * 8; cc < Rgp; cc += 16) {
        const uint32_t tT = tbase + tl0 + (uint32_t)(Rgp * (1 + b) + cc);
        const uint32_t tS = tbase + tl0 + (uint32_t)(Rgp * (1 + nbt + b) + cc);
        float vt[8], vs[8];
        tmem_ld8(tT, vt);
        if (first) {
#pragma unroll
          for (int j = 0; j < 8; ++j) vs[j] = vt[j];
        } else {
          tmem_ld8(tS, vs);
#pragma unroll
          for (int j = 0; j < 8; ++j) vs[j] = fmaf(vs[j], IS_A ? 1.f : colScale[cc + j], vt[j]);
        }
        tmem_st8(tS, vs);
      }
  };
  bool folded = false;

  uint32_t c1_phase = 0, c2_phase = 0;
  bool c2_pending = false, d2_started = false;
  int bail = 0;
  float* St = IS_A ? cd.logA : cd.logB;
  const float aref = 1.f / (float)P;
  const uint32_t tl = (uint32_t)(quarter * 32) << 16;  // this warp's TMEM lane block

  for (int q = 0; q < ntl; ++q) {
    const int i0 = (pg + q * cd.Pg) * kTcTile;
    const int ni = min(kTcTile, N - i0);
    // ---- 1. C = X_tile Panel^T (skipped for the initial passes: c = 0)
    if (do_c1) {
      if (tid == 0 && !flags[0]) {
        bool ok = true;
        for (int j = 0; j < nc1 && ok; ++j) {
          const int kc = j / SUB, part = j - kc * SUB;
          ok = consume([&](unsigned char* st) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t da = desc_sw128(su32(st + ks * 32));
              const uint64_t db = desc_sw128(su32(st + 128 * 128 + ks * 32));
              tc_mma<BF>(tbase, da, db, id, (kc | ks | part) ? 1u : 0u);
              if (SPLIT && part == 0)  // X hi * P lo
                tc_mma<BF>(tbase, da, desc_sw128(su32(st + 128 * 128 + pnl + ks * 32)), id, 1u);
            }
          });
        }
        if (ok) tc_commit(bar_c1);
        else flags[0] = 1;
      }
      __syncthreads();
      const int to = flags[0] ? 1 : (mbar_wait(bar_c1, c1_phase, tmo) ? 0 : 2);
      if (to) atomicOr(bt->status, 1 << (8 + to));  // 9: contraction-1 pipeline, 10: its commit
      if (__syncthreads_or(to)) {
        bail = 1;
        break;
      }
      c1_phase ^= 1;
      tc_fence_after();
    }
    // the previous tile's contraction 2 must finish before W is rewritten or Acc rescaled
    if (c2_pending) {
      const int to = mbar_wait(bar_c2, c2_phase, tmo) ? 0 : 1;
      if (to) atomicOr(bt->status, 1 << 11);  // contraction 2 of the previous tile
      if (__syncthreads_or(to)) {
        bail = 1;
        break;
      }
      c2_phase ^= 1;
      c2_pending = false;
      tc_fence_after();
      if (SPLIT) {
        fold_tile(!folded);
        folded = true;
      }
    }
    // ---- 2. epilogue: warp (quarter, half) = pixels 32*quarter.., runs of parity `half`
    const int il = quarter * 32 + lane;
    const bool valid = il < ni;
    const size_t Nst = (size_t)cd.Nst;
    const size_t gpix = (size_t)c0 * Nst + i0 + il;  // state of column c of this pixel: gpix + c * Nst
    const bool ld_state = !init && valid;
    unsigned char* wl = Wsm + (il / KCH) * wchunk;   // this pixel's 128-byte K chunk of W
    const int kb = (il % KCH) * ESZ;
    auto store_w = [&](int c, float w) {
      unsigned char* dst = wl + c * 128 + (kb ^ ((c & 7) << 4));
      if (BF) {
        *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(w);
      } else if (SPLIT) {
        const float hi = to_tf32(w);
        *reinterpret_cast<float*>(dst) = hi;
        *reinterpret_cast<float*>(dst + NPC * wchunk) = to_tf32(w - hi);
      } else {
        *reinterpret_cast<float*>(dst) = to_tf32(w);
      }
    };
    if (IS_A) {
      // eq. (update_A), K1 steps in base 2 (y = z log2 e); the state and the
      // TMEM row of the next run of this warp are loaded one run ahead
      float zn[P];
      uint32_t cn[8];
#pragma unroll
      for (int j = 0; j < P; ++j) zn[j] = (ld_state && half < nr) ? St[gpix + (half * P + j) * Nst] : 0.f;
      if (do_c1 && half < nr) tmem_ld8_issue(tbase + tl + (uint32_t)(half * P), cn);
      for (int r = half; r < nr; r += 2) {
        float cv[P], zc[P];
        if (do_c1) {
          tmem_wait_ld8(cn);
#pragma unroll
          for (int j = 0; j < P; ++j) cv[j] = __uint_as_float(cn[j]);
        } else {
#pragma unroll
          for (int j = 0; j < P; ++j) cv[j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < P; ++j) zc[j] = zn[j];
        if (r + 2 < nr) {
#pragma unroll
          for (int j = 0; j < P; ++j) zn[j] = ld_state ? St[gpix + ((r + 2) * P + j) * Nst] : 0.f;
          if (do_c1) tmem_ld8_issue(tbase + tl + (uint32_t)((r + 2) * P), cn);
        }
        const float* G = Gs + r * P * P;
        float a[P], wdev[P], znew[P];  // new a, a - 1/p (shifted accumulation), new log frame
        if (SPLIT) {
          // FP32 throughout, as in the CUDA-core pass: a+ = softmax(log a - eta (G a - c)),
          // G = E^T E, c = E^T x; the deviation a - 1/p from d = expm1(z)
          const float eta = runEta[r];
          float ea[P], se = 0.f;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            ea[j] = expf(zc[j]);
            se += ea[j];
          }
          for (int kk = 0; kk < K1; ++kk) {
            const float inv = 1.f / se;
            float at[P], mx = -EDAA_INF;
#pragma unroll
            for (int j = 0; j < P; ++j) at[j] = ea[j] * inv;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              float g = -cv[j];
#pragma unroll
              for (int k = 0; k < P; ++k) g = fmaf(G[j * P + k], at[k], g);
              zc[j] = fmaf(-eta, g, zc[j]);
              mx = fmaxf(mx, zc[j]);
            }
            se = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              zc[j] -= mx;
              ea[j] = expf(zc[j]);
              se += ea[j];
            }
          }
          float d[P], sd = 0.f;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            d[j] = expm1f(zc[j]);
            sd += d[j];
          }
          const float den = 1.f / ((float)P + sd);
#pragma unroll
          for (int j = 0; j < P; ++j) {
            a[j] = valid ? (1.f + d[j]) * den : 0.f;
            wdev[j] = valid ? ((float)P * d[j] - sd) * den * aref : 0.f;
            znew[j] = zc[j];
          }
        } else {
          // the same step in base 2 (y = z log2 e) with the hardware exponential
          const float e2 = runEta[r] * kLog2e;
          float y[P], ea[P], se = 0.f;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            y[j] = zc[j] * kLog2e;
            ea[j] = ex2_approx(y[j]);
            se += ea[j];
          }
          for (int kk = 0; kk < K1; ++kk) {
            const float inv = rcp_approx(se);
            float at[P], mx = -EDAA_INF;
#pragma unroll
            for (int j = 0; j < P; ++j) at[j] = ea[j] * inv;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              float g = -cv[j];
#pragma unroll
              for (int k = 0; k < P; ++k) g = fmaf(G[j * P + k], at[k], g);
              y[j] = fmaf(-e2, g, y[j]);
              mx = fmaxf(mx, y[j]);
            }
            se = 0.f;
#pragma unroll
            for (int j = 0; j < P; ++j) {
              y[j] -= mx;
              ea[j] = ex2_approx(y[j]);
              se += ea[j];
            }
          }
          const float inv = rcp_approx(se);
#pragma unroll
          for (int j = 0; j < P; ++j) {
            a[j] = valid ? ea[j] * inv : 0.f;
            wdev[j] = valid ? a[j] - aref : 0.f;
            znew[j] = y[j] * kLn2;
          }
        }
#pragma unroll
        for (int j = 0; j < P; ++j) {
          if (valid) St[gpix + (r * P + j) * Nst] = znew[j];
          store_w(r * P + j, wdev[j]);
        }
        // A A^T of this tile's pixels: products in 2^-24 fixed point, summed
        // exactly over the warp's 32 pixels (integer warp reduction)
        int e = 0;
#pragma unroll
        for (int j = 0; j < P; ++j)
#pragma unroll
          for (int k = j; k < P; ++k) {
            const int v = __reduce_add_sync(0xffffffffu, __float2int_rn(a[j] * a[k] * 16777216.f));
            if (lane == 0) aaq[(quarter * Rm + r) * PP + e] += (float)v * (1.f / 16777216.f);
            ++e;
          }
      }
    } else {
      // eq. (update_B): u' = u - lse - eta2 g (initial pass: u = 0.1 * SplitMix64
      // uniform).  The old logits and TMEM rows of kRB runs are loaded together.
      for (int r0 = half; r0 < nr; r0 += 2 * kRB) {
        float uo[kRB][P];
        uint32_t gr[kRB][8];
#pragma unroll
        for (int b = 0; b < kRB; ++b)
#pragma unroll
          for (int j = 0; j < P; ++j)
            uo[b][j] = (ld_state && r0 + 2 * b < nr) ? St[gpix + ((r0 + 2 * b) * P + j) * Nst] : 0.f;
        if (do_c1) {
#pragma unroll
          for (int b = 0; b < kRB; ++b)
            if (r0 + 2 * b < nr) tmem_ld8_issue(tbase + tl + (uint32_t)((r0 + 2 * b) * P), gr[b]);
#pragma unroll
          for (int b = 0; b < kRB; ++b)
            if (r0 + 2 * b < nr) tmem_wait_ld8(gr[b]);
        }
#pragma unroll
        for (int b = 0; b < kRB; ++b) {
          const int r = r0 + 2 * b;
          if (r >= nr) break;
          const float eta = runEta[r];
#pragma unroll
          for (int j = 0; j < P; ++j) {
            const int c = r * P + j;
            float u = -EDAA_INF;
            if (valid) {
              if (init) u = 0.1f * uniform24(cd.seeds[m0 + r], (uint64_t)(i0 + il) * P + j + 1);
              else u = uo[b][j] - colLse[c] - eta * (do_c1 ? __uint_as_float(gr[b][j]) : 0.f);
              St[gpix + c * Nst] = u;  // the new logits (read back below for the weights)
            }
            const int key = __reduce_max_sync(0xffffffffu, ord_key(u));
            if (lane == 0) atomicMax(&colKey[c], key);
          }
        }
      }
      __syncthreads();
      // new running exponents, rescale factors for the accumulators, reference weights
      for (int c = tid; c < nc; c += kThreads) {
        const float Mo = colM[c];
        const float Mn = fmaxf(Mo, tile_exp(colKey[c]));
        colScale[c] = (Mo == Mn || Mo == -EDAA_INF) ? 1.f : ldexpf(1.f, (int)(Mo - Mn));
        if (Mo != Mn && Mo != -EDAA_INF) flags[1] = 1;
        colM[c] = Mn;
        colKey[c] = ord_key(-EDAA_INF);
        colRefW[c] = ldexpf(1.f, colRef[c] - (int)Mn);
      }
      __syncthreads();
      if (!SPLIT && flags[1] && d2_started) {  // exact power-of-two rescale of Acc in TMEM, disjoint 8-column chunks
        for (int b = 0; b < nbt; ++b)
          for (int cc = half * 8; cc < Rgp; cc += 16) {
            float v[8];
            const uint32_t ta = tbase + tl + (uint32_t)(Rgp * (1 + b) + cc);
            tmem_ld8(ta, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] *= colScale[cc + j];
            tmem_st8(ta, v);
          }
      }
      // shifted weights e^u 2^-Mn - 2^(k-Mn) (the reference is added back in the merge)
      for (int r0 = half; r0 < nr; r0 += 2 * kRB) {
        float un[kRB][P];
#pragma unroll
        for (int b = 0; b < kRB; ++b)
#pragma unroll
          for (int j = 0; j < P; ++j) un[b][j] = (valid && r0 + 2 * b < nr) ? St[gpix + ((r0 + 2 * b) * P + j) * Nst] : 0.f;
#pragma unroll
        for (int b = 0; b < kRB; ++b) {
          const int r = r0 + 2 * b;
          if (r >= nr) break;
#pragma unroll
          for (int j = 0; j < P; ++j) {
            const int c = r * P + j;
            float w = 0.f;
            if (valid)
              w = SPLIT ? shifted_weight(un[b][j], colM[c], colRef[c])  // FP32, expm1 near the reference
                        : ex2_approx(fmaf(un[b][j], kLog2e, -colM[c])) - colRefW[c];
            store_w(c, w);
          }
        }
      }
    }
    // ---- 3. Acc += X_bands W^T (W from generic-proxy stores -> async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      flags[1] = 0;
      tc_fence_after();
      if (!flags[0]) {
        const bool first = !d2_started;
        bool ok = true;
        for (int j = 0; j < nc2 && ok; ++j) {
          const int kc = j / SUB, part = j - kc * SUB, bti = kc / NPC, pc = kc - bti * NPC;
          ok = consume([&](unsigned char* st) {
            const uint32_t dcol = tbase + (uint32_t)(Rgp * (1 + bti));
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t da = desc_sw128(su32(st + ks * 32));
              const uint64_t db = desc_sw128(su32(Wsm + pc * wchunk + ks * 32));
              tc_mma<BF>(dcol, da, db, id, ((SPLIT || first) && pc == 0 && part == 0 && ks == 0) ? 0u : 1u);
              if (SPLIT && part == 0)  // X hi * W lo
                tc_mma<BF>(dcol, da, desc_sw128(su32(Wsm + (NPC + pc) * wchunk + ks * 32)), id, 1u);
            }
          });
        }
        if (ok) tc_commit(bar_c2);
        else {
          flags[0] = 1;
          atomicOr(bt->status, 1 << 12);  // contraction-2 pipeline
        }
      }
    }
    if (__syncthreads_or(flags[0])) {
      bail = 1;
      break;
    }
    d2_started = true;
    c2_pending = true;
  }

  // ---- end of the pass: wait for the last Acc update, write the partials
  if (!bail && c2_pending) {
    const int to = mbar_wait(bar_c2, c2_phase, tmo) ? 0 : 1;
    if (to) atomicOr(bt->status, 1 << 13);  // last contraction 2
    bail = __syncthreads_or(to);
    tc_fence_after();
    if (SPLIT && !bail) {
      fold_tile(!folded);
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }
  if (bail) {
    // time-out: report it, give in-flight TMA/MMA work a bounded time to drain, then free TMEM
    if (tid == 0) {
      atomicOr(bt->status, kStatTimeout);
      const unsigned long long t0 = global_ns();
      while ((long long)(global_ns() - t0) < 50000000ll) __nanosleep(1000);
    }
  } else if (d2_started) {
    float* part = cd.part + (size_t)pg * (L + 1) * Mp;
    for (int b = 0; b < nbt; ++b) {
      const int l = b * 128 + quarter * 32 + lane;
      for (int r = half; r < nr; r += 2) {
        float v[8];
        tmem_ld8(tbase + tl + (uint32_t)(Rgp * (1 + (SPLIT ? nbt : 0) + b) + r * P), v);  // split: the running sums
        if (l <= L) {
#pragma unroll
          for (int j = 0; j < P; ++j) part[(size_t)(c0 + r * P + j) * (L + 1) + l] = v[j];  // lanes: consecutive bands
        }
      }
    }
  } else {
    // no tile: zero partials
    float* part = cd.part + (size_t)pg * (L + 1) * Mp;
    for (int e = tid; e < (L + 1) * nc; e += kThreads) part[(size_t)c0 * (L + 1) + e] = 0.f;
  }
  __syncthreads();
  if (!bail) {
    if (IS_A) {
      for (int e = tid; e < nr * PP; e += kThreads) {
        const int r = e / PP, pe = e - r * PP;
        float v = 0.f;
        for (int q = 0; q < 4; ++q) v += aaq[(q * Rm + r) * PP + pe];
        int j = 0, rem = pe;
        while (rem >= P - j) {
          rem -= P - j;
          ++j;
        }
        const int k = j + rem;
        float* dst = cd.paa + ((size_t)pg * cd.M + m0 + r) * P * P;
        dst[j * P + k] = v;
        dst[k * P + j] = v;
      }
    } else {
      for (int c = tid; c < nc; c += kThreads) cd.pmax[(size_t)pg * Mp + c0 + c] = colM[c];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512) : "memory");
  // the barriers' shared memory is reused by the next phase: invalidate them first
  if (tid == 0) {
    for (int b = 0; b < 2 * kTcStages + 2; ++b)
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(su32(full + b)) : "memory");
  }
  __syncthreads();
}

}  // namespace edaa
