// The tcgen05 pass work item (see edaa_tc.cuh for the scheme).  Included by
// edaa_pass_p.cu, instantiated per p.
#pragma once
#include "edaa_tc.cuh"

namespace edaa {

// tcgen05.st of P (1..8) consecutive 32-bit TMEM columns from v (32 lanes,
// warp-collective), then the wait for the stores.  The callers store at
// column r*P: for P = 1, 2, 4, 8 that is a multiple of the width and one
// .xP store is used; other P store column by column.
template <int P>
__device__ __forceinline__ void tmem_st_p(uint32_t ta, const float (&v)[P]) {
  if constexpr (P == 8) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
  } else if constexpr (P == 4) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(ta), "r"(__float_as_uint(v[0])),
                 "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3]))
                 : "memory");
  } else if constexpr (P == 2) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(ta), "r"(__float_as_uint(v[0])),
                 "r"(__float_as_uint(v[1]))
                 : "memory");
  } else {
#pragma unroll
    for (int j = 0; j < P; ++j)
      asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(ta + (uint32_t)j), "r"(__float_as_uint(v[j]))
                   : "memory");
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 0.1 u for the P entries of pixel i of a run with seed `seed`: u from
// SplitMix64 outputs i*P + j + 1, top 24 bits (eq. initB0), bit for bit the
// values of the CUDA-core passes (the split-operand pass, which is held to
// the FP32 path's accuracy, draws them here instead of reading the 16-bit
// table).  Consecutive outputs differ by one gamma increment of the state.
template <int P>
__device__ __forceinline__ void initial_logits(uint64_t seed, uint64_t i, float (&u0)[P]) {
  uint64_t z = seed + (i * (uint64_t)P + 1ull) * kSplitMixGamma;
#pragma unroll
  for (int j = 0; j < P; ++j) {
    u0[j] = 0.1f * ((float)(splitmix64_mix(z) >> 40) * (1.0f / 16777216.0f));
    z += kSplitMixGamma;
  }
}

// PREC: 0 TF32, 1 BF16, 2 split TF32 (x = hi + lo; products hi*hi + hi*lo + lo*hi,
// and the element-wise steps in full FP32 as in the CUDA-core pass).
template <int P, bool IS_A, int PREC>
__device__ __noinline__ void tc_pass_item(const Batch* __restrict__ bt, const CubeDev& cd, int rg, int pg,
                                          unsigned char* smem_raw, int K1, bool init) {
  constexpr bool BF = PREC == 1, SPLIT = PREC == 2;
  constexpr int SUB = SPLIT ? 2 : 1;  // stream chunks per 128-byte K chunk (split: high part, then low part)
  constexpr bool TWO = SPLIT || !IS_A;  // contraction 1 reads a high and a low panel part
  constexpr int PP = P * (P + 1) / 2;
  constexpr int ESZ = BF ? 2 : 4;
  constexpr int KCH = 128 / ESZ;   // elements per 128-byte row (32 tf32, 64 bf16)
  constexpr int NPC = 128 / KCH;   // pixel chunks per 128-pixel tile
  constexpr uint32_t FMT = BF ? 1u : 2u;
  // BF16: whole X tiles, contraction 2 reads them as an MN-major operand
  // (TF32 keeps the stage ring and the band-major copy of X)
  constexpr bool MNX = BF;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quarter = warp & 3, half = warp >> 2;
  const int L = cd.L, N = cd.N, Mp = cd.Mp, Rm = cd.Rm;
  const int m0 = rg * Rm, nr = min(Rm, cd.M - m0), c0 = m0 * P, nc = nr * P;
  const int Rgp = cd.tc_rgp, nkc = cd.tc_nkc, nbt = cd.tc_nbt;
  const long long tmo = bt->timeout_ns;
  const CUtensorMap* tmX = cd.tmaps + TM_X;
  const CUtensorMap* tmXT = cd.tmaps + TM_XT;
  const CUtensorMap* tmPan = cd.tmaps + (IS_A ? TM_E : TM_S);
  const CUtensorMap* tmXlo = cd.tmaps + TM_XLO;  // split operands: the low parts
  const CUtensorMap* tmXTlo = cd.tmaps + TM_XTLO;
  const CUtensorMap* tmPanLo = cd.tmaps + (IS_A ? TM_ELO : TM_SLO);
  const CUtensorMap* tmState = cd.tmaps + (IS_A ? TM_STATE : TM_R16);
  const TcSmem S = tc_smem(Rgp, ESZ, SPLIT, P, IS_A, L, bt->smem_bytes);
  const uint32_t NS = S.stages;
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Wsm = sm + (S.w_off - 1024u);
  float* Sst = reinterpret_cast<float*>(sm + (S.state_off - 1024u));  // A: state [column][128 pixels]
  const uint16_t* R16 = reinterpret_cast<const uint16_t*>(Sst);       // B: uniforms [column][128 pixels]
  const uint32_t wchunk = ((uint32_t)Rgp * 128u + 1023u) & ~1023u;
  const uint32_t pnl = wchunk;  // a panel chunk (Rgp rows of 128 B), 1024-byte aligned
  unsigned char* Psm = sm + (S.panel_off - 1024u);  // resident panel: [part][K chunk] chunks of pnl bytes
  unsigned char* ring = Psm + (TWO ? 2u : 1u) * (uint32_t)nkc * pnl;
  unsigned char* misc = sm + (S.misc_off - 1024u);
  const TcMisc ML = tc_misc(Rgp, P, IS_A);
  const int cs = (int)ML.cs;                               // column-array length
  uint64_t* full = reinterpret_cast<uint64_t*>(misc);      // kTcMaxStages (BF16: one per X tile buffer)
  uint64_t* empty = full + kTcMaxStages;                   // kTcMaxStages
  uint64_t* bar_c1 = empty + kTcMaxStages;
  uint64_t* bar_c2 = bar_c1 + 1;
  uint64_t* bar_st = bar_c2 + 1;                           // the tile's table slice (A state, B uniforms)
  uint64_t* bar_pn = bar_st + 1;                           // the resident panel
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_pn + 1);
  int* flags = reinterpret_cast<int*>(tmem_slot + 4);      // [0] bail, [1] rescale needed
  // B: every column keeps its weights as e^u 2^-F in a power-of-two frame F
  // (exact rescales); F starts at the reference exponent k and follows the
  // largest logit seen, one tile late
  float* colF = reinterpret_cast<float*>(misc + ML.cols);  // frame F of Acc and of this tile's weights (B)
  int* colKey = reinterpret_cast<int*>(colF + cs);         // tile maximum logit (B)
  float* colScale = reinterpret_cast<float*>(colKey + cs);  // 2^(F - Fn), the pending rescale (B)
  float* colLam = colScale + cs;                           // Lambda, the logits' offset (B)
  int* colRef = reinterpret_cast<int*>(colLam + cs);       // reference exponent k (B)
  float* colFn = reinterpret_cast<float*>(colRef + cs);    // the frame after this tile (B)
  // (C, 2^(k - F)) per column (B): C = (kR16Scale / 2 - Lambda) log2 e - F and the reference weight
  float2* colCW = reinterpret_cast<float2*>(colFn + cs);
  float* runEta = reinterpret_cast<float*>(misc + ML.eta);  // Rm (<= 128)
  float* Gs = reinterpret_cast<float*>(misc + ML.g);       // Rm x P x P (A)
  float* aaq = reinterpret_cast<float*>(misc + ML.aaq);    // 4 x Rm x PP (A)

  // ---- set-up: barriers, TMEM (512 columns: one CTA per SM), per-run constants
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(512)
                 : "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kTcMaxStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(bar_c1, 1);
    mbar_init(bar_c2, 1);
    mbar_init(bar_st, 1);
    mbar_init(bar_pn, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    flags[0] = 0;
    flags[1] = 0;
    flags[2] = 0;
  }
  for (int c = tid; c < cs; c += kThreads) {
    colKey[c] = ord_key(-EDAA_INF);
    colScale[c] = 1.f;
    colLam[c] = 0.f;
  }
  if (!IS_A)
    for (int c = tid; c < cs; c += kThreads) {
      // k is a lower bound of log2 of the column's mean weight, so its largest
      // weight is at least 2^(k - 1/2): a first frame of k never underflows
      const int k = (!init && c < nc) ? ref_exponent(cd, m0 + c / P, c0 + c) : 0;
      colRef[c] = k;
      colF[c] = (float)k;
      colFn[c] = (float)k;
      colCW[c].y = 1.f;
      if (c < nc) {
        if (!init) colLam[c] = (float)cd.lamd[c0 + c];
        if (pg == 0) cd.bref[c0 + c] = k;
      }
      colCW[c].x = (0.5f * kR16Scale - colLam[c]) * kLog2e - (float)k;
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
  // one TMA box of the tile's table slice: 128 pixels x the group's rows (A: float, B: uint16)
  const uint32_t state_bytes = 128u * (IS_A ? 4u : 2u) * (uint32_t)(Rm * P);

  // ---- the chunk stream (thread 0).  The panel is loaded once, before the
  // first tile.  Per tile: contraction 1 (nkc chunks of the pixel-major X; not
  // in the initial passes), then contraction 2 (nbt * NPC chunks of the
  // band-major X).  Chunk k uses ring stage k % NS.  Loads run up to NS
  // chunks ahead of the MMAs, so contraction 2's X streams in during the
  // epilogue and the next tile's contraction 1 after it.
  const int nc1 = do_c1 ? nkc * SUB : 0;
  const int nc2 = nbt * NPC * SUB;
  const int per_tile = nc1 + nc2;
  const int ntl = pg < cd.ntiles ? (cd.ntiles - pg + cd.Pg - 1) / cd.Pg : 0;
  const uint32_t total = (uint32_t)(ntl * per_tile);
  // Ring bookkeeping of thread 0, all incremental (no divisions: this code
  // runs on one lane on the critical path of every tile).  Chunk k uses
  // stage k % NS in round k / NS; a load waits for the previous round's
  // release of its stage (empty barrier), an issue for its own round's
  // arrival (full barrier).
  constexpr int SUBS = SPLIT ? 1 : 0, NPCS = ESZ == 2 ? 1 : 2;  // log2 SUB, log2 NPC
  uint32_t loaded = 0, issued = 0;
  uint32_t ld_s = 0, ld_round = 0, is_s = 0, is_round = 0;
  int ld_j = 0, ld_ti0 = pg * kTcTile;  // chunk within its tile, first pixel of that tile
  const int ti_step = cd.Pg * kTcTile;
  // Load the next chunk once the MMAs that read its stage's previous chunk
  // are done: `block` waits for them (bounded), otherwise a busy stage
  // returns 0 and nothing is issued.  Returns 1 loaded, 0 busy, -1 timed out.
  auto load_chunk = [&](bool block) -> int {
    if (ld_round > 0) {
      const uint32_t par = (ld_round & 1u) ^ 1u;
      if (block ? !mbar_wait(empty + ld_s, par, tmo) : !mbar_test(empty + ld_s, par)) return block ? -1 : 0;
    }
    unsigned char* dst = ring + ld_s * kTcStageBytes;
    uint64_t* fb = full + ld_s;
    mbar_expect(fb, kTcStageBytes);
    if (ld_j < nc1) {  // X chunk (split: high part, then low part)
      const int kc = ld_j >> SUBS, part = ld_j & SUBS;
      tma2d(dst, part ? tmXlo : tmX, kc * KCH, ld_ti0, fb);
    } else {  // band-major X chunk (split: high part, then low part)
      const int jj = ld_j - nc1, kc = jj >> SUBS, part = jj & SUBS, bti = kc >> NPCS, pc = kc & (NPC - 1);
      tma2d(dst, part ? tmXTlo : tmXT, ld_ti0 + pc * KCH, bti * 128, fb);
    }
    if (++ld_s == NS) {
      ld_s = 0;
      ++ld_round;
    }
    if (++ld_j == per_tile) {
      ld_j = 0;
      ld_ti0 += ti_step;
    }
    ++loaded;
    return 1;
  };
  // Top the ring up without waiting: stops at the first stage still read by
  // MMAs in flight (the just-issued ones, typically), so issuing is never
  // held up by the tensor core's progress.
  auto fill = [&]() {
    while (loaded < total && loaded < issued + NS && load_chunk(false) == 1) {
    }
  };
  // MMAs of the next chunk (loading it first if the ring has not yet); its
  // stage is released by the MMAs' commit
  auto consume = [&](auto&& mma) -> bool {
    while (loaded <= issued)
      if (load_chunk(true) != 1) return false;
    if (!mbar_wait(full + is_s, is_round & 1u, tmo)) return false;
    tc_fence_after();
    mma(ring + is_s * kTcStageBytes);
    tc_commit(empty + is_s);
    if (++is_s == NS) {
      is_s = 0;
      ++is_round;
    }
    ++issued;
    fill();
    return true;
  };
  if (tid == 0) {  // the maps this pass uses, into the descriptor cache before the first copy
    tmap_prefetch(tmX);
    if (!MNX) tmap_prefetch(tmXT);
    tmap_prefetch(tmState);
    if (do_c1) {
      tmap_prefetch(tmPan);
      if (TWO) tmap_prefetch(tmPanLo);
    }
    if (SPLIT) {
      tmap_prefetch(tmXlo);
      tmap_prefetch(tmXTlo);
    }
  }
  if (tid == 0 && do_c1 && total > 0) {  // the resident panel (high part, then low part)
    mbar_expect(bar_pn, (TWO ? 2u : 1u) * (uint32_t)nkc * (uint32_t)Rgp * 128u);
    for (int kc = 0; kc < nkc; ++kc) {
      tma2d(Psm + kc * pnl, tmPan, kc * KCH, c0, bar_pn);
      if (TWO) tma2d(Psm + (nkc + kc) * pnl, tmPanLo, kc * KCH, c0, bar_pn);
    }
  }
  if (!MNX && tid == 0) fill();
  bool panel_ready = !do_c1;

  // Split operands: contraction 2 of each tile restarts a tile accumulator T
  // (TMEM columns Rgp (1 + b)), and the threads add it into the running sums
  // S (columns Rgp (1 + nbt + b)) in FP32, S = S + T (tile and sums share the
  // B-pass frame; frame changes rescale S).  The tensor core's FP32
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
          for (int j = 0; j < 8; ++j) vs[j] += vt[j];
        }
        tmem_st8(tS, vs);
      }
  };
  bool folded = false;


  uint32_t c1_phase = 0, c2_phase = 0, st_phase = 0;
  bool c2_pending = false, d2_started = false, st_stored = false;
  int bail = 0;
  const float aref = 1.f / (float)P;
  const uint32_t tl = (uint32_t)(quarter * 32) << 16;  // this warp's TMEM lane block

  // B: move Acc (split: the running sums) into the frames Fn by the exact
  // powers of two 2^(F - Fn), then F = Fn.  Callers make sure no contraction 2
  // is in flight.
  auto apply_frames = [&]() {
    if (d2_started)
      for (int b = 0; b < nbt; ++b)
        for (int cc = half * 8; cc < Rgp; cc += 16) {
          float v[8];
          const uint32_t ta = tbase + tl0 + (uint32_t)(Rgp * (1 + (SPLIT ? nbt : 0) + b) + cc);
          tmem_ld8(ta, v);
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] *= colScale[cc + j];
          tmem_st8(ta, v);
        }
    __syncthreads();
    for (int c = tid; c < nc; c += kThreads) {
      colF[c] = colFn[c];
      colScale[c] = 1.f;
      colCW[c] = make_float2((0.5f * kR16Scale - colLam[c]) * kLog2e - colF[c], ldexpf(1.f, colRef[c] - (int)colF[c]));
    }
    if (tid == 0) flags[1] = 0;
    __syncthreads();
  };

  // ---- 2. the epilogue of one tile (pixels i0 .. i0 + ni - 1): warp (quarter,
  // half) = pixels 32*quarter.., runs of parity `half`.  False: a wait timed out.
  auto epilogue = [&](int i0, int ni) -> bool {
    const int il = quarter * 32 + lane;
    const bool valid = il < ni;
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
      if (!init) {  // the state tile has landed
        const int to = mbar_wait(bar_st, st_phase, tmo) ? 0 : 1;
        if (to) atomicOr(bt->status, 1 << 14);  // the A state tile's load
        if (__syncthreads_or(to)) return false;
        st_phase ^= 1;
      }
      // eq. (update_A), K1 steps per (pixel, run).  The run's G = E^T E is
      // symmetric: its p (p + 1) / 2 distinct entries are read into registers
      // once per run, so the K1 steps touch no shared memory.
      for (int r = half; r < nr; r += 2) {
        float cv[P], zc[P], gsym[PP];
        if (do_c1) {
          uint32_t ca[8];
          tmem_ld8_issue(tbase + tl + (uint32_t)(r * P), ca);
          tmem_wait_ld8(ca);
#pragma unroll
          for (int j = 0; j < P; ++j) cv[j] = __uint_as_float(ca[j]);
        } else {
#pragma unroll
          for (int j = 0; j < P; ++j) cv[j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < P; ++j) zc[j] = (!init && valid) ? Sst[(r * P + j) * kTcTile + il] : 0.f;
        {
          const float* G = Gs + r * P * P;
          int e = 0;
#pragma unroll
          for (int j = 0; j < P; ++j)
#pragma unroll
            for (int k = j; k < P; ++k) gsym[e++] = G[j * P + k];
        }
        // G[j][k] from the packed upper triangle
        auto gjk = [&](int j, int k) -> float {
          const int lo = j < k ? j : k, hi = j < k ? k : j;
          return gsym[lo * P - lo * (lo - 1) / 2 + (hi - lo)];
        };
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
              for (int k = 0; k < P; ++k) g = fmaf(gjk(j, k), at[k], g);
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
              for (int k = 0; k < P; ++k) g = fmaf(gjk(j, k), at[k], g);
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
          // the new state in place (the initial pass also zeroes the padding pixels)
          if (valid || init) Sst[(r * P + j) * kTcTile + il] = valid ? znew[j] : 0.f;
          store_w(r * P + j, wdev[j]);
        }
        // A A^T of this tile's pixels: products in 2^-24 fixed point, summed
        // exactly over the warp's 32 pixels (integer warp reduction); lane e
        // keeps the sum of entry e and adds it to the run's sums (one
        // read-modify-write per lane instead of one per entry)
        float a24[P];
#pragma unroll
        for (int k = 0; k < P; ++k) a24[k] = a[k] * 16777216.f;
        constexpr int NH = (PP + 31) / 32;  // lane words per entry set (p = 8: 36 entries)
        int mine[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) mine[h] = 0;
        int e = 0;
#pragma unroll
        for (int j = 0; j < P; ++j)
#pragma unroll
          for (int k = j; k < P; ++k) {
            const int v = __reduce_add_sync(0xffffffffu, __float2int_rn(a[j] * a24[k]));
            mine[e >> 5] = (lane == (e & 31)) ? v : mine[e >> 5];
            ++e;
          }
#pragma unroll
        for (int h = 0; h < NH; ++h)
          if (h * 32 + lane < PP) aaq[(quarter * Rm + r) * PP + h * 32 + lane] += (float)mine[h] * (1.f / 16777216.f);
      }
    } else {
      // eq. (update_B) without stored logits: u = 0.1 r - Lambda - x^T (S + eta2 R),
      // the last term from contraction 1 (initial pass: u = 0.1 r), r from the
      // table slice in shared memory, and the shifted weights
      // e^u 2^-F - 2^(k-F) (the reference is added back in the merge), in one
      // loop over the thread's runs, kRB at a time (their TMEM rows load
      // together).  In base 2, u log2 e - F = q s log2 e + C - g log2 e with
      // s = 0.1 / 2^16 and the column constant C = (s/2 - Lambda) log2 e - F.
      // The frames stay at k unless a weight exceeds 2^96 (then sums of N
      // weights could overflow): such a tile forms its exact column maxima
      // and is redone in the raised frames.  Until then no column maximum is
      // needed: at frame k every column's largest weight is at least 2^-1/2.
      if (!SPLIT) {
        const int to = mbar_wait(bar_st, st_phase, tmo) ? 0 : 1;  // the uniforms have landed
        if (to) atomicOr(bt->status, 1 << 14);
        if (__syncthreads_or(to)) return false;
        st_phase ^= 1;
      }
      constexpr int kRB = 2;
      constexpr float kWmax = 79228162514264337593543950336.f;  // 2^96
      constexpr float kQs = kR16Scale * kLog2e;
      auto b_weights = [&](bool exact) -> float {
        float wmax = 0.f;
        for (int r0 = half; r0 < nr; r0 += 2 * kRB) {
          uint32_t gr[kRB][8];
          if (do_c1) {
#pragma unroll
            for (int b = 0; b < kRB; ++b)
              if (r0 + 2 * b < nr) tmem_ld8_issue(tbase + tl + (uint32_t)((r0 + 2 * b) * P), gr[b]);
          }
          // Every shared-memory input of the kRB x P elements is read before
          // any of their W stores: a load cannot be moved across a store to
          // shared memory, and loads interleaved with the stores would chain
          // the elements' latencies one after another.
          float qv[kRB][P], cv[kRB][P], rv[kRB][P];  // table value, column constant, reference weight
          int kv[kRB][P];                             // split: reference exponent
#pragma unroll
          for (int b = 0; b < kRB; ++b) {
            const int rc = r0 + 2 * b < nr ? r0 + 2 * b : r0;  // a missing run recomputes run r0, stores nothing
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const int c = rc * P + j;
              if (SPLIT) {
                cv[b][j] = colLam[c];
                rv[b][j] = colF[c];
                kv[b][j] = colRef[c];
              } else {
                qv[b][j] = (float)R16[c * kTcTile + il];
                const float2 t = colCW[c];
                cv[b][j] = t.x;
                rv[b][j] = t.y;
              }
            }
          }
          if (do_c1) {
#pragma unroll
            for (int b = 0; b < kRB; ++b)
              if (r0 + 2 * b < nr) tmem_wait_ld8(gr[b]);
          }
          float wv[kRB][P];
#pragma unroll
          for (int b = 0; b < kRB; ++b) {
            const int r = r0 + 2 * b;
            const bool live = r < nr;  // warp-uniform
            const bool act = valid && live;
            const int rc = live ? r : r0;
            float u24[P];  // split operands: the exact 24-bit draw
            if (SPLIT) initial_logits<P>(__ldg(cd.seeds + m0 + rc), (uint64_t)(i0 + il), u24);
#pragma unroll
            for (int j = 0; j < P; ++j) {
              const float g = (do_c1 && live) ? __uint_as_float(gr[b][j]) : 0.f;
              float w = 0.f, e;
              if (SPLIT) {  // FP32, expm1 near the reference
                const float u = act ? (u24[j] - cv[b][j]) - g : -EDAA_INF;
                e = ex2_approx(fmaf(u, kLog2e, -rv[b][j]));
                if (act) w = shifted_weight(u, rv[b][j], kv[b][j]);
              } else {
                const float x2 = act ? fmaf(-g, kLog2e, fmaf(qv[b][j], kQs, cv[b][j])) : -EDAA_INF;  // u log2 e - F
                e = ex2_approx(x2);  // 0 where inactive
                if (act) w = e - rv[b][j];
              }
              wmax = fmaxf(wmax, e);
              wv[b][j] = w;
            }
          }
#pragma unroll
          for (int b = 0; b < kRB; ++b)
            if (r0 + 2 * b < nr)
#pragma unroll
              for (int j = 0; j < P; ++j) store_w((r0 + 2 * b) * P + j, wv[b][j]);
          if (exact) {  // the tile's exact column maxima of u (rare: frames about to overflow)
#pragma unroll
            for (int b = 0; b < kRB; ++b) {
              const int r = r0 + 2 * b;
              if (r >= nr) continue;
              float u24[P];
              if (SPLIT) initial_logits<P>(__ldg(cd.seeds + m0 + r), (uint64_t)(i0 + il), u24);
#pragma unroll
              for (int j = 0; j < P; ++j) {
                const int c = r * P + j;
                const float u0 = SPLIT ? u24[j] : (qv[b][j] + 0.5f) * kR16Scale;
                const float g = do_c1 ? __uint_as_float(gr[b][j]) : 0.f;
                const float u = valid ? (u0 - colLam[c]) - g : -EDAA_INF;
                const int key = __reduce_max_sync(0xffffffffu, ord_key(u));
                if (lane == 0) atomicMax(&colKey[c], key);
              }
            }
          }
        }
        return wmax;
      };
      const float wmax = b_weights(false);
      if (__syncthreads_or(!(wmax <= kWmax))) {
        // weights too large for the frames: exact maxima, raised frames
        // (Acc rescaled: the previous contraction 2 has finished), redo
        b_weights(true);
        __syncthreads();
        for (int c = tid; c < nc; c += kThreads) {
          const float te = tile_exp(colKey[c]);
          colKey[c] = ord_key(-EDAA_INF);
          const float Fn = fmaxf(colF[c], te);
          colFn[c] = Fn;
          colScale[c] = ldexpf(1.f, (int)(colF[c] - Fn));
        }
        __syncthreads();
        apply_frames();
        b_weights(false);
      }
    }
    return true;
  };

  if constexpr (MNX) {
    // ---- BF16: whole X tiles in NB (1 or 2) buffers.  Tile q uses buffer
    // q % NB; its X is loaded once and read by both contractions.  Thread 0,
    // after tile q's epilogue: the state store (A) or the next uniforms (B),
    // contraction 2 of tile q, the next state slice (A), contraction 1 of
    // tile q + 1.  The other buffer's next X is loaded at the start of the
    // epilogue, once contraction 2 of the previous tile has read it.
    const uint32_t NB = S.stages;
    const int nkx = tc_nkx(L);
    const uint32_t xtb = (uint32_t)nkx * kTcStageBytes;
    const uint32_t id2 = tc_idesc(128, Rgp, FMT, true);  // contraction 2: A = X^T, MN-major
    const bool need_slice = IS_A ? !init : true;
    auto xbuf = [&](int q) -> uint32_t { return NB == 2 ? (uint32_t)(q & 1) : 0u; };
    auto xpar = [&](int q) -> uint32_t { return (uint32_t)(NB == 2 ? (q >> 1) : q) & 1u; };
    auto load_x = [&](int q) {
      const uint32_t b = xbuf(q);
      unsigned char* dst = ring + b * xtb;
      mbar_expect(full + b, xtb);
      const int ti0 = (pg + q * cd.Pg) * kTcTile;
      for (int kc = 0; kc < nkx; ++kc) tma2d(dst + kc * kTcStageBytes, tmX, kc * KCH, ti0, full + b);
    };
    auto load_slice = [&](int q) {
      mbar_expect(bar_st, state_bytes);
      tma2d(Sst, tmState, (pg + q * cd.Pg) * kTcTile, c0, bar_st);
    };
    // C = X_q Panel^T (B: high and low panel parts)
    auto issue_c1 = [&](int q) -> bool {
      if (!mbar_wait(full + xbuf(q), xpar(q), tmo)) return false;
      tc_fence_after();
      unsigned char* xb = ring + xbuf(q) * xtb;
      for (int kc = 0; kc < nkc; ++kc) {
        const uint64_t da0 = desc_sw128(su32(xb + kc * kTcStageBytes));
        const uint64_t dh0 = desc_sw128(su32(Psm + kc * pnl));
        const uint64_t dl0 = desc_sw128(su32(Psm + (nkc + kc) * pnl));
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          tc_mma<BF>(tbase, da0 + 2u * ks, dh0 + 2u * ks, id, (kc | ks) ? 1u : 0u);
          if (TWO) tc_mma<BF>(tbase, da0 + 2u * ks, dl0 + 2u * ks, id, 1u);
        }
      }
      tc_commit(bar_c1);
      return true;
    };
    // Acc_b += X_q^T W for each 128-band tile b: A is the X tile read MN-major,
    // two consecutive 64-band chunks from chunk cb (the last band tile starts
    // one chunk early when the chunk count is odd: its first 64 rows repeat
    // bands of the tile before and are not written out); K = 16 pixels per MMA
    // (2048 bytes of X, 32 bytes of a W row)
    auto issue_c2 = [&](int q, bool first) -> bool {
      if (!do_c1 && !mbar_wait(full + xbuf(q), xpar(q), tmo)) return false;
      tc_fence_after();
      unsigned char* xb = ring + xbuf(q) * xtb;
      for (int b = 0; b < nbt; ++b) {
        const int cb = min(2 * b, nkx - 2);
        const uint32_t dcol = tbase + (uint32_t)(Rgp * (1 + b));
        const uint64_t da0 = desc_sw128_mn(su32(xb + cb * kTcStageBytes), kTcStageBytes);
        for (int pc = 0; pc < NPC; ++pc) {
          const uint64_t db0 = desc_sw128(su32(Wsm + pc * wchunk));
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            tc_mma<BF>(dcol, da0 + (uint64_t)(pc * 512 + ks * 128), db0 + 2u * ks, id2,
                       (first && pc == 0 && ks == 0) ? 0u : 1u);
        }
      }
      tc_commit(bar_c2);
      return true;
    };
    if (tid == 0 && ntl > 0) {
      load_x(0);
      if (need_slice) load_slice(0);
      if (do_c1) {
        bool ok = mbar_wait(bar_pn, 0, tmo);
        tc_fence_after();
        if (ok) ok = issue_c1(0);
        if (!ok) {
          flags[0] = 1;
          atomicOr(bt->status, 1 << 9);  // contraction-1 pipeline
        }
      }
    }
    __syncthreads();
    for (int q = 0; q < ntl; ++q) {
      const int i0 = (pg + q * cd.Pg) * kTcTile;
      const int ni = min(kTcTile, N - i0);
      // contraction 2 of the previous tile (W and its X buffer are free), then
      // contraction 1 of this tile
      int to = flags[0] ? 1 : 0;
      if (!to && c2_pending) to = mbar_wait(bar_c2, c2_phase, tmo) ? 0 : 2;
      if (!to && do_c1) to = mbar_wait(bar_c1, c1_phase, tmo) ? 0 : 3;
      if (to > 1) atomicOr(bt->status, 1 << (to == 2 ? 11 : 10));
      if (__syncthreads_or(to)) {
        bail = 1;
        break;
      }
      if (c2_pending) {
        c2_phase ^= 1;
        c2_pending = false;
      }
      if (do_c1) c1_phase ^= 1;
      tc_fence_after();
      if (tid == 0 && NB == 2 && q + 1 < ntl) load_x(q + 1);
      if (!epilogue(i0, ni)) {
        bail = 1;
        break;
      }
      // W and the A state from generic-proxy stores -> async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const bool more = q + 1 < ntl;
        if (IS_A) {  // the new state tile back to global memory
          tma2d_store(tmState, i0, c0, Sst);
          bulk_commit();
          st_stored = true;
        } else if (more) {
          load_slice(q + 1);  // the uniforms have been read
        }
        bool ok = issue_c2(q, !d2_started);
        if (!ok) atomicOr(bt->status, 1 << 12);  // contraction-2 X tile
        if (ok && more) {
          if (IS_A) {
            bulk_wait_read();  // the store has read the state buffer
            if (need_slice) load_slice(q + 1);
          }
          if (NB == 1) {  // one buffer: contraction 2 must have read it
            ok = mbar_wait(bar_c2, c2_phase, tmo);
            if (ok) load_x(q + 1);
            else atomicOr(bt->status, 1 << 11);
          }
          if (ok && do_c1) {
            ok = issue_c1(q + 1);
            if (!ok) atomicOr(bt->status, 1 << 9);
          }
        }
        if (!ok) flags[0] = 1;
      }
      d2_started = true;
      c2_pending = true;
      if (__syncthreads_or(flags[0])) {
        bail = 1;
        break;
      }
    }
  } else {
    for (int q = 0; q < ntl; ++q) {
      const int i0 = (pg + q * cd.Pg) * kTcTile;
      const int ni = min(kTcTile, N - i0);
      // the previous tile's state store must have read the buffer before it is
      // rewritten; then the tile's table slice (A: the state, B: the uniforms)
      // by one TMA load
      if (IS_A && tid == 0 && st_stored) bulk_wait_read();
      if ((IS_A ? !init : !SPLIT) && tid == 0 && !flags[0]) {
        mbar_expect(bar_st, state_bytes);
        tma2d(Sst, tmState, i0, c0, bar_st);
      }
      // ---- 1. C = X_tile Panel^T (skipped for the initial passes: c = 0)
      if (do_c1) {
        if (tid == 0 && !flags[0]) {
          bool ok = true;
          if (!panel_ready) {
            ok = mbar_wait(bar_pn, 0, tmo);
            panel_ready = true;
            tc_fence_after();
          }
          for (int j = 0; j < nc1 && ok; ++j) {
            const int kc = j >> SUBS, part = j & SUBS;
            ok = consume([&](unsigned char* st) {
              // descriptors of the chunk's first K step; each further 32-byte K
              // step adds 2 to the start-address field (address / 16)
              const uint64_t da0 = desc_sw128(su32(st));
              const uint64_t dh0 = desc_sw128(su32(Psm + kc * pnl));  // the resident panel's K chunk kc
              const uint64_t dl0 = desc_sw128(su32(Psm + (nkc + kc) * pnl));
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint64_t da = da0 + 2u * ks;
                tc_mma<BF>(tbase, da, dh0 + 2u * ks, id, (kc | ks | part) ? 1u : 0u);
                if (TWO && part == 0)  // X * P lo (split: X hi * P lo)
                  tc_mma<BF>(tbase, da, dl0 + 2u * ks, id, 1u);
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
        if (tid == 0) fill();  // contraction 1's stages are free: stream the next chunks during the epilogue
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
        if (tid == 0) fill();  // the previous contraction 2's stages are free as well
        if (SPLIT) {
          fold_tile(!folded);
          folded = true;
        }
      }
      if (!epilogue(i0, ni)) {
        bail = 1;
        break;
      }
      // ---- 3. Acc += X_bands W^T (W and the A state from generic-proxy stores -> async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        if (IS_A) {  // the new state tile back to global memory
          tma2d_store(tmState, i0, c0, Sst);
          bulk_commit();
          st_stored = true;
        }
        if (!flags[0]) {
          const bool first = !d2_started;
          bool ok = true;
          for (int j = 0; j < nc2 && ok; ++j) {
            const int kc = j >> SUBS, part = j & SUBS, bti = kc >> NPCS, pc = kc & (NPC - 1);
            ok = consume([&](unsigned char* st) {
              const uint32_t dcol = tbase + (uint32_t)(Rgp * (1 + bti));
              const uint64_t da0 = desc_sw128(su32(st));
              const uint64_t db0 = desc_sw128(su32(Wsm + pc * wchunk));
              const uint64_t dl0 = desc_sw128(su32(Wsm + (NPC + pc) * wchunk));
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint64_t da = da0 + 2u * ks;
                tc_mma<BF>(dcol, da, db0 + 2u * ks, id,
                           ((SPLIT || first) && pc == 0 && part == 0 && ks == 0) ? 0u : 1u);
                if (SPLIT && part == 0)  // X hi * W lo
                  tc_mma<BF>(dcol, da, dl0 + 2u * ks, id, 1u);
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
      // TMEM lane 0 of band tile b holds band lb (BF16: the tile's first X chunk)
      const int lb = MNX ? 64 * min(2 * b, tc_nkx(L) - 2) : 128 * b;
      const int l = lb + quarter * 32 + lane;
      for (int r = half; r < nr; r += 2) {
        float v[8];
        tmem_ld8(tbase + tl + (uint32_t)(Rgp * (1 + (SPLIT ? nbt : 0) + b) + r * P), v);  // split: the running sums
        if (l >= 128 * b && l <= L) {
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
  // the state stores complete in global memory before the phase ends (they
  // never wait on other CTAs, so this wait is not bounded)
  if (IS_A && tid == 0 && st_stored) {
    bulk_wait_all();
    asm volatile("fence.proxy.async.global;" ::: "memory");
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
      for (int c = tid; c < nc; c += kThreads) cd.pmax[(size_t)pg * Mp + c0 + c] = colF[c];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512) : "memory");
  // the barriers' shared memory is reused by the next phase: invalidate them first
  if (tid == 0) {
    for (int b = 0; b < 2 * kTcMaxStages + 4; ++b)
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(su32(full + b)) : "memory");
  }
  __syncthreads();
}

}  // namespace edaa
