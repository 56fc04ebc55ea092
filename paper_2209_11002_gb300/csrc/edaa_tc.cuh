// Tensor-core (tcgen05) pass of EDAA for batched ensembles (TF32 or BF16
// operands, FP32 accumulation in tensor memory), sm_103a.
//
// Per CTA: one run group (Rg = Rm*p columns, padded to Rgp, a multiple of
// 16) and the pixel tiles pg, pg + Pg, ... of 128 pixels.  Per tile:
//   1. C (128 px x Rgp) = X_tile (128 x L) * Panel^T by tcgen05.mma (128-byte
//      swizzle, K-major operands), the accumulator in TMEM columns [0, Rgp).
//      The panel stays in shared memory for the whole pass: E for the A-pass;
//      for the B-pass S + eta2 R, the running sum of eta2 times the
//      B-gradient factors R of every B-step so far (eq. update_B), as a high
//      and a low part (two MMAs per K step).
//   2. Epilogue (8 warps; warp w reads TMEM lanes 32*(w%4).. = its pixels and
//      handles the runs of parity w/4):
//      A: the tile's log-abundance state arrives in shared memory by one TMA
//         load; the K1 fused A-steps update it in place and one TMA store
//         writes it back.
//      B: no per-pixel state.  The logits are u = 0.1 r - Lambda - C, with r
//         the B^0 uniforms (eq. initB0) from a 16-bit table slice loaded by
//         TMA with the tile (split operands: the exact 24-bit draw from
//         SplitMix64 in registers); the weights are formed in a fixed
//         power-of-two frame per column.
//      Both write W = weights - reference (shifted accumulation) into shared
//      memory in the swizzled K-major layout the MMA reads.
//   3. Acc (bands x Rgp) += X_bands (128 bands x 128 px) * W^T for each
//      128-band tile; Acc lives in TMEM columns [Rgp*(1+bt), Rgp*(2+bt))
//      across all tiles of the CTA.
// X reaches shared memory in one of two ways:
//   TF32 (and split TF32): a ring of 16 KB stages streams the tile's
//     pixel-major chunks for contraction 1, then the chunks of a band-major
//     copy of X for contraction 2.
//   BF16: the whole pixel-major tile (tc_nkx 64-band chunks) is loaded once
//     into one of two tile buffers, and contraction 2 reads the same chunks
//     as an MN-major operand (bands are the M index: two consecutive 64-band
//     chunks per MMA), so no band-major copy exists.  The next tile's X
//     streams into the other buffer during this tile's epilogue, and the next
//     tile's contraction 1 is issued right behind this tile's contraction 2.
// At the end the accumulators are written as the same per-CTA partials the
// CUDA-core pass writes, so the FP64 merges are shared.  Every mbarrier wait
// is bounded.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "edaa_pass.cuh"

namespace edaa {

constexpr int kTcTile = 128;

// su32, mbar_init, mbar_expect and the bounded mbar_wait live in edaa_pass.cuh
__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* m, int c0, int c1, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          su32(dst)),
      "l"(m), "r"(c0), "r"(c1), "r"(su32(b))
      : "memory");
}
// brings a tensor map (in global memory) into the TMA unit's descriptor cache
__device__ __forceinline__ void tmap_prefetch(const CUtensorMap* m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(m) : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// The same for an MN-major operand with 128-byte swizzle: each 128-byte row
// holds 128 B of consecutive M (or N) indices at one K index, 8 K rows form a
// 1024-byte atom and the atoms follow each other along K (stride 1024 B);
// the next 128 B of M indices start `mn_stride` bytes further on (the
// leading-byte-offset field).
__device__ __forceinline__ uint64_t desc_sw128_mn(uint32_t saddr, uint32_t mn_stride) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((mn_stride >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor: FP32 accumulator, A and B of format fmt (tf32: 2, bf16: 1), K-major
// (a_mn: A is MN-major instead)
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, int fmt, bool a_mn = false) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
template <bool BF>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (BF)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 8 consecutive 32-bit columns (warp-collective)
__device__ __forceinline__ void tmem_ld8(uint32_t ta, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_st8(uint32_t ta, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// the same load without the wait: several loads are issued, then one tmem_wait_ld()
__device__ __forceinline__ void tmem_ld8_issue(uint32_t ta, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
}
// waits for the thread's outstanding TMEM loads; r is tied to the wait so its uses stay after it
__device__ __forceinline__ void tmem_wait_ld8(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

// Hardware base-2 exponential and reciprocal (relative error near 2^-22).
// The tensor-core passes use them: their results feed TF32/BF16 operands
// (2^-11 / 2^-9), so the approximation stays far below the operand rounding.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// element (row, k) of a K-major 128-byte-swizzled tile with 128-byte rows
__device__ __forceinline__ uint32_t sw128_off(int row, int kbyte) {
  return (uint32_t)(row * 128 + (kbyte ^ ((row & 7) << 4)));
}

// TF32 operands are float32 containers rounded to 10 mantissa bits
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}


struct TcSmem {
  uint32_t stages, panel_off, w_off, state_off, misc_off, total;
};
// BF16 X tiles: 128 pixels x kp bands in 64-band (128-byte) chunks, at least
// two (contraction 2 reads two consecutive chunks, 128 bands, per MMA)
__host__ __device__ inline int tc_nkx(int L) {
  const int n = (L + 1 + 63) / 64;
  return n < 2 ? 2 : n;
}
// The misc region: barriers and flags (256 B), eight column arrays of cs
// floats (cs = Rgp rounded up to 32), the run step sizes (128 floats), and for
// the A-pass G = E^T E (Rm x p x p) and the A A^T sums (4 x Rm x p(p+1)/2).
struct TcMisc {
  uint32_t cs, cols, eta, g, aaq, total;
};
__host__ __device__ inline TcMisc tc_misc(int Rgp, int p, bool is_a) {
  TcMisc m;
  const uint32_t rm = (uint32_t)(Rgp / p), pp = (uint32_t)(p * (p + 1) / 2);
  m.cs = ((uint32_t)Rgp + 31u) & ~31u;
  m.cols = 256u;
  m.eta = m.cols + 8u * m.cs * 4u;
  m.g = m.eta + 128u * 4u;
  m.aaq = m.g + (is_a ? rm * (uint32_t)(p * p) * 4u : 0u);
  m.total = (m.aaq + (is_a ? 4u * rm * pp * 4u : 0u) + 1023u) & ~1023u;
  return m;
}
// Shared memory of a tensor-core pass, per pass kind.  The run group's panel
// is resident for the whole pass (nkc K chunks of Rgp rows x 128 B): the
// A-pass's E (split operands: its high and low part), the B-pass's
// S + eta2 R as a high and a low part.  Then the X staging area, in units:
//   TF32 (and split): a ring of stages, each one 128 x 128-byte chunk of X
//     (contraction 1: pixel-major, contraction 2: band-major);
//   BF16: one or two whole 128-pixel X tiles (tc_nkx chunks each), read by
//     both contractions (contraction 2 as an MN-major operand).
// W holds the weights of one 128-pixel tile in 128-byte pixel chunks (split:
// high and low part).  The tile's slice of a per-pixel table follows (Rgp
// rows of 128 pixels): the A-pass's log-abundance state, the B-pass's B^0
// uniforms.  Then the misc region (tc_misc); 1 KB alignment slack first.
constexpr uint32_t kTcStageBytes = 128u * 128u;
constexpr int kTcMaxStages = 8;
__host__ __device__ inline int tc_nkc(int L, int esz) { return (L + 128 / esz - 1) / (128 / esz); }
// bytes of one unit of the X staging area and the most units used
__host__ __device__ inline uint32_t tc_x_unit(int L, int esz) {
  return esz == 2 ? (uint32_t)tc_nkx(L) * kTcStageBytes : kTcStageBytes;
}
// `stages` units of X staging; 0 = as many as fit in `cap` bytes (ring: at
// most kTcMaxStages, at least 2; BF16 tiles: at most 2, at least 1; a layout
// that does not fit says so by its total)
__host__ __device__ inline TcSmem tc_smem_n(int Rgp, int esz, bool split, int p, bool is_a, int L, uint32_t stages,
                                           uint32_t cap) {
  TcSmem s;
  const uint32_t pnl = ((uint32_t)Rgp * 128u + 1023u) & ~1023u;
  const uint32_t pparts = (split || !is_a) ? 2u : 1u;
  const uint32_t wparts = split ? 2u : 1u;
  const uint32_t npc = (uint32_t)esz;  // 128-byte pixel chunks per 128-pixel tile (128 / (128 / esz))
  const uint32_t unit = tc_x_unit(L, esz);
  const uint32_t umax = esz == 2 ? 2u : (uint32_t)kTcMaxStages, umin = esz == 2 ? 1u : 2u;
  s.panel_off = 1024u;
  const uint32_t ring_off = s.panel_off + pparts * (uint32_t)tc_nkc(L, esz) * pnl;
  const uint32_t fixed = wparts * npc * pnl + (((uint32_t)Rgp * (is_a ? 512u : 256u) + 1023u) & ~1023u) +
                         tc_misc(Rgp, p, is_a).total;
  if (stages == 0) {
    const uint32_t room = cap > ring_off + fixed ? cap - ring_off - fixed : 0u;
    stages = room / unit;
    if (stages > umax) stages = umax;
    if (stages < umin) stages = umin;  // does not fit: the total says so
  }
  s.stages = stages;
  s.w_off = ring_off + stages * unit;
  s.state_off = s.w_off + wparts * npc * pnl;
  // the per-tile slice of a per-pixel table: A the state (float), B the B^0 uniforms (uint16)
  s.misc_off = s.state_off + (((uint32_t)Rgp * (is_a ? 512u : 256u) + 1023u) & ~1023u);
  s.total = s.misc_off + tc_misc(Rgp, p, is_a).total;
  return s;
}
// 226 KB: one CTA's 227 KB of shared memory less 1 KB for the program
// kernel's static shared memory
constexpr uint32_t kTcSmemCap = 232448u - 1024u;

// The layout a pass uses: as many stages as fit in the dynamic shared memory
// the kernel was launched with (`cap`, the same for every pass of a batch).
__host__ __device__ inline TcSmem tc_smem(int Rgp, int esz, bool split, int p, bool is_a, int L, uint32_t cap) {
  return tc_smem_n(Rgp, esz, split, p, is_a, L, 0u, cap);
}
__host__ __device__ inline uint32_t tc_smem_max(int Rgp, int esz, bool split, int p, int L, uint32_t cap) {
  const uint32_t a = tc_smem(Rgp, esz, split, p, true, L, cap).total;
  const uint32_t b = tc_smem(Rgp, esz, split, p, false, L, cap).total;
  return a > b ? a : b;
}

// Largest padded run-group width (a multiple of 16): TMEM holds C (Rgp
// columns) and one Acc per 128-band tile (split operands: a per-tile Acc and
// a running sum per band tile), with 8 spare columns so that the 8-wide TMEM
// reads of the last run stay inside the 512 allocated; the shared memory of
// both pass kinds stays within kTcSmemCap with, where that is possible, at
// least three ring stages (TF32) or two X tiles (BF16).
__host__ __device__ inline int tc_rgp_max(int L, int esz, bool split, int p) {
  const int nbt = (L + 1 + 127) / 128;
  int r = ((512 - 8) / (1 + (split ? 2 : 1) * nbt)) & ~15;
  auto fits = [&](int rg, uint32_t st) {
    return tc_smem_n(rg, esz, split, p, true, L, st, kTcSmemCap).total <= kTcSmemCap &&
           tc_smem_n(rg, esz, split, p, false, L, st, kTcSmemCap).total <= kTcSmemCap;
  };
  const uint32_t want = esz == 2 ? 2u : 3u, least = esz == 2 ? 1u : 2u;
  int r3 = r;
  while (r3 > 16 && !fits(r3, want)) r3 -= 16;
  if (fits(r3, want)) return r3;
  while (r > 16 && !fits(r, least)) r -= 16;
  return r;
}

// TMA tensor store shared -> global (bulk group), its commit and waits.
__device__ __forceinline__ void tma2d_store(const CUtensorMap* m, int c0, int c1, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(m), "r"(c0),
               "r"(c1), "r"(su32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the stores' reads of shared memory are done (the buffer may be rewritten)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the stores are complete in global memory
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace edaa
